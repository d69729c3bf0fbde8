"""Column-walk tile lists of the fused level-step (claw_set_tile_walk): CTAs that take contiguous
stretches of tile columns and hand the edge values of shared rows from each tile to the one above
give the same new states, dt and speed maxima, bit for bit, as CTAs striding over the tiles, on
every tiling, with filled, pulled and step-interpolated ghosts, wall and periodic boundaries,
ragged tiles, box stacks that do and do not line up, and runs batched into one launch whose boxes
sit at the same indices; acoustics in a uniform medium and shallow water (a cell-wise medium does
not walk)."""
import numpy as np
import pytest
import torch

from paper_1808_02638_gb300 import inputs

from gpu_helpers import lib_ready, single_grid

pytestmark = pytest.mark.gpu

TILINGS = [(32, 32, 1, 256), (32, 32, 0, 512), (32, 16, 2, 256), (32, 16, 1, 256), (16, 16, 1, 128),
           (16, 16, 0, 128)]

# 128 x 128 in boxes whose columns line up in some stacks and not in others; heights of 40 and
# 48 give ragged tiles (8 rows) in the middle of a walk
MIXED_BOXES = [(0, 0, 64, 40), (0, 40, 32, 40), (32, 40, 32, 40), (0, 80, 32, 48), (32, 80, 32, 48),
               (64, 0, 32, 128), (96, 0, 32, 40), (96, 40, 32, 40), (96, 80, 32, 48)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _same(A, B, levels=None):
    torch.cuda.synchronize()
    for L in range(A.nlev) if levels is None else levels:
        for ri, run in enumerate(A.runs):
            if L >= len(run.levels):
                continue
            for n in range(len(run.levels[L].boxes)):
                assert np.array_equal(A.interior(ri, L, n), B.interior(ri, L, n)), (ri, L, n)
    assert torch.equal(A.dt, B.dt)
    assert A.sync_status() == 0 and B.sync_status() == 0


def _random_velocity(run, q, seed):
    lev = run.levels[0]
    for k, b in enumerate(lev.boxes):
        v = inputs.box_view(q, lev.qoff[k], int(b[2]), int(b[3]), 3)
        v[...] = inputs.uniform(seed + k, v.size).reshape(v.shape) - 0.5


@pytest.mark.parametrize("tiling", TILINGS)
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 2, 2), (2, 0, 1, 1)])
def test_single_level_walk_equals_stride_uniform_medium(tiling, bc):
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(128, pulse=False, seed=300, bc=bc, boxes=MIXED_BOXES)
    _random_velocity(run, q, 300)
    A = Hierarchy([run], [[q]], rho0=1.0, K0=4.0, tiling=tiling, walk=1)
    B = Hierarchy([run], [[q]], rho0=1.0, K0=4.0, tiling=tiling, walk=0)
    for h in (A, B):
        h.init_dt()
        for _ in range(3):
            h.coarse_step()
        h.fused = True   # the one-launch step: pulled ghosts and Eq. cfl on the device
        for _ in range(3):
            h.coarse_step()
    _same(A, B)


SWE_TILINGS = [(16, 16, 1, 256), (16, 16, 0, 256), (32, 16, 1, 512), (32, 16, 0, 512)]


@pytest.mark.parametrize("tiling", SWE_TILINGS)
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 2, 2)])
def test_shallow_water_walk_equals_stride(tiling, bc):
    # the shallow-water step hands over its Roe states, strengths, limited parts and transverse
    # parts of the shared rows the same way
    from paper_1808_02638_gb300.solver import Hierarchy
    run, _ = single_grid(128, bc=bc, boxes=MIXED_BOXES)
    q = inputs.init_swe(run, run.levels[0], u0=0.2, v0=-0.1)
    A = Hierarchy([run], [[q]], tiling=tiling, system="shallow_water", grav=1.0, walk=1)
    B = Hierarchy([run], [[q]], tiling=tiling, system="shallow_water", grav=1.0, walk=0)
    for h in (A, B):
        h.init_dt()
        for _ in range(3):
            h.coarse_step()
        h.fused = True
        for _ in range(3):
            h.coarse_step()
    _same(A, B)


def test_shallow_water_three_levels_walk_equals_stride():
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q = [inputs.init_swe(run, lev, u0=0.2, v0=0.1) for lev in run.levels]
    hs = []
    for walk in (1, 0):
        H = Hierarchy([run], [q], tiling=(16, 16, 1, 256), system="shallow_water", grav=1.0, walk=walk)
        H.init_dt()
        for _ in range(2):
            H.coarse_step()
        hs.append(H)
    _same(*hs)


def test_only_uniform_medium_levels_walk():
    # column walks are built for the uniform medium only: a cell-wise level rejects walk = 1 and
    # keeps striding under the automatic choice
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(128, pulse=False, seed=310, boxes=MIXED_BOXES)
    lev = run.levels[0]
    rho, K = np.ones(lev.csize), np.full(lev.csize, 4.0)
    H = Hierarchy([run], [[q]], [[rho]], [[K]])
    with pytest.raises(claw.ClawError):
        claw.claw_set_tile_walk(H.ctx, 0, 1)
    claw.claw_set_tile_walk(H.ctx, 0, 0)
    claw.claw_set_tile_walk(H.ctx, 0, -1)


@pytest.mark.parametrize("ghosts", ["pull", "pull+interp", "fill"])
def test_three_level_hierarchy_walk_equals_stride(ghosts):
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    hs = []
    for walk in (1, 0):
        H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, tiling=(16, 16, 1, 128), walk=walk)
        H.fuse_interp = [ghosts == "pull+interp"] * H.nlev
        H.pull_levels = [ghosts != "fill"] * H.nlev
        H.init_dt()
        for _ in range(3):
            H.coarse_step()
        hs.append(H)
    _same(*hs)


def test_batched_runs_with_the_same_box_indices_walk_equals_stride():
    # two runs with the same boxes in their own index spaces and different data: no walk may
    # continue from one run's box into the other's
    from paper_1808_02638_gb300.solver import Hierarchy
    runs, qs = [], []
    for seed in (400, 500):
        run, q = single_grid(128, pulse=False, seed=seed, boxes=MIXED_BOXES)
        _random_velocity(run, q, seed)
        runs.append(run)
        qs.append([q])
    A = Hierarchy(runs, qs, rho0=1.0, K0=4.0, tiling=(32, 16, 2, 256), walk=1)
    B = Hierarchy(runs, qs, rho0=1.0, K0=4.0, tiling=(32, 16, 2, 256), walk=0)
    for h in (A, B):
        h.init_dt()
        for _ in range(4):
            h.coarse_step()
    _same(A, B)


@pytest.mark.parametrize("boxes", [[(0, 0, 64, 64)], [(0, 0, 32, 8), (0, 8, 32, 8), (0, 16, 16, 16), (16, 16, 16, 16)]])
def test_walk_on_a_level_with_fewer_tiles_than_ctas(boxes):
    # a forced walk on a tiny level: most CTAs get an empty stretch, chains of one or two tiles
    from paper_1808_02638_gb300.solver import Hierarchy
    n = max(b[0] + b[2] for b in boxes)
    run, q = single_grid(n, pulse=False, seed=600, boxes=boxes)
    _random_velocity(run, q, 600)
    hs = []
    for walk in (1, 0):
        H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0, tiling=(32, 16, 2, 256), walk=walk)
        H.init_dt()
        H.fused = True
        for _ in range(4):
            H.coarse_step()
        hs.append(H)
    _same(*hs)


def test_walk_switch_rejects_bad_values():
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(64)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    for bad in (-2, 2):
        with pytest.raises(claw.ClawError):
            claw.claw_set_tile_walk(H.ctx, 0, bad)
    claw.claw_set_tile_walk(H.ctx, 0, -1)   # automatic
    with pytest.raises(claw.ClawError):
        claw.claw_set_tile_walk(H.ctx, 1, 1)   # level not set
