"""GPU parity of the AMR path (Sec. 2.2-2.3): coarse-to-fine space-time ghost interpolation,
fine-to-coarse averaging and recursive subcycling, and of many independent runs batched into
one launch per level-step, against the oracle's AMR driver."""
import numpy as np
import pytest
import torch

from paper_1808_02638_gb300 import inputs

from gpu_amr_helpers import composite
from gpu_helpers import M, lib_ready, rel_err

pytestmark = pytest.mark.gpu
TOL1, TOLN = 1e-12, 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _compare_all_levels(H, O, run_index, tol):
    run = H.runs[run_index]
    worst = 0.0
    scale = max(np.abs(O.q[L]).max() for L in range(len(run.levels)))
    for L, lev in enumerate(run.levels):
        for n in range(len(lev.boxes)):
            got = H.interior(run_index, L, n)
            want = O.interior(L, n)
            worst = max(worst, float(np.abs(got - want).max()) / scale)
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("ghosts", ["pull", "pull, own fill launches", "pull+interp", "fill"])
def test_three_level_hierarchy_one_and_twenty_coarse_steps(ghosts):
    # 64^2 base, ratio 4 twice, seeded patches of 8..64 cells on the annuli (the uneven AMR
    # workload); uniform medium rho = 1, K = 4; each way the fine levels can get their ghosts
    # (interpolated ones filled by the launch before, or by a launch of their own, evaluated
    # inside the one-launch step, or all filled)
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    H.fuse_interp = [ghosts == "pull+interp"] * H.nlev
    H.pull_levels = [ghosts != "fill"] * H.nlev
    H.fill_ahead = ghosts != "pull, own fill launches"
    O = OracleHierarchy(run, q0, [inputs.const_pool(l, 1.0) for l in run.levels],
                        [inputs.const_pool(l, 4.0) for l in run.levels])
    H.init_dt()
    assert float(H.dt[0]) == pytest.approx(0.9 * (2.0 / 64) / 2.0, rel=1e-15)
    H.coarse_step()
    O.coarse_step()
    _compare_all_levels(H, O, 0, TOL1)
    for _ in range(19):
        H.coarse_step()
        O.coarse_step()
    _compare_all_levels(H, O, 0, TOLN)
    assert H.sync_status() == 0


@pytest.mark.parametrize("medium", ["uniform", "cellwise", "shallow_water"])
def test_fill_ahead_equals_own_fill_launches_with_fewer_launches(medium):
    # the interpolated ghosts of every fine substep written by spare CTAs of the launch before
    # (the previous substep's step, or the coarser level's step for the first substep at tau 0)
    # give the same pools, ghost cells included, as their own fill launches, bit for bit
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    if medium == "uniform":
        kw = dict(rho0=1.0, K0=4.0)
        args = ([run], [q0])
    elif medium == "shallow_water":   # the second system: a flowing ring as depth
        kw = dict(system="shallow_water", grav=1.0)
        args = ([run], [[inputs.init_swe(run, lev, u0=0.2, v0=0.1) for lev in run.levels]])
    else:   # a smooth random medium (the heterogeneous workload's kind), injected per level
        r0 = inputs.smooth_field(11, 64, 64, 0.5, 2.0)
        k0 = inputs.smooth_field(12, 64, 64, 1.0, 6.0)
        rhos = [inputs.coef_pool(lev, r0, 4 ** L) for L, lev in enumerate(run.levels)]
        Ks = [inputs.coef_pool(lev, k0, 4 ** L) for L, lev in enumerate(run.levels)]
        kw = {}
        args = ([run], [q0], [rhos], [Ks])
    Hs = []
    for ahead in (True, False):
        H = Hierarchy(*args, **kw)
        H.fill_ahead = ahead
        H.init_dt()
        n0 = claw.claw_launch_count(H.ctx)
        for _ in range(3):
            H.coarse_step()
        torch.cuda.synchronize()
        Hs.append((H, (claw.claw_launch_count(H.ctx) - n0) / 3))
    (A, la), (B, lb) = Hs
    for L in range(A.nlev):
        assert A.cur[L] == B.cur[L]
        for c in range(2):
            assert torch.equal(A.q[L][c], B.q[L][c]), (L, c)
    assert torch.equal(A.dt, B.dt)
    # 3 levels of ratio 4: 1 + 4 + 16 level-steps, 4 + 16 interpolation fills, 4 + 1 averages, 1 dt
    assert lb == 47 and la == 27, (la, lb)
    assert A.sync_status() == 0 and B.sync_status() == 0
    A.close()
    B.close()


def test_advance_fill_rejects_jobs_it_cannot_run():
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    H.init_dt()
    P = claw.CLAW_ADVANCE_PULL_GHOSTS
    q1, d1 = H.q[1][0], H.q[1][1]
    q0a, q0b = H.q[0][0], H.q[0][1]
    q2 = H.q[2][0]
    bad = [
        [(1, d1, q0a, q0b, 0.25)] * 3,              # more than two jobs
        [(1, q1, q0a, q0b, 0.25)],                  # writes the step's q_old
        [(1, d1, q0a, q0b, 1.5)],                   # tau outside [0, 1]
        [(2, q2, d1, d1, 0.0)],                     # reads the step's q_new as a coarse state
        [(3, q2, q1, q1, 0.0)],                     # not this level nor the next finer one
        [(0, q0a, q1, q1, 0.0)],                    # level 0 has no coarser level
    ]
    for jobs in bad:
        with pytest.raises(claw.ClawError) as e:
            claw.claw_level_advance_fill(H.ctx, 1, q1, d1, H.aux[1], H.dt, H.smax, P, jobs)
        assert e.value.status == claw.CLAW_EINVAL, jobs
    claw.claw_level_advance_fill(H.ctx, 1, q1, d1, H.aux[1], H.dt, H.smax, P,
                                 [(1, d1, q0a, q0b, 0.25), (2, q2, q1, q1, 0.0)])
    torch.cuda.synchronize()
    assert H.sync_status() == 0
    H.close()


def test_fine_level_ghosts_match_oracle_fill():
    # the interpolated and copied ghosts of the finest level at a substep fraction
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    import oracle
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    # a non-trivial coarse pair: perturb level 1 old / new differently
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    L1, L2 = run.levels[1], run.levels[2]
    cold = q0[1] + 0.01 * inputs.uniform(9, q0[1].size)
    cnew = q0[1] - 0.02 * inputs.uniform(10, q0[1].size)
    import torch
    dev = H.q[1][0].device
    tco = torch.from_numpy(np.concatenate([cold, np.zeros(H.q[1][0].numel() - cold.size)])).to(dev)
    tcn = torch.from_numpy(np.concatenate([cnew, np.zeros(H.q[1][0].numel() - cnew.size)])).to(dev)
    fine = H.q[2][0]
    claw.claw_fill_ghost(H.ctx, 2, fine, tco, tcn, 0.25)
    got = fine.cpu().numpy()[:q0[2].size]
    want = q0[2].copy()
    bx = lambda lev: [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(lev.boxes, lev.qoff)]
    oracle.level_fill_ghost(bx(L2), want, 3, L2.NX, L2.NY, run.bc, bx(L1), cold, cnew, 0.25, 4)
    assert rel_err(got, want) <= 1e-14


@pytest.mark.parametrize("tiling", [(32, 32, 1, 256), (32, 16, 2, 256), (16, 16, 1, 128)])
def test_step_evaluating_interpolated_ghosts_equals_fill_then_step(tiling):
    # claw_level_advance_interp (one launch: same-level and boundary ghosts pulled, coarse-fine
    # ghosts interpolated in space and time inside the step) against claw_fill_ghost_interp +
    # claw_level_advance with pulled ghosts: the same arithmetic, bit for bit, on both fine
    # levels of the 3-level hierarchy at a time fraction between two distinct coarse states
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, tiling=tiling)
    H.init_dt()
    H.coarse_step()   # two different coarse states on every level
    flags = claw.CLAW_ADVANCE_PULL_GHOSTS
    for L in (1, 2):
        cold, cnew = H.q[L - 1][1 - H.cur[L - 1]], H.q[L - 1][H.cur[L - 1]]
        q = H.q[L][H.cur[L]].clone()
        a, b = torch.full_like(q, float("nan")), torch.full_like(q, float("nan"))
        claw.claw_level_advance_interp(H.ctx, L, q, a, None, H.dt, H.smax, flags, cold, cnew, 0.25)
        qf = q.clone()
        claw.claw_fill_ghost_interp(H.ctx, L, qf, cold, cnew, 0.25)
        claw.claw_level_advance(H.ctx, L, qf, b, None, H.dt, H.smax, flags)
        torch.cuda.synchronize()
        lev = run.levels[L]
        for n in range(len(lev.boxes)):
            assert np.array_equal(H.interior(0, L, n, pool=a), H.interior(0, L, n, pool=b)), (L, n)
        assert torch.equal(q, H.q[L][H.cur[L]])   # q_old's ghost cells are neither needed nor written
    with pytest.raises(claw.ClawError):   # coarse states are required where interpolated ghosts exist
        claw.claw_level_advance_interp(H.ctx, 1, q, a, None, H.dt, H.smax, flags, None, None, 0.25)
    assert H.sync_status() == 0


def test_batched_independent_runs_two_levels_cellwise():
    # several 2-level problems of different sizes and media advanced together: every
    # level-step is one launch over the boxes of all runs, with per-run dt and CFL scalars
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    runs = inputs.config4_runs(4)
    qs, rhos, Ks, orcs = [], [], [], []
    for run, rho2, K2 in runs:
        q = [inputs.init_q(run, lev) for lev in run.levels]
        r = [inputs.coef_pool(lev, rho2, 4 ** L) for L, lev in enumerate(run.levels)]
        k = [inputs.coef_pool(lev, K2, 4 ** L) for L, lev in enumerate(run.levels)]
        qs.append(q)
        rhos.append(r)
        Ks.append(k)
        orcs.append(OracleHierarchy(run, q, r, k))
    H = Hierarchy([r for r, _, _ in runs], qs, rhos, Ks)
    H.init_dt()
    for ri, O in enumerate(orcs):
        assert float(H.dt[ri]) == pytest.approx(0.9 * min(O.levels[0].dx, O.levels[0].dy) / O.smax, rel=1e-15)
    for step in range(3):
        H.coarse_step()
        for O in orcs:
            O.coarse_step()
    for ri in range(len(runs)):
        _compare_all_levels(H, orcs[ri], ri, TOLN)
    assert H.sync_status() == 0


def test_all_64_batched_runs_one_coarse_step_with_the_tuned_launch():
    # the batched-runs workload at full breadth: all 64 independent 2-level runs (9226 boxes on
    # level 1, per-run heterogeneous media) in one hierarchy, with the tiling and ghost-launch
    # choice the autotuner installs for the benchmark, one coarse step, every run against its
    # own oracle hierarchy
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300 import measure
    from paper_1808_02638_gb300.solver import Hierarchy
    runs = inputs.config4_runs(64)
    qs, rhos, Ks, orcs = [], [], [], []
    for run, rho2, K2 in runs:
        q = [inputs.init_q(run, lev) for lev in run.levels]
        r = [inputs.coef_pool(lev, rho2, 4 ** L) for L, lev in enumerate(run.levels)]
        k = [inputs.coef_pool(lev, K2, 4 ** L) for L, lev in enumerate(run.levels)]
        qs.append(q)
        rhos.append(r)
        Ks.append(k)
        orcs.append(OracleHierarchy(run, q, r, k))
    H = Hierarchy([r for r, _, _ in runs], qs, rhos, Ks)
    H.init_dt()
    measure.tune_all(H)   # times steps into scratch pools; the state keeps its interiors
    H.init_dt()
    H.coarse_step()
    for O in orcs:
        O.coarse_step()
    worst = max(_compare_all_levels(H, orcs[ri], ri, TOL1) for ri in range(len(runs)))
    assert worst <= TOL1
    assert H.sync_status() == 0


# ------------------------------------------------------------ conservation fix (Sec. 2.3)
def _flowing_pulse(run):
    q = []
    for lev in run.levels:
        a = inputs.init_q(run, lev, fn=lambda x, y: inputs.radial_pulse(x - 0.1, y + 0.05)).copy()
        for n, b in enumerate(lev.boxes):
            v = inputs.box_view(a, lev.qoff[n], int(b[2]), int(b[3]), 3)
            v[1] += 0.3
            v[2] -= 0.2
        q.append(a)
    return q


_composite = composite


def test_reflux_three_levels_matches_oracle():
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    O = OracleHierarchy(run, q0, [inputs.const_pool(l, 1.0) for l in run.levels],
                        [inputs.const_pool(l, 4.0) for l in run.levels], reflux=True)
    H.init_dt()
    H.coarse_step()
    O.coarse_step()
    _compare_all_levels(H, O, 0, TOL1)
    for _ in range(19):
        H.coarse_step()
        O.coarse_step()
    _compare_all_levels(H, O, 0, TOLN)
    assert H.sync_status() == 0


def test_reflux_van_leer_matches_oracle():
    # the benchmark's limiter through the conservation fix's own edge solves
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    run.limiter = 3
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    O = OracleHierarchy(run, q0, [inputs.const_pool(l, 1.0) for l in run.levels],
                        [inputs.const_pool(l, 4.0) for l in run.levels], reflux=True)
    H.init_dt()
    for _ in range(6):
        H.coarse_step()
        O.coarse_step()
    _compare_all_levels(H, O, 0, TOLN)
    assert H.sync_status() == 0


def test_reflux_conserves_the_composite_integral_on_a_periodic_domain():
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1))
    run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45)], [2002])
    q0 = _flowing_pulse(run)
    drift = {}
    for reflux in (True, False):
        H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=reflux)
        H.init_dt()
        m0 = _composite(H)
        for _ in range(8):
            H.coarse_step()
        drift[reflux] = np.abs(_composite(H) - m0)
        assert H.sync_status() == 0
    scale = 4.0 * 1.5
    assert (drift[True] <= 1e-13 * scale).all(), drift[True]
    assert drift[False].max() >= 1e-6 * scale, drift[False]


def test_reflux_graph_replay_equals_eager():
    import torch
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    A = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    B = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    for h in (A, B):
        h.init_dt()
        h.coarse_step()
        h.coarse_step()
    g = B.capture(2)
    for _ in range(2):
        A.coarse_step()
        A.coarse_step()
        g.replay()
    torch.cuda.synchronize()
    for L in range(A.nlev):
        assert torch.equal(A.pool(L), B.pool(L))


def test_reflux_needs_the_uniform_medium():
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    runs = inputs.config4_runs(1)
    run, r2, k2 = runs[0]
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)]
    with pytest.raises(ValueError):
        Hierarchy([run], [q], [rho], [K], reflux=True)
    H = Hierarchy([run], [q], [rho], [K])
    buf = H.q[0][0].clone()
    with pytest.raises(claw.ClawError) as e:
        claw.claw_reflux_coarse(H.ctx, 1, H.q[0][0], H.dt, buf)
    assert e.value.status == claw.CLAW_EINVAL
    with pytest.raises(claw.ClawError) as e:
        claw.claw_reflux_buffer_size(H.ctx, 1)
    assert e.value.status == claw.CLAW_EINVAL


# ------------------------------------------------------------ regridding (Sec. 2.2)
def _upload_level(H, L, pool_np):
    import torch
    t = H.q[L][H.cur[L]]
    t.zero_()
    t[:pool_np.size] = torch.from_numpy(pool_np).to(t.device)


def test_flags_match_the_oracle_on_the_same_state():
    import torch
    from oracle import regrid as org
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    O = OracleHierarchy(run, q0, [inputs.const_pool(l, 1.0) for l in run.levels],
                        [inputs.const_pool(l, 4.0) for l in run.levels])
    for _ in range(3):
        O.coarse_step()
    O.fill(0, O.q[0])
    O.fill(1, O.q[1], O.q[0], O.q[0], 0.0)
    H = Hierarchy([run], [O.q], rho0=1.0, K0=4.0)
    for L in (0, 1):
        _upload_level(H, L, O.q[L])          # ghosts included: the same state on both sides
        for tol in (0.005, 0.03):
            flags = torch.zeros(claw.claw_flag_grid_size(H.ctx, L), dtype=torch.uint8, device=H.dev)
            claw.claw_flag_cells(H.ctx, L, H.q[L][H.cur[L]], tol, flags)
            lev = run.levels[L]
            got = flags.cpu().numpy().reshape(lev.NY, lev.NX).astype(bool)
            want = org.flag_level(lev, O.q[L], tol)
            assert np.array_equal(got, want) and want.any()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_clustering_matches_the_oracle(seed):
    from oracle import regrid as org
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    rng = np.random.default_rng(seed)
    for L in (0, 1):
        lev = run.levels[L]
        blobs = np.zeros((lev.NY, lev.NX), bool)
        for _ in range(6):                   # a few random blobs plus sparse noise
            cx, cy, rx, ry = rng.integers(0, lev.NX), rng.integers(0, lev.NY), rng.integers(1, 12), rng.integers(1, 12)
            blobs[max(0, cy - ry):cy + ry, max(0, cx - rx):cx + rx] = True
        flags = blobs | (rng.random((lev.NY, lev.NX)) < 0.01)
        for (buffer, cutoff, cap) in ((2, 0.7, 64), (0, 0.5, 32), (3, 0.9, 260)):
            got = claw.claw_regrid_boxes(H.ctx, L, 0, flags.astype(np.uint8), buffer, 2, cutoff, cap)
            m = org.nest_mask(lev, 2)
            f = org.dilate(flags, buffer) & m
            want = [(i0 * 4, j0 * 4, nx * 4, ny * 4) for (i0, j0, nx, ny) in org.cluster(f, cutoff, max(1, cap // 4), m)]
            assert got == want


def test_clustering_with_more_boxes_than_the_first_output_buffer():
    # a checkerboard with cutoff 1 leaves one box per flagged cell: 131072 boxes, more than the
    # binding's first output buffer holds, so the call is repeated with room for every cell
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 512
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = [inputs.Level(n, n, 2.0 / n, 2.0 / n, [(0, 0, n, n)]),
                  inputs.Level(2 * n, 2 * n, 1.0 / n, 1.0 / n, np.zeros((0, 4), dtype=np.int32), 2)]
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    jj, ii = np.mgrid[0:n, 0:n]
    flags = ((ii + jj) % 2 == 0).astype(np.uint8)
    got = claw.claw_regrid_boxes(H.ctx, 0, 0, flags, 0, 0, 1.0, 1024)
    want = sorted((2 * int(i), 2 * int(j), 2, 2) for j, i in zip(*np.nonzero(flags)))
    assert len(got) == n * n // 2 > 65536
    assert sorted(got) == want


def _run_with_regrid(hier, steps, every, params):
    for k in range(steps):
        hier.coarse_step()
        if (k + 1) % every == 0:
            hier.regrid(**params)


def test_regrid_end_to_end_matches_the_oracle():
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    params = dict(tol=0.02, buffer=2, cutoff=0.7, max_size=64, nest=2)
    run_g, run_o = inputs.config2(), inputs.config2()   # each side rebuilds its own levels
    q0 = [inputs.init_q(run_g, lev) for lev in run_g.levels]
    H = Hierarchy([run_g], [q0], rho0=1.0, K0=4.0)
    O = OracleHierarchy(run_o, q0, [inputs.const_pool(l, 1.0) for l in run_o.levels],
                        [inputs.const_pool(l, 4.0) for l in run_o.levels])
    H.init_dt()
    for k in range(12):
        H.coarse_step()
        O.coarse_step()
        if (k + 1) % 4 == 0:
            H.regrid(**params)
            O.regrid(**params)
            for L in (1, 2):
                assert np.array_equal(run_g.levels[L].boxes, run_o.levels[L].boxes)
            _compare_all_levels(H, O, 0, TOLN)
    _compare_all_levels(H, O, 0, TOLN)
    assert H.sync_status() == 0


def test_regrid_transfer_on_the_device_equals_copy_and_interpolation():
    # the device transfer (index grids painted with the old and the coarse boxes, a gather per
    # new cell) against its definition evaluated on the host: every interior cell of a new box is
    # the old box's value where one covered it, else the minmod-limited linear interpolation from
    # the coarse cell's parent (ghosts filled); old boxes outside their level are rejected
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    H.init_dt()
    H.coarse_step()
    qc = H.q[0][H.cur[0]]
    claw.claw_fill_ghost(H.ctx, 0, qc)
    qc_h = qc.cpu().numpy()
    old_boxes, old_pool = H.boxes[1].copy(), H.q[1][H.cur[1]]
    old_h = old_pool.cpu().numpy()
    lev1 = run.levels[1]
    r = lev1.ratio
    # the new level 1: every old box shifted by one coarse cell (partly over old data, partly not)
    shifted = np.array([(int(b[0]) + r, int(b[1]) + r, int(b[2]), int(b[3])) for b in lev1.boxes], dtype=np.int32)
    run.levels[1] = inputs.Level(lev1.NX, lev1.NY, lev1.dx, lev1.dy, shifted, r)
    boxes, _, qb, _ = H._layout(1)
    claw.claw_set_level(H.ctx, 1, boxes)
    new = torch.zeros(max(qb, inputs.ALIGN), dtype=torch.float64, device=qc.device)
    claw.claw_regrid_transfer(H.ctx, 1, old_boxes, old_pool, new, qc)
    torch.cuda.synchronize()
    got = new.cpu().numpy()
    owner = np.full((lev1.NY, lev1.NX), -1)
    for n, o in enumerate(old_boxes):
        owner[o.jlo:o.jlo + o.ny, o.ilo:o.ilo + o.nx] = n
    (cb,) = H.boxes[0]   # one coarse box covers level 0
    cv = inputs.box_view(qc_h, int(cb.qoff), int(cb.nx), int(cb.ny), 3)

    def minmod(a, b):
        return np.where(a * b > 0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)

    ncopied = 0
    for b in boxes:
        nx, ny = int(b.nx), int(b.ny)
        g = inputs.box_view(got, int(b.qoff), nx, ny, 3)[:, M:-M, M:-M]
        gj, gi = np.meshgrid(np.arange(b.jlo, b.jlo + ny), np.arange(b.ilo, b.ilo + nx), indexing="ij")
        I, J = gi // r, gj // r
        ci, cj = I - int(cb.ilo) + M, J - int(cb.jlo) + M
        q = cv[:, cj, ci]
        sx = minmod(cv[:, cj, ci + 1] - q, q - cv[:, cj, ci - 1])
        sy = minmod(cv[:, cj + 1, ci] - q, q - cv[:, cj - 1, ci])
        xi = ((gi - I * r) + 0.5) / r - 0.5
        eta = ((gj - J * r) + 0.5) / r - 0.5
        want = q + xi * sx + eta * sy
        own = owner[gj, gi]
        for o in np.unique(own[own >= 0]):
            O = old_boxes[o]
            ov = inputs.box_view(old_h, int(O.qoff), int(O.nx), int(O.ny), 3)
            m = own == o
            want[:, m] = ov[:, gj[m] - O.jlo + M, gi[m] - O.ilo + M]
            ncopied += int(m.sum())
        assert np.allclose(g, want, rtol=1e-15, atol=1e-15)
    assert ncopied > 0 and ncopied < sum(int(b.nx) * int(b.ny) for b in boxes)
    bad = claw.box_array(1)
    bad.ilo, bad.jlo, bad.nx, bad.ny = lev1.NX - 4, 0, 8, 8   # sticks out of the level
    with pytest.raises(claw.ClawError):
        claw.claw_regrid_transfer(H.ctx, 1, bad, old_pool, new, qc)
    assert H.sync_status() == 0


def test_regrid_keeps_the_reflux_conservation():
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1))
    run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45)], [2002])
    q0 = _flowing_pulse(run)
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    H.init_dt()
    m0 = _composite(H)
    for k in range(6):
        H.coarse_step()
        if k == 2:
            H.regrid(tol=0.02, buffer=2, cutoff=0.7, max_size=64, nest=2)
    drift = np.abs(_composite(H) - m0)
    # the transfer is conservative where it interpolates and the fine data it drops was
    # averaged into the coarse level: the composite integral survives the regrid
    assert (drift <= 1e-13 * 6.0).all(), drift


def test_section_timing_leaves_the_result_alone():
    # CUDA events around the sections of an eager coarse step change nothing in the state
    import torch
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    A = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    B = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    A.init_dt()
    B.init_dt()
    B.sections = []
    for _ in range(3):
        A.coarse_step()
        B.coarse_step()
    ms = B.section_ms()
    assert set(ms) == {"fill", "advance", "update"} and all(v > 0.0 for v in ms.values())
    assert B.sections == [] and B.section_ms() == {}
    for L in range(len(run.levels)):
        assert torch.equal(A.pool(L), B.pool(L))


def test_benchmark_analog_paths_agree():
    # a small benchmark analog: the batched launch and one launch per patch take the same
    # hierarchy through the same regrids (identical states, hence identical flags and boxes)
    from paper_1808_02638_gb300 import measure
    kw = dict(ncoarse=6, base=160, max_size=48, regrid_every=2, tol=0.01)
    a = measure.e1(**kw)
    b = measure.e1(per_patch=True, **kw)
    assert a["status"] == b["status"] == "ok"
    assert a["cell_updates"] == b["cell_updates"] > 0
    assert a["final_boxes_per_level"] == b["final_boxes_per_level"]
    assert a["final_boxes_per_level"][2] > 0 and a["regrids"] == 3
    for r in (a, b):
        s = r["sections_s"]
        assert min(s[k] for k in ("advance", "ghost_fill", "regrid", "updating")) > 0.0
        assert abs(sum(v for k, v in s.items() if k != "total") - s["total"]) < 1e-9


def _analog_run(base, nlev, ratio):
    """the benchmark analog's hierarchy (Sec. 4.1-4.2): a base level in 4 x 4 patches, van Leer,
    outflow boundaries, finer levels empty until the first regrid"""
    run = inputs.Run(*inputs.PULSE_DOMAIN, limiter=3)
    d0, st = 2.0 / base, base // 4
    run.levels = [inputs.Level(base, base, d0, d0, [(i, j, st, st) for j in range(0, base, st)
                                                     for i in range(0, base, st)])]
    for L in range(1, nlev):
        n = base * ratio ** L
        run.levels.append(inputs.Level(n, n, 2.0 / n, 2.0 / n, np.zeros((0, 4), dtype=np.int32), ratio))
    return run


def test_benchmark_analog_matches_the_oracle():
    # the benchmark analog's combination at a size the oracle finishes in seconds: 3 levels of
    # ratio 2, van Leer, the conservation fix on through the regrids, fine levels built at t = 0
    # by regridding and then set from the initial condition, a regrid every 2 coarse steps with
    # buffer 2 and cutoff 0.7, and patches capped at 24 fine cells so that clustering splits
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    base, nlev, ratio, every = 96, 3, 2, 2
    params = dict(tol=0.01, buffer=every, cutoff=0.7, max_size=24, nest=2)
    run_g, run_o = _analog_run(base, nlev, ratio), _analog_run(base, nlev, ratio)
    q0 = [inputs.init_q(run_g, lev) for lev in run_g.levels]
    H = Hierarchy([run_g], [q0], rho0=1.0, K0=4.0, reflux=True, tiling=((32, 16, 2, 256), (16, 16, 1, 128)))
    O = OracleHierarchy(run_o, q0, [inputs.const_pool(run_o.levels[0], 1.0)] + [np.ones(1)] * (nlev - 1),
                        [inputs.const_pool(run_o.levels[0], 4.0)] + [np.full(1, 4.0)] * (nlev - 1), reflux=True)

    def same_boxes():
        for L in range(1, nlev):
            assert np.array_equal(run_g.levels[L].boxes, run_o.levels[L].boxes), L
        assert len(run_g.levels[2].boxes) > 0
        assert max(int(b[2:].max()) for L in (1, 2) for b in run_g.levels[L].boxes) == 24

    for _ in range(nlev - 1):
        H.regrid(**params)
        O.regrid(**params)
        same_boxes()
    for L, lev in enumerate(run_g.levels):
        a = inputs.init_q(run_g, lev)
        t = H.q[L][H.cur[L]]
        t.zero_()
        t[:a.size] = torch.from_numpy(a).to(t.device)
        O.q[L] = inputs.init_q(run_o, run_o.levels[L])
    H.init_dt()
    for k in range(6):
        H.coarse_step()
        O.coarse_step()
        if (k + 1) % every == 0:
            H.regrid(**params)
            O.regrid(**params)
            same_boxes()
    assert float(H.dt[0]) == pytest.approx(O.dt_history[-1], rel=1e-15)
    _compare_all_levels(H, O, 0, TOLN)
    assert H.sync_status() == 0


def test_coefficient_ghost_tables_of_a_uniform_medium_on_first_use():
    # a uniform-medium context builds the one-plane ghost tables on the first call; they equal
    # the ones a cell-wise context builds with its levels, also after the levels are set again
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.const_pool(l, 1.0) for l in run.levels]
    K = [inputs.const_pool(l, 4.0) for l in run.levels]
    U = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    C = Hierarchy([run], [q0], rho, K)
    g = torch.Generator(device="cuda").manual_seed(5)
    for rebuild in (False, True):
        if rebuild:
            for L in range(len(run.levels)):
                claw.claw_set_level(U.ctx, L, U.boxes[L])
        for L in range(len(run.levels)):
            a = torch.rand(C.rho[L].shape, dtype=torch.float64, device="cuda", generator=g)
            b = a.clone()
            claw.claw_fill_ghost_coef(C.ctx, L, a)
            claw.claw_fill_ghost_coef(U.ctx, L, b)
            torch.cuda.synchronize()
            assert torch.equal(a, b)
            claw.claw_fill_ghost_coef_adjoint(C.ctx, L, a)
            claw.claw_fill_ghost_coef_adjoint(U.ctx, L, b)
            torch.cuda.synchronize()
            assert torch.equal(a, b)
