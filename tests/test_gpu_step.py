"""GPU parity of the fused level-step (C ABI) against the CPU oracle.

Tolerances: max |GPU - oracle| <= 1e-12 max|q| after one step and <= 1e-10 max|q| after 50-100
steps (the GPU uses fused multiply-adds, division-free limiter forms and reciprocal
multiplies; the oracle plain IEEE operations in textbook order)."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

from gpu_helpers import M, lib_ready, oracle_single, rel_err, single_grid

pytestmark = pytest.mark.gpu

TOL1, TOLN = 1e-12, 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _hier(run, q, rho=None, K=None, rho0=1.0, K0=4.0, tiling=None):
    from paper_1808_02638_gb300.solver import Hierarchy
    if rho is None:
        return Hierarchy([run], [[q]], rho0=rho0, K0=K0, tiling=tiling)
    return Hierarchy([run], [[q]], [[rho]], [[K]], tiling=tiling)


def _uniform_planes(n, rho0=1.0, K0=4.0):
    return np.full((n + 4, n + 4), rho0), np.full((n + 4, n + 4), K0)


@pytest.mark.parametrize("tiling", [(32, 32, 1), (32, 32, 0), (32, 16, 1), (32, 16, 2), (16, 16, 0), (16, 16, 1)])
def test_uniform_pulse_100x100_one_and_50_steps(orc, tiling):
    run, q = single_grid(100)
    H = _hier(run, q, tiling=tiling)
    H.init_dt()
    assert float(H.dt[0]) == pytest.approx(0.9 * 0.02 / 2.0, rel=1e-15)
    rho, K = _uniform_planes(100)
    H.coarse_step()
    want, _ = oracle_single(orc, run, q, rho, K, 1, dt=0.009)
    got = H.interior(0, 0, 0)
    assert rel_err(got, want) <= TOL1
    for _ in range(49):
        H.coarse_step()
    want, dts = oracle_single(orc, run, q, rho, K, 50)
    assert rel_err(H.interior(0, 0, 0), want) <= TOLN
    assert H.sync_status() == 0
    assert float(H.smax[0]) == 0.0 and float(H.dt[0]) == pytest.approx(dts[-1], rel=1e-15)


@pytest.mark.parametrize("limiter", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("order,transverse", [(2, 2), (2, 1), (2, 0), (1, 0), (1, 1)])
def test_schemes_random_data_one_step(orc, limiter, order, transverse):
    n = 36
    run, q = single_grid(n, pulse=False, seed=100 + limiter, limiter=limiter, order=order, transverse=transverse)
    H = _hier(run, q, rho0=1.3, K0=2.7, tiling=(16, 16, 1))
    H.dt.fill_(0.004)
    H.coarse_step()
    rho, K = _uniform_planes(n, 1.3, 2.7)
    want, _ = oracle_single(orc, run, q, rho, K, 1, dt=0.004)
    assert rel_err(H.interior(0, 0, 0), want) <= TOL1


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (2, 2, 2, 2), (2, 0, 1, 1)])
def test_boundary_conditions_ten_steps(orc, bc):
    n = 40
    run, q = single_grid(n, pulse=False, seed=7, bc=bc)
    H = _hier(run, q, tiling=(16, 16, 0))
    H.init_dt()
    for _ in range(10):
        H.coarse_step()
    rho, K = _uniform_planes(n)
    want, _ = oracle_single(orc, run, q, rho, K, 10)
    assert rel_err(H.interior(0, 0, 0), want) <= TOLN


@pytest.mark.parametrize("tiling", [(32, 32, 1), (32, 16, 0), (32, 16, 2), (16, 16, 1)])
def test_cellwise_medium_one_and_100_steps(orc, tiling):
    n = 64
    run, rho2, K2 = inputs.config3(n)
    run2, q = single_grid(n)
    lev = run2.levels[0]
    rho = inputs.coef_pool(lev, rho2, 1)
    K = inputs.coef_pool(lev, K2, 1)
    H = _hier(run2, q, rho, K, tiling=tiling)
    H.init_dt()
    rp = inputs.box_view(rho, 0, n, n, 1)[0]
    kp = inputs.box_view(K, 0, n, n, 1)[0]
    smax = float(np.sqrt(K2 / rho2).max())
    assert float(H.dt[0]) == pytest.approx(0.9 * (2.0 / n) / smax, rel=1e-15)
    H.coarse_step()
    want, _ = oracle_single(orc, run2, q, rp, kp, 1)
    assert rel_err(H.interior(0, 0, 0), want) <= TOL1
    for _ in range(99):
        H.coarse_step()
    want, _ = oracle_single(orc, run2, q, rp, kp, 100)
    assert rel_err(H.interior(0, 0, 0), want) <= TOLN
    assert H.sync_status() == 0


@pytest.mark.parametrize("limiter", [0, 1, 2, 3, 4])
def test_uniform_state_preserved_bit_exactly_cellwise(limiter):
    n = 48
    run, rho2, K2 = inputs.config3(n)
    run2, _ = single_grid(n, limiter=limiter)
    lev = run2.levels[0]
    q = np.zeros(lev.qsize)
    v = inputs.box_view(q, 0, n, n, 3)
    v[0], v[1], v[2] = 1.25, -0.5, 0.75
    H = _hier(run2, q, inputs.coef_pool(lev, rho2, 1), inputs.coef_pool(lev, K2, 1), tiling=(16, 16, 1))
    H.init_dt()
    for _ in range(5):
        H.coarse_step()
    got = H.interior(0, 0, 0)
    assert np.all(got[0] == 1.25) and np.all(got[1] == -0.5) and np.all(got[2] == 0.75)


def test_tiled_level_and_patchwise_path_match_oracle_and_each_other(orc):
    # 128 x 128 as 16 patches of 32 x 32 (the uniform-batch layout at a size the oracle
    # finishes quickly): same-level ghost copies + extrapolation, fused vs one launch per box
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config1(128, 32)
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    Hp = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    Hp.patchwise = True
    for h in (H, Hp):
        h.init_dt()
        for _ in range(20):
            h.coarse_step()
    for nb in range(len(lev.boxes)):
        assert np.array_equal(H.interior(0, 0, nb), Hp.interior(0, 0, nb))
    # the oracle on the same single grid
    srun, sq = single_grid(128)
    rho, K = _uniform_planes(128)
    want, _ = oracle_single(orc, srun, sq, rho, K, 20)
    got = np.zeros_like(want)
    for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
        got[:, jlo:jlo + bny, ilo:ilo + bnx] = H.interior(0, 0, nb)
    assert rel_err(got, want) <= TOLN


def test_graph_replay_equals_eager():
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config1(256, 32)
    q = inputs.init_q(run, run.levels[0])
    A = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    B = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    for h in (A, B):
        h.init_dt()
        h.coarse_step()
        h.coarse_step()   # warm-up outside capture (descriptors, attributes)
    g = B.capture(2)
    for _ in range(3):
        g.replay()
        A.coarse_step()
        A.coarse_step()
    import torch
    torch.cuda.synchronize()
    assert np.array_equal(A.level_numpy(0, 0), B.level_numpy(0, 0))


def test_full_size_uniform_batch_sampled_parity_and_symmetry(orc):
    # 2048^2 as 4096 patches of 32 x 32, the configuration the benchmark times: ghosts equal
    # the edge-padded global field, sampled patches equal the oracle's one-patch step from the
    # same input, and after 200 steps the radial pulse keeps its symmetries
    from paper_1808_02638_gb300.solver import Hierarchy
    import torch
    run = inputs.config1()
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    rng = np.random.default_rng(5)
    sample = rng.choice(len(lev.boxes), 48, replace=False)
    ones = np.ones((36, 36))
    for step in range(200):
        check = step in (0, 100, 199)
        if check:
            claw = __import__("paper_1808_02638_gb300.claw", fromlist=["claw"])
            claw.claw_fill_ghost(H.ctx, 0, H.pool(0))
            before = H.pool(0).cpu().numpy()
            dt = float(H.dt[0])
        H.coarse_step()
        if check:
            after = H.pool(0).cpu().numpy()
            if step == 0:
                # ghosts of every patch equal the edge-extrapolated global field
                glob = np.zeros((3, 2048, 2048))
                for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
                    glob[:, jlo:jlo + 32, ilo:ilo + 32] = inputs.box_view(before, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
                gp = np.pad(glob, ((0, 0), (M, M), (M, M)), mode="edge")
                for nb in sample:
                    ilo, jlo = int(lev.boxes[nb][0]), int(lev.boxes[nb][1])
                    assert np.array_equal(inputs.box_view(before, lev.qoff[nb], 32, 32, 3),
                                          gp[:, jlo:jlo + 36, ilo:ilo + 36])
            for nb in sample:
                qin = inputs.box_view(before, lev.qoff[nb], 32, 32, 3).copy()
                want, _ = orc.step(qin, ones, 4 * ones, lev.dx, lev.dy, dt)
                got = inputs.box_view(after, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
                scale = np.abs(after).max()
                assert np.abs(got - want[:, M:-M, M:-M]).max() <= TOL1 * scale
    glob = np.zeros((3, 2048, 2048))
    final = H.pool(0).cpu().numpy()
    for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
        glob[:, jlo:jlo + 32, ilo:ilo + 32] = inputs.box_view(final, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
    p, u, v = glob
    tol = 1e-12 * np.abs(glob).max()
    assert np.abs(p - p.T).max() <= tol and np.abs(p - p[:, ::-1]).max() <= tol
    assert np.abs(u - v.T).max() <= tol and np.abs(u + u[:, ::-1]).max() <= tol
    assert H.sync_status() == 0


def _tilings():
    from paper_1808_02638_gb300 import tune
    return ["tuned"] + [tuple(c) for c in tune.CANDIDATES]


@pytest.mark.parametrize("tiling", _tilings())
def test_full_size_bench_launch_path_sampled_parity(orc, tiling):
    # the launch path bench.py times, at its full size: 2048^2 as 4096 patches, the tiling the
    # autotuner picks (or each candidate), CUDA-graph replays of the one launch per step: the
    # persistent level-step that takes every ghost from its source cell and applies the device
    # Eq. cfl update.  The pools' ghost cells are poisoned with NaN first: the step must never
    # read them.  At steps 0, 100 and 199 sampled patches equal the oracle's one-patch step from
    # the same input, whose ghosts are the edge-extrapolated global field; after 200 steps the
    # symmetries hold.
    from paper_1808_02638_gb300 import claw, tune
    from paper_1808_02638_gb300.solver import Hierarchy
    import torch
    run = inputs.config1()
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    if tiling == "tuned":
        tune.tune_level(H, 0, use_cache=False, pull=True)
    else:
        claw.claw_set_tiling(H.ctx, 0, *tiling)
    H.coarse_step()
    H.coarse_step()
    ghost = np.ones(lev.qsize, bool)
    for nb in range(len(lev.boxes)):
        inputs.box_view(ghost, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M] = False
    gmask = torch.from_numpy(np.concatenate([ghost, np.zeros(H.q[0][0].numel() - ghost.size, bool)])).to(H.dev)
    for k in range(2):
        H.q[0][k][gmask] = float("nan")
    st = H.fused_stepper()
    assert st.launches_per_step == 1
    rng = np.random.default_rng(7)
    sample = rng.choice(len(lev.boxes), 32, replace=False)
    ones = np.ones((36, 36))

    def glob_of(pool):
        g = np.zeros((3, 2048, 2048))
        for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
            g[:, jlo:jlo + 32, ilo:ilo + 32] = inputs.box_view(pool, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
        return g

    for step in range(200):
        check = step in (0, 100, 199)
        if check:
            torch.cuda.synchronize()
            gp = np.pad(glob_of(H.pool(0).cpu().numpy()), ((0, 0), (M, M), (M, M)), mode="edge")
            dt = float(H.dt[0])
        st.step()
        if check:
            torch.cuda.synchronize()
            after = H.pool(0).cpu().numpy()
            scale = np.nanmax(np.abs(after))
            for nb in sample:
                ilo, jlo = int(lev.boxes[nb][0]), int(lev.boxes[nb][1])
                qin = np.ascontiguousarray(gp[:, jlo:jlo + 36, ilo:ilo + 36])
                want, _ = orc.step(qin, ones, 4 * ones, lev.dx, lev.dy, dt)
                got = inputs.box_view(after, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
                assert np.abs(got - want[:, M:-M, M:-M]).max() <= TOL1 * scale
    g = glob_of(H.pool(0).cpu().numpy())
    assert np.isfinite(g).all()
    p, u, v = g
    tol = 1e-12 * max(np.abs(p).max(), 1.0)
    assert np.abs(p - p.T).max() <= tol and np.abs(p - p[:, ::-1]).max() <= tol
    assert np.abs(u - v.T).max() <= tol and np.abs(u + u[:, ::-1]).max() <= tol
    assert H.sync_status() == 0


def test_pulled_ghosts_equal_filled_ghosts_on_amr_and_walls():
    # the pulled path against fill + step on boxes of mixed sizes with periodic and wall
    # boundaries (sign flips), and on the finer level of a hierarchy (interpolated ghosts are
    # filled, copied ones are pulled): bit for bit the same new state
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    for bc in ((1, 1, 2, 2), (2, 0, 1, 1)):
        run = inputs.Run(*inputs.PULSE_DOMAIN, bc=bc)
        run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45)], [2002])
        q = [inputs.init_q(run, lev) for lev in run.levels]
        for L, lev in enumerate(run.levels):
            for nb, b in enumerate(lev.boxes):   # a velocity field so that the wall flips matter
                v = inputs.box_view(q[L], lev.qoff[nb], int(b[2]), int(b[3]), 3)
                v[1] = 0.3 * v[0]
                v[2] = -0.2 * v[0]
        H = Hierarchy([run], [q], rho0=1.0, K0=4.0)
        H.init_dt()
        for L in range(2):
            qc = H.q[L - 1][H.cur[L - 1]] if L else None
            a = H.q[L][H.cur[L]]
            claw.claw_fill_ghost(H.ctx, L, a, qc, qc, 0.0)
            ref = torch.zeros_like(a)
            claw.claw_level_step(H.ctx, L, a, ref, None, H.dt, H.smax)
            # pulled: the copied ghosts of a poisoned copy must not matter
            b = a.clone()
            ring_cells = torch.zeros_like(a, dtype=torch.bool)
            lev = run.levels[L]
            qbase = [qb for (ri, qb, _) in H.layout[L] if ri == 0][0]
            mask = np.zeros(lev.qsize, bool)
            for nb, bx in enumerate(lev.boxes):
                nx, ny = int(bx[2]), int(bx[3])
                m = inputs.box_view(mask, lev.qoff[nb], nx, ny, 3)
                m[...] = True
                m[:, M:-M, M:-M] = False
            if L == 0:   # level 0 has no interpolated ghosts: poison them all
                ring_cells[qbase:qbase + lev.qsize] = torch.from_numpy(mask).to(a.device)
                b[ring_cells] = float("nan")
            out = torch.zeros_like(a)
            claw.claw_level_advance(H.ctx, L, b, out, None, H.dt, H.smax, claw.CLAW_ADVANCE_PULL_GHOSTS)
            torch.cuda.synchronize()
            inner = torch.from_numpy(~mask).to(a.device)
            sl = slice(qbase, qbase + lev.qsize)
            assert torch.equal(out[sl][inner], ref[sl][inner]), (bc, L)
        assert H.sync_status() == 0


def test_host_resident_steps_equal_device_steps():
    # the pipelined host loop (state copied in and out every step, the level stepped in pieces
    # of boxes as they arrive) produces bit for bit the states of the same steps on the device
    import torch
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config1(256, 32)
    q = inputs.init_q(run, run.levels[0])
    A = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    B = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    for h in (A, B):
        h.init_dt()
        h.fused = True
    ha = torch.empty_like(B.q[0][0], device="cpu").pin_memory()
    hb = torch.empty_like(ha).pin_memory()
    ha.copy_(B.q[0][B.cur[0]])
    for _ in range(6):
        A.coarse_step()
    out = B.steps_from_host(ha, hb, 6, bands=5)
    torch.cuda.synchronize()
    assert torch.equal(out, A.pool(0).cpu()) and float(A.dt[0]) == float(B.dt[0])


def test_pack_unpack_and_pieces_on_mixed_boxes():
    # packed interiors of boxes of mixed sizes: pack then unpack restores the interiors and
    # leaves ghost cells alone; stepping the level in pieces of boxes equals one launch
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    boxes = [(0, 0, 40, 24), (40, 0, 24, 24), (0, 24, 64, 40)]
    run, q = single_grid(64, boxes=boxes, pulse=False, seed=41)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    n = H.packed_size()
    assert n == 3 * (40 * 24 + 24 * 24 + 64 * 40)
    packed = H.pack()
    lev = run.levels[0]
    off = 0
    for nb, (i0, j0, nx, ny) in enumerate(boxes):
        got = packed[off:off + 3 * nx * ny].view(3, ny, nx).cpu().numpy()
        assert np.array_equal(got, H.interior(0, 0, nb))
        off += 3 * nx * ny
    pool = H.pool(0)
    poisoned = torch.full_like(pool, float("nan"))
    claw.claw_unpack_interiors(H.ctx, 0, 0, 3, packed, poisoned)
    for nb in range(3):
        assert np.array_equal(H.interior(0, 0, nb, pool=poisoned), H.interior(0, 0, nb))
    assert torch.isnan(poisoned).any()   # ghost cells untouched
    # pieces: boxes [0, 2) then [2, 3) against the whole level
    claw.claw_fill_ghost(H.ctx, 0, pool)
    whole, parts = torch.zeros_like(pool), torch.zeros_like(pool)
    sm = torch.zeros_like(H.smax)
    claw.claw_level_step(H.ctx, 0, pool, whole, None, H.dt, sm)
    sm2 = torch.zeros_like(H.smax)
    flags = claw.CLAW_ADVANCE_PULL_GHOSTS
    claw.claw_level_advance_boxes(H.ctx, 0, 2, 3, pool, parts, None, H.dt, sm2, flags)
    claw.claw_level_advance_boxes(H.ctx, 0, 0, 2, pool, parts, None, H.dt, sm2, flags)
    torch.cuda.synchronize()
    for nb in range(3):
        assert np.array_equal(H.interior(0, 0, nb, pool=parts), H.interior(0, 0, nb, pool=whole))
    assert float(sm2[0]) == float(sm[0])
    with pytest.raises(claw.ClawError):
        claw.claw_level_advance_boxes(H.ctx, 0, 2, 4, pool, parts, None, H.dt, sm2, flags)
    with pytest.raises(claw.ClawError):
        claw.claw_level_advance_boxes(H.ctx, 0, 0, 1, pool, parts, None, H.dt, sm2, claw.CLAW_ADVANCE_UPDATE_DT)


def test_host_resident_packed_interiors():
    # the same loop with the host state in packed form (interiors only): unpacked into the pool
    # and packed out of it piece by piece; equal to the device steps bit for bit
    import torch
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config1(256, 32)
    run.bc = (1, 1, 0, 0)
    q = inputs.init_q(run, run.levels[0])
    A = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    B = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    for h in (A, B):
        h.init_dt()
        h.fused = True
    assert B.packed_size() == 3 * 256 * 256
    ha = B.pack().cpu().pin_memory()
    hb = torch.empty_like(ha).pin_memory()
    for _ in range(7):
        A.coarse_step()
    out = B.steps_from_host(ha, hb, 7, bands=4)
    torch.cuda.synchronize()
    assert torch.equal(out, A.pack().cpu())
    lev = run.levels[0]
    v = out.numpy()
    for nb, b in enumerate(lev.boxes):   # packed layout: box after box, three 32 x 32 planes
        got = v[nb * 3 * 1024:(nb + 1) * 3 * 1024].reshape(3, 32, 32)
        assert np.array_equal(got, A.interior(0, 0, nb))
    assert float(A.dt[0]) == float(B.dt[0]) and B.sync_status() == 0


@pytest.mark.parametrize("bc,bands", [((1, 1, 1, 1), 7), ((2, 0, 2, 2), 3)])
def test_host_resident_bands_follow_ghost_sources(bc, bands):
    # periodic and wall boundaries: a piece waits for the pieces its ghosts come from,
    # including the periodic images; the result equals the one-launch device steps bit for bit
    import torch
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config1(256, 32)
    run.bc = bc
    q = inputs.init_q(run, run.levels[0])
    v = q.reshape(-1)
    A = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    B = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    for h in (A, B):
        h.init_dt()
        h.fused = True
    _, _, needs = B._bands(bands)
    if bc[0] == 1:   # the first piece reads the last one across the periodic boundary
        assert len(needs) - 1 in needs[0]
    ha = torch.empty_like(B.q[0][0], device="cpu").pin_memory()
    hb = torch.empty_like(ha).pin_memory()
    ha.copy_(B.q[0][B.cur[0]])
    for _ in range(5):
        A.coarse_step()
    out = B.steps_from_host(ha, hb, 5, bands=bands)
    torch.cuda.synchronize()
    lev = run.levels[0]
    for nb, b in enumerate(lev.boxes):
        got = inputs.box_view(out.numpy(), lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
        assert np.array_equal(got, A.interior(0, 0, nb)), nb
    assert float(A.dt[0]) == float(B.dt[0]) and A.sync_status() == 0 and B.sync_status() == 0


def test_errors_are_status_codes():
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(32)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    bad = claw.claw_box()
    bad.run, bad.ilo, bad.jlo, bad.nx, bad.ny, bad.qoff, bad.coff = 0, 16, 0, 32, 32, 0, 0
    with pytest.raises(claw.ClawError) as e:
        claw.claw_set_level(H.ctx, 0, [bad])          # outside the domain
    assert e.value.status == claw.CLAW_EINVAL
    b1 = claw.claw_box()
    b1.run, b1.ilo, b1.jlo, b1.nx, b1.ny, b1.qoff, b1.coff = 0, 0, 0, 16, 16, 0, 0
    b2 = claw.claw_box()
    b2.run, b2.ilo, b2.jlo, b2.nx, b2.ny, b2.qoff, b2.coff = 0, 8, 8, 16, 16, 4096, 4096
    with pytest.raises(claw.ClawError) as e:
        claw.claw_set_level(H.ctx, 0, [b1, b2])       # overlapping boxes
    assert e.value.status == claw.CLAW_EINVAL
    with pytest.raises(claw.ClawError) as e:
        claw.claw_set_level(H.ctx, 1, [b1])           # level 0 was cleared by the failed set
    assert e.value.status in (claw.CLAW_ESTATE, claw.CLAW_EINVAL)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (33, 17), (4096, 8), (8, 4096)])
def test_tiny_and_extreme_box_shapes_match_oracle(orc, shape):
    # boxes smaller than a tile, odd sizes (cooperative staging), and the widest and tallest
    # boxes the tables accept: 5 steps of random data against the oracle's single grid
    from paper_1808_02638_gb300.solver import Hierarchy
    nx, ny = shape
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = [inputs.Level(nx, ny, 2.0 / nx, 2.0 / ny, [(0, 0, nx, ny)])]
    lev = run.levels[0]
    q = np.zeros(lev.qsize)
    v = inputs.box_view(q, 0, nx, ny, 3)
    v[...] = inputs.uniform(60 + nx + 7 * ny, v.size).reshape(v.shape) - 0.5
    v[0] += 1.0
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    for _ in range(5):
        H.coarse_step()
    got = H.interior(0, 0, 0)
    ones = np.ones((ny + 4, nx + 4))
    want, _ = oracle_single(orc, run, q, ones, 4.0 * ones, 5)
    assert rel_err(got, want) <= TOLN
    assert H.sync_status() == 0


def test_empty_level_and_box_limits():
    # a level without boxes is a valid no-op for every entry point; boxes past 4096 cells per
    # side are rejected before any launch
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(32)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    claw.claw_set_level(H.ctx, 0, [])
    a, b, c = (torch.zeros(64, dtype=torch.float64, device=H.dev) for _ in range(3))
    before = claw.claw_launch_count(H.ctx)
    claw.claw_fill_ghost(H.ctx, 0, a)
    claw.claw_level_step(H.ctx, 0, a, b, None, H.dt, H.smax)   # distinct buffers (no aliasing)
    claw.claw_cfl_max(H.ctx, 0, None, H.smax)
    claw.claw_level_step_adjoint(H.ctx, 0, a, b, c, None, None, H.dt)
    assert claw.claw_launch_count(H.ctx) == before
    assert all(bool((t == 0).all()) for t in (a, b, c))
    assert H.sync_status() == 0
    big = inputs.Run(*inputs.PULSE_DOMAIN)
    big.levels = [inputs.Level(4104, 8, 2.0 / 4104, 0.25, [(0, 0, 4104, 8)])]
    with pytest.raises(claw.ClawError) as e:
        Hierarchy([big], [[np.zeros(big.levels[0].qsize)]], rho0=1.0, K0=4.0)
    assert e.value.status == claw.CLAW_EINVAL


def test_nan_input_is_reported_not_trapped():
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(32)
    inputs.box_view(q, 0, 32, 32, 3)[0, 10, 10] = np.nan
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    H.coarse_step()
    assert H.sync_status() == claw.CLAW_ENAN
    assert H.sync_status() == claw.CLAW_OK   # reading clears the flag


def test_cfl_violation_is_reported():
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    run, q = single_grid(32)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    H.dt.mul_(1.5)                      # nu = 1.35 > 1
    H.coarse_step()
    assert H.sync_status() == claw.CLAW_ECFL


def test_autotuner_installs_a_valid_tiling_and_keeps_parity(orc):
    from paper_1808_02638_gb300 import tune
    from paper_1808_02638_gb300.solver import Hierarchy
    run = inputs.config1(256, 32)
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    H = Hierarchy([run], [[q]], rho0=1.0, K0=4.0)
    H.init_dt()
    best, timings = tune.tune_level(H, 0, use_cache=False)
    assert best in timings and len(timings) >= 4 and all(v > 0 for v in timings.values())
    for _ in range(5):
        H.coarse_step()
    srun, sq = single_grid(256)
    rho, K = _uniform_planes(256)
    want, _ = oracle_single(orc, srun, sq, rho, K, 5)
    got = np.zeros_like(want)
    for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
        got[:, jlo:jlo + bny, ilo:ilo + bnx] = H.interior(0, 0, nb)
    assert rel_err(got, want) <= TOLN


@pytest.mark.parametrize("case", ["tiled_extrap", "tiled_periodic", "single_wall_16", "cellwise_32x16"])
def test_fused_advance_equals_fill_step_update(case):
    # the fused one-launch step (ghosts pulled from their sources, Eq. cfl on the last CTA)
    # reproduces fill + step + dt update bit for bit: interiors, dt and the reset speed maximum;
    # one more step with the ghost push as well gives q_new's ghosts equal to a fill
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    import torch
    tiling, medium = None, None
    if case.startswith("tiled"):
        run = inputs.config1(128, 32)
        if case == "tiled_periodic":
            run.bc = (1, 1, 1, 1)
    elif case == "single_wall_16":
        run, _ = single_grid(100, bc=(2, 2, 0, 2))
        tiling = (16, 16, 1)
    else:
        run, _ = single_grid(64)
        tiling = (32, 16, 1)
        medium = inputs.config3(64)
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    if medium is not None:
        _, r2, k2 = medium
        mk = lambda: Hierarchy([run], [[q]], [[inputs.coef_pool(lev, r2, 1)]], [[inputs.coef_pool(lev, k2, 1)]],
                               tiling=tiling)
    else:
        mk = lambda: Hierarchy([run], [[q]], rho0=1.0, K0=4.0, tiling=tiling)
    A, B = mk(), mk()
    B.fused = True
    for h in (A, B):
        h.init_dt()
    for _ in range(7):
        A.coarse_step()
        B.coarse_step()
    torch.cuda.synchronize()
    a, b = A.pool(0).cpu().numpy(), B.pool(0).cpu().numpy()
    for n, box in enumerate(lev.boxes):
        va = inputs.box_view(a, lev.qoff[n], int(box[2]), int(box[3]), 3)[:, 2:-2, 2:-2]
        vb = inputs.box_view(b, lev.qoff[n], int(box[2]), int(box[3]), 3)[:, 2:-2, 2:-2]
        assert np.array_equal(va, vb)
    assert float(A.dt[0]) == float(B.dt[0]) and float(B.smax[0]) == 0.0
    # push as well: the ghosts of q_new are those a fill gives
    A.coarse_step()
    src, dst = B.q[0][B.cur[0]], B.q[0][1 - B.cur[0]]
    claw.claw_level_advance(B.ctx, 0, src, dst, B.aux[0], B.dt, B.smax,
                            claw.CLAW_ADVANCE_PULL_GHOSTS | claw.CLAW_ADVANCE_PUSH_GHOSTS |
                            claw.CLAW_ADVANCE_UPDATE_DT)
    B.cur[0] ^= 1
    claw.claw_fill_ghost(A.ctx, 0, A.pool(0))
    torch.cuda.synchronize()
    assert torch.equal(A.pool(0), B.pool(0))
    assert A.sync_status() == 0 and B.sync_status() == 0


def test_captured_graph_survives_descriptor_cache_churn(orc):
    # a staged step captured into a CUDA graph reads the tensor-map descriptors of its pool; the
    # context caches descriptors per pool and evicts old ones, but never one a capture has seen:
    # after eager steps from more other pools than the cache holds, the graph still steps the
    # right pool (equal to the eager step bit for bit)
    import torch
    from paper_1808_02638_gb300 import claw
    from paper_1808_02638_gb300.solver import Hierarchy
    n = 64
    run, q = single_grid(n, pulse=False, seed=5)
    H = Hierarchy([run], [[q]], rho0=1.3, K0=2.7, tiling=(32, 32, 1))
    H.dt.fill_(0.005)
    src, dst = H.q[0][0], H.q[0][1]
    flags = claw.CLAW_ADVANCE_PULL_GHOSTS
    claw.claw_level_advance(H.ctx, 0, src, dst, None, H.dt, H.smax, flags)   # descriptor of src cached
    torch.cuda.synchronize()
    want = dst.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        claw.claw_level_advance(H.ctx, 0, src, dst, None, H.dt, H.smax, flags, s)
    torch.cuda.current_stream().wait_stream(s)
    others = [src.clone() + 0.25 * k for k in range(1, 7)]
    for o in others:   # six more pools through the cache
        claw.claw_level_advance(H.ctx, 0, o, torch.empty_like(o), None, H.dt, H.smax, flags)
    dst.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(H.interior(0, 0, 0, pool=dst), H.interior(0, 0, 0, pool=want))
    assert H.sync_status() == 0
