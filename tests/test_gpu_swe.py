"""GPU parity of the shallow-water level-step (the second system through the same fused step,
ghost filling, averaging and CFL control) against the shallow-water oracle, through the C ABI.

Tolerances as for acoustics: max |GPU - oracle| <= 1e-12 max|q| after one step, <= 1e-10 max|q|
after 100 steps; the time steps (Eq. cfl from the largest Roe speed of the previous step) agree
to 1e-13.  The GPU takes Roe averages with one reciprocal per edge and reciprocal square roots,
the oracle plain IEEE divisions and square roots in textbook order."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

from gpu_helpers import M, lib_ready, rel_err

pytestmark = pytest.mark.gpu

TOL1, TOLN = 1e-12, 1e-10
G = 1.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _run(n, boxes=None, bc=(0, 0, 0, 0), limiter=4, order=2, transverse=2):
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=bc, limiter=limiter, order=order, transverse=transverse)
    d = 2.0 / n
    run.levels = [inputs.Level(n, n, d, d, [(0, 0, n, n)] if boxes is None else boxes)]
    return run


def _hier(run, q, tiling=None, grav=G):
    from paper_1808_02638_gb300.solver import Hierarchy
    qs = q if isinstance(q, list) else [q]
    return Hierarchy([run], [qs], tiling=tiling, system="shallow_water", grav=grav)


def _oracle(run, q, grav=G):
    from oracle.amr import OracleHierarchy
    qs = q if isinstance(q, list) else [q]
    return OracleHierarchy(run, qs, system="shallow_water", grav=grav)


def _interiors(run, pool_of, L=0):
    lev = run.levels[L]
    return [inputs.box_view(pool_of(L), lev.qoff[n], int(b[2]), int(b[3]), 3)[:, M:-M, M:-M]
            for n, b in enumerate(lev.boxes)]


def _compare(run, H, O, tol):
    scale = max(np.abs(O.q[L]).max() for L in range(len(run.levels)))
    for L in range(len(run.levels)):
        got = _interiors(run, lambda l: H.level_numpy(0, l), L)
        want = _interiors(run, lambda l: O.q[l], L)
        for g, w in zip(got, want):
            assert np.abs(g - w).max() <= tol * scale


def _random_wet(run, seed):
    lev = run.levels[0]
    q = np.zeros(lev.qsize)
    for k, b in enumerate(lev.boxes):
        v = inputs.box_view(q, lev.qoff[k], int(b[2]), int(b[3]), 3)
        u = inputs.uniform(seed + k, v.size).reshape(v.shape)
        v[0] = 0.5 + u[0]
        v[1] = u[1] - 0.5
        v[2] = u[2] - 0.5
    return q


@pytest.mark.parametrize("tiling", [(16, 16, 1), (16, 16, 0), (32, 16, 1), (32, 16, 0)])
def test_ring_with_mean_flow_one_and_100_steps(orc, tiling):
    # 100^2 single box (ragged against both tile shapes), ring-pulse depth 1..2 with a mean flow
    run = _run(100)
    q = inputs.init_swe(run, run.levels[0], u0=0.3, v0=-0.2)
    H = _hier(run, q, tiling=tiling)
    O = _oracle(run, q)
    H.init_dt()
    dt0 = run.cfl * run.levels[0].dx / O.smax
    assert float(H.dt[0]) == pytest.approx(dt0, rel=1e-15)
    H.coarse_step()
    O.coarse_step()
    _compare(run, H, O, TOL1)
    for _ in range(99):
        H.coarse_step()
        O.coarse_step()
    _compare(run, H, O, TOLN)
    assert float(H.dt[0]) == pytest.approx(run.cfl * run.levels[0].dx / O.smax, rel=1e-13)
    assert H.sync_status() == 0


@pytest.mark.parametrize("limiter", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("order,transverse", [(2, 2), (2, 1), (2, 0), (1, 0), (1, 1)])
def test_schemes_random_wet_data_one_step(orc, limiter, order, transverse):
    n = 36
    run = _run(n, limiter=limiter, order=order, transverse=transverse)
    q = _random_wet(run, 300 + limiter)
    H = _hier(run, q, tiling=(16, 16, 1))
    O = _oracle(run, q)
    H.dt.fill_(0.004)
    H.coarse_step()
    O.coarse_step(dt=0.004)
    _compare(run, H, O, TOL1)


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (2, 2, 2, 2), (2, 0, 1, 1)])
def test_boundary_conditions_ten_steps(orc, bc):
    n = 40
    run = _run(n, bc=bc)
    q = _random_wet(run, 17)
    H = _hier(run, q, tiling=(32, 16, 1))
    O = _oracle(run, q)
    H.init_dt()
    for _ in range(10):
        H.coarse_step()
        O.coarse_step()
    _compare(run, H, O, TOLN)


def test_many_patches_with_same_level_ghosts(orc):
    # 96^2 as 9 patches of 32 x 32 and one run of mixed boxes: ghost copies between patches
    run = _run(96, boxes=inputs.uniform_tiling(96, 96, 32, 32))
    q = inputs.init_swe(run, run.levels[0], u0=-0.25, v0=0.1)
    H = _hier(run, q)
    O = _oracle(run, q)
    H.init_dt()
    for _ in range(30):
        H.coarse_step()
        O.coarse_step()
    _compare(run, H, O, TOLN)


def test_three_level_amr_two_coarse_steps(orc):
    # the 3-level ratio-4 hierarchy of the AMR workload with a shallow-water ring: subcycling,
    # space-time interpolated fine ghosts and averaging, all through the same kernels
    run = inputs.config2()
    q = [inputs.init_swe(run, lev, u0=0.2, v0=0.1) for lev in run.levels]
    H = _hier(run, q)
    O = _oracle(run, q)
    H.init_dt()
    assert float(H.dt[0]) == pytest.approx(run.cfl * run.levels[0].dx / O.smax, rel=1e-15)
    H.coarse_step()
    O.coarse_step()
    _compare(run, H, O, TOL1 * 10)
    H.coarse_step()
    O.coarse_step()
    _compare(run, H, O, TOLN)
    assert H.sync_status() == 0


def test_conservation_fix_three_levels_matches_oracle(orc):
    # the conservation fix of Sec. 2.3 for shallow water (flux form with the equations' flux):
    # the 3-level hierarchy with a flowing ring, GPU against the oracle over 6 coarse steps
    run = inputs.config2()
    q = [inputs.init_swe(run, lev, u0=0.2, v0=0.1) for lev in run.levels]
    from paper_1808_02638_gb300.solver import Hierarchy
    from oracle.amr import OracleHierarchy
    H = Hierarchy([run], [q], system="shallow_water", grav=G, reflux=True)
    O = OracleHierarchy(run, q, reflux=True, system="shallow_water", grav=G)
    H.init_dt()
    H.coarse_step()
    O.coarse_step()
    _compare(run, H, O, TOL1 * 10)
    for _ in range(5):
        H.coarse_step()
        O.coarse_step()
    _compare(run, H, O, TOLN)
    assert H.sync_status() == 0


def test_conservation_fix_conserves_the_composite_integral():
    from gpu_amr_helpers import composite
    from paper_1808_02638_gb300.solver import Hierarchy
    # the inward half of the ring focuses and the speeds grow by up to 9 % within a coarse step:
    # CFL 0.7 keeps every step's CFL number below 1
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1), cfl=0.7)
    run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45)], [2002])
    q = [inputs.init_swe(run, lev, depth=lambda x, y: inputs.radial_pulse(x - 0.1, y + 0.05), u0=0.3, v0=-0.2)
         for lev in run.levels]
    drift = {}
    for reflux in (True, False):
        H = Hierarchy([run], [q], system="shallow_water", grav=G, reflux=reflux)
        H.init_dt()
        m0 = composite(H)
        for _ in range(8):
            H.coarse_step()
        drift[reflux] = np.abs(composite(H) - m0)
        assert H.sync_status() == 0
    scale = 4.0 * 2.0
    assert (drift[True] <= 1e-13 * scale).all(), drift[True]
    assert drift[False].max() >= 1e-6 * scale, drift[False]


def test_regridding_matches_the_oracle(orc):
    # flags, Berger-Rigoutsos boxes and the transfer are system-independent: the shallow-water
    # hierarchy regridded every 4 coarse steps follows the oracle's
    from oracle.amr import OracleHierarchy
    from paper_1808_02638_gb300.solver import Hierarchy
    params = dict(tol=0.02, buffer=2, cutoff=0.7, max_size=64, nest=2)
    run_g, run_o = inputs.config2(), inputs.config2()   # each side rebuilds its own levels
    q = [inputs.init_swe(run_g, lev, u0=0.2, v0=0.1) for lev in run_g.levels]
    H = Hierarchy([run_g], [q], system="shallow_water", grav=G, reflux=True)
    O = OracleHierarchy(run_o, q, reflux=True, system="shallow_water", grav=G)
    H.init_dt()
    for k in range(8):
        H.coarse_step()
        O.coarse_step()
        if (k + 1) % 4 == 0:
            H.regrid(**params)
            O.regrid(**params)
            for L in (1, 2):
                assert np.array_equal(run_g.levels[L].boxes, run_o.levels[L].boxes)
            _compare(run_g, H, O, TOLN)
    _compare(run_g, H, O, TOLN)
    assert H.sync_status() == 0


@pytest.mark.parametrize("bc", [(2, 2, 2, 2), (1, 1, 0, 0)])
def test_pulled_ghosts_equal_filled_ghosts(bc):
    # the one-launch path (ghosts pulled from their sources, wall flips of hu and hv) against
    # fill + step + dt update on 9 patches: bit for bit over 10 steps
    import torch
    run = _run(96, boxes=inputs.uniform_tiling(96, 96, 32, 32), bc=bc)
    q = inputs.init_swe(run, run.levels[0], u0=0.25, v0=-0.15)
    A, B = _hier(run, q), _hier(run, q)
    B.fused = True
    for h in (A, B):
        h.init_dt()
    for _ in range(10):
        A.coarse_step()
        B.coarse_step()
    torch.cuda.synchronize()
    for nb in range(len(run.levels[0].boxes)):
        assert np.array_equal(A.interior(0, 0, nb), B.interior(0, 0, nb))
    assert torch.equal(A.dt, B.dt) and A.sync_status() == 0 and B.sync_status() == 0


def test_graph_replay_equals_eager():
    import torch
    run = inputs.config1(256, 32)
    q = inputs.init_swe(run, run.levels[0], u0=0.1)
    A, B = _hier(run, q), _hier(run, q)
    for h in (A, B):
        h.init_dt()
        h.coarse_step()
        h.coarse_step()
    g = B.capture(2)
    for _ in range(3):
        g.replay()
        A.coarse_step()
        A.coarse_step()
    torch.cuda.synchronize()
    assert np.array_equal(A.level_numpy(0, 0), B.level_numpy(0, 0))
    assert torch.equal(A.dt, B.dt)


def test_full_size_bench_path_sampled_parity(orc):
    # 2048^2 as 4096 patches of 32 x 32, the shallow-water bench workload, through the fused
    # stepper (graphs of the one launch per step: the persistent step with ghosts pulled from
    # their source cells and the device Eq. cfl update) with the tuned tiling: sampled patches
    # equal the oracle's one-patch step from the same input (ghosts: the edge-extrapolated
    # global field) at steps 0, 40 and 79, and the radial symmetry holds at the end
    import torch
    from paper_1808_02638_gb300 import tune
    run = inputs.config1()
    lev = run.levels[0]
    q = inputs.init_swe(run, lev)
    H = _hier(run, q)
    H.init_dt()
    tune.tune_level(H, 0, use_cache=False, pull=True)
    H.coarse_step()
    st = H.fused_stepper()
    assert st.launches_per_step == 1
    rng = np.random.default_rng(9)
    sample = rng.choice(len(lev.boxes), 32, replace=False)

    def glob_of(pool):
        g = np.zeros((3, 2048, 2048))
        for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
            g[:, jlo:jlo + 32, ilo:ilo + 32] = inputs.box_view(pool, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
        return g

    for step in range(80):
        check = step in (0, 40, 79)
        if check:
            torch.cuda.synchronize()
            gp = np.pad(glob_of(H.pool(0).cpu().numpy()), ((0, 0), (M, M), (M, M)), mode="edge")
            dt = float(H.dt[0])
        st.step()
        if check:
            torch.cuda.synchronize()
            after = H.pool(0).cpu().numpy()
            scale = np.abs(after).max()
            for nb in sample:
                ilo, jlo = int(lev.boxes[nb][0]), int(lev.boxes[nb][1])
                qin = np.ascontiguousarray(gp[:, jlo:jlo + 36, ilo:ilo + 36])
                want, _ = orc.swe_step(qin, lev.dx, lev.dy, dt, G)
                got = inputs.box_view(after, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
                assert np.abs(got - want[:, M:-M, M:-M]).max() <= TOL1 * scale
    final = H.pool(0).cpu().numpy()
    glob = np.zeros((3, 2048, 2048))
    for nb, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
        glob[:, jlo:jlo + 32, ilo:ilo + 32] = inputs.box_view(final, lev.qoff[nb], 32, 32, 3)[:, M:-M, M:-M]
    h, hu, hv = glob
    tol = 1e-12 * np.abs(glob).max()
    assert np.abs(h - h.T).max() <= tol and np.abs(h - h[:, ::-1]).max() <= tol
    assert np.abs(hu - hv.T).max() <= tol and np.abs(hu + hu[:, ::-1]).max() <= tol
    assert H.sync_status() == 0


def test_dry_cell_is_reported_not_faulted():
    from paper_1808_02638_gb300 import claw
    run = _run(32)
    q = inputs.init_swe(run, run.levels[0])
    inputs.box_view(q, 0, 32, 32, 3)[0, 10, 12] = 0.0
    H = _hier(run, q)
    H.dt.fill_(0.01)
    H.coarse_step()
    assert H.sync_status() == claw.CLAW_ENAN


def test_acoustics_only_entry_points_reject_shallow_water():
    import torch
    from paper_1808_02638_gb300 import claw
    run = _run(32, boxes=inputs.uniform_tiling(32, 32, 16, 16))
    q = inputs.init_swe(run, run.levels[0])
    H = _hier(run, q)
    lam = torch.zeros_like(H.pool(0))
    for fn, args in ((claw.claw_cfl_max, (H.ctx, 0, None, H.smax)),
                     (claw.claw_set_tiling, (H.ctx, 0, 32, 16, 2, 256)),
                     (claw.claw_level_step_adjoint, (H.ctx, 0, H.pool(0), lam, lam.clone(), None, None, H.dt)),
                     (claw.claw_set_tiling, (H.ctx, 0, 32, 32, 1, 256)),
                     (claw.claw_set_tiling, (H.ctx, 0, 16, 16, 1, 128))):
        with pytest.raises(claw.ClawError) as e:
            fn(*args)
        assert e.value.status == claw.CLAW_EINVAL
    # a non-positive gravity or a medium is refused at creation
    from paper_1808_02638_gb300.solver import Hierarchy
    with pytest.raises(claw.ClawError):
        Hierarchy([run], [[q]], system="shallow_water", grav=0.0)
    with pytest.raises(ValueError):
        Hierarchy([run], [[q]], [[np.ones(1)]], [[np.ones(1)]], system="shallow_water")
