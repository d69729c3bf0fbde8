"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

Each test names the property it checks; none re-types the oracle's formulas.  A plausible
mistake in the oracle (a dropped term, a wrong sign, a transposed operand, a wrong index)
should fail at least one of them.
"""
import os

import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

M = 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def padded(nx, ny, ncomp=None, fill=0.0):
    shape = (ny + 2 * M, nx + 2 * M) if ncomp is None else (ncomp, ny + 2 * M, nx + 2 * M)
    return np.full(shape, fill, dtype=np.float64)


def interior(a):
    return a[..., M:-M, M:-M]


# ---------------------------------------------------------------- P1, P8

def test_p1_hand_worked_first_order_4x4(orc):
    q = padded(4, 4, 3)
    q[0, 1 + M, 1 + M] = 1.0
    rho = padded(4, 4, fill=1.0)
    K = padded(4, 4, fill=1.0)
    orc.fill_bc(q, (0, 0, 0, 0))
    qn, smax = orc.step(q, rho, K, 1.0, 1.0, 0.5, order=1, transverse=0, limiter=0)
    want = np.zeros((3, 4, 4))
    for line in open(os.path.join(GOLDEN, "p1_hand_4x4.txt")):
        if line.startswith("#") or not line.strip():
            continue
        m, i, j, v = line.split()
        want[int(m), int(j), int(i)] = float(v)
    assert np.array_equal(interior(qn), want)
    assert interior(qn)[0].sum() == 1.0
    assert smax == 1.0


def test_p8_limiter_tables(orc):
    for line in open(os.path.join(GOLDEN, "limiter_tables.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, th, phi = line.split()
        assert orc.philim(name, float(th)) == pytest.approx(float(phi), abs=2e-16), (name, th)


# ---------------------------------------------------------------- P7 Riemann

def test_p7_riemann_waves_sum_to_jump(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        pl, ul, pr, ur = rng.normal(size=4)
        rl, rr = rng.uniform(0.5, 2.0, 2)
        kl, kr = rng.uniform(1.0, 8.0, 2)
        w, s = orc.riemann_x(pl, ul, rl, kl, pr, ur, rr, kr)
        jump = np.array([pr - pl, ur - ul, 0.0])
        assert np.allclose(w.sum(axis=0), jump, rtol=0, atol=8e-16 * (1 + np.abs(jump).max()))
        assert s[0] == -np.sqrt(kl / rl) and s[1] == np.sqrt(kr / rr)


def test_p7_riemann_constant_medium_is_eigendecomposition(orc):
    # Z_L = Z_R: waves are eigenvectors of A (Sec. 4.1) with eigenvalues -c, +c and the
    # fluctuation sum equals A dQ
    rng = np.random.default_rng(8)
    rho, K = 1.7, 3.1
    A = np.array([[0.0, K, 0.0], [1.0 / rho, 0.0, 0.0], [0.0, 0.0, 0.0]])
    for _ in range(50):
        pl, ul, pr, ur = rng.normal(size=4)
        w, s = orc.riemann_x(pl, ul, rho, K, pr, ur, rho, K)
        for k in range(2):
            assert np.allclose(A @ w[k], s[k] * w[k], atol=1e-14)
        dq = np.array([pr - pl, ur - ul, 0.0])
        assert np.allclose(s[0] * w[0] + s[1] * w[1], A @ dq, atol=1e-14)


def test_p6_interface_reflection_transmission(orc):
    # right-going pulse hits a material interface: pressure reflection (Z_R-Z_L)/(Z_R+Z_L),
    # transmission 2 Z_R/(Z_L+Z_R) (textbook acoustics); checked on the peaks
    nx, ny = 1600, 2
    dx = 2.0 / nx
    rho = padded(nx, ny)
    K = padded(nx, ny)
    x = (np.arange(-M, nx + M) + 0.5) * dx
    left = x < 1.0
    rho[:, left], K[:, left] = 1.0, 1.0          # Z_L = 1, c_L = 1
    rho[:, ~left], K[:, ~left] = 2.0, 8.0        # Z_R = 4, c_R = 2
    zl, zr = 1.0, 4.0
    w = np.exp(-((x - 0.5) / 0.05) ** 2)
    q = padded(nx, ny, 3)
    q[0] = zl * w
    q[1] = w
    T = 0.8
    dt0 = 0.9 * dx / 2.0
    n = int(np.ceil(T / dt0))
    from oracle.amr import run_single_grid
    qf, _ = run_single_grid(q, rho, K, dx, dx, n, bc=(0, 0, 0, 0), dt=T / n, limiter=4)
    p = qf[0, M]
    refl = p[left].min()
    trans = p[~left].max()
    R = (zr - zl) / (zr + zl)
    Tc = 2 * zr / (zl + zr)
    assert abs(p[left].max() - R * zl) < 0.02 * zl          # reflected pulse: 0.6 x incident
    assert abs(trans - Tc * zl) < 0.02 * Tc * zl            # transmitted: 1.6 x incident
    assert refl > -1e-3


# ---------------------------------------------------------------- P2 uniform state

@pytest.mark.parametrize("limiter", [0, 1, 2, 3, 4])
def test_p2_uniform_state_is_preserved_bit_exactly(orc, limiter):
    nx, ny = 13, 9
    run, rho, K = inputs.config3(32)
    rho = np.pad(rho[:ny, :nx], M, mode="edge")
    K = np.pad(K[:ny, :nx], M, mode="edge")
    q = padded(nx, ny, 3)
    q[0], q[1], q[2] = 1.25, -0.5, 0.75
    qn, _ = orc.step(q, rho, K, 0.1, 0.07, 0.004, limiter=limiter)
    assert np.array_equal(qn, q)


# ---------------------------------------------------------------- P3 plane waves

def _plane_wave_error(orc, N, limiter, theta_deg, T, w):
    from oracle.amr import run_single_grid
    th = np.deg2rad(theta_deg)
    rho0, K0 = 1.0, 4.0
    c, Z = 2.0, 2.0
    if theta_deg == 0:
        Lx, Nx, Ny = 1.0, N, 4
        Ly = Ny * Lx / Nx
    else:
        # anisotropic cells (dy close to dx/2) so that dx and dy enter the update separately
        Lx, Ly = 1 / np.cos(th), 1 / np.sin(th)
        Nx, Ny = N, int(round(2 * N * Ly / Lx))
    dx, dy = Lx / Nx, Ly / Ny
    x = (np.arange(-M, Nx + M) + 0.5) * dx
    y = (np.arange(-M, Ny + M) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    xi = X * np.cos(th) + Y * np.sin(th)
    q = np.zeros((3, Ny + 2 * M, Nx + 2 * M))
    q[0], q[1], q[2] = Z * w(xi), np.cos(th) * w(xi), np.sin(th) * w(xi)
    dt0 = 0.9 * min(dx, dy) / c
    n = int(np.ceil(T / dt0))
    qf, _ = run_single_grid(q, np.full(X.shape, rho0), np.full(X.shape, K0), dx, dy, n,
                            bc=(1, 1, 1, 1), dt=T / n, limiter=limiter)
    exact = Z * w(xi - c * T)
    return np.abs(interior(qf[0]) - interior(exact)).mean()


@pytest.mark.parametrize("limiter,rate", [(0, 1.9), (4, 1.8)])
def test_p3_plane_wave_second_order_along_x(orc, limiter, rate):
    w = lambda s: np.sin(2 * np.pi * s) + 0.5 * np.exp(-40 * np.sin(np.pi * (s - 0.3)) ** 2)
    e = [_plane_wave_error(orc, N, limiter, 0, 0.5, w) for N in (50, 100, 200, 400)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert rates[-1] >= rate and rates[-2] >= rate - 0.05, rates


@pytest.mark.parametrize("limiter,rate", [(0, 1.9), (4, 1.8)])
def test_p3_plane_wave_second_order_oblique_30deg(orc, limiter, rate):
    w = lambda s: np.sin(2 * np.pi * s)
    e = [_plane_wave_error(orc, N, limiter, 30, 0.25, w) for N in (20, 40, 80, 160)]
    rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert rates[-1] >= rate and rates[-2] >= rate, rates


def test_p3_transverse_terms_are_needed_for_second_order(orc):
    # with the transverse terms off the unsplit method is only first order for an oblique
    # wave: guards against a transverse solver that silently contributes nothing
    from oracle.amr import run_single_grid
    th = np.deg2rad(30)
    errs = []
    for N in (40, 80):
        Lx, Ly = 1 / np.cos(th), 1 / np.sin(th)
        Nx, Ny = N, int(round(N * Ly / Lx))
        dx, dy = Lx / Nx, Ly / Ny
        X, Y = np.meshgrid((np.arange(-M, Nx + M) + 0.5) * dx, (np.arange(-M, Ny + M) + 0.5) * dy)
        xi = X * np.cos(th) + Y * np.sin(th)
        q = np.zeros((3,) + X.shape)
        q[0], q[1], q[2] = 2 * np.sin(2 * np.pi * xi), np.cos(th) * np.sin(2 * np.pi * xi), \
            np.sin(th) * np.sin(2 * np.pi * xi)
        n = int(np.ceil(0.25 / (0.9 * min(dx, dy) / 2)))
        qf, _ = run_single_grid(q, np.ones(X.shape), np.full(X.shape, 4.0), dx, dy, n,
                                bc=(1, 1, 1, 1), dt=0.25 / n, limiter=0, transverse=0)
        errs.append(np.abs(interior(qf[0]) - interior(2 * np.sin(2 * np.pi * (xi - 0.5)))).mean())
    assert np.log2(errs[0] / errs[1]) < 1.5


@pytest.mark.parametrize("limiter", [1, 2, 3, 4])
def test_limited_scheme_is_tvd_for_a_simple_wave(orc, limiter):
    # a right-going simple wave with a square profile: with constant coefficients each
    # characteristic variable is advected by the scalar high-resolution scheme, which is TVD
    # for upwind-ratio limiters at CFL <= 1 -- no new extrema, total variation not increasing
    from oracle.amr import run_single_grid
    nx, ny = 200, 2
    dx = 1.0 / nx
    x = (np.arange(-M, nx + M) + 0.5) * dx
    w = ((x > 0.2) & (x < 0.4)).astype(float) + 0.5 * ((x > 0.55) & (x < 0.6))
    q = padded(nx, ny, 3)
    q[0], q[1] = 2.0 * w, w
    qf, _ = run_single_grid(q, padded(nx, ny, fill=1.0), padded(nx, ny, fill=4.0), dx, dx, 60,
                            bc=(1, 1, 1, 1), dt=0.8 * dx / 2.0, limiter=limiter)
    p = interior(qf[0])[0]
    assert p.max() <= 2.0 + 1e-12 and p.min() >= -1e-12
    tv0 = np.abs(np.diff(2.0 * w[M:-M])).sum()
    assert np.abs(np.diff(p)).sum() <= tv0 + 1e-12


# ---------------------------------------------------------------- P4 conservation

def test_p4_conservation_periodic_constant_medium(orc):
    nx = ny = 48
    rng_q = inputs.uniform(11, 3 * (nx + 4) * (ny + 4)).reshape(3, ny + 4, nx + 4) - 0.5
    q = np.ascontiguousarray(rng_q)
    orc.fill_bc(q, (1, 1, 1, 1))
    rho = padded(nx, ny, fill=1.3)
    K = padded(nx, ny, fill=2.9)
    s0 = interior(q).sum(axis=(1, 2))
    amax = np.abs(q).max()
    for _ in range(20):
        q, _ = orc.step(q, rho, K, 0.1, 0.1, 0.9 * 0.1 / np.sqrt(2.9 / 1.3))
        orc.fill_bc(q, (1, 1, 1, 1))
    s1 = interior(q).sum(axis=(1, 2))
    assert np.all(np.abs(s1 - s0) <= 20 * 1e-13 * nx * ny * amax), s1 - s0


def test_first_order_heterogeneous_conserves_p_over_K_and_momentum(orc):
    # with variable rho, K the fluctuations of the normal solver conserve sum(p/K) and
    # sum(rho u), sum(rho v) on a periodic grid (p_t + K div u = 0, rho u_t + grad p = 0);
    # a wrong impedance in the normal Riemann solver breaks this
    nx = ny = 40
    run, rho0, K0 = inputs.config3(64)
    rho = np.pad(rho0[:ny, :nx], M, mode="wrap")
    K = np.pad(K0[:ny, :nx], M, mode="wrap")
    q = padded(nx, ny, 3)
    q[:, M:-M, M:-M] = inputs.uniform(5, 3 * nx * ny).reshape(3, ny, nx) - 0.5
    orc.fill_bc(q, (1, 1, 1, 1))

    def inv(q):
        i = interior(q)
        return np.array([(i[0] / interior(K)).sum(), (interior(rho) * i[1]).sum(),
                         (interior(rho) * i[2]).sum()])

    a0 = inv(q)
    for _ in range(10):
        q, _ = orc.step(q, rho, K, 0.05, 0.05, 0.01, order=1, transverse=0, limiter=0)
        orc.fill_bc(q, (1, 1, 1, 1))
    assert np.allclose(inv(q), a0, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- P5 symmetry

def _pulse_run(orc, nsteps):
    from oracle.amr import run_single_grid
    run = inputs.config0()
    lev = run.levels[0]
    q = inputs.box_view(inputs.init_q(run, lev), 0, 100, 100, 3).copy()
    rho = padded(100, 100, fill=1.0)
    K = padded(100, 100, fill=4.0)
    qf, dts = run_single_grid(q, rho, K, lev.dx, lev.dy, nsteps)
    return interior(qf), dts


def test_p5_radial_pulse_symmetries(orc):
    q, _ = _pulse_run(orc, 30)
    p, u, v = q
    tol = 1e-13 * np.abs(q).max()
    assert np.abs(p - p[:, ::-1]).max() <= tol
    assert np.abs(p - p[::-1, :]).max() <= tol
    assert np.abs(p - p.T).max() <= tol
    assert np.abs(u + u[:, ::-1]).max() <= tol
    assert np.abs(v + v[::-1, :]).max() <= tol
    assert np.abs(u - v.T).max() <= tol


def test_symmetric_heterogeneous_medium_keeps_symmetry(orc):
    # a medium symmetric under x -> -x, y -> -y and transposition keeps the pulse symmetric:
    # pins the variable-coefficient transverse solver against lo/hi or sweep mix-ups
    from oracle.amr import run_single_grid
    n = 40
    run, r0, k0 = inputs.config3(n)
    sym = lambda a: (a + a[::-1] + a[:, ::-1] + a[::-1, ::-1] + a.T + a.T[::-1] + a.T[:, ::-1]
                     + a.T[::-1, ::-1]) / 8
    rho = np.pad(sym(r0), M, mode="edge")
    K = np.pad(sym(k0), M, mode="edge")
    lev = inputs.Level(n, n, 2 / n, 2 / n, [(0, 0, n, n)])
    q = inputs.box_view(inputs.init_q(run, lev), 0, n, n, 3).copy()
    qf, _ = run_single_grid(q, rho, K, 2 / n, 2 / n, 15)
    p, u, v = interior(qf)
    tol = 1e-13 * np.abs(interior(qf)).max()
    assert np.abs(p - p[:, ::-1]).max() <= tol
    assert np.abs(p - p[::-1]).max() <= tol
    assert np.abs(p - p.T).max() <= tol
    assert np.abs(u - v.T).max() <= tol
    assert np.abs(u + u[:, ::-1]).max() <= tol


def test_solid_wall_equals_mirror_image_problem(orc):
    # method of images: a wall at x = 0 (and at y = top) acts exactly like the mirrored
    # problem on the doubled domain with the normal velocity reversed
    nx, ny = 12, 10
    half = padded(nx, ny, 3)
    half[:, M:-M, M:-M] = inputs.uniform(31, 3 * nx * ny).reshape(3, ny, nx)
    full = padded(2 * nx, 2 * ny, 3)
    body = half[:, M:-M, M:-M].copy()
    full[:, M:M + ny, M + nx:M + 2 * nx] = body                     # lower right: original
    full[:, M:M + ny, M:M + nx] = body[:, :, ::-1] * np.array([1, -1, 1])[:, None, None]
    top = full[:, M:M + ny, M:M + 2 * nx]
    full[:, M + ny:M + 2 * ny, M:M + 2 * nx] = top[:, ::-1, :] * np.array([1, 1, -1])[:, None, None]
    ones_h, ones_f = padded(nx, ny, fill=1.0), padded(2 * nx, 2 * ny, fill=1.0)
    for _ in range(4):
        orc.fill_bc(half, (2, 0, 0, 2))
        orc.fill_bc(full, (0, 0, 0, 0))
        half, _ = orc.step(half, ones_h, 4 * ones_h, 0.1, 0.1, 0.02)
        full, _ = orc.step(full, ones_f, 4 * ones_f, 0.1, 0.1, 0.02)
    # the mirrored half accumulates its flux terms in another order: equal to rounding
    assert np.abs(interior(half) - interior(full)[:, :ny, nx:]).max() <= 1e-14 * np.abs(full).max()


# ---------------------------------------------------------------- P9 CFL

def test_p9_cfl_speed_is_max_cell_speed(orc):
    q, dts = _pulse_run(orc, 3)
    assert dts == [0.9 * 0.02 / 2.0] * 3
    run, rho0, K0 = inputs.config3(24)
    rho = np.pad(rho0, M, mode="edge")
    K = np.pad(K0, M, mode="edge")
    s_cells = orc.cfl_max(rho, K)
    qq = padded(24, 24, 3)
    qq[0, M:-M, M:-M] = inputs.uniform(3, 24 * 24).reshape(24, 24)
    orc.fill_bc(qq)
    _, s_edges = orc.step(qq, rho, K, 2 / 24, 2 / 24, 0.01)
    assert s_edges == s_cells == np.sqrt(K0 / rho0).max()


# ---------------------------------------------------------------- multi-box levels

def _level_from_single(orc, run_lev_boxes, qfull, nx, ny):
    lev = inputs.Level(nx, ny, 1.0 / nx, 1.0 / ny, run_lev_boxes)
    pool = np.zeros(lev.qsize)
    for n, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
        v = inputs.box_view(pool, lev.qoff[n], int(bnx), int(bny), 3)
        v[:, M:-M, M:-M] = qfull[:, M + jlo:M + jlo + bny, M + ilo:M + ilo + bnx]
    return lev, pool


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 2, 0, 1), (2, 0, 0, 2)])
def test_multibox_level_equals_single_grid_bitwise(orc, bc):
    # same-level ghost copies + physical boundaries make a tiled level identical to one box
    from oracle.amr import OracleHierarchy
    nx, ny = 24, 16
    q = padded(nx, ny, 3)
    q[:, M:-M, M:-M] = inputs.uniform(21, 3 * nx * ny).reshape(3, ny, nx)
    rho = padded(nx, ny, fill=1.0)
    K = padded(nx, ny, fill=4.0)
    boxes = [(0, 0, 8, 8), (8, 0, 16, 4), (8, 4, 8, 12), (16, 4, 8, 12), (0, 8, 8, 8)]
    lev, pool = _level_from_single(orc, boxes, q, nx, ny)
    run = inputs.Run(0, 0, 1, 1, [lev], bc=bc)
    H = OracleHierarchy(run, [pool], [inputs.const_pool(lev, 1.0)], [inputs.const_pool(lev, 4.0)])
    single = q.copy()
    for _ in range(3):
        H.coarse_step(dt=0.01)
        orc.fill_bc(single, bc)
        single, _ = orc.step(single, rho, K, lev.dx, lev.dy, 0.01)
    for n, (ilo, jlo, bnx, bny) in enumerate(lev.boxes):
        assert np.array_equal(H.interior(0, n), interior(single)[:, jlo:jlo + bny, ilo:ilo + bnx])


# ---------------------------------------------------------------- P10 AMR

def _two_level(coarse_n=8, r=4, fine_boxes=((8, 8, 8, 8),)):
    run = inputs.Run(-1, -1, 1, 1)
    d = 2.0 / coarse_n
    L0 = inputs.Level(coarse_n, coarse_n, d, d, [(0, 0, coarse_n, coarse_n)])
    L1 = inputs.Level(coarse_n * r, coarse_n * r, d / r, d / r, fine_boxes, ratio=r)
    run.levels = [L0, L1]
    return run


def test_p10_interp_conservative_and_exact_for_linear(orc):
    run = _two_level()
    L0, L1 = run.levels
    c = np.zeros(L0.qsize)
    v = inputs.box_view(c, 0, 8, 8, 3)
    I, J = np.meshgrid(np.arange(-M, 8 + M), np.arange(-M, 8 + M))
    v[0] = 0.3 * I - 0.7 * J + 2.0                    # linear
    v[1] = np.sin(I) * np.cos(0.3 * J)               # arbitrary
    v[2] = (I * J) % 5
    cb = [(0, 0, 8, 8, 0)]
    for (I0, J0) in [(3, 4), (1, 1), (6, 2)]:
        kids = np.array([orc.interp_cell(cb, c, c, 0.0, 4, 3, 8, 8, (0, 0, 0, 0), 4 * I0 + a, 4 * J0 + b)
                         for b in range(4) for a in range(4)])
        assert np.allclose(kids.mean(axis=0), v[:, J0 + M, I0 + M], atol=1e-15)
        for k, (a, b) in enumerate([(a, b) for b in range(4) for a in range(4)]):
            xf = I0 + (a + 0.5) / 4 - 0.5
            yf = J0 + (b + 0.5) / 4 - 0.5
            assert kids[k, 0] == pytest.approx(0.3 * xf - 0.7 * yf + 2.0, abs=1e-14)


def test_p10_interp_time_fraction(orc):
    run = _two_level()
    L0 = run.levels[0]
    a = np.zeros(L0.qsize)
    b = np.zeros(L0.qsize)
    inputs.box_view(a, 0, 8, 8, 3)[:] = 1.0
    inputs.box_view(b, 0, 8, 8, 3)[:] = 3.0
    cb = [(0, 0, 8, 8, 0)]
    assert np.all(orc.interp_cell(cb, a, b, 0.0, 4, 3, 8, 8, (0,) * 4, 9, 9) == 1.0)
    assert np.all(orc.interp_cell(cb, a, b, 0.25, 4, 3, 8, 8, (0,) * 4, 9, 9) == 1.5)
    assert np.all(orc.interp_cell(cb, a, b, 1.0, 4, 3, 8, 8, (0,) * 4, 9, 9) == 3.0)


def test_p10_interp_minmod_limits_at_extremum(orc):
    # a coarse local maximum gets zero slope: no new extrema from the interpolation
    run = _two_level()
    c = np.zeros(run.levels[0].qsize)
    v = inputs.box_view(c, 0, 8, 8, 3)
    v[0, M + 4, M + 4] = 1.0
    vals = [orc.interp_cell([(0, 0, 8, 8, 0)], c, c, 0.0, 4, 3, 8, 8, (0,) * 4, 16 + a, 16 + b)[0]
            for a in range(4) for b in range(4)]
    assert np.all(np.array(vals) == 1.0)


def test_p10_average_then_interp_constant_exact_and_uniform_preserved(orc):
    from oracle.amr import OracleHierarchy
    run = _two_level(fine_boxes=[(8, 8, 8, 8), (16, 8, 8, 12)])
    L0, L1 = run.levels
    q0 = np.zeros(L0.qsize)
    q1 = np.zeros(L1.qsize)
    for pool, lev in ((q0, L0), (q1, L1)):
        for n, b in enumerate(lev.boxes):
            v = inputs.box_view(pool, lev.qoff[n], int(b[2]), int(b[3]), 3)
            v[0], v[1], v[2] = 0.75, -0.25, 0.5
    H = OracleHierarchy(run, [q0, q1], [inputs.const_pool(L, 1.0) for L in run.levels],
                        [inputs.const_pool(L, 4.0) for L in run.levels])
    for _ in range(2):
        H.coarse_step()
    for L, lev in enumerate(run.levels):
        for n in range(len(lev.boxes)):
            i = H.interior(L, n)
            assert np.all(i[0] == 0.75) and np.all(i[1] == -0.25) and np.all(i[2] == 0.5)


def test_p10_full_cover_fine_level_equals_single_fine_grid(orc):
    # a fine level covering the whole domain has no interpolated ghosts: after a coarse step
    # its solution is the single fine grid's after r fine steps, and the coarse level holds
    # the average of it
    from oracle.amr import OracleHierarchy
    r = 2
    run = _two_level(coarse_n=8, r=r, fine_boxes=[(0, 0, 8, 16), (8, 0, 8, 8), (8, 8, 8, 8)])
    L0, L1 = run.levels
    q0 = inputs.init_q(run, L0)
    q1 = inputs.init_q(run, L1)
    H = OracleHierarchy(run, [q0, q1], [inputs.const_pool(L, 1.0) for L in run.levels],
                        [inputs.const_pool(L, 4.0) for L in run.levels])
    single = np.zeros((3, 20, 20))
    for n, (ilo, jlo, bnx, bny) in enumerate(L1.boxes):
        single[:, M + jlo:M + jlo + bny, M + ilo:M + ilo + bnx] = \
            inputs.box_view(q1, L1.qoff[n], int(bnx), int(bny), 3)[:, M:-M, M:-M]
    rho = np.ones((20, 20))
    K = np.full((20, 20), 4.0)
    dt = H.coarse_step()
    for _ in range(r):
        orc.fill_bc(single)
        single, _ = orc.step(single, rho, K, L1.dx, L1.dy, dt / r)
    for n, (ilo, jlo, bnx, bny) in enumerate(L1.boxes):
        assert np.array_equal(H.interior(1, n), interior(single)[:, jlo:jlo + bny, ilo:ilo + bnx])
    avg = interior(single).reshape(3, 8, 2, 8, 2).mean(axis=(2, 4))
    assert np.allclose(H.interior(0, 0), avg, atol=1e-15)


def test_amr_hierarchy_generator_is_nested_and_disjoint():
    run = inputs.config2()
    L0, L1, L2 = run.levels
    for lev in (L1, L2):
        b = lev.boxes
        assert np.all(b[:, 2] >= 8) and np.all(b[:, 2] <= 64) and np.all(b[:, 3] >= 8) and np.all(b[:, 3] <= 64)
        assert np.all(b % 4 == 0)
        cover = np.zeros((lev.NY, lev.NX), dtype=int)
        for ilo, jlo, nx, ny in b:
            cover[jlo:jlo + ny, ilo:ilo + nx] += 1
        assert cover.max() == 1
    # level 2 boxes (grown by two level-1 cells) lie inside level 1
    c1 = np.zeros((L1.NY, L1.NX), dtype=bool)
    for ilo, jlo, nx, ny in L1.boxes:
        c1[jlo:jlo + ny, ilo:ilo + nx] = True
    need = inputs.box_mask(L2.boxes, L1.NX, L1.NY, grow=2, scale_down=4)
    assert np.all(c1[need])
    assert 8000 < L1.ncells < 16000 and 45000 < L2.ncells < 90000


def test_splitmix64_published_sequence():
    # first outputs of splitmix64 seeded with 1234567 (the generator's reference sequence)
    z = inputs.splitmix64(1234567, 5)
    assert [int(v) for v in z] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                   4593380528125082431, 16408922859458223821]


# ------------------------------------------------- transverse correction weight (reading 4)

def _split_parts(rho, K, axis):
    """the acoustics matrix of Sec. 4.1 for direction `axis` (0: A, 1: B) and its positive,
    negative and absolute parts, from numpy's eigen-decomposition"""
    Mat = np.zeros((3, 3))
    Mat[0, 1 + axis] = K
    Mat[1 + axis, 0] = 1.0 / rho
    lam, R = np.linalg.eig(Mat)
    lam, R = lam.real, R.real
    Ri = np.linalg.inv(R)
    plus = R @ np.diag(np.maximum(lam, 0.0)) @ Ri
    minus = R @ np.diag(np.minimum(lam, 0.0)) @ Ri
    return plus, minus, plus - minus


def _scheme_symbol(rho, K, nux, nuy, thx, thy, transverse, cw):
    """Amplification matrix of the unlimited (Lax-Wendroff) unsplit wave-propagation step with
    constant coefficients, derived in Fourier space from Eq. wave_form_2d_2nd_order:
      Q+ = Q - nux (A+ dQ_{i-1/2} + A- dQ_{i+1/2}) - nuy (B+ dQ_{j-1/2} + B- dQ_{j+1/2})
             - nux (F_{i+1/2} - F_{i-1/2}) - nuy (G_{j+1/2} - G_{j-1/2}),
    F = 1/2 |A|(I - nux|A|) dQ, the fluctuation D into a cell (A+dQ - cw C from its left edge,
    A-dQ + cw C from its right edge, C = |A|(I - nux|A|) dQ) split by B+ onto its upper edge
    and B- onto its lower edge with weight -nux/2 (and x <-> y).  Every edge quantity is
    written relative to the cell right of / above it; a shift by one cell is a factor e^{i th}."""
    I3 = np.eye(3)
    Ap, Am, Aa = _split_parts(rho, K, 0)
    Bp, Bm, Ba = _split_parts(rho, K, 1)
    ex, ey = np.exp(1j * thx), np.exp(1j * thy)
    jxl, jxr = 1 - 1 / ex, ex - 1        # Q_i - Q_{i-1} and Q_{i+1} - Q_i over Q_i
    jyl, jyr = 1 - 1 / ey, ey - 1
    Cx = Aa @ (I3 - nux * Aa)
    Cy = Ba @ (I3 - nuy * Ba)
    F = 0.5 * Cx * jxl                  # correction flux at the cell's left edge
    G = 0.5 * Cy * jyl
    if transverse:
        D = (Ap - cw * Cx) * jxl + (Am + cw * Cx) * jxr
        E = (Bp - cw * Cy) * jyl + (Bm + cw * Cy) * jyr
        F = F - 0.5 * nuy * (Ap @ E / ex + Am @ E)   # from the cells left of and right of the edge
        G = G - 0.5 * nux * (Bp @ D / ey + Bm @ D)
    return I3 - nux * (Ap * jxl + Am * jxr) - nuy * (Bp * jyl + Bm * jyr) - nux * jxr * F - nuy * jyr * G


def _oracle_amplification(orc, rho, K, dx, dy, dt, Nx, Ny, mx, my, transverse):
    """one oracle step of e_m cos(phi) and e_m sin(phi), phi = th . (i, j), on a periodic grid;
    returns the amplification matrix and its spread over the cells"""
    thx, thy = 2 * np.pi * mx / Nx, 2 * np.pi * my / Ny
    I, J = np.meshgrid(np.arange(-M, Nx + M), np.arange(-M, Ny + M))
    phase = thx * I + thy * J
    rh = padded(Nx, Ny, fill=rho)
    kk = padded(Nx, Ny, fill=K)
    G = np.zeros((3, 3), dtype=complex)
    spread = 0.0
    for m in range(3):
        out = []
        for wave in (np.cos(phase), np.sin(phase)):
            q = padded(Nx, Ny, 3)
            q[m] = wave
            orc.fill_bc(q, (1, 1, 1, 1))
            qn, _ = orc.step(q, rh, kk, dx, dy, dt, order=2, transverse=transverse, limiter=0)
            out.append(interior(qn))
        col = (out[0] + 1j * out[1]) * np.exp(-1j * interior(phase))[None]
        G[:, m] = col.reshape(3, -1).mean(axis=1)
        spread = max(spread, np.abs(col - G[:, m][:, None, None]).max())
    return G, spread, thx, thy


@pytest.mark.parametrize("mode", [(1, 1), (3, 2), (5, 4), (7, 5), (2, 6)])
def test_transverse_correction_weight_fourier_symbol(orc, mode):
    # With constant rho, K, periodic boundaries and no limiter the step is linear and shift
    # invariant, so each Fourier mode is multiplied by a 3x3 matrix.  The oracle's matrix,
    # measured by stepping cos / sin modes, must equal the symbol derived above with the
    # correction propagated at full weight for transverse = 2 and at zero weight for
    # transverse = 1; at these parameters the half weight is measurably different.
    rho, K = 1.7, 3.1
    c = np.sqrt(K / rho)
    Nx, Ny = 16, 12
    dx, dy = 0.1, 0.07
    dt = 0.5 * dx / c
    nux, nuy = dt / dx, dt / dy
    assert nuy * c < 1.0
    for transverse, cw in ((2, 1.0), (1, 0.0), (0, 0.0)):
        G, spread, thx, thy = _oracle_amplification(orc, rho, K, dx, dy, dt, Nx, Ny, *mode, transverse)
        assert spread < 1e-13                      # one mode in, the same mode out
        want = _scheme_symbol(rho, K, nux, nuy, thx, thy, transverse, cw)
        assert np.abs(G - want).max() < 1e-13, (transverse, np.abs(G - want).max())
        if transverse == 2:
            half = _scheme_symbol(rho, K, nux, nuy, thx, thy, transverse, 0.5)
            assert np.abs(half - want).max() > 1e-3


def test_scheme_symbol_is_second_order_accurate():
    # the derived symbol against the exact propagator exp(-dt (i kx A + i ky B)) of the
    # acoustics system: the one-step error falls like h^3 (second order) -- checks the
    # derivation itself, independently of the oracle
    from scipy.linalg import expm
    rho, K = 1.7, 3.1
    c = np.sqrt(K / rho)
    kx, ky = 2.0, 1.3
    A = np.array([[0, K, 0], [1 / rho, 0, 0], [0, 0, 0]])
    B = np.array([[0, 0, K], [0, 0, 0], [1 / rho, 0, 0]])
    errs = []
    for h in (0.02, 0.01, 0.005):
        dx, dy = h, 0.7 * h
        dt = 0.5 * dx / c
        want = expm(-dt * (1j * kx * A + 1j * ky * B))
        got = _scheme_symbol(rho, K, dt / dx, dt / dy, kx * dx, ky * dy, 2, 1.0)
        errs.append(np.abs(got - want).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), rates


# ------------------------------------------------- subcycling time fraction (reading 8)

def test_subcycling_time_fraction_exact_on_linear_data(orc):
    # q linear in x and y solves q_t + A q_x + B q_y = 0 exactly as q(t) = q(0) - t (A qx + B qy)
    # (constant gradients).  On such data every step of the method is exact up to rounding:
    # each wave is the same on every edge (theta = 1, MC phi = 1), the correction and transverse
    # terms are constant and cancel in the update, the minmod slopes of the interpolation are the
    # gradient, and the time-linear coarse state is exact -- but only at the fine level's own time.
    # So fine ghosts interpolated at the right fraction of the coarse step leave every fine cell
    # and every coarse cell away from the (extrapolating) domain edge exact.
    from oracle.amr import OracleHierarchy
    r, Nc = 4, 32
    d = 2.0 / Nc
    run = inputs.Run(-1.0, -1.0, 1.0, 1.0)
    L0 = inputs.Level(Nc, Nc, d, d, [(0, 0, Nc, Nc)])
    L1 = inputs.Level(Nc * r, Nc * r, d / r, d / r, [(48, 52, 24, 20), (72, 52, 16, 28)], ratio=r)
    run.levels = [L0, L1]
    rho, K = 1.3, 2.9
    g = np.array([[0.3, -0.2], [0.05, 0.2], [0.1, -0.15]])      # (p, u, v) x (d/dx, d/dy)
    q0 = np.array([1.0, 0.1, -0.2])
    rate = np.array([K * (g[1, 0] + g[2, 1]), g[0, 0] / rho, g[0, 1] / rho])   # A qx + B qy

    def exact(x, y, t):
        return (q0 - t * rate)[:, None, None] + g[:, 0, None, None] * x + g[:, 1, None, None] * y

    pools = []
    for lev in run.levels:
        pool = np.zeros(lev.qsize)
        for n, b in enumerate(lev.boxes):
            x, y = inputs.cell_centres(run, lev, b)
            inputs.box_view(pool, lev.qoff[n], int(b[2]), int(b[3]), 3)[:] = exact(x, y, 0.0)
        pools.append(pool)
    H = OracleHierarchy(run, pools, [inputs.const_pool(L, rho) for L in run.levels],
                        [inputs.const_pool(L, K) for L in run.levels])
    nsteps = 2
    for _ in range(nsteps):
        H.coarse_step()
    t = float(np.sum(H.dt_history))
    scale = np.abs(q0).max() + 1.0
    for n, b in enumerate(L1.boxes):
        x, y = inputs.cell_centres(run, L1, b)
        err = np.abs(H.interior(1, n) - interior(exact(x, y, t))).max()
        assert err < 1e-13 * scale, (n, err)
    x, y = inputs.cell_centres(run, L0, L0.boxes[0])
    e = np.abs(H.interior(0, 0) - interior(exact(x, y, t))).max(axis=0)
    m = 2 * (nsteps + 1)
    assert e[m:-m, m:-m].max() < 1e-13 * scale
    assert e.max() > 1e-6           # the extrapolating edge is not exact: the data is not trivial
