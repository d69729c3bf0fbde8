"""Pins of the shallow-water oracle (the second system through the same step, Sec. 3.3: a
system enters the framework through its normal and transverse Riemann solvers).  Each pin
comes from the equations or from mathematics, not from the oracle's own formulas:

  - Roe property: the fluctuations of an edge sum to the flux difference f(Q_R) - f(Q_L) of the
    shallow water equations, the waves sum to the jump, and each wave lies along an eigenvector
    of the form (1, s, v) / (0, 0, 1);
  - a uniform state is preserved bit for bit, and the step is conservative (periodic domain);
  - reflection and transpose symmetry of a radial hump;
  - the 1D dam break converges to the exact Riemann solution (rarefaction plus shock);
  - small-amplitude waves about a lake at rest obey linear acoustics with rho = 1/H, K = g
    (p = g (h - H), u = hu, v = hv); the difference to the pinned acoustics oracle is O(eps);
  - second-order self-convergence on a smooth 2D flow with a mean velocity, which fails if any
    term of the transverse solve is wrong.
"""
import numpy as np
import pytest

MBC = 2


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def flux_x(q, g):
    h, hu, hv = q
    return np.array([hu, hu * hu / h + 0.5 * g * h * h, hu * hv / h])


def test_roe_property_and_eigenvectors(orc):
    rng = np.random.default_rng(11)
    for _ in range(200):
        g = rng.uniform(0.5, 10.0)
        L = np.array([rng.uniform(0.1, 3.0), rng.normal(), rng.normal()])
        R = np.array([rng.uniform(0.1, 3.0), rng.normal(), rng.normal()])
        w, s = orc.swe_roe_x(L, R, g)
        scale = np.abs(flux_x(L, g)).max() + np.abs(flux_x(R, g)).max()
        assert np.allclose(w.sum(0), R - L, rtol=0, atol=1e-14 * np.abs(R - L).max() * 8)
        assert np.allclose((s[:, None] * w).sum(0), flux_x(R, g) - flux_x(L, g), rtol=0, atol=1e-13 * scale)
        assert s[0] < s[1] < s[2]
        # W1, W3 along (1, s_p, v), W2 along (0, 0, 1), with the same v for both
        assert w[1, 0] == 0.0 and w[1, 1] == 0.0
        assert np.isclose(w[0, 1] / w[0, 0], s[0], rtol=1e-12) and np.isclose(w[2, 1] / w[2, 0], s[2], rtol=1e-12)
        assert np.isclose(w[0, 2] / w[0, 0], w[2, 2] / w[2, 0], rtol=1e-10, atol=1e-12)
        # celerity of the linearisation: (s3 - s1) / 2 = sqrt(g (h_L + h_R) / 2)
        assert np.isclose((s[2] - s[0]) / 2, np.sqrt(g * (L[0] + R[0]) / 2), rtol=1e-14)
    # no jump: no waves, speeds u -+ sqrt(g h) of the state
    w, s = orc.swe_roe_x((1.5, 0.6, -0.3), (1.5, 0.6, -0.3), 2.0)
    assert not w.any()
    assert np.allclose(s, [0.4 - np.sqrt(3.0), 0.4, 0.4 + np.sqrt(3.0)], rtol=1e-15)


def _periodic(q, orc):
    return orc.fill_bc(q, bc=(1, 1, 1, 1))


def _smooth_state(N, amp=0.2, u0=0.3, v0=-0.2):
    x = (np.arange(-MBC, N + MBC) + 0.5) / N
    X, Y = np.meshgrid(x, x)
    h = 1.0 + amp * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) + 0.5 * amp * np.cos(2 * np.pi * (X + Y))
    return np.ascontiguousarray(np.stack([h, h * u0, h * v0]))


def test_uniform_state_is_preserved_bit_for_bit(orc):
    q = np.empty((3, 12, 16))
    q[0], q[1], q[2] = 1.7, -0.4, 0.9
    for lim in ("none", "minmod", "superbee", "vanleer", "mc"):
        qn, sm = orc.swe_step(q, 0.1, 0.1, 0.01, 9.81, limiter=lim)
        assert np.array_equal(qn, q)
    assert sm == pytest.approx(abs(0.9 / 1.7) + np.sqrt(9.81 * 1.7), rel=1e-15)


@pytest.mark.parametrize("limiter", ["mc", "none", "vanleer"])
def test_step_is_conservative_on_a_periodic_domain(orc, limiter):
    N, g = 24, 9.81
    q = _periodic(_smooth_state(N, amp=0.3), orc)
    dx = 1.0 / N
    tot0 = q[:, MBC:-MBC, MBC:-MBC].sum(axis=(1, 2))
    for _ in range(5):
        dt = 0.9 * dx / orc.swe_cfl_max(q, g)
        q, _ = orc.swe_step(q, dx, dx, dt, g, limiter=limiter)
        q = _periodic(q, orc)
    tot = q[:, MBC:-MBC, MBC:-MBC].sum(axis=(1, 2))
    assert np.abs(tot - tot0).max() <= 1e-13 * N * N * np.abs(q).max()


def test_radial_hump_keeps_its_symmetries(orc):
    N, g = 40, 1.0
    x = (np.arange(-MBC, N + MBC) + 0.5) / N - 0.5
    X, Y = np.meshgrid(x, x)
    r = np.sqrt(X * X + Y * Y)
    h = 1.0 + np.where(r < 0.2, 0.5, 0.0)    # radial dam break
    q = np.ascontiguousarray(np.stack([h, 0 * h, 0 * h]))
    q = orc.fill_bc(q, bc=(0, 0, 0, 0))
    dx = 1.0 / N
    for _ in range(6):
        dt = 0.9 * dx / orc.swe_cfl_max(q, g)
        q, _ = orc.swe_step(q, dx, dx, dt, g)
        q = orc.fill_bc(q, bc=(0, 0, 0, 0))
    h, hu, hv = (c[MBC:-MBC, MBC:-MBC] for c in q)
    tol = 1e-13 * np.abs(q).max()
    assert np.abs(h - h[:, ::-1]).max() <= tol and np.abs(h - h[::-1, :]).max() <= tol
    assert np.abs(h - h.T).max() <= tol
    assert np.abs(hu + hu[:, ::-1]).max() <= tol and np.abs(hu - hu[::-1, :]).max() <= tol
    assert np.abs(hu - hv.T).max() <= tol
    assert np.abs(hu).max() > 1e-3


def _dam_break_exact(x, t, hl, hr, g):
    """exact solution (left rarefaction, right shock) of the 1D dam break, u = 0 on both sides"""
    cl = np.sqrt(g * hl)
    lo, hi = hr, hl
    for _ in range(200):   # bisection on h*: rarefaction speed change equals shock speed change
        hs = 0.5 * (lo + hi)
        f = 2 * (cl - np.sqrt(g * hs)) - (hs - hr) * np.sqrt(g * (hs + hr) / (2 * hs * hr))
        lo, hi = (hs, hi) if f > 0 else (lo, hs)
    us = 2 * (cl - np.sqrt(g * hs))
    S = hs * us / (hs - hr)
    xi = x / t
    h = np.where(xi < -cl, hl, np.where(xi < us - np.sqrt(g * hs), (2 * cl - xi) ** 2 / (9 * g),
                                          np.where(xi < S, hs, hr)))
    u = np.where(xi < -cl, 0.0, np.where(xi < us - np.sqrt(g * hs), 2 * (xi + cl) / 3,
                                           np.where(xi < S, us, 0.0)))
    return h, h * u


@pytest.mark.parametrize("limiter,order", [("mc", 2), ("none", 1)])
def test_dam_break_converges_to_the_exact_solution(orc, limiter, order):
    g, hl, hr, T = 1.0, 2.0, 1.0, 0.25
    errs = []
    for N in (100, 200, 400):
        x = (np.arange(-MBC, N + MBC) + 0.5) / N - 0.5
        ny = 2
        h = np.tile(np.where(x < 0, hl, hr), (ny + 2 * MBC, 1))
        q = np.ascontiguousarray(np.stack([h, 0 * h, 0 * h]))
        q = orc.fill_bc(q, bc=(0, 0, 1, 1))
        dx, t = 1.0 / N, 0.0
        while t < T - 1e-14:
            dt = min(0.9 * dx / orc.swe_cfl_max(q, g), T - t)
            q, _ = orc.swe_step(q, dx, dx, dt, g, order=order, limiter=limiter)
            q = orc.fill_bc(q, bc=(0, 0, 1, 1))
            t += dt
        assert not q[2].any()                                   # no transverse momentum
        assert (q[:, MBC:-MBC] == q[:, MBC:MBC + 1]).all()      # y-uniform, bit for bit
        he, hue = _dam_break_exact(x[MBC:-MBC], T, hl, hr, g)
        errs.append(dx * (np.abs(q[0, MBC, MBC:-MBC] - he).sum() + np.abs(q[1, MBC, MBC:-MBC] - hue).sum()))
    assert errs[0] / errs[1] > 1.4 and errs[1] / errs[2] > 1.4, errs
    assert errs[2] < (0.006 if order == 2 else 0.02), errs


@pytest.mark.parametrize("limiter", ["mc", "none"])
def test_small_amplitude_limit_is_linear_acoustics(orc, limiter):
    # h = H + eps eta, hu = eps m, hv = eps n  ~  acoustics with rho = 1/H, K = g:
    # p = g eps eta, u = eps m, v = eps n; the difference of the scaled steps is O(eps)
    N, g, H = 32, 2.0, 1.5
    x = (np.arange(-MBC, N + MBC) + 0.5) / N
    X, Y = np.meshgrid(x, x)
    eta = np.exp(-60 * ((X - 0.45) ** 2 + (Y - 0.55) ** 2))
    m = 0.7 * np.exp(-50 * ((X - 0.5) ** 2 + (Y - 0.4) ** 2))
    n = -0.4 * np.sin(2 * np.pi * X) * np.exp(-40 * (Y - 0.5) ** 2)
    dx = 1.0 / N
    dt = 0.8 * dx / np.sqrt(g * H)
    rho, K = np.full_like(X, 1.0 / H), np.full_like(X, g)
    qa = np.ascontiguousarray(np.stack([g * eta, m, n]))
    ref, _ = orc.step(qa, rho, K, dx, dx, dt, limiter=limiter)
    ref = ref[:, MBC:-MBC, MBC:-MBC]
    errs = []
    for eps in (1e-3, 1e-4):
        q = np.ascontiguousarray(np.stack([H + eps * eta, eps * m, eps * n]))
        qn, _ = orc.swe_step(q, dx, dx, dt, g, limiter=limiter)
        lin = np.stack([g * (qn[0] - H), qn[1], qn[2]])[:, MBC:-MBC, MBC:-MBC] / eps
        errs.append(np.abs(lin - ref).max() / np.abs(ref).max())
    assert errs[0] < 1e-3 and 9 < errs[0] / errs[1] < 11, errs


def test_second_order_self_convergence_on_a_smooth_flow(orc):
    # unlimited (Lax-Wendroff with transverse terms) on a smooth flow with a mean velocity:
    # differences of successive grids shrink by about 4
    g, T = 1.0, 0.15
    sol = {}
    for N in (32, 64, 128):
        q = _periodic(_smooth_state(N, amp=0.1), orc)
        dx = 1.0 / N
        nsteps = int(np.ceil(T / (0.8 * dx / 1.5)))
        dt = T / nsteps
        for _ in range(nsteps):
            q, _ = orc.swe_step(q, dx, dx, dt, g, limiter="none")
            q = _periodic(q, orc)
        sol[N] = q[:, MBC:-MBC, MBC:-MBC]

    def coarsen(a):
        return 0.25 * (a[:, ::2, ::2] + a[:, 1::2, ::2] + a[:, ::2, 1::2] + a[:, 1::2, 1::2])

    d1 = np.abs(sol[32] - coarsen(sol[64])).mean()
    d2 = np.abs(sol[64] - coarsen(sol[128])).mean()
    assert d1 / d2 > 2 ** 1.8, (d1, d2)


def test_cfl_speed_and_dry_cells(orc):
    q = np.empty((3, 8, 8))
    q[0], q[1], q[2] = 2.0, 0.0, 0.0
    q[1, 4, 3] = -3.0        # u = -1.5 in one ring cell
    assert orc.swe_cfl_max(q, 2.0) == 1.5 + 2.0
    q[0, 3, 3] = 0.0
    with pytest.raises(ValueError):
        orc.swe_step(q, 0.1, 0.1, 0.01, 2.0)
