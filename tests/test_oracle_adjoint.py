"""Pins of the oracle's reverse mode (pin P11): brute-force Jacobian of the linear scheme,
central differences of the limited scheme, dot-product identities of the AMR transfers."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

M = 2


def interior(a):
    return a[..., M:-M, M:-M]


def _medium(nx, ny, seed=3):
    run, r0, k0 = inputs.config3(32)
    return (np.ascontiguousarray(np.pad(r0[:ny, :nx], M, mode="edge")),
            np.ascontiguousarray(np.pad(k0[:ny, :nx], M, mode="edge")))


@pytest.mark.parametrize("transverse", [0, 2])
def test_adjoint_equals_bruteforce_jacobian_linear_scheme(orc, transverse):
    # limiter off: the step is linear in q; its Jacobian built column by column from unit
    # vectors equals the transpose built row by row by the reverse mode
    nx, ny = 6, 6
    rho, K = _medium(nx, ny)
    H, W = ny + 2 * M, nx + 2 * M
    nin, nout = 3 * H * W, 3 * nx * ny
    dx, dy, dt = 0.1, 0.13, 0.012
    J = np.zeros((nout, nin))
    for k in range(nin):
        e = np.zeros(nin)
        e[k] = 1.0
        qn, _ = orc.step(e.reshape(3, H, W), rho, K, dx, dy, dt, limiter=0, transverse=transverse)
        J[:, k] = interior(qn).ravel()
    JT = np.zeros((nin, nout))
    for i in range(nout):
        lam = np.zeros((3, H, W))
        unit = np.zeros(nout)
        unit[i] = 1.0
        lam[:, M:-M, M:-M] = unit.reshape(3, ny, nx)
        lq, _, _ = orc.step_adjoint(np.zeros((3, H, W)), rho, K, lam, dx, dy, dt, limiter=0,
                                    transverse=transverse)
        JT[:, i] = lq.ravel()
    assert np.abs(J - JT.T).max() <= 1e-14 * np.abs(J).max()


@pytest.mark.parametrize("limiter", [4, 3, 1])
def test_adjoint_matches_central_differences_limited_scheme(orc, limiter):
    nx, ny = 10, 8
    rho, K = _medium(nx, ny)
    H, W = ny + 2 * M, nx + 2 * M
    q = inputs.uniform(41, 3 * H * W).reshape(3, H, W) - 0.5
    lam = inputs.uniform(42, 3 * H * W).reshape(3, H, W) - 0.5
    dq = inputs.uniform(43, 3 * H * W).reshape(3, H, W) - 0.5
    dr = inputs.uniform(44, H * W).reshape(H, W) - 0.5
    dk = inputs.uniform(45, H * W).reshape(H, W) - 0.5
    dx, dy, dt = 0.1, 0.1, 0.015
    lq, gr, gk = orc.step_adjoint(q, rho, K, lam, dx, dy, dt, limiter=limiter)
    h = 1e-6

    def J(qq, rr, kk):
        qn, _ = orc.step(qq, rr, kk, dx, dy, dt, limiter=limiter)
        return (interior(qn) * interior(lam)).sum()

    fd_q = (J(q + h * dq, rho, K) - J(q - h * dq, rho, K)) / (2 * h)
    fd_r = (J(q, rho + h * dr, K) - J(q, rho - h * dr, K)) / (2 * h)
    fd_k = (J(q, rho, K + h * dk) - J(q, rho, K - h * dk)) / (2 * h)
    assert (lq * dq).sum() == pytest.approx(fd_q, rel=1e-6)
    assert (gr * dr).sum() == pytest.approx(fd_r, rel=1e-6)
    assert (gk * dk).sum() == pytest.approx(fd_k, rel=1e-6)


def test_multistep_adjoint_with_boundary_fill_matches_fd(orc):
    # J = sum p^2 over a receiver after n steps of (fill ghosts, step): reverse sweep
    # through step_adjoint and fill_bc_adjoint against central differences
    nx = ny = 16
    rho, K = _medium(nx, ny)
    H, W = ny + 2 * M, nx + 2 * M
    x = (np.arange(-M, nx + M) + 0.5) / nx * 2 - 1
    X, Y = np.meshgrid(x, x)
    q0 = np.zeros((3, H, W))
    q0[0] = np.exp(-20 * (X ** 2 + Y ** 2))
    dx = dy = 2.0 / nx
    dt = 0.9 * dx / np.sqrt(K / rho).max()
    nsteps = 6
    rec = (slice(M + 9, M + 13), slice(M + 3, M + 8))

    def forward(q, r, k):
        qs = []
        for _ in range(nsteps):
            q = q.copy()
            orc.fill_bc(q)
            qs.append(q)
            q, _ = orc.step(q, r, k, dx, dy, dt)
        return q, qs

    def Jf(q, r, k):
        qf, _ = forward(q, r, k)
        return (qf[0][rec] ** 2).sum()

    qf, qs = forward(q0, rho, K)
    lam = np.zeros_like(q0)
    lam[0][rec] = 2 * qf[0][rec]
    g_r = np.zeros_like(rho)
    g_k = np.zeros_like(K)
    for n in reversed(range(nsteps)):
        lq, gr, gk = orc.step_adjoint(qs[n], rho, K, lam, dx, dy, dt)
        g_r += gr
        g_k += gk
        orc.fill_bc_adjoint(lq)
        lam = lq
    # smooth directions (R19: the q direction lives where the pulse is)
    dq = np.zeros_like(q0)
    dq[0] = np.exp(-20 * (X ** 2 + Y ** 2)) * np.cos(3 * X)
    dq[1] = 0.3 * np.exp(-20 * (X ** 2 + Y ** 2))
    dr = np.cos(2 * X + Y)
    dk = np.sin(X - 2 * Y)
    h = 1e-6
    fd_q = (Jf(q0 + h * dq, rho, K) - Jf(q0 - h * dq, rho, K)) / (2 * h)
    fd_r = (Jf(q0, rho + h * dr, K) - Jf(q0, rho - h * dr, K)) / (2 * h)
    fd_k = (Jf(q0, rho, K + h * dk) - Jf(q0, rho, K - h * dk)) / (2 * h)
    assert (lam * dq).sum() == pytest.approx(fd_q, rel=1e-6)
    assert (g_r * dr).sum() == pytest.approx(fd_r, rel=1e-6)
    assert (g_k * dk).sum() == pytest.approx(fd_k, rel=1e-6)


def _amr_two_level():
    run = inputs.Run(-1, -1, 1, 1)
    L0 = inputs.Level(12, 12, 2 / 12, 2 / 12, [(0, 0, 12, 12)])
    L1 = inputs.Level(48, 48, 2 / 48, 2 / 48, [(12, 12, 12, 8), (24, 12, 8, 16), (12, 20, 12, 12)], ratio=4)
    run.levels = [L0, L1]
    return run


def _bx(lev):
    return [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(lev.boxes, lev.qoff)]


def test_fill_ghost_adjoint_dot_product(orc):
    # <G(x), y> = <x, G^T y> where G is the level ghost fill (copies + space-time
    # interpolation, piecewise linear through minmod: the identity holds at a fixed point)
    run = _amr_two_level()
    L0, L1 = run.levels
    cold = inputs.uniform(51, L0.qsize)
    cnew = inputs.uniform(52, L0.qsize)
    f = inputs.uniform(53, L1.qsize)

    def ghost_only(pool):
        out = np.zeros_like(pool)
        for n, b in enumerate(L1.boxes):
            src = inputs.box_view(pool, L1.qoff[n], int(b[2]), int(b[3]), 3)
            dst = inputs.box_view(out, L1.qoff[n], int(b[2]), int(b[3]), 3)
            dst[...] = src
            dst[:, M:-M, M:-M] = 0
        return out

    tau = 0.25
    filled = f.copy()
    orc.level_fill_ghost(_bx(L1), filled, 3, 48, 48, (0, 0, 0, 0), _bx(L0), cold, cnew, tau, 4)
    y = ghost_only(inputs.uniform(54, L1.qsize))
    lhs = (ghost_only(filled) * y).sum()
    gf = y.copy()
    gco = np.zeros(L0.qsize)
    gcn = np.zeros(L0.qsize)
    orc.level_fill_ghost_adjoint(_bx(L1), gf, 3, 48, 48, (0, 0, 0, 0), _bx(L0), gco, gcn, cold, cnew,
                                 tau, 4)
    # the forward ghost values are linear in (f interiors, cold, cnew) along the branch taken
    # by minmod; evaluate the same linear map on the inputs themselves
    rhs = (gf * f).sum() + (gco * cold).sum() + (gcn * cnew).sum()
    assert lhs == pytest.approx(rhs, rel=1e-13)
    assert np.all(ghost_only(gf) == 0)


def test_average_down_adjoint_dot_product(orc):
    run = _amr_two_level()
    L0, L1 = run.levels
    f = inputs.uniform(61, L1.qsize)
    c = np.zeros(L0.qsize)
    orc.average_down(_bx(L1), f, _bx(L0), c, 3, 4)
    y = inputs.uniform(62, L0.qsize)
    # only the covered coarse cells are written: mask them
    covered = np.zeros(L0.qsize, dtype=bool)
    probe = np.zeros(L0.qsize)
    orc.average_down(_bx(L1), np.ones(L1.qsize), _bx(L0), probe, 3, 4)
    covered = probe != 0
    y = np.where(covered, y, 0.0)
    gc = y.copy()
    gf = np.zeros(L1.qsize)
    orc.average_down_adjoint(_bx(L1), gf, _bx(L0), gc, 3, 4)
    assert (c * y).sum() == pytest.approx((gf * f).sum(), rel=1e-13)
    assert np.all(gc == 0)
