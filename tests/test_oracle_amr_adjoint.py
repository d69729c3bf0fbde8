"""Pin of the oracle's AMR reverse mode: central differences of a receiver functional over two
coarse steps of a two-level hierarchy (interpolated ghosts, averaging, subcycling), in smooth
directions of q0 (inside the pulse ring, even in x and y), rho and K, with the time steps frozen.

The q0 directions are even in x and y: the pulse is, and on the symmetric grid the waves across
the lines x = 0 and y = 0 vanish exactly at t = 0; an odd perturbation would excite them where
the limited wave is odd-homogeneous in its two strengths, and central differences would
average two one-sided slopes there."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

M = 2


def _hier():
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = inputs.amr_levels(run, 16, 4, [(0.2, 0.45)], [77])
    n = 16
    rho2 = inputs.smooth_field(11, n, n, 0.5, 2.0, sigma=2.0)
    K2 = inputs.smooth_field(12, n, n, 1.0, 8.0, sigma=2.0)
    q = [inputs.init_q(run, lev) for lev in run.levels]
    rho = [inputs.coef_pool(lev, rho2, 4 ** L) for L, lev in enumerate(run.levels)]
    K = [inputs.coef_pool(lev, K2, 4 ** L) for L, lev in enumerate(run.levels)]
    return run, q, rho, K


def _J(run, q, rho, K, nsteps, dts):
    from oracle.amr import OracleHierarchy
    O = OracleHierarchy(run, q, rho, K)
    for n in range(nsteps):
        O.coarse_step(dt=dts[n])
    v = inputs.box_view(O.q[0], 0, 16, 16, 3)
    return float((v[0, M + 8:M + 12, M + 9:M + 13] ** 2).sum())


def test_oracle_amr_reverse_mode_matches_central_differences(orc):
    from oracle.amr import OracleHierarchy
    run, q, rho, K = _hier()
    nsteps = 2

    def final_adjoint(qs):
        lam = [np.zeros_like(a) for a in qs]
        v = inputs.box_view(qs[0], 0, 16, 16, 3)
        lv = inputs.box_view(lam[0], 0, 16, 16, 3)
        lv[0, M + 8:M + 12, M + 9:M + 13] = 2 * v[0, M + 8:M + 12, M + 9:M + 13]
        return lam

    O = OracleHierarchy(run, q, rho, K)
    gq, gr, gk = O.gradient(nsteps, final_adjoint)
    dts = O.dt_history
    # smooth directions: q0 windowed to the ring on every level, rho / K global
    dq, dr, dk = [], [], []
    for L, lev in enumerate(run.levels):
        d = np.zeros(lev.qsize)
        e = np.zeros(lev.csize)
        f = np.zeros(lev.csize)
        for nb, b in enumerate(lev.boxes):
            x, y = inputs.cell_centres(run, lev, b)
            r = np.sqrt(x * x + y * y)
            win = np.where(np.abs(r - 0.3) < 0.1, 0.5 * (1 + np.cos(np.pi * (r - 0.3) / 0.1)), 0.0)
            inputs.box_view(d, lev.qoff[nb], int(b[2]), int(b[3]), 3)[0] = win * np.cos(2 * x) * np.cos(3 * y)
            inputs.box_view(e, lev.coff[nb], int(b[2]), int(b[3]), 1)[0] = np.sin(x - 2 * y)
            inputs.box_view(f, lev.coff[nb], int(b[2]), int(b[3]), 1)[0] = np.cos(3 * x * y)
        dq.append(d)
        dr.append(e)
        dk.append(f)
    h = 1e-6
    ip = lambda a, b: sum(float((x * y).sum()) for x, y in zip(a, b))
    add = lambda a, b, s: [x + s * y for x, y in zip(a, b)]
    fd_q = (_J(run, add(q, dq, h), rho, K, nsteps, dts) - _J(run, add(q, dq, -h), rho, K, nsteps, dts)) / (2 * h)
    fd_r = (_J(run, q, add(rho, dr, h), K, nsteps, dts) - _J(run, q, add(rho, dr, -h), K, nsteps, dts)) / (2 * h)
    fd_k = (_J(run, q, rho, add(K, dk, h), nsteps, dts) - _J(run, q, rho, add(K, dk, -h), nsteps, dts)) / (2 * h)
    assert ip(gq, dq) == pytest.approx(fd_q, rel=1e-6)
    assert ip(gr, dr) == pytest.approx(fd_r, rel=1e-6)
    assert ip(gk, dk) == pytest.approx(fd_k, rel=1e-6)
