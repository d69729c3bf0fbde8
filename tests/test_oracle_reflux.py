"""Pins of the oracle's conservation fix (Sec. 2.3, "refluxing"): with periodic boundaries the
composite integral of q (every cell not covered by a finer level, times its area) is a conserved
quantity of the uniform-medium scheme, which the fix must keep to rounding while the plain AMR
step does not; the interface records follow the box geometry; the fix is a no-op without an
interface and on a uniform state."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _composite(O):
    from oracle.amr import _view
    tot = np.zeros(3)
    for L, lev in enumerate(O.levels):
        for n, b in enumerate(lev.boxes):
            nx, ny = int(b[2]), int(b[3])
            v = _view(O.q[L], lev.qoff[n], nx, ny, 3)[:, 2:2 + ny, 2:2 + nx]
            mask = np.ones((ny, nx), bool)
            if L + 1 < len(O.levels):
                r = O.levels[L + 1].ratio
                for fb in O.levels[L + 1].boxes:
                    i0, j0 = int(fb[0]) // r - int(b[0]), int(fb[1]) // r - int(b[1])
                    i1, j1 = i0 + int(fb[2]) // r, j0 + int(fb[3]) // r
                    mask[max(j0, 0):max(min(j1, ny), 0), max(i0, 0):max(min(i1, nx), 0)] = False
            tot += (v * mask).sum(axis=(1, 2)) * lev.dx * lev.dy
    return tot


def _flowing_pulse(run):
    """off-centre pulse with a mean flow (u, v) = (0.3, -0.2), so all three integrals move"""
    q = []
    for lev in run.levels:
        a = inputs.init_q(run, lev, fn=lambda x, y: inputs.radial_pulse(x - 0.1, y + 0.05)).copy()
        for n, b in enumerate(lev.boxes):
            v = inputs.box_view(a, lev.qoff[n], int(b[2]), int(b[3]), 3)
            v[1] += 0.3
            v[2] -= 0.2
        q.append(a)
    return q


def _hier(run, q, reflux):
    from oracle.amr import OracleHierarchy
    return OracleHierarchy(run, q, [inputs.const_pool(l, 1.0) for l in run.levels],
                           [inputs.const_pool(l, 4.0) for l in run.levels], reflux=reflux)


@pytest.mark.parametrize("nlev,ncoarse,limiter", [(2, 8, 4), (3, 2, 4), (2, 6, 3), (2, 6, 1), (2, 6, 2)])
def test_reflux_conserves_the_composite_integral_on_a_periodic_domain(orc, nlev, ncoarse, limiter):
    # MC, and van Leer (the benchmark's limiter), minmod and superbee
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1), limiter=limiter)
    annuli, seeds = [(0.2, 0.45), (0.25, 0.35)][:nlev - 1], [2002, 2003][:nlev - 1]
    run.levels = inputs.amr_levels(run, 32, 4, annuli, seeds)
    q0 = _flowing_pulse(run)
    drift = {}
    for reflux in (True, False):
        O = _hier(run, q0, reflux)
        m0 = _composite(O)
        for _ in range(ncoarse):
            O.coarse_step()
        drift[reflux] = np.abs(_composite(O) - m0)
    scale = 4.0 * 1.5   # domain area x max |q|
    assert (drift[True] <= 1e-13 * scale).all(), drift[True]
    assert drift[False].max() >= 1e-6 * scale, drift[False]


@pytest.mark.parametrize("nlev,ncoarse", [(2, 6), (3, 2)])
def test_shallow_water_reflux_conserves_the_composite_integral(orc, nlev, ncoarse):
    # the same fix with the shallow-water flux f: the Roe solver is conservative
    # (A-dQ + A+dQ = f(Q_R) - f(Q_L)), so the flux form holds with f(Q_F) - f(Q_C) for A dQ
    from oracle.amr import OracleHierarchy
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1), cfl=0.7)   # speeds grow as the ring focuses
    annuli, seeds = [(0.2, 0.45), (0.25, 0.35)][:nlev - 1], [2002, 2003][:nlev - 1]
    run.levels = inputs.amr_levels(run, 32, 4, annuli, seeds)
    q0 = [inputs.init_swe(run, lev, depth=lambda x, y: inputs.radial_pulse(x - 0.1, y + 0.05), u0=0.3, v0=-0.2)
          for lev in run.levels]
    drift = {}
    for reflux in (True, False):
        O = OracleHierarchy(run, q0, reflux=reflux, system="shallow_water", grav=1.0)
        m0 = _composite(O)
        for _ in range(ncoarse):
            O.coarse_step()
        drift[reflux] = np.abs(_composite(O) - m0)
    scale = 4.0 * 2.0   # domain area x max |q|
    assert (drift[True] <= 1e-13 * scale).all(), drift[True]
    assert drift[False].max() >= 1e-6 * scale, drift[False]


def test_interface_records_follow_the_box_geometry(orc):
    from oracle.amr import interface
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = [inputs.Level(16, 16, 0.125, 0.125, [(0, 0, 16, 16)]),
                  inputs.Level(64, 64, 0.03125, 0.03125, [(16, 16, 16, 8), (32, 16, 8, 8)], ratio=4)]
    recs = interface(run.levels, 1, run.bc)
    # union of the two boxes: coarse cells [4, 10) x [4, 6); the shared edge at coarse x = 8 is fine-fine
    got = sorted((ci, cj, d, side) for (n_c, ci, cj, d, side, n_f, cells) in recs)
    want = sorted([(3, 4, 0, 1), (3, 5, 0, 1), (10, 4, 0, -1), (10, 5, 0, -1)] +
                  [(i, 3, 1, 1) for i in range(4, 10)] + [(i, 6, 1, -1) for i in range(4, 10)])
    assert got == want
    for (n_c, ci, cj, d, side, n_f, cells) in recs:
        assert len(cells) == 4
        fb = run.levels[1].boxes[n_f]
        for fi, fj in cells:       # fine cells inside their box, on the side facing the coarse cell
            assert 0 <= fi < fb[2] and 0 <= fj < fb[3]
            if d == 0:
                assert fi == (0 if side > 0 else fb[2] - 1)
            else:
                assert fj == (0 if side > 0 else fb[3] - 1)


def test_reflux_is_a_no_op_without_interface_and_on_a_uniform_state(orc):
    # a fine level over the whole domain has no coarse-fine interface
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1))
    run.levels = [inputs.Level(8, 8, 0.25, 0.25, [(0, 0, 8, 8)]),
                  inputs.Level(32, 32, 0.0625, 0.0625, [(0, 0, 32, 32)], ratio=4)]
    q0 = _flowing_pulse(run)
    A, B = _hier(run, q0, True), _hier(run, q0, False)
    for _ in range(2):
        A.coarse_step()
        B.coarse_step()
    assert all(np.array_equal(a, b) for a, b in zip(A.q, B.q))
    # a uniform state stays uniform bit for bit with the fix applied at a real interface
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=(1, 1, 1, 1))
    run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45)], [2002])
    q = [np.where(np.arange(inputs.init_q(run, l).size) >= 0, 0.0, 0.0) for l in run.levels]
    for L, lev in enumerate(run.levels):
        for n, b in enumerate(lev.boxes):
            v = inputs.box_view(q[L], lev.qoff[n], int(b[2]), int(b[3]), 3)
            v[0], v[1], v[2] = 1.25, 0.5, -0.75
    O = _hier(run, q, True)
    O.coarse_step()
    for L, lev in enumerate(run.levels):
        for n, b in enumerate(lev.boxes):
            v = inputs.box_view(O.q[L], lev.qoff[n], int(b[2]), int(b[3]), 3)[:, 2:-2, 2:-2]
            assert (v[0] == 1.25).all() and (v[1] == 0.5).all() and (v[2] == -0.75).all()
