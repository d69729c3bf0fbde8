"""Pins of the oracle's regridding (Sec. 2.2, Sec. 4.3): flag criterion, buffer, nesting mask,
Berger-Rigoutsos clustering (coverage, disjointness, efficiency >= cutoff, size cap, exact
boxes on simple patterns) and the data transfer (identity on unchanged boxes, exact on uniform
states, conservative where new fine cells are interpolated)."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs


@pytest.fixture(scope="module")
def rg():
    import oracle
    from oracle import regrid
    oracle.build()
    return regrid


def test_flags_mark_the_cells_next_to_a_jump(rg):
    q = np.zeros((3, 12, 14))
    q[0, :, :9] = 1.0                     # jump in p between padded columns 8 and 9
    f = rg.flag_box(q, 0.5)               # interior columns 0..9 are padded 2..11
    want = np.zeros((8, 10), bool)
    want[:, 6] = want[:, 7] = True
    assert np.array_equal(f, want)
    assert not rg.flag_box(q, 1.0).any()  # the criterion is strict: |diff| > tol


def test_dilate_grows_a_square_clipped_to_the_domain(rg):
    f = np.zeros((10, 10), bool)
    f[5, 5] = f[0, 9] = True
    g = rg.dilate(f, 2)
    want = np.zeros((10, 10), bool)
    want[3:8, 3:8] = True
    want[0:3, 7:10] = True
    assert np.array_equal(g, want)


def test_nest_mask_erodes_inside_the_domain_only(rg):
    lev = inputs.Level(16, 16, 0.125, 0.125, [(4, 4, 8, 8)])
    m = rg.nest_mask(lev, 2)
    want = np.zeros((16, 16), bool)
    want[6:10, 6:10] = True
    assert np.array_equal(m, want)
    full = inputs.Level(16, 16, 0.125, 0.125, [(0, 0, 16, 16)])
    assert rg.nest_mask(full, 2).all()


def test_cluster_exact_on_rectangles(rg):
    f = np.zeros((20, 30), bool)
    f[3:8, 4:12] = True
    assert rg.cluster(f, 0.7, 100) == [(4, 3, 8, 5)]
    f[12:18, 20:27] = True
    assert sorted(rg.cluster(f, 0.7, 100)) == [(4, 3, 8, 5), (20, 12, 7, 6)]
    g = np.zeros((20, 20), bool)
    g[2:10, 2:4] = True
    g[8:10, 2:12] = True                  # an L: two full rectangles
    assert sorted(rg.cluster(g, 0.8, 100)) == [(2, 2, 2, 6), (2, 8, 10, 2)]
    assert rg.cluster(np.zeros((5, 5), bool), 0.7, 10) == []


def test_cluster_splits_to_the_size_cap(rg):
    f = np.ones((40, 40), bool)           # efficiency 1: only the cap splits (halving 40 -> 20 -> 10)
    boxes = rg.cluster(f, 0.7, 16)
    assert sorted(boxes) == sorted((i, j, 10, 10) for i in range(0, 40, 10) for j in range(0, 40, 10))


def test_cluster_keeps_boxes_inside_the_allowed_region(rg):
    allowed = np.zeros((30, 30), bool)
    allowed[2:28, 2:10] = True
    allowed[20:28, 2:28] = True           # an L-shaped region (nesting mask)
    flags = allowed.copy()
    flags[5:7, 5:7] = False               # efficiency below 1 everywhere near the corner
    for cutoff in (0.5, 0.7, 0.9):
        boxes = rg.cluster(flags, cutoff, 100, allowed)
        cov = np.zeros_like(flags)
        for (i0, j0, nx, ny) in boxes:
            assert allowed[j0:j0 + ny, i0:i0 + nx].all()
            cov[j0:j0 + ny, i0:i0 + nx] = True
        assert (cov | ~flags).all()
    # without the region the same flags give a box reaching outside it
    assert any(not allowed[j0:j0 + ny, i0:i0 + nx].all() for (i0, j0, nx, ny) in rg.cluster(flags, 0.5, 100))


@pytest.mark.parametrize("seed,density,cutoff,cap", [(1, 0.05, 0.5, 16), (2, 0.2, 0.7, 8), (3, 0.6, 0.9, 64)])
def test_cluster_properties_on_random_flags(rg, seed, density, cutoff, cap):
    h = np.random.default_rng(seed).random((48, 40)) < density
    boxes = rg.cluster(h, cutoff, cap)
    cov = np.zeros_like(h)
    for (i0, j0, nx, ny) in boxes:
        assert nx <= cap and ny <= cap
        assert not cov[j0:j0 + ny, i0:i0 + nx].any()          # disjoint
        cov[j0:j0 + ny, i0:i0 + nx] = True
        sub = h[j0:j0 + ny, i0:i0 + nx]
        assert sub[0].any() and sub[-1].any() and sub[:, 0].any() and sub[:, -1].any()   # tight
        assert sub.mean() >= cutoff
    assert (cov | ~h).all()                                       # every flag covered


def _two_level_run(bc=(1, 1, 1, 1)):
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=bc)
    run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45)], [2002])
    return run


def _hier(run, reflux=False):
    from oracle.amr import OracleHierarchy
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    return OracleHierarchy(run, q0, [inputs.const_pool(l, 1.0) for l in run.levels],
                           [inputs.const_pool(l, 4.0) for l in run.levels], reflux=reflux)


def test_transfer_is_the_identity_on_unchanged_boxes_and_exact_on_a_uniform_state(rg):
    run = _two_level_run()
    O = _hier(run)
    O.coarse_step()
    c, f = O.levels
    same = rg.transfer(f, O.q[1], f, c, O.q[0], run.bc)
    for n, b in enumerate(f.boxes):
        a = inputs.box_view(same, f.qoff[n], int(b[2]), int(b[3]), 3)[:, 2:-2, 2:-2]
        w = inputs.box_view(O.q[1], f.qoff[n], int(b[2]), int(b[3]), 3)[:, 2:-2, 2:-2]
        assert np.array_equal(a, w)
    u = np.zeros_like(O.q[0])
    for n, b in enumerate(c.boxes):
        inputs.box_view(u, c.qoff[n], int(b[2]), int(b[3]), 3)[...] = np.array([1.5, -0.25, 0.75])[:, None, None]
    moved = type(f)(f.NX, f.NY, f.dx, f.dy, [(40, 40, 16, 24)], f.ratio)
    t = rg.transfer(None, None, moved, c, u, run.bc)
    v = inputs.box_view(t, 0, 16, 24, 3)[:, 2:-2, 2:-2]
    assert (v[0] == 1.5).all() and (v[1] == -0.25).all() and (v[2] == 0.75).all()


def test_transfer_is_conservative_where_it_interpolates(rg):
    run = _two_level_run()
    O = _hier(run)
    O.coarse_step()
    c, f = O.levels
    r = f.ratio
    box = (40, 44, 20, 12)                # fine cells of coarse cells [10, 15) x [11, 14)
    new = type(f)(f.NX, f.NY, f.dx, f.dy, [box], r)
    t = rg.transfer(None, None, new, c, O.q[0], run.bc)
    fine_sum = inputs.box_view(t, 0, 20, 12, 3)[:, 2:-2, 2:-2].sum(axis=(1, 2)) * f.dx * f.dy
    cv = inputs.box_view(O.q[0], c.qoff[0], int(c.boxes[0][2]), int(c.boxes[0][3]), 3)
    coarse_sum = cv[:, 2 + 11:2 + 14, 2 + 10:2 + 15].sum(axis=(1, 2)) * c.dx * c.dy
    assert np.abs(fine_sum - coarse_sum).max() <= 1e-14 * np.abs(coarse_sum).max()


def test_regrid_follows_the_flags_and_keeps_nesting(rg):
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = inputs.amr_levels(run, 32, 4, [(0.2, 0.45), (0.25, 0.35)], [2002, 2003])
    O = _hier(run)
    for _ in range(3):
        O.coarse_step()
    O.regrid(tol=0.02, buffer=2, cutoff=0.7, max_size=64, nest=2)
    c0, l1, l2 = O.levels
    # every flagged (and grown) level-0 cell is refined
    O.fill(0, O.q[0])
    want = rg.dilate(rg.flag_level(c0, O.q[0], 0.02), 2)
    cov = np.zeros((c0.NY, c0.NX), bool)
    for b in l1.boxes:
        cov[int(b[1]) // 4:(int(b[1]) + int(b[3])) // 4, int(b[0]) // 4:(int(b[0]) + int(b[2])) // 4] = True
    assert (cov | ~want).all()
    # level 2 lies two level-1 cells inside level 1 (or against the domain)
    m = rg.nest_mask(l1, 2)
    for b in l2.boxes:
        I0, J0 = int(b[0]) // 4, int(b[1]) // 4
        assert m[J0:J0 + int(b[3]) // 4, I0:I0 + int(b[2]) // 4].all()
    # the state keeps stepping
    O.coarse_step()
    assert all(np.isfinite(q).all() for q in O.q)


def test_reaches_wider_than_the_level():
    # a buffer or nesting square wider than the level, clipped to the domain, is the whole level:
    # one flag grows over everything; one uncovered cell disallows every cell, full coverage none
    from oracle import regrid as org
    flags = np.zeros((7, 9), bool)
    flags[3, 4] = True
    assert org.dilate(flags, 12).all()
    full = inputs.Level(9, 7, 1.0, 1.0, np.array([(0, 0, 9, 7)], dtype=np.int32))
    assert org.nest_mask(full, 15).all()
    holed = inputs.Level(9, 7, 1.0, 1.0, np.array([(0, 0, 9, 3), (0, 3, 4, 4), (5, 3, 4, 4), (4, 4, 1, 3)],
                                                  dtype=np.int32))   # cell (4, 3) uncovered
    assert not org.nest_mask(holed, 15).any()
    assert org.nest_mask(holed, 0).sum() == 9 * 7 - 1


def test_regrid_of_an_initially_empty_level_takes_the_uniform_medium_of_level_0():
    # a level that starts without boxes has no coefficient value of its own: the regrid gives
    # the new boxes the uniform medium of the base level
    from oracle.amr import OracleHierarchy
    run = inputs.Run(*inputs.PULSE_DOMAIN)
    run.levels = [inputs.Level(32, 32, 2 / 32, 2 / 32, [(0, 0, 32, 32)]),
                  inputs.Level(64, 64, 2 / 64, 2 / 64, np.zeros((0, 4), dtype=np.int32), 2)]
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    O = OracleHierarchy(run, q0, [inputs.const_pool(run.levels[0], 1.7), np.zeros(32)],
                        [inputs.const_pool(run.levels[0], 3.1), np.zeros(32)])
    O.regrid(tol=0.02, buffer=2, cutoff=0.7, max_size=64)
    assert len(run.levels[1].boxes) > 0
    assert np.all(O.rho[1] == 1.7) and np.all(O.K[1] == 3.1)
