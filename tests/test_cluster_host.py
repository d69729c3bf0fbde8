"""The library's clustering (claw_cluster_flags: host code, no GPU) against the oracle's
buffer, nesting and Berger-Rigoutsos steps of Sec. 2.2 on random flag grids and coverages:
identical boxes, in the same order."""
import numpy as np
import pytest

from paper_1808_02638_gb300 import inputs


def _case(rng, NX, NY):
    # coverage: a tiling of the level with some tiles missing (or the whole level)
    bx, by = int(rng.integers(8, 40)), int(rng.integers(8, 40))
    cover = [(i, j, min(bx, NX - i), min(by, NY - j)) for j in range(0, NY, by) for i in range(0, NX, bx)]
    if rng.random() < 0.7:
        cover = [b for b in cover if rng.random() < 0.8]
    flags = np.zeros((NY, NX), bool)
    for _ in range(int(rng.integers(0, 7))):   # blobs of varying density, plus sparse noise
        cx, cy, rx, ry = rng.integers(0, NX), rng.integers(0, NY), rng.integers(1, 20), rng.integers(1, 20)
        blob = np.zeros_like(flags)
        blob[max(0, cy - ry):cy + ry, max(0, cx - rx):cx + rx] = True
        flags |= blob & (rng.random(flags.shape) < rng.random())
    flags |= rng.random(flags.shape) < 0.003 * rng.random()
    return cover, flags


@pytest.mark.parametrize("seed", range(20))
def test_clustering_matches_the_oracle(seed):
    from oracle import regrid as org
    from paper_1808_02638_gb300 import build, claw
    build.build()
    rng = np.random.default_rng(1000 + seed)
    for _ in range(6):
        NX, NY = int(rng.integers(20, 140)), int(rng.integers(20, 140))
        cover, flags = _case(rng, NX, NY)
        ratio = int(rng.choice([2, 4]))
        buffer, nest = int(rng.integers(0, 5)), int(rng.integers(0, 3))
        cutoff, cap = float(rng.choice([0.5, 0.7, 0.9, 1.0])), int(rng.integers(8, 200))
        got = claw.claw_cluster_flags(NX, NY, ratio, cover, flags.astype(np.uint8), buffer, nest, cutoff, cap)
        lev = inputs.Level(NX, NY, 1.0, 1.0, np.array(cover, dtype=np.int32).reshape(-1, 4))
        m = org.nest_mask(lev, nest)
        f = org.dilate(flags, buffer) & m
        want = [(i0 * ratio, j0 * ratio, nx * ratio, ny * ratio)
                for (i0, j0, nx, ny) in org.cluster(f, cutoff, max(1, cap // ratio), m)]
        assert got == want


def test_clustering_argument_errors():
    from paper_1808_02638_gb300 import build, claw
    build.build()
    flags = np.ones((8, 8), np.uint8)
    with pytest.raises(claw.ClawError):
        claw.claw_cluster_flags(8, 8, 2, [(0, 0, 8, 8)], flags, 1, 1, 1.5, 16)   # cutoff above 1
    with pytest.raises(claw.ClawError):
        claw.claw_cluster_flags(8, 8, 0, [(0, 0, 8, 8)], flags, 1, 1, 0.7, 16)   # ratio 0
    assert claw.claw_cluster_flags(8, 8, 2, [(0, 0, 8, 8)], np.zeros((8, 8), np.uint8), 1, 1, 0.7, 16) == []


def test_more_boxes_than_the_first_output_buffer():
    # a checkerboard with cutoff 1 leaves one box per flagged cell: 131072 boxes, more than the
    # binding's first output buffer, so the call is repeated with room for every cell
    from paper_1808_02638_gb300 import build, claw
    build.build()
    n = 512
    jj, ii = np.mgrid[0:n, 0:n]
    flags = ((ii + jj) % 2 == 0).astype(np.uint8)
    got = claw.claw_cluster_flags(n, n, 2, [(0, 0, n, n)], flags, 0, 0, 1.0, 1024)
    assert len(got) == n * n // 2 > 65536
    assert sorted(got) == sorted((2 * int(i), 2 * int(j), 2, 2) for j, i in zip(*np.nonzero(flags)))


@pytest.mark.parametrize("NX,NY,fill,nest,buffer", [(1, 40, 0.5, 0, 0), (40, 1, 0.5, 1, 2), (17, 23, 1.0, 0, 0),
                                                     (12, 12, 0.3, 20, 1), (64, 64, 0.02, 1, 30)])
def test_clustering_degenerate_grids(NX, NY, fill, nest, buffer):
    # one-cell-wide levels, a fully flagged level, a nesting reach wider than the level and a buffer
    # wider than it: still the oracle's boxes
    from oracle import regrid as org
    from paper_1808_02638_gb300 import build, claw
    build.build()
    rng = np.random.default_rng(NX * 100 + NY)
    flags = rng.random((NY, NX)) < fill
    cover = [(0, 0, NX, NY)]
    for cutoff, cap in ((0.7, 8), (1.0, 64), (0.5, 1000)):
        got = claw.claw_cluster_flags(NX, NY, 2, cover, flags.astype(np.uint8), buffer, nest, cutoff, cap)
        lev = inputs.Level(NX, NY, 1.0, 1.0, np.array(cover, dtype=np.int32))
        m = org.nest_mask(lev, nest)
        f = org.dilate(flags, buffer) & m
        want = [(2 * i0, 2 * j0, 2 * nx, 2 * ny) for (i0, j0, nx, ny) in org.cluster(f, cutoff, max(1, cap // 2), m)]
        assert got == want
