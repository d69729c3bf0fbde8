"""Host logic of the solver (no GPU).  Stepping a level in pieces: the pieces partition the boxes
in pool order, their pool ranges cover each box's planes, and a piece waits exactly for the pieces
whose boxes its two ghost layers touch, periodic images included.  Per-level tilings."""
import numpy as np

from paper_1808_02638_gb300 import inputs
from paper_1808_02638_gb300.solver import band_plan


def _boxes(n, patch):
    lev = inputs.Level(n, n, 2.0 / n, 2.0 / n, inputs.uniform_tiling(n, n, patch, patch))
    return [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(lev.boxes, lev.qoff)]


def test_pieces_partition_the_boxes_and_cover_their_planes():
    boxes = _boxes(256, 32)   # 64 boxes, row-major
    pieces, ranges, _ = band_plan(boxes, 4, 256, 256, (0, 0, 0, 0))
    assert pieces == [(0, 16), (16, 32), (32, 48), (48, 64)]
    for (b0, b1), (a, b) in zip(pieces, ranges):
        for (_, _, nx, ny, qoff) in boxes[b0:b1]:
            assert a <= qoff and qoff + 3 * (nx + 4) * (ny + 4) <= b
    assert all(ranges[k][1] <= ranges[k + 1][0] for k in range(len(ranges) - 1))


def test_needs_follow_neighbours_and_periodic_images():
    boxes = _boxes(256, 32)
    # two box rows per piece: each piece touches its neighbours above and below only
    _, _, needs = band_plan(boxes, 4, 256, 256, (0, 0, 0, 0))
    assert needs == [[0, 1], [0, 1, 2], [1, 2, 3], [2, 3]]
    # periodic in y: the first and the last pieces see each other across the boundary
    _, _, needs = band_plan(boxes, 4, 256, 256, (0, 0, 1, 1))
    assert needs[0] == [0, 1, 3] and needs[3] == [0, 2, 3]
    # periodic in x only: a band of full box rows is its own image
    _, _, needs = band_plan(boxes, 4, 256, 256, (1, 1, 0, 0))
    assert needs == [[0, 1], [0, 1, 2], [1, 2, 3], [2, 3]]


def test_more_pieces_than_rows_and_uneven_boxes():
    boxes = [(0, 0, 64, 8, 0), (0, 8, 64, 56, 3 * 68 * 12), (64, 0, 64, 64, 3 * 68 * 12 + 3 * 68 * 60)]
    pieces, ranges, needs = band_plan(boxes, 8, 128, 64, (0, 0, 0, 0))
    assert sorted(b for p in pieces for b in range(*p)) == [0, 1, 2]
    # the big second box dominates the cell count: no empty pieces, every box in one piece
    assert all(b1 > b0 for b0, b1 in pieces)
    for k, (b0, b1) in enumerate(pieces):
        assert k in needs[k]
    assert np.all(np.diff([a for a, _ in ranges]) > 0)


def test_level_tiling_per_level_or_shared():
    # Hierarchy.level_tiling: one tuple for every level, or one per level with the last one
    # standing for the levels beyond the sequence
    from types import SimpleNamespace

    from paper_1808_02638_gb300.solver import Hierarchy
    one = SimpleNamespace(tiling=(32, 16, 2, 256))
    assert [Hierarchy.level_tiling(one, L) for L in range(3)] == [(32, 16, 2, 256)] * 3
    per = SimpleNamespace(tiling=((32, 16, 2, 256), [16, 16, 1, 128]))
    assert [Hierarchy.level_tiling(per, L) for L in range(3)] == [(32, 16, 2, 256), (16, 16, 1, 128),
                                                                   (16, 16, 1, 128)]
    assert Hierarchy.level_tiling(SimpleNamespace(tiling=None), 0) is None


def test_cell_updates_count_every_level_step():
    # the metric's unit: one interior cell advanced one step on its level, so a coarse step of a
    # level-1 box counts r times its cells, of a level-2 box r^2 times
    from paper_1808_02638_gb300.measure import cell_updates_per_coarse_step
    from types import SimpleNamespace
    run = inputs.Run(-1.0, -1.0, 1.0, 1.0)
    run.levels = [inputs.Level(16, 16, 1.0, 1.0, [(0, 0, 16, 16)]),
                  inputs.Level(64, 64, 1.0, 1.0, [(8, 8, 16, 8), (24, 8, 8, 8)], 4),
                  inputs.Level(256, 256, 1.0, 1.0, [(40, 40, 8, 8)], 4)]
    H = SimpleNamespace(runs=[run, run])
    assert cell_updates_per_coarse_step(H) == 2 * (256 + 4 * (128 + 64) + 16 * 64)
