"""Shared helper of the AMR GPU tests: the composite integral of a hierarchy."""
import numpy as np


def composite(H, run_index=0):
    """sum over every cell not covered by a finer level of q times the cell area"""
    run = H.runs[run_index]
    tot = np.zeros(3)
    for L, lev in enumerate(run.levels):
        for n, b in enumerate(lev.boxes):
            nx, ny = int(b[2]), int(b[3])
            v = H.interior(run_index, L, n)
            mask = np.ones((ny, nx), bool)
            if L + 1 < len(run.levels):
                r = run.levels[L + 1].ratio
                for fb in run.levels[L + 1].boxes:
                    i0, j0 = int(fb[0]) // r - int(b[0]), int(fb[1]) // r - int(b[1])
                    i1, j1 = i0 + int(fb[2]) // r, j0 + int(fb[3]) // r
                    mask[max(j0, 0):max(min(j1, ny), 0), max(i0, 0):max(min(i1, nx), 0)] = False
            tot += (v * mask).sum(axis=(1, 2)) * lev.dx * lev.dy
    return tot
