"""Oracle regridding (Sec. 2.2: every K steps the finer levels are regenerated; cells are flagged
by a gradient criterion and clustered into rectangles with the algorithm of Berger and Rigoutsos;
Sec. 4.3: `cutoff` is the least fraction of flagged cells a new patch may hold, and with a regrid
interval of a the flags are grown by a cells so that waves stay inside the refined region).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python and numpy, written from those
definitions:
  flag_level      cell flagged when some component differs from a face neighbour by more than tol
  dilate          flags grown by `buffer` cells (square neighbourhood), clipped to the domain
  nest_mask       cells of level L at least `nest` cells inside level L's coverage (domain
                  edges do not count as coverage edges)
  cluster         Berger-Rigoutsos: accept the flags' bounding box when its efficiency reaches
                  cutoff, it fits max_size and all its cells are allowed (nesting); otherwise cut
                  at a hole of a signature (the one nearest the middle), else at the strongest
                  inflection of a signature's second difference, else at the middle of the longer
                  side; recurse on both parts
  regrid          levels 1.. rebuilt top-down; new fine cells copy old fine values where the old
                  level had them, else the conservative space interpolation from the coarse level
"""
from __future__ import annotations

import numpy as np

from . import MBC, interp_cell


def _view(pool, off, nx, ny, ncomp):
    n = ncomp * (nx + 2 * MBC) * (ny + 2 * MBC)
    return pool[off:off + n].reshape(ncomp, ny + 2 * MBC, nx + 2 * MBC)


def flag_box(qb, tol):
    """flags (ny, nx) of one padded box (3, ny+4, nx+4) whose ghosts are filled"""
    c = qb[:, MBC:-MBC, MBC:-MBC]
    diffs = [np.abs(qb[:, MBC:-MBC, MBC + 1:qb.shape[2] - MBC + 1] - c),   # east
             np.abs(qb[:, MBC:-MBC, MBC - 1:qb.shape[2] - MBC - 1] - c),   # west
             np.abs(qb[:, MBC + 1:qb.shape[1] - MBC + 1, MBC:-MBC] - c),   # north
             np.abs(qb[:, MBC - 1:qb.shape[1] - MBC - 1, MBC:-MBC] - c)]   # south
    return np.any([(d > tol).any(axis=0) for d in diffs], axis=0)


def flag_level(lev, pool, tol):
    """level-wide flags (NY, NX) of a level whose ghosts are filled"""
    f = np.zeros((lev.NY, lev.NX), bool)
    for n, b in enumerate(lev.boxes):
        i0, j0, nx, ny = (int(v) for v in b)
        f[j0:j0 + ny, i0:i0 + nx] |= flag_box(_view(pool, lev.qoff[n], nx, ny, 3), tol)
    return f


def dilate(flags, buffer):
    out = flags.copy()
    NY, NX = flags.shape
    for dj in range(-buffer, buffer + 1):
        for di in range(-buffer, buffer + 1):
            if abs(dj) >= NY or abs(di) >= NX:   # the shifted grid lies outside the domain
                continue
            src = flags[max(0, -dj):NY - max(0, dj), max(0, -di):NX - max(0, di)]
            out[max(0, dj):NY - max(0, -dj), max(0, di):NX - max(0, -di)] |= src
    return out


def nest_mask(lev, nest):
    """cells of lev (level-wide grid) whose square neighbourhood of radius `nest`, clipped to the
    domain, lies inside the level's boxes"""
    cov = np.zeros((lev.NY, lev.NX), bool)
    for b in lev.boxes:
        i0, j0, nx, ny = (int(v) for v in b)
        cov[j0:j0 + ny, i0:i0 + nx] = True
    ok = cov.copy()
    NY, NX = cov.shape
    for dj in range(-nest, nest + 1):
        for di in range(-nest, nest + 1):
            if abs(dj) >= NY or abs(di) >= NX:   # all outside the domain: covered
                continue
            sh = np.ones_like(cov)   # outside the domain counts as covered
            sh[max(0, -dj):NY - max(0, dj), max(0, -di):NX - max(0, di)] = \
                cov[max(0, dj):NY - max(0, -dj), max(0, di):NX - max(0, -di)]
            ok &= sh
    return ok


def _cut(sig):
    """cut position (between sig[k-1] and sig[k], 0 < k < len) of a signature, or None"""
    n = len(sig)
    holes = [k for k in range(1, n - 1) if sig[k] == 0]
    if holes:
        mid = n / 2.0
        best = min(holes, key=lambda k: (abs(k + 0.5 - mid), k))
        # cut on the side of the hole nearer the middle, at the hole's edge
        return best if best + 0.5 >= mid else best + 1
    return None


def _inflection(sig):
    """(strength, cut) of the strongest sign change of the second difference, or None"""
    n = len(sig)
    if n < 4:
        return None
    lap = [sig[k - 1] - 2 * sig[k] + sig[k + 1] for k in range(1, n - 1)]   # at k = 1..n-2
    best = None
    for t in range(len(lap) - 1):
        a, b = lap[t], lap[t + 1]
        if a * b < 0:
            s = abs(a - b)
            k = t + 2          # cut between cells t+1 and t+2
            if best is None or s > best[0]:
                best = (s, k)
    return best


def cluster(flags, cutoff, max_size, allowed=None):
    """boxes (i0, j0, nx, ny) covering every flagged cell of `flags` (NY, NX); with `allowed`
    (flags must lie inside it) every box lies inside it too"""
    out = []
    stack = [(0, 0, flags.shape[1], flags.shape[0])]
    while stack:
        i0, j0, nx, ny = stack.pop()
        sub = flags[j0:j0 + ny, i0:i0 + nx]
        cols = np.nonzero(sub.any(axis=0))[0]
        if len(cols) == 0:
            continue
        rows = np.nonzero(sub.any(axis=1))[0]
        i0, nx = i0 + int(cols[0]), int(cols[-1] - cols[0] + 1)
        j0, ny = j0 + int(rows[0]), int(rows[-1] - rows[0] + 1)
        sub = flags[j0:j0 + ny, i0:i0 + nx]
        eff = sub.sum() / float(nx * ny)
        inside = allowed is None or bool(allowed[j0:j0 + ny, i0:i0 + nx].all())
        if eff >= cutoff and nx <= max_size and ny <= max_size and inside:
            out.append((i0, j0, nx, ny))
            continue
        sx = [int(v) for v in sub.sum(axis=0)]
        sy = [int(v) for v in sub.sum(axis=1)]
        cut = None
        if eff < cutoff:
            kx, ky = _cut(sx), _cut(sy)
            if kx is not None:
                cut = ("x", kx)
            elif ky is not None:
                cut = ("y", ky)
            else:
                ix, iy = _inflection(sx), _inflection(sy)
                if ix is not None and (iy is None or ix[0] >= iy[0]):
                    cut = ("x", ix[1])
                elif iy is not None:
                    cut = ("y", iy[1])
        if cut is None:   # bisect the longer side
            cut = ("x", nx // 2) if nx >= ny else ("y", ny // 2)
        d, k = cut
        if d == "x":
            stack.append((i0 + k, j0, nx - k, ny))
            stack.append((i0, j0, k, ny))
        else:
            stack.append((i0, j0 + k, nx, ny - k))
            stack.append((i0, j0, nx, k))
    return out


def new_boxes(coarse, cpool, tol, buffer, cutoff, max_size, nest, ratio):
    """fine boxes (fine index space) for the level above `coarse` from its state (ghosts filled)"""
    m = nest_mask(coarse, nest)
    f = dilate(flag_level(coarse, cpool, tol), buffer) & m
    return [(i0 * ratio, j0 * ratio, nx * ratio, ny * ratio) for (i0, j0, nx, ny) in
            cluster(f, cutoff, max(1, max_size // ratio), m)]


def transfer(fine_old, fpool_old, fine_new, coarse, cpool, bc):
    """new fine pool: old fine values where the old level had the cell, otherwise the
    conservative interpolation from the coarse pool (time fraction 0)"""
    r = fine_new.ratio
    out = np.zeros(fine_new.qsize)
    cb = [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(coarse.boxes, coarse.qoff)]
    old = [(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(o)) for b, o in zip(fine_old.boxes, fine_old.qoff)] \
        if fine_old is not None else []
    for n, b in enumerate(fine_new.boxes):
        i0, j0, nx, ny = (int(v) for v in b)
        v = _view(out, fine_new.qoff[n], nx, ny, 3)
        for j in range(ny):
            for i in range(nx):
                gi, gj = i0 + i, j0 + j
                src = None
                for (oi, oj, onx, ony, oo) in old:
                    if oi <= gi < oi + onx and oj <= gj < oj + ony:
                        src = _view(fpool_old, oo, onx, ony, 3)[:, MBC + gj - oj, MBC + gi - oi]
                        break
                if src is None:
                    src = interp_cell(cb, cpool, cpool, 0.0, r, 3, coarse.NX, coarse.NY, bc, gi, gj)
                v[:, MBC + j, MBC + i] = src
    return out
