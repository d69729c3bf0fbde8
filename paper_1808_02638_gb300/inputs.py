"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module draws random numbers, lays out patch pools and builds the synthetic
workloads (radial pulse, smoothed random media, patch tilings).  It holds none of the
wave-propagation arithmetic, so both sides can consume identical arrays without sharing
any method code.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014): state += 0x9E3779B97F4A7C15,
z = (z ^ z>>30) * 0xBF58476D1CE4E5B9, z = (z ^ z>>27) * 0x94D049BB133111EB, z ^ z>>31;
the i-th draw (i = 1, 2, ...) of a stream with seed s is the mix of s + i * gamma, and a
uniform double is (z >> 11) * 2^-53.

Patch storage: each box is stored padded with MBC = 2 ghost layers as planes of
(nx + 4) x (ny + 4) doubles, x fastest; q = (p, u, v) is three consecutive planes.  Box
blocks start at multiples of 32 doubles (256 B) so every row and plane is 16-byte aligned
whenever nx is even (all generated boxes have nx, ny multiples of 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MBC = 2
ALIGN = 32

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start+1 .. start+n of the splitmix64 stream of `seed` as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from the splitmix64 stream of `seed`."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class Stream:
    """Sequential reader of a splitmix64 stream."""

    def __init__(self, seed: int):
        self.seed, self.k = seed, 0

    def next(self) -> float:
        v = float(uniform(self.seed, 1, self.k)[0])
        self.k += 1
        return v

    def randint(self, lo: int, hi: int) -> int:
        """uniform integer in [lo, hi]"""
        return lo + min(hi - lo, int(self.next() * (hi - lo + 1)))


# ------------------------------------------------------------------ hierarchy

@dataclass
class Level:
    """One AMR level of one run: boxes in the level's own index space [0,NX) x [0,NY)."""
    NX: int
    NY: int
    dx: float
    dy: float
    boxes: np.ndarray            # (nb, 4) int32: ilo, jlo, nx, ny
    ratio: int = 1               # refinement ratio to the next coarser level (1 on level 0)
    qoff: np.ndarray = None      # (nb,) int64 element offset of the box's p plane in the q pool
    coff: np.ndarray = None      # (nb,) int64 element offset of the box's plane in 1-plane pools
    qsize: int = 0
    csize: int = 0

    def __post_init__(self):
        self.boxes = np.asarray(self.boxes, dtype=np.int32).reshape(-1, 4)
        self.qoff, self.qsize = layout(self.boxes, 3)
        self.coff, self.csize = layout(self.boxes, 1)

    @property
    def ncells(self) -> int:
        return int(np.sum(self.boxes[:, 2].astype(np.int64) * self.boxes[:, 3]))


@dataclass
class Run:
    xlo: float
    ylo: float
    xhi: float
    yhi: float
    levels: list = field(default_factory=list)
    bc: tuple = (0, 0, 0, 0)
    cfl: float = 0.9
    limiter: int = 4
    order: int = 2
    transverse: int = 2


def layout(boxes: np.ndarray, ncomp: int, align: int = ALIGN):
    """Element offsets of each box's first plane in a pool of `ncomp` planes per box."""
    b = np.asarray(boxes, dtype=np.int64).reshape(-1, 4)
    sizes = ncomp * (b[:, 2] + 2 * MBC) * (b[:, 3] + 2 * MBC)
    sizes = (sizes + align - 1) // align * align   # every box starts on an aligned offset
    ends = np.cumsum(sizes)
    offs = (ends - sizes).astype(np.int64)
    return offs, int(max(int(ends[-1]) if len(ends) else 0, align))


def box_view(pool: np.ndarray, off: int, nx: int, ny: int, ncomp: int) -> np.ndarray:
    """(ncomp, ny+4, nx+4) view of one box inside a flat pool."""
    n = ncomp * (nx + 2 * MBC) * (ny + 2 * MBC)
    return pool[off:off + n].reshape(ncomp, ny + 2 * MBC, nx + 2 * MBC)


def cell_centres(run: Run, lev: Level, box) -> tuple:
    """x, y of the cell centres of a box's padded region, shapes (ny+4, nx+4)."""
    ilo, jlo, nx, ny = (int(v) for v in box)
    i = np.arange(ilo - MBC, ilo + nx + MBC)
    j = np.arange(jlo - MBC, jlo + ny + MBC)
    x = run.xlo + (i + 0.5) * lev.dx
    y = run.ylo + (j + 0.5) * lev.dy
    return np.meshgrid(x, y)


# ------------------------------------------------------------- initial data

def radial_pulse(x: np.ndarray, y: np.ndarray, r0=0.3, width=0.1, amp=0.5, base=1.0):
    """p = base + amp (1 + cos(pi (r - r0)/width)) for |r - r0| < width, else base;
    point values at cell centres (the ring pulse of the benchmark, Sec. 4.1)."""
    r = np.sqrt(x * x + y * y)
    p = np.full_like(r, base)
    inside = np.abs(r - r0) < width
    p[inside] = base + amp * (1.0 + np.cos(np.pi * (r[inside] - r0) / width))
    return p


def init_q(run: Run, lev: Level, fn=radial_pulse) -> np.ndarray:
    """q pool of a level: p from `fn` at cell centres (ghosts included), u = v = 0."""
    pool = np.zeros(lev.qsize)
    for n, b in enumerate(lev.boxes):
        x, y = cell_centres(run, lev, b)
        v = box_view(pool, lev.qoff[n], int(b[2]), int(b[3]), 3)
        v[0] = fn(x, y)
    return pool


def init_swe(run: Run, lev: Level, depth=radial_pulse, u0: float = 0.0, v0: float = 0.0) -> np.ndarray:
    """shallow-water q pool of a level: h = depth(x, y) at cell centres (ghosts included),
    hu = h u0, hv = h v0.  The default depth is the benchmark's ring pulse (1 <= h <= 2)."""
    pool = np.zeros(lev.qsize)
    for n, b in enumerate(lev.boxes):
        x, y = cell_centres(run, lev, b)
        v = box_view(pool, lev.qoff[n], int(b[2]), int(b[3]), 3)
        v[0] = depth(x, y)
        v[1] = v[0] * u0
        v[2] = v[0] * v0
    return pool


def gaussian_smooth(a: np.ndarray, sigma: float, truncate: float = 4.0) -> np.ndarray:
    """Separable Gaussian filter, kernel truncated at truncate*sigma, edges mirrored with
    the edge cell repeated (d c b a | a b c d | d c b a)."""
    rad = int(truncate * sigma + 0.5)
    k = np.arange(-rad, rad + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / sigma) ** 2)
    w /= w.sum()
    out = a.astype(np.float64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (rad, rad)
        ap = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for t, wt in enumerate(w):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(t, t + n)
            acc += wt * ap[tuple(sl)]
        out = acc
    return out


def smooth_field(seed: int, nx: int, ny: int, lo: float, hi: float, sigma: float = 8.0) -> np.ndarray:
    """U[lo,hi] white noise (seeded), Gaussian-smoothed (sigma cells, 4 sigma cut-off) and
    affinely rescaled so that its minimum is lo and its maximum hi.  Shape (ny, nx)."""
    a = lo + (hi - lo) * uniform(seed, nx * ny).reshape(ny, nx)
    s = gaussian_smooth(a, sigma)
    smin, smax = s.min(), s.max()
    return lo + (hi - lo) * (s - smin) / (smax - smin)


def coef_pool(lev: Level, field_l0: np.ndarray, ratio_to_l0: int) -> np.ndarray:
    """One-plane pool of a cell coefficient on a level: the level-0 field (shape
    (NY0, NX0)) injected piecewise-constant, the index clamped to the domain in ghosts."""
    NY0, NX0 = field_l0.shape
    pool = np.zeros(lev.csize)
    for n, b in enumerate(lev.boxes):
        ilo, jlo, nx, ny = (int(v) for v in b)
        i = np.clip(np.arange(ilo - MBC, ilo + nx + MBC), 0, lev.NX - 1) // ratio_to_l0
        j = np.clip(np.arange(jlo - MBC, jlo + ny + MBC), 0, lev.NY - 1) // ratio_to_l0
        v = box_view(pool, lev.coff[n], nx, ny, 1)
        v[0] = field_l0[np.ix_(np.clip(j, 0, NY0 - 1), np.clip(i, 0, NX0 - 1))]
    return pool


def const_pool(lev: Level, value: float) -> np.ndarray:
    pool = np.zeros(lev.csize)
    for n, b in enumerate(lev.boxes):
        box_view(pool, lev.coff[n], int(b[2]), int(b[3]), 1)[...] = value
    return pool


def fourier_field(seed: int, nx: int, ny: int, kmax: int = 4, even: bool = False) -> np.ndarray:
    """Smooth random field on the cell centres of [-1,1]^2 (shape (ny, nx)): a sum of
    cos/sin modes with wave numbers |kx|, |ky| <= kmax (in units of pi) and seeded U[-1,1]
    coefficients, normalised to max |f| = 1.  even=True keeps the cos(kx x) cos(ky y) modes
    only (even in x and in y)."""
    x = -1.0 + (np.arange(nx) + 0.5) * (2.0 / nx)
    y = -1.0 + (np.arange(ny) + 0.5) * (2.0 / ny)
    X, Y = np.meshgrid(x, y)
    k = np.arange(0, kmax + 1)
    coef = 2.0 * uniform(seed, 4 * len(k) ** 2) - 1.0
    f = np.zeros((ny, nx))
    n = 0
    for a in k:
        for b in k:
            if even:
                f += coef[n] * np.cos(np.pi * a * X) * np.cos(np.pi * b * Y)
            else:
                ph = np.pi * (a * X + b * Y)
                f += coef[n] * np.cos(ph) + coef[n + 1] * np.sin(ph)
                ph2 = np.pi * (a * X - b * Y)
                f += coef[n + 2] * np.cos(ph2) + coef[n + 3] * np.sin(ph2)
            n += 4
    return f / np.abs(f).max()


def annulus_window(nx: int, ny: int, r0: float = 0.3, width: float = 0.1) -> np.ndarray:
    """(1 + cos(pi (r - r0)/width))/2 inside |r - r0| < width, else 0, at cell centres of
    [-1,1]^2: a smooth bump over the pulse's ring."""
    x = -1.0 + (np.arange(nx) + 0.5) * (2.0 / nx)
    y = -1.0 + (np.arange(ny) + 0.5) * (2.0 / ny)
    X, Y = np.meshgrid(x, y)
    r = np.sqrt(X * X + Y * Y)
    w = np.zeros_like(r)
    inside = np.abs(r - r0) < width
    w[inside] = 0.5 * (1.0 + np.cos(np.pi * (r[inside] - r0) / width))
    return w


# ---------------------------------------------------------------- tilings

def uniform_tiling(NX: int, NY: int, bx: int, by: int) -> np.ndarray:
    """NX x NY cells as (NX/bx) x (NY/by) patches, row-major."""
    assert NX % bx == 0 and NY % by == 0
    return np.array([(i * bx, j * by, bx, by) for j in range(NY // by) for i in range(NX // bx)],
                    dtype=np.int32)


def guillotine(stream: Stream, x0: int, y0: int, w: int, h: int, smin: int = 2, smax: int = 16,
               p_split: float = 0.5):
    """Seeded guillotine split of a w x h rectangle (in units) into rectangles whose sides
    are in [smin, smax] units.  Returns a list of (x, y, w, h) in units."""
    out = []

    def rec(x, y, w, h):
        must = [ax for ax, n in ((0, w), (1, h)) if n > smax]
        can = [ax for ax, n in ((0, w), (1, h)) if n >= 2 * smin]
        if must:
            ax = must[0] if len(must) == 1 else (0 if w >= h else 1)
        elif can and stream.next() < p_split:
            ax = can[0] if len(can) == 1 else (0 if stream.next() < 0.5 else 1)
        else:
            out.append((x, y, w, h))
            return
        n = w if ax == 0 else h
        k = stream.randint(smin, n - smin)
        if ax == 0:
            rec(x, y, k, h)
            rec(x + k, y, w - k, h)
        else:
            rec(x, y, w, k)
            rec(x, y + k, w, h - k)

    rec(x0, y0, w, h)
    return out


def cover_boxes(flag: np.ndarray, unit: int, seed: int, smin: int = 2, smax: int = 16) -> np.ndarray:
    """Disjoint boxes (cell index space of `flag`, shape (NY, NX)) covering every flagged
    cell: the bounding box of the flagged units (unit x unit cells) is guillotine-split into
    rectangles with sides of smin..smax units and those holding a flagged cell are kept."""
    NY, NX = flag.shape
    assert NX % unit == 0 and NY % unit == 0
    fu = flag.reshape(NY // unit, unit, NX // unit, unit).any(axis=(1, 3))
    js, is_ = np.nonzero(fu)
    if len(is_) == 0:
        return np.zeros((0, 4), dtype=np.int32)
    NXu, NYu = NX // unit, NY // unit
    x0, x1 = int(is_.min()), int(is_.max()) + 1
    y0, y1 = int(js.min()), int(js.max()) + 1
    # widen to at least smin units, staying inside the domain
    while x1 - x0 < smin:
        x1 = min(NXu, x1 + 1) if x1 < NXu else x1
        x0 = max(0, x0 - 1) if x1 - x0 < smin else x0
    while y1 - y0 < smin:
        y1 = min(NYu, y1 + 1) if y1 < NYu else y1
        y0 = max(0, y0 - 1) if y1 - y0 < smin else y0
    rects = guillotine(Stream(seed), x0, y0, x1 - x0, y1 - y0, smin, smax)
    keep = [(x * unit, y * unit, w * unit, h * unit) for (x, y, w, h) in rects
            if fu[y:y + h, x:x + w].any()]
    return np.array(keep, dtype=np.int32).reshape(-1, 4)


def annulus_flag(run: Run, NX: int, NY: int, dx: float, dy: float, r_lo: float, r_hi: float):
    x = run.xlo + (np.arange(NX) + 0.5) * dx
    y = run.ylo + (np.arange(NY) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    r = np.sqrt(X * X + Y * Y)
    return (r > r_lo) & (r < r_hi)


def box_mask(boxes: np.ndarray, NX: int, NY: int, grow: int = 0, scale_down: int = 1):
    """Cells of a level (NX x NY) covered by boxes given on a level `scale_down` times finer,
    grown by `grow` cells of this level and clipped to the domain."""
    m = np.zeros((NY, NX), dtype=bool)
    for ilo, jlo, nx, ny in boxes:
        i0 = ilo // scale_down - grow
        j0 = jlo // scale_down - grow
        i1 = -(-(ilo + nx) // scale_down) + grow
        j1 = -(-(jlo + ny) // scale_down) + grow
        m[max(0, j0):min(NY, j1), max(0, i0):min(NX, i1)] = True
    return m


def amr_levels(run: Run, N1: int, ratio: int, annuli, seeds) -> list:
    """Levels of a nested hierarchy over [xlo,xhi] x [ylo,yhi]: level 0 is one N1 x N1 box;
    level L >= 1 covers annuli[L-1] (cell centres with r_lo < r < r_hi) with seeded
    guillotine boxes of 8..64 cells per side aligned to coarse cells, and is grown so that
    it holds every finer box plus two of its own cells (proper nesting for two ghost layers
    and one slope cell).  The finest level is built first."""
    nlev = len(annuli) + 1
    N = [N1 * ratio ** L for L in range(nlev)]
    dx = [(run.xhi - run.xlo) / n for n in N]
    dy = [(run.yhi - run.ylo) / n for n in N]
    boxes = [None] * nlev
    finer = None
    for L in range(nlev - 1, 0, -1):
        flag = annulus_flag(run, N[L], N[L], dx[L], dy[L], *annuli[L - 1])
        if finer is not None:
            flag |= box_mask(finer, N[L], N[L], grow=2, scale_down=ratio)
        boxes[L] = cover_boxes(flag, ratio, seeds[L - 1], smin=8 // ratio if ratio <= 4 else 1,
                               smax=64 // ratio)
        finer = boxes[L]
    boxes[0] = np.array([(0, 0, N1, N1)], dtype=np.int32)
    return [Level(N[L], N[L], dx[L], dy[L], boxes[L], ratio if L else 1) for L in range(nlev)]


# ---------------------------------------------------------------- workloads

PULSE_DOMAIN = (-1.0, -1.0, 1.0, 1.0)


def config0() -> Run:
    """100 x 100 single grid on [-1,1]^2, rho = 1, K = 4, radial pulse, MC, 50 steps."""
    run = Run(*PULSE_DOMAIN)
    run.levels = [Level(100, 100, 0.02, 0.02, [(0, 0, 100, 100)])]
    return run


def config1(n: int = 2048, patch: int = 32) -> Run:
    """n x n on [-1,1]^2 tiled as (n/patch)^2 patches of patch x patch."""
    run = Run(*PULSE_DOMAIN)
    d = 2.0 / n
    run.levels = [Level(n, n, d, d, uniform_tiling(n, n, patch, patch))]
    return run


def config2() -> Run:
    """3 levels, ratio 4: 64^2 base, level 2 on 0.2<r<0.45 (seed 2002), level 3 on
    0.25<r<0.35 (seed 2003)."""
    run = Run(*PULSE_DOMAIN)
    run.levels = amr_levels(run, 64, 4, [(0.2, 0.45), (0.25, 0.35)], [2002, 2003])
    return run


def config3(n: int = 256) -> tuple:
    """n x n heterogeneous medium: rho ~ U[0.5,2] (seed 3001), K ~ U[1,8] (seed 3002), each
    Gaussian-smoothed (sigma 8 cells) and rescaled to its interval.  Returns (run, rho, K)
    with rho, K of shape (n, n)."""
    run = Run(*PULSE_DOMAIN)
    d = 2.0 / n
    run.levels = [Level(n, n, d, d, [(0, 0, n, n)])]
    rho = smooth_field(3001, n, n, 0.5, 2.0)
    K = smooth_field(3002, n, n, 1.0, 8.0)
    return run, rho, K


def receiver_box(n: int, x0: float = 0.5, y0: float = -0.0625, size: int = 16):
    """Level-0 cells (i0, j0, size) of the receiver: size x size cells whose lower-left cell
    contains (x0, y0) on an n x n grid of [-1,1]^2."""
    d = 2.0 / n
    i0 = int(math.floor((x0 + 1.0) / d))
    j0 = int(math.floor((y0 + 1.0) / d))
    return i0, j0, size


def config4_runs(nruns: int = 64, base_seed: int = 4000) -> list:
    """Independent 2-level problems: N uniform in [64,256] rounded to a multiple of 4 (seed
    4000+r), level 2 of ratio 4 on 0.2<r<0.45 tiled with seed 4000+r, rho/K as in the
    heterogeneous workload on N^2 with seeds 40000+2r, 40000+2r+1."""
    out = []
    for r in range(nruns):
        st = Stream(base_seed + r)
        N = 4 * st.randint(16, 64)
        run = Run(*PULSE_DOMAIN)
        run.levels = amr_levels(run, N, 4, [(0.2, 0.45)], [base_seed + r])
        rho = smooth_field(40000 + 2 * r, N, N, 0.5, 2.0)
        K = smooth_field(40000 + 2 * r + 1, N, N, 1.0, 8.0)
        out.append((run, rho, K))
    return out
