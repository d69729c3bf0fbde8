"""Plain CPU FP64 oracle of the wave-propagation level-step of arXiv:1808.02638.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use this package;
the product path (``paper_1808_02638_gb300``) never imports it and shares no code
with it.  The numerics live in ``claw_oracle.c`` (plain C, -O2 -ffp-contract=off);
this module compiles it with gcc on first use and wraps it for numpy arrays.

Array convention: a patch is a float64 array of shape (ncomp, ny + 2*mbc, nx + 2*mbc)
(x fastest), q = (p, u, v) stacked on the first axis, mbc = 2 ghost layers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "claw_oracle.c")
_SRC_SWE = os.path.join(_HERE, "swe_oracle.c")
_HDR = os.path.join(_HERE, "claw_oracle.h")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MBC = 2
LIMITERS = {"none": 0, "minmod": 1, "superbee": 2, "vanleer": 3, "mc": 4}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, strict IEEE)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_SWE), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, _SRC_SWE, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Box(ctypes.Structure):
    _fields_ = [("ilo", ctypes.c_int32), ("jlo", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("off", ctypes.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            dbl = ctypes.c_double
            BP = ctypes.POINTER(Box)
            IP = ctypes.POINTER(ctypes.c_int)
            L.orc_philim.argtypes = [I, dbl]
            L.orc_philim.restype = dbl
            L.orc_riemann_x.argtypes = [dbl] * 8 + [D, D]
            L.orc_step.argtypes = [I, I, I, dbl, dbl, dbl, I, I, I, D, D, D, D, D]
            L.orc_step_edges.argtypes = [I, I, I, dbl, dbl, dbl, I, I, I, D, D, D, D, D, D]
            L.orc_step_adjoint.argtypes = [I, I, I, dbl, dbl, dbl, I, I, I, D, D, D, D, D, D, D]
            L.orc_fill_bc.argtypes = [I, I, I, I, IP, D]
            L.orc_fill_bc_adjoint.argtypes = [I, I, I, I, IP, D]
            L.orc_cfl_max.argtypes = [I, I, I, D, D]
            L.orc_cfl_max.restype = dbl
            L.orc_level_fill_ghost.argtypes = [I, BP, D, I, I, I, I, IP, I, BP, D, D, dbl, I, I]
            L.orc_average_down.argtypes = [I, BP, D, I, BP, D, I, I, I]
            L.orc_interp_cell.argtypes = [I, BP, D, D, dbl, I, I, I, I, I, IP, I, I, D]
            L.orc_level_fill_ghost_adjoint.argtypes = [I, BP, D, I, I, I, I, IP, I, BP, D, D, D, D,
                                                       dbl, I, I]
            L.orc_average_down_adjoint.argtypes = [I, BP, D, I, BP, D, I, I, I]
            L.orc_swe_step.argtypes = [I, I, I, dbl, dbl, dbl, I, I, I, dbl, D, D, D]
            L.orc_swe_step_edges.argtypes = [I, I, I, dbl, dbl, dbl, I, I, I, dbl, D, D, D, D]
            L.orc_swe_roe_x.argtypes = [dbl] * 7 + [D, D]
            L.orc_swe_cfl_max.argtypes = [I, I, I, dbl, D]
            L.orc_swe_cfl_max.restype = dbl
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(v):
    arr = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return arr


def _lim(limiter) -> int:
    return LIMITERS[limiter] if isinstance(limiter, str) else int(limiter)


def philim(limiter, theta: float) -> float:
    return lib().orc_philim(_lim(limiter), float(theta))


def riemann_x(pl, ul, rhol, Kl, pr, ur, rhor, Kr):
    """Waves (2, 3) and speeds (2,) of the normal Riemann problem at one x-edge."""
    w = np.zeros(6)
    s = np.zeros(2)
    lib().orc_riemann_x(pl, ul, rhol, Kl, pr, ur, rhor, Kr, _p(w), _p(s))
    return w.reshape(2, 3), s


def step(q, rho, K, dx, dy, dt, order=2, transverse=2, limiter="mc"):
    """One level-step on one patch whose ghosts are filled.

    q: (3, H, W); rho, K: (H, W).  Returns (qnew, smax); qnew has the interior advanced
    and the ghost cells of q copied unchanged."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    _, H, W = q.shape
    nx, ny = W - 2 * MBC, H - 2 * MBC
    qn = q.copy()
    sm = ctypes.c_double(0.0)
    rc = lib().orc_step(nx, ny, MBC, dx, dy, dt, order, transverse, _lim(limiter),
                        _p(q), _p(rho), _p(K), _p(qn), ctypes.byref(sm))
    if rc:
        raise ValueError(f"orc_step failed ({rc})")
    return qn, sm.value


def step_edges(q, rho, K, dx, dy, dt, order=2, transverse=2, limiter="mc"):
    """:func:`step` that also returns the step's per-edge quantities (Sec. 2.3 conservation fix).

    Returns (qnew, smax, edges) with edges a dict of (3, H, W) arrays: "amx", "apx" (A-dQ, A+dQ
    of the x-edge between cells (i-1, j) and (i, j), stored at (i, j)), "amy", "apy" (y-edges,
    stored at the upper cell), "F" and "G" (the correction-plus-transverse fluxes of the x- and
    y-edges, same storage)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    _, H, W = q.shape
    nx, ny = W - 2 * MBC, H - 2 * MBC
    qn = q.copy()
    sm = ctypes.c_double(0.0)
    e = np.zeros((6, 3, H, W))
    rc = lib().orc_step_edges(nx, ny, MBC, dx, dy, dt, order, transverse, _lim(limiter),
                              _p(q), _p(rho), _p(K), _p(qn), ctypes.byref(sm), _p(e))
    if rc:
        raise ValueError(f"orc_step_edges failed ({rc})")
    return qn, sm.value, dict(zip(("amx", "apx", "amy", "apy", "F", "G"), e))


def step_adjoint(q, rho, K, lam_new, dx, dy, dt, order=2, transverse=2, limiter="mc"):
    """Reverse mode of :func:`step` with dt frozen.

    Returns (lam_q, g_rho, g_K) over all cells of the patch (ghosts included); only the
    interior of lam_new is read."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    lam_new = np.ascontiguousarray(lam_new, dtype=np.float64)
    _, H, W = q.shape
    nx, ny = W - 2 * MBC, H - 2 * MBC
    lq = np.zeros_like(q)
    gr = np.zeros_like(rho)
    gk = np.zeros_like(K)
    rc = lib().orc_step_adjoint(nx, ny, MBC, dx, dy, dt, order, transverse, _lim(limiter),
                                _p(q), _p(rho), _p(K), _p(lam_new), _p(lq), _p(gr), _p(gk))
    if rc:
        raise ValueError(f"orc_step_adjoint failed ({rc})")
    return lq, gr, gk


def swe_step(q, dx, dy, dt, grav, order=2, transverse=2, limiter="mc"):
    """One shallow-water step (q = (h, hu, hv), Roe solver) on one patch whose ghosts are
    filled.  Returns (qnew, smax) like :func:`step`."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    _, H, W = q.shape
    qn = q.copy()
    sm = ctypes.c_double(0.0)
    rc = lib().orc_swe_step(W - 2 * MBC, H - 2 * MBC, MBC, dx, dy, dt, order, transverse,
                            _lim(limiter), float(grav), _p(q), _p(qn), ctypes.byref(sm))
    if rc:
        raise ValueError(f"orc_swe_step failed ({rc})")
    return qn, sm.value


def swe_step_edges(q, dx, dy, dt, grav, order=2, transverse=2, limiter="mc"):
    """:func:`swe_step` that also returns the per-edge quantities, like :func:`step_edges`."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    _, H, W = q.shape
    qn = q.copy()
    sm = ctypes.c_double(0.0)
    e = np.zeros((6, 3, H, W))
    rc = lib().orc_swe_step_edges(W - 2 * MBC, H - 2 * MBC, MBC, dx, dy, dt, order, transverse,
                                  _lim(limiter), float(grav), _p(q), _p(qn), ctypes.byref(sm), _p(e))
    if rc:
        raise ValueError(f"orc_swe_step_edges failed ({rc})")
    return qn, sm.value, dict(zip(("amx", "apx", "amy", "apy", "F", "G"), e))


def swe_roe_x(left, right, grav):
    """Waves (3, 3) and speeds (3,) of the Roe solve at one x-edge; states are (h, hu, hv)."""
    w = np.zeros(9)
    s = np.zeros(3)
    lib().orc_swe_roe_x(*[float(v) for v in left], *[float(v) for v in right], float(grav),
                        _p(w), _p(s))
    return w.reshape(3, 3), s


def swe_cfl_max(q, grav) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    _, H, W = q.shape
    return lib().orc_swe_cfl_max(W - 2 * MBC, H - 2 * MBC, MBC, float(grav), _p(q))


def fill_bc(a, bc=(0, 0, 0, 0)):
    """Physical-boundary ghosts of a single patch covering the domain (in place)."""
    a3 = a if a.ndim == 3 else a[None]
    nc, H, W = a3.shape
    assert a3.flags["C_CONTIGUOUS"]
    lib().orc_fill_bc(W - 2 * MBC, H - 2 * MBC, MBC, nc, _ip(bc), _p(a3))
    return a


def fill_bc_adjoint(g, bc=(0, 0, 0, 0)):
    g3 = g if g.ndim == 3 else g[None]
    nc, H, W = g3.shape
    lib().orc_fill_bc_adjoint(W - 2 * MBC, H - 2 * MBC, MBC, nc, _ip(bc), _p(g3))
    return g


def cfl_max(rho, K) -> float:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    H, W = rho.shape
    return lib().orc_cfl_max(W - 2 * MBC, H - 2 * MBC, MBC, _p(rho), _p(K))


# ----------------------------------------------------------------- AMR helpers

def boxes_array(boxes):
    """boxes: iterable of (ilo, jlo, nx, ny, off) -> ctypes array of Box."""
    boxes = list(boxes)
    arr = (Box * max(1, len(boxes)))()
    for n, b in enumerate(boxes):
        arr[n] = Box(int(b[0]), int(b[1]), int(b[2]), int(b[3]), int(b[4]))
    return arr, len(boxes)


def level_fill_ghost(boxes, pool, ncomp, NX, NY, bc, cboxes=None, cold=None, cnew=None,
                     tau=0.0, r=0, copy_only=False):
    """Fill the ghosts of every box of a level in place (Sec. 2.2 ghost rules)."""
    b, nb = boxes_array(boxes)
    if cboxes is None:
        cb, ncb = boxes_array([])
        ncb = 0
        dummy = np.zeros(1)
        cold = cnew = dummy
    else:
        cb, ncb = boxes_array(cboxes)
    rc = lib().orc_level_fill_ghost(nb, b, _p(pool), ncomp, MBC, NX, NY, _ip(bc), ncb, cb,
                                    _p(cold), _p(cnew), float(tau), int(r), int(copy_only))
    if rc:
        raise ValueError(f"level_fill_ghost failed ({rc}): improper nesting")
    return pool


def level_fill_ghost_adjoint(boxes, gpool, ncomp, NX, NY, bc, cboxes=None, gcold=None,
                             gcnew=None, cold=None, cnew=None, tau=0.0, r=0, copy_only=False):
    b, nb = boxes_array(boxes)
    if cboxes is None:
        cb, _ = boxes_array([])
        ncb = 0
        dummy = np.zeros(1)
        gcold = gcnew = cold = cnew = dummy
    else:
        cb, ncb = boxes_array(cboxes)
    rc = lib().orc_level_fill_ghost_adjoint(nb, b, _p(gpool), ncomp, MBC, NX, NY, _ip(bc), ncb,
                                            cb, _p(gcold), _p(gcnew), _p(cold), _p(cnew),
                                            float(tau), int(r), int(copy_only))
    if rc:
        raise ValueError(f"level_fill_ghost_adjoint failed ({rc})")
    return gpool


def average_down(fboxes, fpool, cboxes, cpool, ncomp, r):
    fb, nf = boxes_array(fboxes)
    cb, nc = boxes_array(cboxes)
    lib().orc_average_down(nf, fb, _p(fpool), nc, cb, _p(cpool), ncomp, MBC, int(r))
    return cpool


def average_down_adjoint(fboxes, gfpool, cboxes, gcpool, ncomp, r):
    fb, nf = boxes_array(fboxes)
    cb, nc = boxes_array(cboxes)
    lib().orc_average_down_adjoint(nf, fb, _p(gfpool), nc, cb, _p(gcpool), ncomp, MBC, int(r))
    return gfpool


def interp_cell(cboxes, cold, cnew, tau, r, ncomp, cNX, cNY, bc, fi, fj):
    cb, ncb = boxes_array(cboxes)
    out = np.zeros(ncomp)
    rc = lib().orc_interp_cell(ncb, cb, _p(cold), _p(cnew), float(tau), int(r), ncomp, MBC,
                               cNX, cNY, _ip(bc), int(fi), int(fj), _p(out))
    if rc:
        raise ValueError("interp_cell: coarse cell not covered")
    return out
