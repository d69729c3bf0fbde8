"""ctypes binding of libclaw.so (include/claw.h): the same entry points, with torch tensors
(device memory) and torch streams marshalled to pointers.  Every step of the level-step path
runs in the library's CUDA kernels; this module only converts arguments and raises
:class:`ClawError` on a non-zero status.  Loading fails loudly when the library is missing or
no CUDA device is present: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libclaw.so")

CLAW_OK, CLAW_EINVAL, CLAW_ECUDA, CLAW_ENOMEM, CLAW_ECFL, CLAW_ENAN, CLAW_ETIMEOUT, CLAW_ESTATE = range(8)
CLAW_MBC = 2
CLAW_MAXLEV = 8
CLAW_NAUX = 10
LIMITERS = {"none": 0, "minmod": 1, "superbee": 2, "vanleer": 3, "mc": 4}
CLAW_SYS_ACOUSTICS, CLAW_SYS_SHALLOW_WATER = 0, 1
SYSTEMS = {"acoustics": CLAW_SYS_ACOUSTICS, "shallow_water": CLAW_SYS_SHALLOW_WATER}


class ClawError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn}: {strerror(status)} (status {status})")


class claw_problem(ctypes.Structure):
    _fields_ = [("xlo", ctypes.c_double), ("ylo", ctypes.c_double), ("xhi", ctypes.c_double),
                ("yhi", ctypes.c_double), ("nx0", ctypes.c_int32), ("ny0", ctypes.c_int32),
                ("nlev", ctypes.c_int32), ("ratio", ctypes.c_int32 * CLAW_MAXLEV),
                ("cfl", ctypes.c_double), ("limiter", ctypes.c_int32), ("order", ctypes.c_int32),
                ("transverse", ctypes.c_int32), ("bc", ctypes.c_int32 * 4), ("medium", ctypes.c_int32),
                ("rho0", ctypes.c_double), ("K0", ctypes.c_double), ("system", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("grav", ctypes.c_double)]


class claw_box(ctypes.Structure):
    _fields_ = [("run", ctypes.c_int32), ("ilo", ctypes.c_int32), ("jlo", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("qoff", ctypes.c_int64), ("coff", ctypes.c_int64)]


class claw_fill_job(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("reserved", ctypes.c_int32), ("q", ctypes.c_void_p),
                ("qc_old", ctypes.c_void_p), ("qc_new", ctypes.c_void_p), ("tau", ctypes.c_double)]


_lib = None
VP = ctypes.c_void_p
I32 = ctypes.c_int32
DBL = ctypes.c_double

_SIGNATURES = {
    "claw_create": ([ctypes.POINTER(VP), ctypes.POINTER(claw_problem), I32, I32], ctypes.c_int),
    "claw_destroy": ([VP], None),
    "claw_set_level": ([VP, I32, VP, I32], ctypes.c_int),
    "claw_set_tiling": ([VP, I32, I32, I32, I32, I32], ctypes.c_int),
    "claw_set_tile_walk": ([VP, I32, I32], ctypes.c_int),
    "claw_limiter_eval": ([I32, ctypes.c_int64, VP, VP, VP, VP], ctypes.c_int),
    "claw_set_wait_limit": ([VP, ctypes.c_uint32], ctypes.c_int),
    "claw_medium_aux": ([VP, I32, VP, VP, VP, VP], ctypes.c_int),
    "claw_medium_aux_adjoint": ([VP, I32, VP, VP, VP, VP, VP, VP], ctypes.c_int),
    "claw_flag_grid_size": ([VP, I32], ctypes.c_longlong),
    "claw_flag_cells": ([VP, I32, VP, ctypes.c_double, VP, VP], ctypes.c_int),
    "claw_regrid_boxes": ([VP, I32, I32, VP, I32, I32, ctypes.c_double, I32, VP, I32], ctypes.c_int),
    "claw_cluster_flags": ([I32, I32, I32, VP, I32, VP, I32, I32, ctypes.c_double, I32, VP, I32], ctypes.c_int),
    "claw_regrid_transfer": ([VP, I32, VP, I32, VP, VP, VP, VP], ctypes.c_int),
    "claw_reflux_count": ([VP, I32], ctypes.c_int),
    "claw_reflux_buffer_size": ([VP, I32], ctypes.c_int),
    "claw_reflux_coarse": ([VP, I32, VP, VP, VP, VP], ctypes.c_int),
    "claw_reflux_fine": ([VP, I32, VP, VP, VP, VP, VP], ctypes.c_int),
    "claw_reflux_apply": ([VP, I32, VP, VP, VP, VP], ctypes.c_int),
    "claw_fill_ghost": ([VP, I32, VP, VP, VP, DBL, VP], ctypes.c_int),
    "claw_fill_ghost_adjoint": ([VP, I32, VP, VP, VP, VP, VP, DBL, VP], ctypes.c_int),
    "claw_fill_ghost_interp_adjoint": ([VP, I32, VP, VP, VP, VP, VP, DBL, VP], ctypes.c_int),
    "claw_fill_ghost_coef": ([VP, I32, VP, VP], ctypes.c_int),
    "claw_fill_ghost_interp": ([VP, I32, VP, VP, VP, DBL, VP], ctypes.c_int),
    "claw_fill_ghost_coef_adjoint": ([VP, I32, VP, VP], ctypes.c_int),
    "claw_cfl_max": ([VP, I32, VP, VP, VP], ctypes.c_int),
    "claw_cfl_max_state": ([VP, I32, VP, VP, VP], ctypes.c_int),
    "claw_dt_update": ([VP, I32, VP, VP, VP], ctypes.c_int),
    "claw_level_step": ([VP, I32, VP, VP, VP, VP, VP, VP], ctypes.c_int),
    "claw_level_step_patchwise": ([VP, I32, VP, VP, VP, VP, VP, VP], ctypes.c_int),
    "claw_level_advance": ([VP, I32, VP, VP, VP, VP, VP, I32, VP], ctypes.c_int),
    "claw_level_advance_boxes": ([VP, I32, I32, I32, VP, VP, VP, VP, VP, I32, VP], ctypes.c_int),
    "claw_level_advance_interp": ([VP, I32, VP, VP, VP, VP, VP, I32, VP, VP, DBL, VP], ctypes.c_int),
    "claw_level_advance_fill": ([VP, I32, VP, VP, VP, VP, VP, I32, VP, I32, VP], ctypes.c_int),
    "claw_packed_size": ([VP, I32], ctypes.c_longlong),
    "claw_pack_interiors": ([VP, I32, I32, I32, VP, VP, VP], ctypes.c_int),
    "claw_unpack_interiors": ([VP, I32, I32, I32, VP, VP, VP], ctypes.c_int),
    "claw_level_step_noalloc": ([I32, I32, DBL, DBL, I32, I32, I32, DBL, DBL, VP, VP, VP, VP, VP, VP],
                                ctypes.c_int),
    "claw_average_down": ([VP, I32, VP, VP, VP], ctypes.c_int),
    "claw_average_down_adjoint": ([VP, I32, VP, VP, VP], ctypes.c_int),
    "claw_level_step_adjoint": ([VP, I32, VP, VP, VP, VP, VP, VP, VP], ctypes.c_int),
    "claw_level_advance_adjoint": ([VP, I32, VP, VP, VP, VP, VP, VP, I32, VP], ctypes.c_int),
    "claw_level_advance_record": ([VP, I32, VP, VP, VP, VP, VP, I32, VP, VP], ctypes.c_int),
    "claw_level_advance_adjoint_tape": ([VP, I32, VP, VP, VP, VP, VP, VP, I32, VP], ctypes.c_int),
    "claw_sync_status": ([VP], ctypes.c_int),
    "claw_launch_count": ([VP], ctypes.c_int64),
    "claw_strerror": ([I32], ctypes.c_char_p),
}


def load(path: str = LIB_PATH):
    """Load libclaw.so (built by paper_1808_02638_gb300.build) and declare its signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1808_02638_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return load().claw_strerror(int(status)).decode()


def _check(fn: str, status: int):
    if status != CLAW_OK:
        raise ClawError(fn, status)


def _ptr(t):
    """device pointer of a torch tensor (or None)"""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("libclaw takes device tensors")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ------------------------------------------------------------------ entry points

def claw_create(runs, device: int = 0):
    arr = (claw_problem * len(runs))(*runs)
    h = VP()
    _check("claw_create", load().claw_create(ctypes.byref(h), arr, len(runs), device))
    return h


def claw_destroy(ctx):
    load().claw_destroy(ctx)


def box_array(n):
    """a numpy record array of n boxes laid out like claw_box (fields run, ilo, jlo, nx, ny,
    reserved, qoff, coff), which the box-taking calls pass without conversion"""
    import numpy as np
    return np.zeros(n, dtype=BOX_DTYPE()).view(np.recarray)


def BOX_DTYPE():
    import numpy as np
    dt = np.dtype([("run", "<i4"), ("ilo", "<i4"), ("jlo", "<i4"), ("nx", "<i4"), ("ny", "<i4"),
                   ("reserved", "<i4"), ("qoff", "<i8"), ("coff", "<i8")], align=True)
    assert dt.itemsize == ctypes.sizeof(claw_box)
    return dt


def _boxes_arg(boxes):
    """(keep-alive object, pointer, count) of a list of claw_box or a box_array"""
    import numpy as np
    if isinstance(boxes, np.ndarray) and boxes.dtype == BOX_DTYPE():
        a = np.ascontiguousarray(boxes)
        return a, ctypes.c_void_p(a.ctypes.data if len(a) else 0), len(a)
    arr = (claw_box * max(1, len(boxes)))(*boxes)
    return arr, ctypes.cast(arr, ctypes.c_void_p), len(boxes)


def claw_set_level(ctx, level: int, boxes):
    keep, ptr, n = _boxes_arg(boxes)
    _check("claw_set_level", load().claw_set_level(ctx, level, ptr, n))


def claw_set_tiling(ctx, level: int, tx: int, ty: int, staging: int, threads: int = 0):
    _check("claw_set_tiling", load().claw_set_tiling(ctx, level, tx, ty, staging, threads))


def claw_set_tile_walk(ctx, level: int, walk: int):
    _check("claw_set_tile_walk", load().claw_set_tile_walk(ctx, level, int(walk)))


def claw_limiter_eval(limiter: int, a, b, out, stream=None):
    n = a.numel()
    if b.numel() != n or out.numel() != n:
        raise ValueError("a, b and out must have the same size")
    _check("claw_limiter_eval", load().claw_limiter_eval(int(limiter), n, _ptr(a), _ptr(b), _ptr(out), _stream(stream)))


def claw_set_wait_limit(ctx, polls: int):
    _check("claw_set_wait_limit", load().claw_set_wait_limit(ctx, int(polls)))


def claw_medium_aux(ctx, level, rho, K, aux, stream=None):
    _check("claw_medium_aux", load().claw_medium_aux(ctx, level, _ptr(rho), _ptr(K), _ptr(aux), _stream(stream)))


def claw_flag_grid_size(ctx, level):
    n = load().claw_flag_grid_size(ctx, level)
    if n < 0:
        raise ClawError("claw_flag_grid_size", int(-n))
    return int(n)


def claw_flag_cells(ctx, level, q, tol, flags, stream=None):
    _check("claw_flag_cells", load().claw_flag_cells(ctx, level, _ptr(q), float(tol), _ptr(flags), _stream(stream)))


def _boxes_out(name, f, call):
    """call(out pointer, capacity) -> count; room for 65536 boxes first, and a grid that makes more
    (at most one per cell) is clustered again with room for all of them"""
    import numpy as np
    for cap in (min(65536, max(16, f.size)), max(16, f.size)):
        out = np.empty(4 * cap, dtype=np.int32)
        n = call(out.ctypes.data_as(ctypes.c_void_p), cap)
        if n != -CLAW_ENOMEM:
            break
    if n < 0:
        raise ClawError(name, -n)
    return [tuple(int(v) for v in out[4 * k:4 * k + 4]) for k in range(n)]


def claw_regrid_boxes(ctx, level, run, flags_host, buffer, nest, cutoff, max_size):
    """new (ilo, jlo, nx, ny) boxes of level+1 for one run from its host flag grid (numpy uint8)"""
    import numpy as np
    f = np.ascontiguousarray(flags_host, dtype=np.uint8)
    return _boxes_out("claw_regrid_boxes", f, lambda out, cap: load().claw_regrid_boxes(
        ctx, level, run, f.ctypes.data_as(ctypes.c_void_p), int(buffer), int(nest), float(cutoff), int(max_size),
        out, cap))


def claw_cluster_flags(nx, ny, ratio, cover, flags_host, buffer, nest, cutoff, max_size):
    """the same clustering without a context: cover = the level's (ilo, jlo, nx, ny) boxes"""
    import numpy as np
    f = np.ascontiguousarray(flags_host, dtype=np.uint8)
    arr = (claw_box * max(1, len(cover)))()
    for k, (i0, j0, bx, by) in enumerate(cover):
        arr[k].ilo, arr[k].jlo, arr[k].nx, arr[k].ny = int(i0), int(j0), int(bx), int(by)
    return _boxes_out("claw_cluster_flags", f, lambda out, cap: load().claw_cluster_flags(
        int(nx), int(ny), int(ratio), ctypes.cast(arr, ctypes.c_void_p), len(cover), f.ctypes.data_as(ctypes.c_void_p),
        int(buffer), int(nest), float(cutoff), int(max_size), out, cap))


def claw_regrid_transfer(ctx, level, old_boxes, q_old, q_new, q_coarse, stream=None):
    keep, ptr, n = _boxes_arg(old_boxes)
    _check("claw_regrid_transfer", load().claw_regrid_transfer(ctx, level, ptr, n, _ptr(q_old), _ptr(q_new),
                                                               _ptr(q_coarse), _stream(stream)))


def claw_reflux_count(ctx, fine_level):
    n = load().claw_reflux_count(ctx, fine_level)
    if n < 0:
        raise ClawError("claw_reflux_count", -n)
    return n


def claw_reflux_buffer_size(ctx, fine_level):
    n = load().claw_reflux_buffer_size(ctx, fine_level)
    if n < 0:
        raise ClawError("claw_reflux_buffer_size", -n)
    return n


def claw_reflux_coarse(ctx, fine_level, q_c_old, dt, buf, stream=None):
    _check("claw_reflux_coarse", load().claw_reflux_coarse(ctx, fine_level, _ptr(q_c_old), _ptr(dt), _ptr(buf),
                                                           _stream(stream)))


def claw_reflux_fine(ctx, fine_level, q_f, q_c_old, dt, buf, stream=None):
    _check("claw_reflux_fine", load().claw_reflux_fine(ctx, fine_level, _ptr(q_f), _ptr(q_c_old), _ptr(dt), _ptr(buf),
                                                       _stream(stream)))


def claw_reflux_apply(ctx, fine_level, buf, dt, q_c_new, stream=None):
    _check("claw_reflux_apply", load().claw_reflux_apply(ctx, fine_level, _ptr(buf), _ptr(dt), _ptr(q_c_new),
                                                         _stream(stream)))


def claw_medium_aux_adjoint(ctx, level, rho, K, g_aux, g_rho, g_K, stream=None):
    _check("claw_medium_aux_adjoint", load().claw_medium_aux_adjoint(
        ctx, level, _ptr(rho), _ptr(K), _ptr(g_aux), _ptr(g_rho), _ptr(g_K), _stream(stream)))


def claw_fill_ghost_interp(ctx, level, q, qc_old=None, qc_new=None, tau=0.0, stream=None):
    _check("claw_fill_ghost_interp", load().claw_fill_ghost_interp(ctx, level, _ptr(q), _ptr(qc_old), _ptr(qc_new),
                                                                   DBL(tau), _stream(stream)))


def claw_fill_ghost(ctx, level, q, qc_old=None, qc_new=None, tau=0.0, stream=None):
    _check("claw_fill_ghost", load().claw_fill_ghost(ctx, level, _ptr(q), _ptr(qc_old), _ptr(qc_new),
                                                     float(tau), _stream(stream)))


def claw_fill_ghost_adjoint(ctx, level, lam, lam_c_old=None, lam_c_new=None, qc_old=None, qc_new=None,
                            tau=0.0, stream=None):
    _check("claw_fill_ghost_adjoint", load().claw_fill_ghost_adjoint(
        ctx, level, _ptr(lam), _ptr(lam_c_old), _ptr(lam_c_new), _ptr(qc_old), _ptr(qc_new), float(tau),
        _stream(stream)))


def claw_fill_ghost_interp_adjoint(ctx, level, lam, lam_c_old=None, lam_c_new=None, qc_old=None, qc_new=None,
                                   tau=0.0, stream=None):
    _check("claw_fill_ghost_interp_adjoint", load().claw_fill_ghost_interp_adjoint(
        ctx, level, _ptr(lam), _ptr(lam_c_old), _ptr(lam_c_new), _ptr(qc_old), _ptr(qc_new), float(tau),
        _stream(stream)))


def claw_fill_ghost_coef(ctx, level, a, stream=None):
    _check("claw_fill_ghost_coef", load().claw_fill_ghost_coef(ctx, level, _ptr(a), _stream(stream)))


def claw_fill_ghost_coef_adjoint(ctx, level, g, stream=None):
    _check("claw_fill_ghost_coef_adjoint", load().claw_fill_ghost_coef_adjoint(ctx, level, _ptr(g), _stream(stream)))


def claw_cfl_max(ctx, level, aux, smax, stream=None):
    _check("claw_cfl_max", load().claw_cfl_max(ctx, level, _ptr(aux), _ptr(smax), _stream(stream)))


def claw_cfl_max_state(ctx, level, q, smax, stream=None):
    _check("claw_cfl_max_state", load().claw_cfl_max_state(ctx, level, _ptr(q), _ptr(smax), _stream(stream)))


def claw_dt_update(ctx, level, smax, dt, stream=None):
    _check("claw_dt_update", load().claw_dt_update(ctx, level, _ptr(smax), _ptr(dt), _stream(stream)))


def claw_level_step(ctx, level, q_old, q_new, aux, dt, smax, stream=None):
    _check("claw_level_step", load().claw_level_step(ctx, level, _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt),
                                                     _ptr(smax), _stream(stream)))


CLAW_ADVANCE_PUSH_GHOSTS = 1
CLAW_ADVANCE_PULL_GHOSTS = 4
CLAW_ADVANCE_UPDATE_DT = 2


def claw_packed_size(ctx, level):
    n = load().claw_packed_size(ctx, level)
    if n < 0:
        raise ClawError("claw_packed_size", -n)
    return n


def claw_pack_interiors(ctx, level, box_begin, box_end, q, packed, stream=None):
    _check("claw_pack_interiors", load().claw_pack_interiors(ctx, level, int(box_begin), int(box_end), _ptr(q),
                                                             _ptr(packed), _stream(stream)))


def claw_unpack_interiors(ctx, level, box_begin, box_end, packed, q, stream=None):
    _check("claw_unpack_interiors", load().claw_unpack_interiors(ctx, level, int(box_begin), int(box_end),
                                                                 _ptr(packed), _ptr(q), _stream(stream)))


def claw_level_advance_boxes(ctx, level, box_begin, box_end, q_old, q_new, aux, dt, smax, flags, stream=None):
    _check("claw_level_advance_boxes", load().claw_level_advance_boxes(
        ctx, level, int(box_begin), int(box_end), _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt), _ptr(smax),
        int(flags), _stream(stream)))


def claw_level_advance(ctx, level, q_old, q_new, aux, dt, smax, flags, stream=None):
    _check("claw_level_advance", load().claw_level_advance(
        ctx, level, _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt), _ptr(smax), int(flags), _stream(stream)))


def claw_level_advance_interp(ctx, level, q_old, q_new, aux, dt, smax, flags, qc_old=None, qc_new=None, tau=0.0,
                              stream=None):
    _check("claw_level_advance_interp", load().claw_level_advance_interp(
        ctx, level, _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt), _ptr(smax), int(flags), _ptr(qc_old), _ptr(qc_new),
        DBL(tau), _stream(stream)))


def claw_level_advance_fill(ctx, level, q_old, q_new, aux, dt, smax, flags, jobs=(), stream=None):
    """claw_level_advance plus, in the same launch, the interpolated-ghost fills `jobs`: tuples
    (fine level, pool, coarse old, coarse new, tau)"""
    arr = (claw_fill_job * max(len(jobs), 1))()
    for n, (lev, q, qc_old, qc_new, tau) in enumerate(jobs):
        arr[n] = claw_fill_job(int(lev), 0, _ptr(q), _ptr(qc_old), _ptr(qc_new), float(tau))
    _check("claw_level_advance_fill", load().claw_level_advance_fill(
        ctx, level, _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt), _ptr(smax), int(flags),
        ctypes.cast(arr, VP), len(jobs), _stream(stream)))


def claw_level_step_patchwise(ctx, level, q_old, q_new, aux, dt, smax, stream=None):
    _check("claw_level_step_patchwise", load().claw_level_step_patchwise(
        ctx, level, _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt), _ptr(smax), _stream(stream)))


def claw_level_step_noalloc(nx, ny, dx, dy, limiter, order, transverse, rho0, K0, q_old, q_new, aux, dt, smax,
                            stream=None):
    _check("claw_level_step_noalloc", load().claw_level_step_noalloc(
        nx, ny, float(dx), float(dy), limiter, order, transverse, float(rho0), float(K0), _ptr(q_old), _ptr(q_new),
        _ptr(aux), _ptr(dt), _ptr(smax), _stream(stream)))


def claw_average_down(ctx, fine_level, q_fine, q_coarse, stream=None):
    _check("claw_average_down", load().claw_average_down(ctx, fine_level, _ptr(q_fine), _ptr(q_coarse),
                                                         _stream(stream)))


def claw_average_down_adjoint(ctx, fine_level, lam_fine, lam_coarse, stream=None):
    _check("claw_average_down_adjoint", load().claw_average_down_adjoint(
        ctx, fine_level, _ptr(lam_fine), _ptr(lam_coarse), _stream(stream)))


def claw_level_step_adjoint(ctx, level, q_old, lam_new, lam_old, aux, g_aux, dt, stream=None):
    _check("claw_level_step_adjoint", load().claw_level_step_adjoint(
        ctx, level, _ptr(q_old), _ptr(lam_new), _ptr(lam_old), _ptr(aux), _ptr(g_aux), _ptr(dt),
        _stream(stream)))


def claw_level_advance_adjoint(ctx, level, q_old, lam_new, lam_old, aux, g_aux, dt, flags, stream=None):
    _check("claw_level_advance_adjoint", load().claw_level_advance_adjoint(
        ctx, level, _ptr(q_old), _ptr(lam_new), _ptr(lam_old), _ptr(aux), _ptr(g_aux), _ptr(dt), int(flags),
        _stream(stream)))


def claw_level_advance_record(ctx, level, q_old, q_new, aux, dt, smax, flags, tape, stream=None):
    _check("claw_level_advance_record", load().claw_level_advance_record(
        ctx, level, _ptr(q_old), _ptr(q_new), _ptr(aux), _ptr(dt), _ptr(smax), int(flags), _ptr(tape),
        _stream(stream)))


def claw_level_advance_adjoint_tape(ctx, level, tape, lam_new, lam_old, aux, g_aux, dt, flags, stream=None):
    _check("claw_level_advance_adjoint_tape", load().claw_level_advance_adjoint_tape(
        ctx, level, _ptr(tape), _ptr(lam_new), _ptr(lam_old), _ptr(aux), _ptr(g_aux), _ptr(dt), int(flags),
        _stream(stream)))


def claw_sync_status(ctx) -> int:
    return int(load().claw_sync_status(ctx))


def claw_launch_count(ctx) -> int:
    return int(load().claw_launch_count(ctx))
