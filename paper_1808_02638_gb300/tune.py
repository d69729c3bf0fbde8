"""Autotuner of the fused level-step's tiling (tile shape, threads per CTA, staging).

For each level it times every supported tiling of the fused launch on the level's own pools
(into a scratch q_new) with CUDA events, keeps the fastest, and caches the choice per
(medium, limiter, histogram of box sizes) in a JSON file next to the library, so that later
hierarchies with the same patch-size mix reuse it without timing.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

import torch

from . import claw

CANDIDATES = [(32, 32, 1, 256), (32, 32, 1, 512), (32, 32, 0, 256), (32, 32, 0, 512),
              (32, 16, 1, 256), (32, 16, 2, 256), (16, 16, 1, 128)]
CANDIDATES_SWE = [(16, 16, 1, 256), (16, 16, 0, 256), (32, 16, 1, 512), (32, 16, 0, 512)]


def candidates_for(H):
    """the tilings the level-step of H's system supports"""
    return CANDIDATES_SWE if getattr(H, "system", 0) == claw.CLAW_SYS_SHALLOW_WATER else CANDIDATES
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")
_lock = threading.Lock()


def _key(H, L):
    sizes = sorted(zip(H.boxes[L].nx.tolist(), H.boxes[L].ny.tolist()))
    hist = {}
    for s in sizes:
        hist[s] = hist.get(s, 0) + 1
    blob = json.dumps([H.medium, getattr(H, "system", 0), H.runs[0].limiter, H.runs[0].order, H.runs[0].transverse,
                       sorted((f"{a}x{b}", n) for (a, b), n in hist.items()),
                       torch.cuda.get_device_name(H.dev)])
    return hashlib.sha256(blob.encode()).hexdigest()[:24]


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def time_tiling(H, L, tiling, reps=5, pull=False):
    """mean device time (ms) of one fused launch of level L with `tiling` (pull: with the ghosts
    taken from their source cells, as the one-level fused path steps)"""
    flags = claw.CLAW_ADVANCE_PULL_GHOSTS if pull else 0
    tx, ty, staging, threads = tiling
    claw.claw_set_tiling(H.ctx, L, tx, ty, staging, threads)
    H.drop_graphs()
    src = H.q[L][H.cur[L]]
    dst = torch.empty_like(src)
    smax = torch.zeros_like(H.smax)
    for _ in range(2):
        claw.claw_level_advance(H.ctx, L, src, dst, H.aux[L], H.dt, smax, flags)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        claw.claw_level_advance(H.ctx, L, src, dst, H.aux[L], H.dt, smax, flags)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_level(H, L, use_cache=True, candidates=None, pull=False):
    """pick the fastest tiling for level L of hierarchy H, install it and return it with the
    timings (an empty dict when the choice came from the cache)"""
    key = _key(H, L) + ("-pull" if pull else "")
    if use_cache:
        with _lock:
            hit = _load().get(key)
        if hit:
            try:
                claw.claw_set_tiling(H.ctx, L, *hit)
                H.drop_graphs()
                return tuple(hit), {}
            except claw.ClawError:
                pass
    if float(H.dt.max()) <= 0.0:
        H.init_dt()
    timings = {}
    for c in candidates or candidates_for(H):
        try:
            timings[c] = time_tiling(H, L, c, pull=pull)
        except claw.ClawError:
            continue   # e.g. bulk-copy staging not allowed for this level
    best = min(timings, key=timings.get)
    claw.claw_set_tiling(H.ctx, L, *best)
    H.drop_graphs()
    with _lock:
        d = _load()
        d[key] = list(best)
        _save(d)
    return best, timings


def choose_pull(H, L, reps=5):
    """how level L of H gets its ghosts, timed with the installed tiling, the fastest recorded in
    H.pull_levels[L] and H.fuse_interp[L]: every ghost filled by the copy and interpolation
    launches before the step ("fill"), the interpolated ghosts filled (by spare CTAs of the launch
    before when H.fill_ahead, timed as a step launch carrying one such fill) and the others pulled
    by the step ("pull"), or one launch that pulls the copied ghosts and evaluates the
    interpolated ones ("pull+interp").  Small boxes put many ghosts in every tile's frame, where
    the separate launches can win."""
    src = H.q[L][H.cur[L]]
    dst = torch.empty_like(src)
    smax = torch.zeros_like(H.smax)
    qc = H.q[L - 1][H.cur[L - 1]] if L else None
    if float(H.dt.max()) <= 0.0:
        H.init_dt()
    flags = claw.CLAW_ADVANCE_PULL_GHOSTS

    def fill_step():
        claw.claw_fill_ghost(H.ctx, L, src, qc, qc, 0.0)
        claw.claw_level_step(H.ctx, L, src, dst, H.aux[L], H.dt, smax)

    def pull_step():
        if H.fill_ahead and L:   # the fill rides on the step launch before: one launch with its job
            claw.claw_level_advance_fill(H.ctx, L, src, dst, H.aux[L], H.dt, smax, flags, [(L, dst, qc, qc, 0.0)])
            return
        claw.claw_fill_ghost_interp(H.ctx, L, src, qc, qc, 0.0)
        claw.claw_level_advance(H.ctx, L, src, dst, H.aux[L], H.dt, smax, flags)

    def fused_step():
        claw.claw_level_advance_interp(H.ctx, L, src, dst, H.aux[L], H.dt, smax, flags, qc, qc, 0.0)

    options = (("fill", fill_step), ("pull", pull_step)) + ((("pull+interp", fused_step),) if L else ())
    times = {}
    for name, fn in options:
        fn()
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    H.pull_levels[L] = best != "fill"
    H.fuse_interp[L] = best == "pull+interp"
    H.drop_graphs()
    return H.pull_levels[L], times


def tune(H, use_cache=True):
    return [tune_level(H, L, use_cache) for L in range(H.nlev)]
