"""Per-workload GPU measurements: the fused batched level-steps (CUDA-graph replays) against the
plain path (one launch per patch, eager) on the same hierarchy, and the adjoint's cost.

  python -m paper_1808_02638_gb300.measure [names...] [--nruns N] [--ncoarse N] [--every N] [--no-plain]

(names: c0 c2 c3 c4 e1 swe1 swe2; default all; the options shrink the batched workload for a profiler)

Each workload reports interior cell-updates per second (a cell advanced one step on its level;
ghost cells and halo recomputation are not counted), algorithmic HBM bytes per second (q read
and written, 48 B per cell-update; 64 B with the cell-wise medium's rho, K), the fraction of the
measured copy bandwidth, and the fraction of the FP64 pipe's issue rate used by the algorithmic
FP64 instructions of the step (42 per cell-update uniform, 78 cell-wise, 324 shallow water; the
kernel sources state how they are counted).  Times are CUDA events around graph replays of whole coarse steps
(ghost fill, every level-step with its substeps, averaging, the Eq. cfl update).
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np
import torch

from . import claw, inputs
from .solver import Hierarchy

FP64_INSTR_UNIFORM = 42
FP64_INSTR_CELLWISE = 78
FP64_INSTR_SWE = 324     # shallow water, Roe solvers (claw_step_swe.cu states the count)
BYTES_UNIFORM = 48.0
BYTES_CELLWISE = 64.0
FP64_ISSUE_PEAK_G = 152 * 2 * 2.07   # G FP64 instructions / s: 152 SMs x 2 per clock x 2.07 GHz


def _hbm_peak():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(root, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def cell_updates_per_coarse_step(H):
    total = 0
    for run in H.runs:
        sub = 1
        for L, lev in enumerate(run.levels):
            if L:
                sub *= lev.ratio
            total += sub * sum(int(b[2]) * int(b[3]) for b in lev.boxes)
    return total


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def tune_all(H, pull=False):
    """autotuned tiling of every level (installed on H), keyed by level (pull: timed with the
    ghosts taken from their source cells, as the one-level fused stepper runs); for the coarse
    steps of a hierarchy, also whether each level pulls its copied ghosts or fills them first"""
    from . import tune
    out = {str(L): list(tune.tune_level(H, L, use_cache=False, pull=pull)[0]) for L in range(H.nlev)}
    if not pull:
        for L in range(H.nlev):
            tune.choose_pull(H, L)
            out[str(L)].append("pull+interp" if H.fuse_interp[L] else "pull" if H.pull_levels[L] else "fill")
    return out


def time_fused(H, ncoarse, warm=2):
    """ms per coarse step over graph replays of two coarse steps"""
    H.coarse_step()
    H.coarse_step()
    g = H.capture(2)
    for _ in range(warm):
        g.replay()
    torch.cuda.synchronize()
    reps = max(1, ncoarse // 2)
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (2 * reps)


def time_plain(H, ncoarse):
    """ms per coarse step with one eager launch per patch per level-step"""
    H.patchwise = True
    try:
        H.coarse_step()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        for _ in range(ncoarse):
            H.coarse_step()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / ncoarse
    finally:
        H.patchwise = False


def _report(name, H, ms, plain_ms, fp64_per_cell, bytes_per_cell, extra=None):
    hbm, hbm_src = _hbm_peak()
    cells = cell_updates_per_coarse_step(H)
    rate = cells / (ms * 1e-3)
    gbs = rate * bytes_per_cell / 1e9
    gops = rate * fp64_per_cell / 1e9
    out = {"workload": name, "cell_updates_per_coarse_step": cells, "ms_per_coarse_step": ms,
           "cell_updates_per_s": rate, "alg_gbs": gbs, "hbm_frac": gbs / hbm, "hbm_peak_source": hbm_src,
           "fp64_gops": gops, "fp64_issue_frac": gops / FP64_ISSUE_PEAK_G,
           "launches_per_coarse_step": H.launches_per_coarse_step(), "status": claw.strerror(H.sync_status())}
    if plain_ms is not None:
        out["plain_ms_per_coarse_step"] = plain_ms
        out["plain_cell_updates_per_s"] = cells / (plain_ms * 1e-3)
        out["fused_over_plain"] = plain_ms / ms
    if extra:
        out.update(extra)
    return out


# ----------------------------------------------------------------- workloads
def config0():
    run = inputs.config0()
    H = Hierarchy([run], [[inputs.init_q(run, run.levels[0])]], rho0=1.0, K0=4.0)
    H.init_dt()
    tiling = tune_all(H, pull=True)
    ms = time_stepper(H, 50)
    plain = time_plain(H, 10)
    return _report("100x100 single grid, radial pulse, rho=1, K=4, MC, 50 steps", H, ms, plain,
                   FP64_INSTR_UNIFORM, BYTES_UNIFORM, {"l2": "L2-resident (0.3 MB)", "tiling": tiling,
                                                       "path": "one launch per step (pulled ghosts)"})


def config2():
    run = inputs.config2()
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0)
    H.init_dt()
    tiling = tune_all(H)
    ms = time_fused(H, 20)
    plain = time_plain(H, 2)
    boxes = [len(l.boxes) for l in run.levels]
    # the same hierarchy with the conservation fix of Sec. 2.3 (same tilings)
    R = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True)
    for L, t in tiling.items():
        claw.claw_set_tiling(R.ctx, int(L), *t[:4])
    R.init_dt()
    ms_r = time_fused(R, 20)
    nrec = [claw.claw_reflux_count(R.ctx, L) for L in range(1, R.nlev)]
    return _report("3-level AMR, 64^2 base, ratio 4 twice, seeded 8..64 patches on the annuli "
                   f"(boxes per level {boxes}), radial pulse, rho=1, K=4, 20 coarse steps",
                   H, ms, plain, FP64_INSTR_UNIFORM, BYTES_UNIFORM,
                   {"l2": "L2-resident (about 30 MB)", "tiling": tiling,
                    "reflux": {"ms_per_coarse_step": ms_r, "overhead": ms_r / ms - 1.0,
                               "interface_records_per_level": nrec,
                               "launches_per_coarse_step": R.launches_per_coarse_step()}})


def _cellwise_single(n):
    run, r2, k2 = inputs.config3(n)
    lev = run.levels[0]
    q = inputs.init_q(run, lev)
    rho, K = inputs.coef_pool(lev, r2, 1), inputs.coef_pool(lev, k2, 1)
    return run, q, rho, K


def _tensors(H, pools, kind):
    """per-level device copies of the per-run pools (requires_grad), in the hierarchy's layout"""
    out = []
    for L in range(H.nlev):
        ref = H.q[L][0] if kind == "q" else H.rho[L]
        a = np.zeros(ref.numel()) if kind == "q" else np.ones(ref.numel())
        for (ri, qb, cb) in H.layout[L]:
            base = qb if kind == "q" else cb
            p = pools[ri][L]
            a[base:base + p.size] = p
        out.append(torch.from_numpy(a).to(ref.device).requires_grad_(True))
    return out


def _receiver_energy(H, outs):
    """sum over runs of sum p^2 over each run's 16 x 16 level-0 receiver box"""
    J = 0.0
    for ri, run in enumerate(H.runs):
        lev = run.levels[0]
        qbase = [qb for (r, qb, _) in H.layout[0] if r == ri][0]
        nx, ny = int(lev.boxes[0][2]), int(lev.boxes[0][3])
        i0, j0, n = inputs.receiver_box(nx)
        v = outs[0][qbase:qbase + 3 * (nx + 4) * (ny + 4)].view(3, ny + 4, nx + 4)
        J = J + (v[0, 2 + j0:2 + j0 + n, 2 + i0:2 + i0 + n] ** 2).sum()
    return J


def time_adjoint(H, q, rho, K, ncoarse, every, passes=2):
    """(forward ms, backward ms, gradients finite) of a checkpointed rollout (every=None: with the
    recorded tape) and its reverse sweep (eager launches); the last of `passes` passes is
    reported (the first warms up)"""
    from .adjoint import rollout
    for _ in range(passes):
        tq, tr, tk = _tensors(H, q, "q"), _tensors(H, rho, "c"), _tensors(H, K, "c")
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record()
        outs = rollout(H, tq, tr, tk, ncoarse=ncoarse, every=every)
        J = _receiver_energy(H, outs)
        e1.record()
        torch.cuda.synchronize()
        b0, b1 = _events()
        b0.record()
        J.backward()
        b1.record()
        torch.cuda.synchronize()
    finite = all(bool(torch.isfinite(t.grad).all()) for t in tq + tr + tk)
    return e0.elapsed_time(e1), b0.elapsed_time(b1), finite


def config3(nsteps=400, every=20):
    run, q, rho, K = _cellwise_single(256)
    H = Hierarchy([run], [[q]], [[rho]], [[K]])
    H.init_dt()
    tiling = tune_all(H, pull=True)
    ms = time_stepper(H, 40)
    H.init_dt()
    fwd, bwd, ok = time_adjoint(H, [[q]], [[rho]], [[K]], nsteps, every)
    H.drop_graphs(buffers=True)   # the segment tapes, before the whole-rollout tape
    tf, tb, tok = time_adjoint(H, [[q]], [[rho]], [[K]], nsteps, None)
    return _report("256x256 heterogeneous medium, 400 steps, checkpoints every 20, J = sum p^2 over the "
                   "16x16 receiver", H, ms, None, FP64_INSTR_CELLWISE, BYTES_CELLWISE,
                   {"tiling": tiling, "path": "one launch per step (pulled ghosts)",
                    "adjoint": {"forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
                                "gradients_finite": ok,
                                "note": "eager launches; backward = segment recompute + adjoint steps"},
                    "adjoint_tape": {"forward_ms": tf, "backward_ms": tb, "backward_over_forward": tb / tf,
                                     "gradients_finite": tok,
                                     "note": "the forward records every level-step's input (HBM); "
                                             "backward = adjoint steps only"}})


def config4(nruns=64, ncoarse=100, every=20, plain=True):
    runs = inputs.config4_runs(nruns)
    qs = [[inputs.init_q(run, lev) for lev in run.levels] for run, _, _ in runs]
    rhos = [[inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(run.levels)] for run, r2, _ in runs]
    Ks = [[inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(run.levels)] for run, _, k2 in runs]
    H = Hierarchy([r for r, _, _ in runs], qs, rhos, Ks)
    H.init_dt()
    tiling = tune_all(H)
    ms = time_fused(H, 20)
    plain = time_plain(H, 2) if plain else None
    H.init_dt()
    fwd, bwd, ok = time_adjoint(H, qs, rhos, Ks, ncoarse, every)
    H.drop_graphs(buffers=True)   # the segment tapes, before the whole-rollout tape
    H.init_dt()
    tf, tb, tok = time_adjoint(H, qs, rhos, Ks, ncoarse, None)
    nbox = [sum(len(r.levels[L].boxes) for r, _, _ in runs) for L in range(2)]
    return _report(f"{nruns} independent 2-level runs (N in [64,256], ratio 4 on seeded annuli; boxes per "
                   f"level {nbox}), per-run heterogeneous media, all runs in one launch per level-step",
                   H, ms, plain, FP64_INSTR_CELLWISE, BYTES_CELLWISE,
                   {"tiling": tiling,
                    "adjoint": {"coarse_steps": ncoarse, "every": every, "forward_ms": fwd, "backward_ms": bwd,
                                "backward_over_forward": bwd / fwd, "gradients_finite": ok,
                                "functional": "sum over runs of sum p^2 over each run's 16x16 receiver"},
                    "adjoint_tape": {"forward_ms": tf, "backward_ms": tb, "backward_over_forward": tb / tf,
                                     "gradients_finite": tok,
                                     "note": "the forward records every level-step's input (HBM); "
                                             "backward = adjoint steps only"}})


def host_copy_bandwidth(nbytes=100 * 2 ** 20, reps=20, device=0):
    """Pinned host <-> device copy rates (GB/s) with CUDA events: host to device alone, device to
    host alone, and both at once on two streams (the aggregate bytes of both directions over the
    time both take), each over `reps` copies of `nbytes` after two warm-up copies."""
    dev = torch.device("cuda", device)
    n = nbytes // 8
    h_in = torch.empty(n, dtype=torch.float64).pin_memory()
    h_out = torch.empty(n, dtype=torch.float64).pin_memory()
    d_a = torch.empty(n, dtype=torch.float64, device=dev)
    d_b = torch.empty(n, dtype=torch.float64, device=dev)
    h_in.fill_(1.0)
    d_b.fill_(2.0)
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = _events()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) * 1e-3

    def h2d():
        d_a.copy_(h_in, non_blocking=True)

    def d2h():
        h_out.copy_(d_b, non_blocking=True)

    def both():
        cur = torch.cuda.current_stream(dev)
        s_in.wait_stream(cur)
        s_out.wait_stream(cur)
        with torch.cuda.stream(s_in):
            d_a.copy_(h_in, non_blocking=True)
        with torch.cuda.stream(s_out):
            h_out.copy_(d_b, non_blocking=True)
        cur.wait_stream(s_in)
        cur.wait_stream(s_out)

    t_in, t_out, t_both = timed(h2d), timed(d2h), timed(both)
    return {"bytes": nbytes, "reps": reps, "h2d_gbs": reps * nbytes / t_in / 1e9,
            "d2h_gbs": reps * nbytes / t_out / 1e9, "both_gbs": 2 * reps * nbytes / t_both / 1e9,
            "method": "pinned host memory, CUDA events around reps copies on the current stream (both: "
                      "one copy each way per rep on two streams)"}


def time_stepper(H, nsteps, warm=3):
    """ms per step of a one-level hierarchy through its fused stepper (graph replays of the
    persistent step with the device Eq. cfl update, then of the ghost copy)"""
    st = H.fused_stepper()
    for _ in range(warm):
        st.step()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(nsteps):
        st.step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / nsteps


def swe1(nsteps=50, n=2048):
    """The second system through the same path: shallow water (g = 1) on the bench's 2048^2 as
    4096 patches of 32^2, the ring pulse as depth (1 <= h <= 2), at rest, MC, transverse 2."""
    run = inputs.config1(n)
    H = Hierarchy([run], [[inputs.init_swe(run, run.levels[0])]], system="shallow_water", grav=1.0)
    H.init_dt()
    tiling = tune_all(H, pull=True)
    ms = time_stepper(H, nsteps)
    plain = time_plain(H, 5)
    return _report(f"shallow water, {n}^2 as {(n // 32) ** 2} patches of 32^2, ring-pulse depth, g = 1, MC, "
                   f"{nsteps} steps", H, ms, plain, FP64_INSTR_SWE, BYTES_UNIFORM,
                   {"l2": "streams from HBM (254 MB of q pools)", "tiling": tiling,
                    "dt_final": float(H.dt[0])})


def swe2():
    """Shallow water through the AMR path: config 2's 3-level hierarchy (ratio 4 twice) with the
    ring as depth and a mean flow (0.2, 0.1), with and without the conservation fix."""
    run = inputs.config2()
    q0 = [inputs.init_swe(run, lev, u0=0.2, v0=0.1) for lev in run.levels]
    H = Hierarchy([run], [q0], system="shallow_water", grav=1.0)
    H.init_dt()
    tiling = tune_all(H)
    ms = time_fused(H, 20)
    plain = time_plain(H, 2)
    R = Hierarchy([run], [q0], system="shallow_water", grav=1.0, reflux=True)
    for L, t in tiling.items():
        claw.claw_set_tiling(R.ctx, int(L), *t[:4])
    R.init_dt()
    ms_r = time_fused(R, 20)
    boxes = [len(l.boxes) for l in run.levels]
    return _report(f"shallow water, 3-level AMR (boxes per level {boxes}), ring depth with a mean flow, "
                   "20 coarse steps", H, ms, plain, FP64_INSTR_SWE, BYTES_UNIFORM,
                   {"l2": "L2-resident", "tiling": tiling,
                    "reflux": {"ms_per_coarse_step": ms_r, "overhead": ms_r / ms - 1.0,
                               "launches_per_coarse_step": R.launches_per_coarse_step(),
                               "status": claw.strerror(R.sync_status())}})


def e1(ncoarse=200, base=1000, nlev=3, ratio=2, cutoff=0.7, regrid_every=8, tol=0.002, max_size=260,
       reflux=True, per_patch=False, tiling=((32, 16, 2, 256), (16, 16, 1, 128))):
    """Analog of the paper's benchmark (Sec. 4.1-4.2): radial pulse in a uniform medium, outflow
    (extrapolation) boundaries, van Leer, 3 levels of ratio 2 over a 1000^2 base tiled in 4 x 4
    patches of 250^2, patches of at most 260^2 generated by regridding (tol on neighbour
    differences, buffer = regrid interval, cutoff 0.7, every 8 coarse steps), the conservation
    fix on; the fine levels are built at t = 0 by regridding and set from the initial condition.
    Times whole coarse steps (eager launches: the hierarchy changes every regrid) including the
    regrids, and splits the time into the sections of the paper's Fig. 4: advancing the solution
    (with the conservation fix's flux records), ghost fill, regridding, updating (averaging and
    the fix's corrections) and the rest.  per_patch: one step launch per patch instead of the
    batched launch (the paper's launch pattern).  tiling: (tx, ty, staging, threads) per level,
    kept through the regrids (default: 32 x 16 tiles on the base level's 250^2 patches, 16 x 16 on
    the finer levels' smaller ones, the faster choices in a trial of five tilings)."""
    import time
    run = inputs.Run(*inputs.PULSE_DOMAIN, limiter=3)
    d0 = 2.0 / base
    step = base // 4
    b0 = [(i, j, step, step) for j in range(0, base, step) for i in range(0, base, step)]
    run.levels = [inputs.Level(base, base, d0, d0, b0)]
    for L in range(1, nlev):
        n = base * ratio ** L
        run.levels.append(inputs.Level(n, n, 2.0 / n, 2.0 / n, np.zeros((0, 4), dtype=np.int32), ratio))
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=reflux, tiling=tiling)
    H.patchwise = bool(per_patch)
    params = dict(tol=tol, buffer=regrid_every, cutoff=cutoff, max_size=max_size, nest=2)
    for _ in range(nlev - 1):       # refine level by level at t = 0
        H.regrid(**params)
    for L, lev in enumerate(run.levels):   # the new levels take the initial condition itself
        a = inputs.init_q(run, lev)
        t = H.q[L][H.cur[L]]
        t.zero_()
        t[:a.size] = torch.from_numpy(a).to(t.device)
    H.init_dt()
    torch.cuda.synchronize()
    H.sections = []
    cells = 0
    patches = 0
    regrid_s = 0.0
    t0 = time.perf_counter()
    for k in range(ncoarse):
        cells += cell_updates_per_coarse_step(H)
        patches += sum(len(lev.boxes) for lev in run.levels)
        H.coarse_step()
        if (k + 1) % regrid_every == 0:
            torch.cuda.synchronize()
            r0 = time.perf_counter()
            H.regrid(**params)
            torch.cuda.synchronize()
            regrid_s += time.perf_counter() - r0
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    sec = H.section_ms()
    H.sections = None
    sections = {"advance": sec.get("advance", 0.0) / 1e3, "ghost_fill": sec.get("fill", 0.0) / 1e3,
                "regrid": regrid_s, "updating": sec.get("update", 0.0) / 1e3}
    sections["other"] = wall - sum(sections.values())
    sections["total"] = wall
    boxes = [len(lev.boxes) for lev in run.levels]
    ncells = [int(lev.ncells) for lev in run.levels]
    status = claw.strerror(H.sync_status())
    H.close()
    return {"workload": f"{base}^2 base, {nlev} levels of ratio {ratio}, patches <= {max_size}^2 by regridding "
                        f"(tol {tol}, cutoff {cutoff}, every {regrid_every} coarse steps), van Leer, radial pulse, "
                        f"conservation fix {'on' if reflux else 'off'}, {ncoarse} coarse steps, "
                        f"{'one launch per patch' if per_patch else 'batched level-step launches'}",
            "coarse_steps": ncoarse, "simulated_time": float(ncoarse) * float(H.dt[0]),
            "cell_updates": cells, "wall_s": wall, "cell_updates_per_s": cells / wall,
            "mean_patches_per_coarse_step": patches / ncoarse,
            "regrid_s": regrid_s, "regrids": ncoarse // regrid_every,
            "sections_s": sections,
            "final_boxes_per_level": boxes, "final_cells_per_level": ncells,
            "status": status,
            "note": "eager launches (the hierarchy changes at every regrid); wall clock includes the regrids; "
                    "advance, ghost fill and updating are CUDA-event spans, regrid is host wall time with "
                    "synchronisation, other = total - the rest"}


def e3(ncoarse=200, cutoffs=(0.5, 0.7, 0.9), intervals=(2, 8, 16), paths=("batched", "per_patch"), tiling=None):
    """Analog of the paper's parameter study (Sec. 4.3): the benchmark analog for every cutoff x
    regrid interval, with the batched level-step launch and with one launch per patch.  Per
    combination: cells advanced, mean patches over all levels per coarse step, and the time of
    each section (Figs. 5-7).  tiling: as in e1 (default here: the library's 32 x 32 tiles)."""
    rows = []
    for cutoff in cutoffs:
        for every in intervals:
            for path in paths:
                r = e1(ncoarse, cutoff=cutoff, regrid_every=every, per_patch=(path == "per_patch"), tiling=tiling)
                rows.append({"cutoff": cutoff, "regrid_interval": every, "path": path,
                             "cell_updates": r["cell_updates"],
                             "mean_patches_per_coarse_step": r["mean_patches_per_coarse_step"],
                             "sections_s": {k: round(v, 4) for k, v in r["sections_s"].items()},
                             "cell_updates_per_s": r["cell_updates_per_s"], "status": r["status"]})
                torch.cuda.empty_cache()
    return {"workload": f"benchmark analog (1000^2 base, 3 levels of ratio 2, van Leer, conservation fix), "
                        f"{ncoarse} coarse steps per combination",
            "runs": rows}


WORKLOADS = {"c0": config0, "c2": config2, "c3": config3, "c4": config4, "e1": e1, "swe1": swe1, "swe2": swe2}
# (bench.py reports every workload above; e1 runs 200 coarse steps there)
SWEEPS = {"e3": e3}   # run on request only: python -m paper_1808_02638_gb300.measure e3


def run_all(names=None):
    out = {}
    for name in names or WORKLOADS:
        out[name] = WORKLOADS[name]()
        torch.cuda.empty_cache()
    return out


def main():
    import argparse
    from .build import build
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*")
    ap.add_argument("--nruns", type=int, default=64)
    ap.add_argument("--ncoarse", type=int, default=100)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--no-plain", action="store_true")
    a = ap.parse_args()
    build()
    torch.cuda.set_device(0)
    if a.names == ["c4"]:
        print(json.dumps({"c4": config4(a.nruns, a.ncoarse, a.every, not a.no_plain)}, indent=1))
    elif a.names and all(n in SWEEPS for n in a.names):
        print(json.dumps({n: SWEEPS[n]() for n in a.names}, indent=1))
    else:
        print(json.dumps(run_all(a.names or None), indent=1))


if __name__ == "__main__":
    main()
