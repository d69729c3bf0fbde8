"""Benchmark of the fused batched FP64 level-step: 2048 x 2048 cells as 4096 patches of 32 x 32
(radial pulse, rho = 1, K = 4, MC limiter, transverse corrections, same-level ghost copy and
device CFL rule; one step = ghost fill + one persistent fused level-step + dt update, each a
CUDA graph replay).  Prints one JSON line (see the keys below).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl claw|reference]

N > 1 runs under torch.distributed.run, one rank per GPU, each advancing its own replica of
the workload (the path has no data exchange between independent runs): weak scaling.
--impl reference times the CPU oracle on the host cores on a bounded sample of the same
workload (same metric and unit).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the problem both arms time (the GPU arm adds its launch, the reference arm its sample)
WORKLOAD = ("2048x2048 cells on [-1,1]^2 as 4096 patches of 32x32 (+2 ghost layers), radial pulse, rho=1, "
            "K=4, MC limiter, transverse corrections, same-level ghosts, extrapolation boundaries, Eq. cfl "
            "time step")
METRIC = "FP64 cell-updates/s fused-batched vs plain per-patch launch; % of HBM peak"
UNIT = "cell-updates/s"
N_CELLS = 2048 * 2048
PATCH = 32
# Algorithmic FP64 work of one cell-update of the uniform-medium MC scheme with transverse
# corrections, every edge solved once (the halo edges a tile recomputes are not counted):
#   per x-edge and per y-edge  2 DADD + 2 DFMA (Riemann: dp, du, two wave strengths)
#                              4 DADD (two MC limiters, one add each; limited sum and difference)
#   per cell                   8 DADD + 10 DFMA (normal update with the centre transverse term,
#                              transverse pressures D, E)
#                              5 DADD + 3 DFMA (rest of the transverse update)
# = 25 DADD + 17 DFMA: 42 FP64-pipe instructions, 59 flops (an FMA counts 2).
ALG_FP64_INSTR_PER_CELL = 42
ALG_FLOPS_PER_CELL = 59
BYTES_PER_CELL = 48.0     # read q^n (p, u, v) + write q^{n+1}: algorithmic HBM traffic
# The FP64 pipe of the part issues 2 FP64 instructions (any of DADD, DMUL, DFMA) per SM per
# clock: 152 SMs x 2 x 2.07 GHz = 629 G instructions/s; 1.259 TFLOP/s if all were FMAs.
FP64_ISSUE_PEAK_G = 152 * 2 * 2.07
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.index = str(device)
        try:   # nvidia-smi numbering may differ from CUDA's: address the GPU by its UUID
            import torch
            u = str(torch.cuda.get_device_properties(device).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle leg
def _oracle_chunk(args):
    """oracle steps of a chunk of filled 32 x 32 patches (runs in a spawned worker)"""
    import numpy as np

    import oracle
    patches, dx, dt = args
    ones = np.ones((PATCH + 4, PATCH + 4))
    for qb in patches:
        oracle.step(qb, ones, 4.0 * ones, dx, dx, dt)
    return len(patches)


def oracle_sample(npatch: int):
    """the first `npatch` patches of the workload with their ghosts filled (host only)"""
    import numpy as np

    from paper_1808_02638_gb300 import inputs
    run = inputs.config1()
    lev = run.levels[0]
    glob = np.ones((3, 2048 + 4, 2048 + 4))
    x = run.xlo + (np.arange(-2, 2048 + 2) + 0.5) * lev.dx
    X, Y = np.meshgrid(x, x)
    glob[0] = inputs.radial_pulse(np.clip(X, x[2], x[-3]), np.clip(Y, x[2], x[-3]))
    glob[1:] = 0.0
    # patches spread evenly over the domain (the ring and the quiet background alike)
    stride = max(1, len(lev.boxes) // max(1, npatch))
    out = []
    for nb in range(0, len(lev.boxes), stride):
        ilo, jlo = int(lev.boxes[nb][0]), int(lev.boxes[nb][1])
        out.append(np.ascontiguousarray(glob[:, jlo:jlo + PATCH + 4, ilo:ilo + PATCH + 4]))
        if len(out) == npatch:
            break
    return out, lev.dx, 0.9 * lev.dx / 2.0


def time_oracle(npatch: int, workers: int, reps: int = 1):
    """wall time of the oracle on `npatch` patches with `workers` spawned processes"""
    import multiprocessing as mp

    import oracle
    oracle.build()
    patches, dx, dt = oracle_sample(npatch)
    chunks = [patches[k::workers] for k in range(workers)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_chunk, [(c[:1], dx, dt) for c in chunks])   # warm the workers
        times = []
        for _ in range(reps):
            t0 = time.perf_counter()
            pool.map(_oracle_chunk, [(c, dx, dt) for c in chunks])
            times.append(time.perf_counter() - t0)
    return len(patches) * PATCH * PATCH, times


STAGINGS = {0: "cooperative", 1: "tensor bulk-copy (two buffers)",
            2: "tensor bulk-copy (one buffer, three CTAs per SM)"}


def cpu_baseline(target_s: float = 15.0):
    workers = os.cpu_count() or 1
    # calibrate on one full level-step, then repeat it to fill ~target_s of wall time
    cells, t = time_oracle(4096, workers)
    reps = max(1, int(target_s / max(t[0], 1e-3)))
    cells, ts = time_oracle(4096, workers, reps=reps)
    wall = sum(ts)
    return {"value": cells * reps / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{reps} level-steps of all 4096 32x32 patches (ghosts filled, the same input each "
                      f"time), {workers} spawned worker processes each running the single-threaded C "
                      f"oracle on a share of the patches, {wall:.1f} s wall"}


def cpu_per_config():
    """single-threaded oracle rates on bounded samples of the other workloads (cell-updates/s)"""
    import numpy as np

    import oracle
    from oracle.amr import OracleHierarchy, run_single_grid
    from paper_1808_02638_gb300 import inputs
    oracle.build()
    out = {}

    def cells_per_coarse(run):
        tot, sub = 0, 1
        for L, lev in enumerate(run.levels):
            sub *= lev.ratio if L else 1
            tot += sub * sum(int(b[2]) * int(b[3]) for b in lev.boxes)
        return tot

    def single(name, run, rho, K, nsteps, sample):
        lev = run.levels[0]
        q = inputs.box_view(inputs.init_q(run, lev), 0, lev.NX, lev.NY, 3)
        t0 = time.perf_counter()
        run_single_grid(q, rho, K, lev.dx, lev.dy, nsteps, bc=run.bc)
        dt = time.perf_counter() - t0
        out[name] = {"value": lev.NX * lev.NY * nsteps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                     "sample": sample, "seconds": dt}

    def amr(name, run, rho, K, ncoarse, sample):
        q0 = [inputs.init_q(run, lev) for lev in run.levels]
        O = OracleHierarchy(run, q0, rho, K)
        t0 = time.perf_counter()
        for _ in range(ncoarse):
            O.coarse_step()
        dt = time.perf_counter() - t0
        out[name] = {"value": cells_per_coarse(run) * ncoarse / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                     "sample": sample, "seconds": dt}

    run = inputs.config0()
    one = np.ones((104, 104))
    single("c0", run, one, 4.0 * one, 50, "all 50 steps of the 100x100 grid")
    run = inputs.config2()
    amr("c2", run, [inputs.const_pool(l, 1.0) for l in run.levels], [inputs.const_pool(l, 4.0) for l in run.levels],
        2, "2 of the 20 coarse steps of the 3-level hierarchy")
    run, r2, k2 = inputs.config3(256)
    lev = run.levels[0]
    rho = inputs.box_view(inputs.coef_pool(lev, r2, 1), 0, 256, 256, 1)[0]
    K = inputs.box_view(inputs.coef_pool(lev, k2, 1), 0, 256, 256, 1)[0]
    single("c3", run, rho, K, 20, "20 of the 400 forward steps of the 256x256 heterogeneous grid")
    run, r2, k2 = inputs.config4_runs(1)[0]
    amr("c4", run, [inputs.coef_pool(l, r2, 4 ** L) for L, l in enumerate(run.levels)],
        [inputs.coef_pool(l, k2, 4 ** L) for L, l in enumerate(run.levels)], 1,
        "1 coarse step of the first of the 64 runs")
    # shallow water: 64 of the 4096 32x32 patches of the 2048^2 workload, one step each
    run = inputs.config1()
    lev = run.levels[0]
    qs = inputs.init_swe(run, lev)
    t0 = time.perf_counter()
    for nb in range(64):
        qb = inputs.box_view(qs, lev.qoff[nb], 32, 32, 3).copy()
        oracle.swe_step(qb, lev.dx, lev.dy, 5e-4, 1.0)
    dt = time.perf_counter() - t0
    out["swe1"] = {"value": 64 * 32 * 32 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "one step of 64 of the 4096 32x32 patches of the shallow-water workload",
                   "seconds": dt}
    return out


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    cells, t = time_oracle(8 * workers, workers)
    rate = cells / max(t[0], 1e-9)
    # each step: a bounded sample sized so that warmup + steps stay within ~2 minutes
    per_step_s = min(10.0, 120.0 / max(1, args.steps + args.warmup))
    npatch = int(min(4096, max(workers, rate * per_step_s / (PATCH * PATCH))))
    _, tw = time_oracle(npatch, workers, reps=args.warmup)
    cells, ts = time_oracle(npatch, workers, reps=args.steps)
    total = sum(ts)
    value = cells * len(ts) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": N_CELLS,
                       "parallelism": f"{workers} host processes",
                       "launch": f"the C oracle on {npatch} of the 4096 patches per step (a bounded sample of "
                                 f"the level-step; ghosts filled, the same input each step)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"{npatch} of the 4096 patches per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU leg
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="claw", choices=["claw", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the per-workload measurements (0, 2, 3 with its adjoint, 4 with its adjoint)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_1808_02638_gb300 import claw, inputs, replicas
    from paper_1808_02638_gb300.build import build
    from paper_1808_02638_gb300.solver import Hierarchy

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build()
    replicas.barrier(dist)
    build()   # no-op once built

    run = inputs.config1()
    lev = run.levels[0]
    q0 = inputs.init_q(run, lev)
    H = Hierarchy([run], [[q0]], rho0=1.0, K0=4.0, device=local)
    H.init_dt()
    from paper_1808_02638_gb300 import tune
    tiling, tune_ms = tune.tune_level(H, 0, use_cache=False, pull=True)
    stream = torch.cuda.current_stream()
    ctx = H.ctx
    H.coarse_step()
    H.coarse_step()
    torch.cuda.synchronize()

    # per buffer parity one graph: the persistent level-step launch that advances every patch,
    # takes the same-level / boundary ghosts from their source cells and applies Eq. cfl on its
    # last CTA; events bracket each replay so the kernel is timed on its launching stream
    stepper = H.fused_stepper()
    per_step_launches = stepper.launches_per_step

    def one_step(k, ev=None):
        stepper.step(ev)

    for k in range(args.warmup):
        one_step(k)
    torch.cuda.synchronize()

    K = args.steps
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(2)) for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    replicas.barrier(dist)
    torch.cuda.synchronize()
    start.record()
    for k in range(K):
        one_step(args.warmup + k, evs[k])
    end.record()
    torch.cuda.synchronize()
    replicas.barrier(dist)
    clocks = sampler.stop()
    kern_ms = [a.elapsed_time(b) for a, b in evs]
    # every rank advances its own replica: the job's cell-updates over its slowest rank's time
    dev = torch.device("cuda", local)
    value, total_ms, _ = replicas.whole_job_rate(K * N_CELLS, start.elapsed_time(end), dist, dev)
    status = H.sync_status()
    kern_avg_s = statistics.mean(kern_ms) * 1e-3

    # plain path: one launch per patch (4096 launches per level-step), eager, same stream
    plain = None
    if args.plain_steps > 0:
        H.patchwise = True
        H.coarse_step()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record()
        for _ in range(args.plain_steps):
            H.coarse_step()
        p1.record()
        torch.cuda.synchronize()
        H.patchwise = False
        pv = args.plain_steps * N_CELLS / (p0.elapsed_time(p1) * 1e-3)
        plain = {"value": pv, "unit": UNIT, "launches_per_step": len(lev.boxes) + 2,
                 "path": "ghost fill + one launch per patch (4096) + dt update, eager",
                 "fused_over_plain": value / world / pv}

    # end to end: the state lives on the host (pinned); every step copies q in, runs the
    # level-step through the C ABI and copies q^{n+1} back (Hierarchy.steps_from_host: the level
    # is stepped in pieces of boxes as they arrive, so copies in both directions and the steps
    # overlap)
    H.fused = True          # one launch per step, ghosts pulled from their source cells
    e2e_steps = max(3, min(100, K // 2))
    # the host holds the state in packed form (interiors only, 3 x 2048^2 doubles): the bytes
    # each way per step
    host_in = H.pack().cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    qbytes = host_in.numel() * 8
    H.steps_from_host(host_in, host_out, 2)   # warm-up: piece tables, streams, events
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    H.steps_from_host(host_in, host_out, e2e_steps)
    e1.record()
    torch.cuda.synchronize()
    e2e_value, _, _ = replicas.whole_job_rate(e2e_steps * N_CELLS, e0.elapsed_time(e1), dist, dev)
    # the copy bound of that loop: qbytes each way per step at the measured pinned-copy rates
    # (each direction alone, and the aggregate of both at once)
    from paper_1808_02638_gb300 import measure as _m
    copies = _m.host_copy_bandwidth(device=dev.index if dev.index is not None else 0)
    bound_s = max(qbytes / (copies["h2d_gbs"] * 1e9), qbytes / (copies["d2h_gbs"] * 1e9),
                  2 * qbytes / (copies["both_gbs"] * 1e9))
    copy_bound = world * N_CELLS / bound_s

    per_config = None
    if rank == 0 and not args.no_configs:
        from paper_1808_02638_gb300 import measure
        per_config = measure.run_all()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    achieved_gops = ALG_FP64_INSTR_PER_CELL * N_CELLS / kern_avg_s / 1e9
    achieved_tflops = ALG_FLOPS_PER_CELL * N_CELLS / kern_avg_s / 1e12
    achieved_gbs = BYTES_PER_CELL * N_CELLS / kern_avg_s / 1e9
    # DRAM traffic of one launch from the last profiler capture, only while the kernel source
    # is unchanged since that capture
    traffic = None
    tf = os.path.join(ROOT, "profiles", "step_uniform_2048x2048_traffic.json")
    if os.path.exists(tf):
        try:
            import hashlib
            rec = json.load(open(tf))
            src = open(os.path.join(ROOT, "paper_1808_02638_gb300", "csrc", "claw_step.cuh"), "rb").read()
            if hashlib.sha256(src).hexdigest()[:16] == rec.get("source_sha256_16"):
                traffic = rec.get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "global_batch": world * N_CELLS, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (254 MB of q pools per replica)",
                   "launch": "per step one persistent level-step launch (ghosts pulled, Eq. cfl on its last "
                             "CTA) replayed from a CUDA graph"},
        "step": "one CUDA-graph replay of the persistent level-step launch (all 4096 patches, each tile's "
                "ghosts pulled from their source cells, Eq. cfl on the last CTA)",
        "ghosts": "pulled by the step kernel from their source cells (no ghost-copy launch)",
        "roofline": {"bound": "alu", "achieved": achieved_gops, "peak": FP64_ISSUE_PEAK_G,
                     "unit": "G FP64 instructions/s", "frac": achieved_gops / FP64_ISSUE_PEAK_G, "traffic": traffic,
                     "per_cell_update": f"{ALG_FP64_INSTR_PER_CELL} FP64 instructions (25 DADD + 17 DFMA), "
                                        f"{ALG_FLOPS_PER_CELL} flops, {BYTES_PER_CELL:.0f} B",
                     "kernel": "level-step (uniform medium, MC), autotuned tiling "
                               f"{tiling[0]}x{tiling[1]} tiles, {tiling[3]} threads, "
                               f"{STAGINGS[tiling[2]]} staging",
                     "kernel_ms": kern_avg_s * 1e3,
                     "peak_source": "FP64 pipe: 152 SMs x 2 instructions/clk x 2.07 GHz (derived; independent "
                                    "DFMA, DADD or DMUL loops measured 1.684 per SM per clk, 530 G/s)",
                     "flops": {"achieved_tflops": achieved_tflops, "peak_tflops": FP64_PEAK_TFLOPS,
                               "frac": achieved_tflops / FP64_PEAK_TFLOPS}},
        "hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": hbm, "frac": achieved_gbs / hbm,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"},
        "plain_per_patch": plain,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": qbytes, "d2h_bytes_per_step": qbytes,
                "copy_bound": copy_bound, "frac_of_copy_bound": e2e_value / copy_bound, "host_copies": copies,
                "note": "copy bound = cell-updates per step / max(bytes/h2d, bytes/d2h, 2 bytes/both) with the "
                        "host_copies rates measured in this run"},
        "gpu_launches": per_step_launches * K,
        "tuning_ms": {f"{a}x{b}/s{c}/t{d}": round(v, 4) for (a, b, c, d), v in tune_ms.items()},
        "clocks": clocks,
        "status": claw.strerror(status),
        "adjoint": per_config["c3"]["adjoint"] if per_config else None,
        "adjoint_tape": per_config["c3"]["adjoint_tape"] if per_config else None,
        "per_config": per_config,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["per_config"] = cpu_per_config()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
