"""Profiling driver: a few eager level-steps of the 2048 x 2048 workload as 4096 patches of
32 x 32, for a profiler to capture single kernel launches.

  python -m paper_1808_02638_gb300.profile_step [uniform|cellwise|swe] [nsteps] [fused|split] [tx,ty,staging,threads] [limiter] [walk]
  python -m paper_1808_02638_gb300.profile_step adjoint [nruns] [ncoarse] [every]
  python -m paper_1808_02638_gb300.profile_step regrid [ncoarse]
  python -m paper_1808_02638_gb300.profile_step amr [ncoarse]

adjoint: the first `nruns` runs of the batched two-level workload (cell-wise media), autotuned,
a checkpointed rollout of `ncoarse` coarse steps and its reverse sweep, twice; the second
reverse sweep (recording steps and tape adjoint kernels, CUDA-graph replays) runs between
cudaProfilerStart and cudaProfilerStop, for `ncu --profile-from-start off`.

amr: `ncoarse` eager coarse steps of the 3-level hierarchy (64^2 base, ratio 4 twice, 194 boxes),
16 x 16 tiles, same-level ghosts pulled, interpolated ones filled by their own launch.

regrid: the benchmark analog (1000^2 base, 3 levels of ratio 2, van Leer, conservation fix, regrid
every 8 coarse steps, cutoff 0.7), `ncoarse` coarse steps after the initial refinement; prints the
host wall time per regrid of each library call the regrid makes (each bracketed by device
synchronisation).

uniform: radial pulse, rho = 1, K = 4; cellwise: the same tiling over the smoothed random
medium of the heterogeneous workload; swe: shallow water (g = 1) with the ring pulse as depth.
fused (default): one claw_level_advance per step (ghosts pulled from their source cells, Eq. cfl
on its last CTA); split: fill, step, dt update.  The tiling defaults to 32 x 32 tiles, tensor
bulk-copy staging, 256 threads; the limiter to MC (4; 3 is van Leer); walk (claw_set_tile_walk) to
the library's default.
"""
import sys

import torch

from . import inputs
from .solver import Hierarchy


def adjoint(nruns, ncoarse, every):
    import time
    from . import measure
    from .adjoint import rollout
    runs = inputs.config4_runs(nruns)
    qs = [[inputs.init_q(r, lev) for lev in r.levels] for r, _, _ in runs]
    rhos = [[inputs.coef_pool(lev, r2, 4 ** L) for L, lev in enumerate(r.levels)] for r, r2, _ in runs]
    Ks = [[inputs.coef_pool(lev, k2, 4 ** L) for L, lev in enumerate(r.levels)] for r, _, k2 in runs]
    H = Hierarchy([r for r, _, _ in runs], qs, rhos, Ks)
    H.init_dt()
    tiling = measure.tune_all(H)
    H.init_dt()
    for p in range(2):
        tq, tr, tk = measure._tensors(H, qs, "q"), measure._tensors(H, rhos, "c"), measure._tensors(H, Ks, "c")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = rollout(H, tq, tr, tk, ncoarse=ncoarse, every=every)
        J = measure._receiver_energy(H, outs)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if p:
            torch.cuda.profiler.start()
        J.backward()
        torch.cuda.synchronize()
        if p:
            torch.cuda.profiler.stop()
        t2 = time.perf_counter()
    print("tiling", tiling, "forward ms", 1e3 * (t1 - t0), "backward ms", 1e3 * (t2 - t1), "status", H.sync_status())


def regrid(ncoarse):
    import time
    import numpy as np
    from . import claw
    spent = {}

    def timed(name, fn):
        def call(*a, **k):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn(*a, **k)
            torch.cuda.synchronize()
            spent[name] = spent.get(name, 0.0) + time.perf_counter() - t0
            return out
        return call

    names = ("claw_fill_ghost", "claw_flag_cells", "claw_regrid_boxes", "claw_set_level", "claw_regrid_transfer",
             "claw_set_tiling", "claw_set_tile_walk")
    saved = {n: getattr(claw, n) for n in names}
    base, nlev, ratio, every = 1000, 3, 2, 8
    run = inputs.Run(*inputs.PULSE_DOMAIN, limiter=3)
    step = base // 4
    run.levels = [inputs.Level(base, base, 2.0 / base, 2.0 / base,
                               [(i, j, step, step) for j in range(0, base, step) for i in range(0, base, step)])]
    for L in range(1, nlev):
        n = base * ratio ** L
        run.levels.append(inputs.Level(n, n, 2.0 / n, 2.0 / n, np.zeros((0, 4), dtype=np.int32), ratio))
    q0 = [inputs.init_q(run, lev) for lev in run.levels]
    H = Hierarchy([run], [q0], rho0=1.0, K0=4.0, reflux=True, tiling=((32, 16, 2, 256), (16, 16, 1, 128)))
    params = dict(tol=0.002, buffer=every, cutoff=0.7, max_size=260, nest=2)
    for _ in range(nlev - 1):
        H.regrid(**params)
    for L, lev in enumerate(run.levels):
        a = inputs.init_q(run, lev)
        t = H.q[L][H.cur[L]]
        t.zero_()
        t[:a.size] = torch.from_numpy(a).to(t.device)
    H.init_dt()
    total, count = 0.0, 0
    for k in range(ncoarse):
        H.coarse_step()
        if (k + 1) % every == 0:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:   # the library calls timed inside the regrid only
                for n in names:
                    setattr(claw, n, timed(n, saved[n]))
                H.regrid(**params)
            finally:
                for n in names:
                    setattr(claw, n, saved[n])
            torch.cuda.synchronize()
            total += time.perf_counter() - t0
            count += 1
    count = max(count, 1)
    print(f"regrids {count}, ms per regrid {1e3 * total / count:.2f}, boxes per level "
          f"{[len(lev.boxes) for lev in run.levels]}")
    for n, v in sorted(spent.items(), key=lambda kv: -kv[1]):
        print(f"  {n:24s} {1e3 * v / count:8.2f} ms per regrid")
    print(f"  {'the rest (Python)':24s} {1e3 * (total - sum(spent.values())) / count:8.2f} ms per regrid")


def amr(ncoarse):
    run = inputs.config2()
    H = Hierarchy([run], [[inputs.init_q(run, lev) for lev in run.levels]], rho0=1.0, K0=4.0,
                  tiling=(16, 16, 1, 128))
    H.init_dt()
    for _ in range(ncoarse):
        H.coarse_step()
    torch.cuda.synchronize()
    print("status", H.sync_status(), "launches per coarse step", H.launches_per_coarse_step())


def main():
    medium = sys.argv[1] if len(sys.argv) > 1 else "uniform"
    if medium == "amr":
        amr(int(sys.argv[2]) if len(sys.argv) > 2 else 3)
        return
    if medium == "regrid":
        regrid(int(sys.argv[2]) if len(sys.argv) > 2 else 80)
        return
    if medium == "adjoint":
        args = [int(v) for v in sys.argv[2:5]]
        adjoint(*(args + [8, 4, 2][len(args):]))
        return
    nsteps = int(sys.argv[2]) if len(sys.argv) > 2 else 3
    fused = (sys.argv[3] if len(sys.argv) > 3 else "fused") == "fused"
    tiling = tuple(int(v) for v in sys.argv[4].split(",")) if len(sys.argv) > 4 else None
    limiter = int(sys.argv[5]) if len(sys.argv) > 5 and sys.argv[5] != "-" else None
    walk = int(sys.argv[6]) if len(sys.argv) > 6 else None
    n = 2048
    if medium == "uniform":
        run = inputs.config1()
        if limiter is not None:
            run.limiter = limiter
        H = Hierarchy([run], [[inputs.init_q(run, run.levels[0])]], rho0=1.0, K0=4.0, tiling=tiling, walk=walk)
    elif medium == "swe":
        run = inputs.config1()
        H = Hierarchy([run], [[inputs.init_swe(run, run.levels[0])]], tiling=tiling, system="shallow_water",
                      grav=1.0, walk=walk)
    else:
        run, r2, k2 = inputs.config3(n)
        run.levels = [inputs.Level(n, n, 2.0 / n, 2.0 / n, inputs.uniform_tiling(n, n, 32, 32))]
        lev = run.levels[0]
        H = Hierarchy([run], [[inputs.init_q(run, lev)]], [[inputs.coef_pool(lev, r2, 1)]],
                      [[inputs.coef_pool(lev, k2, 1)]], tiling=tiling, walk=walk)
    H.fused = fused
    H.init_dt()
    for _ in range(nsteps):
        H.coarse_step()
    torch.cuda.synchronize()
    print("status", H.sync_status(), "dt", float(H.dt[0]))


if __name__ == "__main__":
    main()
