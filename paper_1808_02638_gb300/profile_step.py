"""Profiling driver: a few eager level-steps of the 2048 x 2048 workload as 4096 patches of
32 x 32, for a profiler to capture single kernel launches.

  python -m paper_1808_02638_gb300.profile_step [uniform|cellwise|swe] [nsteps] [fused|split] [tx,ty,staging,threads] [limiter]

uniform: radial pulse, rho = 1, K = 4; cellwise: the same tiling over the smoothed random
medium of the heterogeneous workload; swe: shallow water (g = 1) with the ring pulse as depth.
fused (default): one claw_level_advance per step (ghosts pulled from their source cells, Eq. cfl
on its last CTA); split: fill, step, dt update.  The tiling defaults to 32 x 32 tiles, tensor
bulk-copy staging, 256 threads; the limiter to MC (4; 3 is van Leer).
"""
import sys

import torch

from . import inputs
from .solver import Hierarchy


def main():
    medium = sys.argv[1] if len(sys.argv) > 1 else "uniform"
    nsteps = int(sys.argv[2]) if len(sys.argv) > 2 else 3
    fused = (sys.argv[3] if len(sys.argv) > 3 else "fused") == "fused"
    tiling = tuple(int(v) for v in sys.argv[4].split(",")) if len(sys.argv) > 4 else None
    limiter = int(sys.argv[5]) if len(sys.argv) > 5 else None
    n = 2048
    if medium == "uniform":
        run = inputs.config1()
        if limiter is not None:
            run.limiter = limiter
        H = Hierarchy([run], [[inputs.init_q(run, run.levels[0])]], rho0=1.0, K0=4.0, tiling=tiling)
    elif medium == "swe":
        run = inputs.config1()
        H = Hierarchy([run], [[inputs.init_swe(run, run.levels[0])]], tiling=tiling, system="shallow_water",
                      grav=1.0)
    else:
        run, r2, k2 = inputs.config3(n)
        run.levels = [inputs.Level(n, n, 2.0 / n, 2.0 / n, inputs.uniform_tiling(n, n, 32, 32))]
        lev = run.levels[0]
        H = Hierarchy([run], [[inputs.init_q(run, lev)]], [[inputs.coef_pool(lev, r2, 1)]],
                      [[inputs.coef_pool(lev, k2, 1)]], tiling=tiling)
    H.fused = fused
    H.init_dt()
    for _ in range(nsteps):
        H.coarse_step()
    torch.cuda.synchronize()
    print("status", H.sync_status(), "dt", float(H.dt[0]))


if __name__ == "__main__":
    main()
