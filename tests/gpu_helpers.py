"""Shared set-up of the GPU parity tests: build the CUDA library, move seeded inputs to the
device through the C ABI, and run the same inputs through the oracle."""
import numpy as np

from paper_1808_02638_gb300 import inputs

M = 2


def lib_ready():
    import torch
    from paper_1808_02638_gb300 import build
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    build.build()


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(1e-300, np.abs(b).max()))


def single_grid(n, d=None, rho=None, K=None, pulse=True, seed=None, bc=(0, 0, 0, 0), limiter=4, order=2,
                transverse=2, boxes=None):
    """(run, q pool) of an n x n grid on [-1,1]^2 with one box (or `boxes`)."""
    run = inputs.Run(*inputs.PULSE_DOMAIN, bc=bc, limiter=limiter, order=order, transverse=transverse)
    d = 2.0 / n if d is None else d
    run.levels = [inputs.Level(n, n, d, d, [(0, 0, n, n)] if boxes is None else boxes)]
    lev = run.levels[0]
    if pulse:
        q = inputs.init_q(run, lev)
    else:
        q = np.zeros(lev.qsize)
        for k, b in enumerate(lev.boxes):
            v = inputs.box_view(q, lev.qoff[k], int(b[2]), int(b[3]), 3)
            v[...] = inputs.uniform(seed + k, v.size).reshape(v.shape) - 0.5
    return run, q


def oracle_single(orc, run, q, rho, K, nsteps, dt=None):
    """oracle steps of a single-box run; rho, K: (H, W) padded planes."""
    from oracle.amr import run_single_grid
    lev = run.levels[0]
    b = lev.boxes[0]
    qb = inputs.box_view(q, 0, int(b[2]), int(b[3]), 3).copy()
    qf, dts = run_single_grid(qb, rho, K, lev.dx, lev.dy, nsteps, bc=run.bc, cfl=run.cfl, dt=dt,
                              order=run.order, transverse=run.transverse, limiter=run.limiter)
    return qf[:, M:-M, M:-M], dts
