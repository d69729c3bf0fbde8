"""Host-side logic of runs on several GPUs (one process per GPU).

The level-step has no data exchange between independent runs (Sec. 3: each run is its own
problem; patches exchange ghosts only within a run), so N GPUs either advance N replicas of
a workload or split a batch of independent runs into contiguous shards, one per rank.  The
only collectives are on the host path: a barrier around the timed region and the maximum of
the per-rank times (the job ends when its slowest rank does), plus the sum of the units the
ranks processed.
"""
from __future__ import annotations


def shard(n: int, world: int, rank: int) -> range:
    """contiguous block of the units 0..n-1 owned by `rank` (sizes differ by at most one)"""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def _reduce(x: float, op, dist, device):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, dist=None, device=None) -> float:
    return _reduce(x, dist.ReduceOp.MAX if dist is not None else None, dist, device)


def sum_over_ranks(x: float, dist=None, device=None) -> float:
    return _reduce(x, dist.ReduceOp.SUM if dist is not None else None, dist, device)


def whole_job_rate(units_local: float, ms_local: float, dist=None, device=None):
    """(units of all ranks / slowest rank's time in s, slowest time in ms, units of all ranks)"""
    ms = max_over_ranks(ms_local, dist, device)
    units = sum_over_ranks(units_local, dist, device)
    return units / (ms * 1e-3), ms, units


def barrier(dist=None):
    """all ranks meet (a process group bound to a device at init uses that device)"""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
