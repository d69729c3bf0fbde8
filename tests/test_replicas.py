"""Multi-rank host logic of the replicated / sharded runs: world_size-2 gloo process groups on
the CPU (the level-step itself has no exchange between ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1808_02638_gb300 import replicas


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 4097):
        for world in (1, 2, 3, 8):
            got = [u for r in range(world) for u in replicas.shard(n, world, r)]
            assert got == list(range(n))
            sizes = [len(replicas.shard(n, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_reductions_are_identity():
    rate, ms, units = replicas.whole_job_rate(300.0, 20.0)
    assert (rate, ms, units) == (300.0 / 0.02, 20.0, 300.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.barrier(dist)
        # rank r processed 100 (r + 1) units in 10 (r + 1) ms: the job takes the slowest time
        rate, ms, units = replicas.whole_job_rate(100.0 * (rank + 1), 10.0 * (rank + 1), dist)
        mine = list(replicas.shard(64, world, rank))
        out.put((rank, rate, ms, units, mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_whole_job_timing_and_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms, units, mine in res:
        assert ms == 20.0 and units == 300.0 and rate == pytest.approx(300.0 / 0.02)
    assert res[0][4] + res[1][4] == list(range(64))


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    bench.run_reference(argparse.Namespace(steps=1, warmup=3), rank=1, world=2)
    assert capsys.readouterr().out == ""
