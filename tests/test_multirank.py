"""The multi-rank path of the benchmark on CPU: two gloo ranks (127.0.0.1)
reduce their timings to the slowest rank, report the whole-job rate from it
and draw different fields.  The step itself shards by walkers and has no
collective on its data path, so these reductions are all the ranks share."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    walkers, steps = 1024, 3
    t = bench.slowest_rank(1.5 + rank, world, torch.device("cpu"))   # rank 1 is slower
    rate = bench.job_rate(walkers * steps, world, t)
    seed = bench.shard_seed(1234, rank)
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(4, generator=g)
    dist.barrier()
    q.put((rank, t, rate, seed, x.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_slowest_time_job_rate_and_distinct_fields():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, rate0, s0, x0), (r1, t1, rate1, s1, x1) = out
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.5                       # both ranks see the slowest time
    assert rate0 == rate1 == pytest.approx(world * 1024 * 3 / 2.5)
    assert s0 != s1 and x0 != x1                 # each rank its own fields


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(0.75, 1, torch.device("cpu")) == 0.75
    assert bench.job_rate(1024 * 20, 1, 0.5) == 1024 * 20 / 0.5
    assert bench.shard_seed(1234, 0) == 1234
