"""The multi-GPU path of bench.py, exercised on CPU with two gloo ranks: each
rank gets its own holograms (no hologram computed twice, no data-path
collective), the job's time is the slowest rank's, and the whole-job
throughput counts every rank's holograms."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.argv = ["bench.py", "--batch", "5", "--P", "64", "--N", "7", "--iters", "3"]
    args = bench.parse()
    pbs = bench.problems(args, rank)
    seeds = torch.tensor([pb.seed for pb in pbs], dtype=torch.int64)
    gathered = [torch.empty_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    my_time = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    slowest = bench.max_over_ranks(my_time, world, "cpu")
    value = bench.job_throughput(len(pbs), world, 4, slowest)
    out.put((rank, [g.tolist() for g in gathered], slowest, value,
             [pb.xyz.sum() for pb in pbs]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_holograms_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, g0, s0, v0, x0), (r1, g1, s1, v1, x1) = res
    assert g0 == g1                                     # every rank sees the same assignment
    assert not set(g0[0]) & set(g0[1])                  # no hologram on two ranks
    assert s0 == s1 == 15.0                             # the slowest rank's time
    assert v0 == v1 == pytest.approx(5 * 2 * 4 / 15.0e-3)
    assert x0 != x1                                     # different spot clouds
