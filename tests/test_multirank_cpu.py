"""The multi-GPU path of bench.py is independent replicas: every rank solves
its own system, and the job time is the slowest rank's.  The host logic of that
path (rank seeds, max over ranks) is checked here with two gloo ranks on CPU."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(1001, rank))
        out[rank] = (slow, seeds)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_reduce_max_and_use_distinct_seeds():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert res[0][1] == res[1][1] and len(set(res[0][1])) == 2


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, None) == 3.5
