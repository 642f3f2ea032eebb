"""Host logic of the weak-scaling bench on world-size-2 gloo ranks (CPU): each
rank scores its own query sets, and the job time is the slowest rank's."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_query_seed(1236, rank)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    t = bench._max_over_ranks(dist, 10.0 + 5.0 * rank)
    out.put((rank, t, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_distinct_queries_and_max_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, seeds in res:
        assert t == 15.0                       # max over ranks
        assert len(set(seeds)) == 2            # ranks score different query sets
        assert seeds[0] == 1236 + 7919         # rank 0 keeps the workload's own queries
