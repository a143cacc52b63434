"""bench.py's multi-GPU path is replicas: check its rank aggregation on CPU (gloo, 2 ranks)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist

    class Args:
        gpus = world

    w, r, local = bench.dist_setup(Args())
    assert (w, r, local) == (world, rank, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
    t = bench.max_over_ranks(ms, w)
    nodes_per_s = 1e9 * (rank + 1)
    total = bench.sum_over_ranks(nodes_per_s, w)
    q.put((rank, t, total))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_take_max_time_and_sum_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, t, total in out:
        assert t == 15.0  # the max over ranks
        assert total == 3e9  # every rank's work counts
