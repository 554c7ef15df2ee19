"""Multi-GPU runs are replicas (a single simulation does not shard: the demag
convolution is global).  The bench's cross-rank aggregation - slowest rank's
time, summed work - is checked here with two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.aggregate_ranks(10.0 + rank, 100.0 * (rank + 1), "cpu")
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 11.0                                   # the slowest rank's time
        assert value == pytest.approx(300.0 / 11e-3)        # all ranks' work over it
