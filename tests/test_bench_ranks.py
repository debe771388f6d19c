"""The multi-GPU path of bench.py is independent replicas (one process per
GPU, no collective on the data path): its timing takes the maximum over
ranks and its work the sum.  Checked with two gloo ranks on CPU."""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.reduce_across_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), dist, "cpu")
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_two_rank_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, units in res:
        assert ms == pytest.approx(15.0) and units == pytest.approx(3000.0)


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_across_ranks(3.0, 7.0) == (3.0, 7.0)
