"""The multi-GPU path of bench.py (one process per GPU, an independent index
per partition, no data exchange) is covered on CPU: two gloo ranks run the
same timing aggregation bench.py uses under torchrun."""

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r answered its queries in (10 + 5r) ms and its steps took (100 + r) ms
    value, q_sum, tot = bench.weak_scaling_value(world, 3, 1000, 10.0 + 5.0 * rank,
                                                 100.0 + rank, "cpu")
    q.put((rank, value, q_sum, tot))
    dist.destroy_process_group()


def test_weak_scaling_aggregation_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, q_sum, tot in out:
        assert q_sum == 15.0 and tot == 101.0          # the slowest rank decides
        assert value == pytest.approx(2 * 3 * 1000 / 0.015)
