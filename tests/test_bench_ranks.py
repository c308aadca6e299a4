"""The multi-GPU path of bench.py is N independent replicas: disjoint Philox
counter ranges per rank, and the reported step time is the maximum over
ranks. Checked here with two gloo ranks on the CPU (no GPU)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
        out[rank] = (ms, bench.counter_base(rank))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_disjoint_counters():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 15.0
    # a replica draws counters [base, base + steps * n_x): disjoint for any run below 2^40 families
    assert out[1][1] - out[0][1] == 1 << 40


def test_single_process_is_a_no_op():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
