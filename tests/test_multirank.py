"""The bench's multi-GPU mode runs independent replicas (one per GPU, no exchange in
the data path); its only collective is the aggregation of the timed region: the
slowest rank's time and the sum of the work of all ranks.  Checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 (r + 1) ms for 100 (r + 1) products
        ms, units = bench.aggregate_ranks(torch, 10.0 * (rank + 1), 100 * (rank + 1), "cpu")
        out[rank] = (ms, units)
    finally:
        dist.destroy_process_group()


def test_aggregation_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    # the manager process is spawned too: forking a process that already runs threads
    # (BLAS, FFT workers of earlier tests) can deadlock the child
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, units = res[r]
        assert ms == 20.0            # the slowest rank's time
        assert units == 300.0        # 100 + 200 products
    assert 300.0 / (20.0 / 1000.0) == pytest.approx(15000.0)


def test_single_process_aggregation_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(torch, 12.5, 7, "cpu") == (12.5, 7.0)
