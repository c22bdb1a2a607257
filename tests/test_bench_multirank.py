"""The benchmark's multi-GPU path is independent replicas: whole-job
throughput = work summed over ranks / slowest rank's time.  Checked with two
gloo ranks on the CPU (no GPU collective involved)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [100.0, 300.0][rank]
    secs = [2.0, 4.0][rank]
    v = bench.aggregate(units, secs, world)
    m = bench.barrier_max(secs, world)
    out[rank] = (v, m)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_replicas():
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        v, m = res[rank]
        assert v == pytest.approx((100.0 + 300.0) / 4.0)
        assert m == 4.0


def test_single_rank_needs_no_process_group():
    assert bench.aggregate(10.0, 2.0, 1) == 5.0
    assert bench.barrier_max(3.0, 1) == 3.0
