"""The multi-GPU form of the bench is replicas only (no collective on the data
path): every rank advances its own grid and the job time is the maximum over
ranks.  This checks that aggregation with two gloo ranks on CPU."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.5, 2.0][rank]
    t_max, value = bench.aggregate_replicas(local, steps=10, world_size=world)
    dist.barrier()
    out[rank] = (t_max, value)
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        t_max, value = out[rank]
        assert t_max == pytest.approx(2.0)
        assert value == pytest.approx(world * 10 / 2.0)


def test_single_rank_needs_no_process_group():
    t_max, value = bench.aggregate_replicas(0.25, steps=5, world_size=1)
    assert t_max == 0.25 and value == pytest.approx(20.0)
