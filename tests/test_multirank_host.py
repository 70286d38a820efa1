"""The N > 1 bench path on CPU: independent replicas, timing = max over
ranks, whole-job MLUPS = ranks x nodes x steps / max time.  Run as two gloo
ranks (no GPU, no data-path collective: only the timing reduction)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = [0.5, 2.0][rank]
    t_max = bench.max_over_ranks(t_local, dist, "cpu")
    out[rank] = (t_max, bench.aggregate_mlups(1000, 10, world, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_is_max_and_value_aggregates():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        t_max, value = out[r]
        assert t_max == 2.0
        assert value == pytest.approx(world * 1000 * 10 / 2.0 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.aggregate_mlups(2048 * 2048, 100, 1, 0.5) == pytest.approx(838.8608)
