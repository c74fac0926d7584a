"""The benchmark's multi-rank path (independent replicas, one per GPU: the
contraction needs no data-path collective) on CPU with the gloo backend,
world size 2: the slowest rank's time sets the whole-job throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.replica_throughput(10.0 + 5.0 * rank, 1e12, world)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 15.0  # the max over ranks
    assert value == pytest.approx(2 * 1e12 / 15e-3 / 1e12)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.replica_throughput(4.0, 2e12, 1) == (4.0, pytest.approx(500.0))
