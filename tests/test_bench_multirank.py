"""Host logic of the multi-rank bench (replica lattices, one per rank): the slowest rank's
time is taken by an all-reduce MAX and the whole-job MLUPS counts every rank's sites.
Runs two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slower one
    slowest = bench.max_over_ranks(local_ms)
    out[rank] = (slowest, bench.whole_job_mlups(1_000_000, 10, world, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_job_throughput():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, mlups = res[0]
    assert slowest == 150.0
    assert abs(mlups - 2 * 1_000_000 * 10 / 0.150 / 1e6) < 1e-9


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_mlups(100, 2, 1, 1.0) == pytest.approx(0.2)
