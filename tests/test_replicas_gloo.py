"""The multi-GPU form of the bench is replicas: every rank integrates its own
lattice and only the timing barrier and the whole-job totals cross ranks.
This checks that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from paper_1611_00298_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank-dependent times and byte counts; the job takes the slowest time and the sum
    t, b = bench.replica_totals(dist, 1.0 + rank, 10.0 * (rank + 1), "cpu")
    U = inputs.gauge_field((2, 2, 2, 2), 0.5, bench.replica_seed(3, rank))
    out[rank] = (t, b, float(abs(U).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    # spawn, not fork: the test process may already run OpenMP threads (C oracle)
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:2] == res[1][:2] == (2.0, 30.0)
    assert res[0][2] != res[1][2]  # independent replicas: different lattices
    assert torch is not None


def test_single_rank_totals_pass_through():
    import bench
    assert bench.replica_totals(None, 1.5, 7.0, "cpu") == (1.5, 7.0)
