"""The multi-rank host logic of bench.py (replicas: barrier, max over ranks, whole-job rate)
on two CPU ranks over gloo; no GPU is touched."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), HPHI_BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup(world)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    # rank k "took" 10 + k seconds: every rank must see the slowest
    slowest = bench.max_over_ranks(10.0 + rank, w)
    out[rank] = (slowest, bench.whole_job_rate(2e9, w, slowest))
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for slowest, rate in res.values():
        assert slowest == 11.0
        assert abs(rate - world * 2e9 / 11.0 / 1e9) < 1e-12


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1e9, 1, 2.0) == 0.5
