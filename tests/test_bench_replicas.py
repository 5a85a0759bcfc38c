"""bench.py on N > 1 ranks runs independent replicas (one per GPU): the ranks meet at a barrier
around the timed region and the job's time is the slowest rank's.  This checks that host logic
with two gloo ranks on the CPU (no GPU, no kernels)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_init()
    try:
        bench.barrier(w)
        out[r] = (w, bench.allmax(w, 10.0 + 5.0 * r))
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:       # no fork of a threaded test process
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res == {0: (2, 15.0), 1: (2, 15.0)}


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench

    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_init() == (1, 0, 0)
    assert bench.allmax(1, 3.5) == 3.5
