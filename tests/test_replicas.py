"""Multi-GPU form (replicas only): every rank searches its own queries and the
job's time is the slowest rank's.  The rendezvous, barrier and max-over-ranks
helpers of bench.py run here as two gloo processes on the CPU."""
from __future__ import annotations

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank: int, ws: int, port: int, out) -> None:
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        impl = "reference"  # gloo: the CPU arm's backend

    r, w, _ = bench.dist_init(Args)
    bench.barrier(w)
    # each rank's own elapsed time; the job takes the slowest
    slowest = bench.max_over_ranks(10.0 * (r + 1), w)
    out.put((r, w, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 20.0), (1, 2, 20.0)]
