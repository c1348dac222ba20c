"""CPU checks of the multi-rank path of bench.py (replicas only): two gloo
ranks agree on the max-over-ranks timing, the per-replica value divides by
the rank count, and a non-zero rank of the reference arm exits without work."""

import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    m = bench.max_over_ranks([1.0 + rank, 10.0 * (world - rank)])
    printed = None
    if rank != 0:
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.reference_arm(None)
        printed = buf.getvalue()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, r, w, m, printed))


def test_two_gloo_ranks_max_and_reference_rank_exit():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, m, printed in out:
        assert (r, w) == (rank, 2)
        assert m == [2.0, 20.0]          # max over ranks of [1 + rank, 10 (2 - rank)]
    assert out[1][4] == ""               # rank 1 of the reference arm printed nothing


def test_per_replica_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.per_replica(0.8, 4) == pytest.approx(0.2)
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]   # no process group
