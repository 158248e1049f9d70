"""The multi-rank host logic of bench.py on CPU: world size 2 over gloo (127.0.0.1).  Every
timed quantity is the maximum over the ranks, and the reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                          LOCAL_RANK=str(rank))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist

        import bench

        dist.init_process_group("gloo", rank=rank, world_size=ws)
        got = bench.max_over_ranks(10.0 + rank, ws, "cpu")
        assert bench.dist_env() == (ws, rank, rank)
        # the reference arm: ranks other than 0 leave at once, without work
        ref_rc = bench.run_reference(bench.parse([])) if rank != 0 else 0
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, got, ref_rc))
    except Exception as e:  # pragma: no cover - reported through the queue
        q.put((rank, repr(e), -1))


def test_max_over_ranks_and_reference_rank_gloo():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert out == [(0, 11.0, 0), (1, 11.0, 0)], out


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
