"""The host side of the sharded evaluation (one tree-code velocity spread over GPUs, the
GPU counterpart of the paper's MPI evaluation in Sec. 4.1), on CPU with world size 2 over gloo
(127.0.0.1): the leaves are split into contiguous ranges by their exact PC + PP interaction
counts, each rank contributes the velocities of its ranges' targets as a block in sorted slot
order, and the all-gathered blocks, put back in the particles' order, are the full result.
The velocities here are the FP64 oracle's (the CUDA path is covered by test_gpu_shard.py)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, LEAF, THETA, DEG = 3000, 24, 0.7, 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2401_07361_gb300 import workloads as W

    pos = W.uniform_points(N, 31)
    rng = np.random.default_rng(32)
    zeta, area = rng.standard_normal(N), W.equal_areas(N)
    tr = O.Tree(pos, LEAF)
    ex, li = tr.export(), tr.lists(THETA)
    vel = tr.velocity(zeta, area, THETA, DEG)
    M = O.nbasis(DEG)
    cnt = ex["count"]
    work = np.array([cnt[L] * (M * (li["far_off"][k + 1] - li["far_off"][k])
                               + cnt[li["near_idx"][li["near_off"][k]:li["near_off"][k + 1]]].sum())
                     for k, L in enumerate(ex["leaves"])], dtype=np.int64)
    return ex, work, vel


def _rank(rank, ws, port, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
        sys.path.insert(0, ROOT)
        import torch.distributed as dist

        from paper_2401_07361_gb300 import shard

        dist.init_process_group("gloo", rank=rank, world_size=ws)
        ex, work, vel = _case()
        parts = shard.partition(work, ws)
        leaves, start, count, perm = ex["leaves"], ex["start"], ex["count"], ex["perm"]
        slots = [(int(start[leaves[a]]), int(start[leaves[b - 1]] + count[leaves[b - 1]])) if b > a else (0, 0)
                 for a, b in parts]
        s0, s1 = slots[rank]
        block = torch.from_numpy(vel[perm[s0:s1]].copy())  # this rank's targets, sorted slot order
        full = shard.gather_rows(block, [b - a for a, b in slots]).numpy()
        out = np.empty_like(full)
        out[perm] = full  # back to the particles' order
        dist.destroy_process_group()
        q.put((rank, bool(np.array_equal(out, vel)), parts))
    except Exception as e:  # pragma: no cover - reported through the queue
        q.put((rank, repr(e), None))


def test_partition_is_contiguous_and_balanced():
    sys.path.insert(0, ROOT)
    from paper_2401_07361_gb300 import shard

    _, work, _ = _case()
    for nparts in (1, 2, 3, 8):
        parts = shard.partition(work, nparts)
        assert parts[0][0] == 0 and parts[-1][1] == len(work)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        loads = [int(work[a:b].sum()) for a, b in parts]
        # each boundary is the nearest one to its share: no part exceeds its share by more
        # than one leaf on each side
        assert max(loads) <= work.sum() / nparts + 2 * work.max(), (nparts, loads)
    rng = np.random.default_rng(5)
    w = rng.integers(1, 100, 1000)
    for nparts in (2, 4, 7):
        loads = [w[a:b].sum() for a, b in shard.partition(w, nparts)]
        assert max(loads) - min(loads) <= 2 * w.max()
    assert shard.partition([], 3) == [(0, 0)] * 3


def test_sharded_gather_reassembles_the_full_velocity_gloo():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert [o[1] for o in out] == [True, True], out
    parts = out[0][2]
    assert parts == out[1][2] and parts[0][1] > parts[0][0] and parts[1][1] > parts[1][0]
