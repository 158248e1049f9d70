"""One tree-code velocity spread over several GPUs, one process per GPU.

The paper parallelises the convolution of Sec. 3 over MPI ranks (Sec. 4.1).  Here every rank
builds the same tree (an O(N log N) sort, cheap next to the evaluation), evaluates the targets
of one contiguous range of depth-first leaves, and the ranks all-gather their blocks of
velocities, which are contiguous in sorted slot order; each rank then puts the rows back in the
caller's order.  The ranges balance the exact per-leaf interaction counts of the lists
(sts_leaf_work).  This module is host logic only: the arithmetic is in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def partition(work, nparts: int):
    """Contiguous ranges [(lo, hi), ...] of the leaves 0 .. len(work) - 1, one per part, whose
    summed work is as even as the leaf granularity allows: part k starts at the leaf boundary
    whose running sum of work lies nearest to k / nparts of the total."""
    work = np.asarray(work, dtype=np.int64)
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    L = len(work)
    cum = np.concatenate([[0], np.cumsum(work)])
    total = int(cum[-1])
    bounds = [0]
    for k in range(1, nparts):
        if total > 0:
            t = total * k / nparts
            b = int(np.searchsorted(cum, t, side="left"))
            if b > 0 and (b > L or abs(cum[b - 1] - t) <= abs(cum[b] - t)):
                b -= 1
        else:
            b = (L * k) // nparts
        bounds.append(min(max(b, bounds[-1]), L))
    bounds.append(L)
    return [(bounds[k], bounds[k + 1]) for k in range(nparts)]


def gather_rows(block, counts, group=None):
    """All-gathers per-rank row blocks of different lengths (counts[r] rows on rank r, this
    rank's block first dimension = counts[rank]) into one array of sum(counts) rows in rank
    order.  Blocks are padded to the longest so that one all-gather of equal-sized tensors
    carries them (NCCL's all-gather needs equal sizes)."""
    import torch
    import torch.distributed as dist

    counts = [int(c) for c in counts]
    world = len(counts)
    width = block.shape[1:] if block.dim() > 1 else ()
    mx = max(counts) if counts else 0
    pad = torch.zeros((mx,) + tuple(width), dtype=block.dtype, device=block.device)
    pad[: block.shape[0]] = block
    out = torch.empty((world * mx,) + tuple(width), dtype=block.dtype, device=block.device)
    if world == 1:
        out.copy_(pad)
    else:
        dist.all_gather_into_tensor(out, pad, group=group)
    return torch.cat([out[r * mx: r * mx + counts[r]] for r in range(world)])


def sharded_velocity(ctx, zeta, area, p, rank: int, world: int, group=None, vel=None):
    """The tree-code velocity of the tree last built in ctx (built identically on every
    rank), this rank evaluating its share of the leaves; returns vel[n,3] in the caller's
    order on every rank."""
    import torch

    from . import sts

    # the lists (and the per-leaf work they imply) are built by an empty range evaluation
    sts.sts_velocity_range(ctx, zeta, area, p, 0, 0, out_sorted=True)
    work = sts.sts_leaf_work(ctx, p.degree)
    parts = partition(work, world)
    slots = [sts.sts_leaf_range(ctx, lo, hi) for lo, hi in parts]
    lo, hi = parts[rank]
    mine = sts.sts_velocity_range(ctx, zeta, area, p, lo, hi, out_sorted=True)
    full = gather_rows(mine, [b - a for a, b in slots], group)
    return sts.sts_unpermute(ctx, full, vel)
