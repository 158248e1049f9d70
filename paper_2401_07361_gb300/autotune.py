"""Autotuner for the tree-code parameters under a fixed error budget.

The tree code trades accuracy for speed through the MAC parameter theta (Sec. 3.4), the
interpolation degree d (Sec. 3.2), the leaf size N_T (Sec. 3) and the traversal (target-leaf
lists with PC + PP, or the dual traversal with PP, PC, CP and CC).  For one particle set,
``autotune`` times the whole path (tree build + velocity, through the C ABI, CUDA events on
the caller's stream) for every candidate and measures its error against the FP64 direct sum
on sampled targets (relative l2, area weighted as in Sec. 4.1).  It returns the fastest
candidate whose error is within the budget.  Every evaluation runs in the CUDA library; this
module only chooses parameters.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

from . import sts


@dataclass
class TuneResult:
    theta: float
    degree: int
    leaf_size: int
    ms: float
    error: float
    table: list = field(default_factory=list)  # (theta, degree, leaf, ms, error, dual) per candidate
    dual: bool = False  # the dual traversal (apply with sts.sts_set_traversal)

    def params(self, precision=sts.STS_MIXED, near_fp64_tau=0.0, max_level=16):
        return sts.params(self.theta, self.degree, self.leaf_size, max_level, precision, near_fp64_tau)


def _rel_l2(v, ref, w):
    num = float(np.sum(np.sum((v - ref) ** 2, axis=1) * w))
    den = float(np.sum(np.sum(ref ** 2, axis=1) * w))
    return math.sqrt(num / den) if den > 0 else math.sqrt(num)


def autotune(pos, zeta, area, budget=1e-4, thetas=(0.5, 0.6, 0.7, 0.8), degrees=(4, 6, 8, 10),
             leaf_sizes=(64, 128, 256), precision=sts.STS_MIXED, tau_c=0.01, offsets=None,
             samples=2048, repeats=3, seed=0, ctx=None, stream=None, traversals=(False, True)) -> TuneResult:
    """Fastest (theta, degree, leaf_size, traversal) with rel l2 error <= budget vs the FP64
    direct sum (traversals: False = target-leaf lists, True = dual traversal).

    pos, zeta, area: CUDA float64 tensors ([n,3], [n], [n]).  offsets: instance offsets of a
    batched (forest) set, or None.  The error is measured at ``samples`` random targets (all
    targets if n is smaller); for a forest, each sampled target's direct sum runs over its own
    instance.  Raises ValueError if no candidate meets the budget.
    """
    import torch

    own = ctx is None
    if own:
        ctx_obj = sts.Context()
        ctx = ctx_obj.h
    n = pos.shape[0]
    rng = np.random.default_rng(seed)
    off = np.array([0, n], dtype=np.int64) if offsets is None else np.asarray(offsets, dtype=np.int64)
    # reference: FP64 direct sum per instance on sampled targets
    tg_all, ref_all = [], []
    per = max(1, samples // (len(off) - 1))
    for b in range(len(off) - 1):
        lo, hi = int(off[b]), int(off[b + 1])
        if hi - lo < 2:
            continue
        k = min(per, hi - lo)
        tg = np.sort(rng.choice(hi - lo, k, replace=False)).astype(np.int64)
        vb = sts.sts_direct_targets(ctx, pos[lo:hi].contiguous(), zeta[lo:hi].contiguous(),
                                    area[lo:hi].contiguous(), torch.from_numpy(tg).to(pos.device), sts.STS_FP64,
                                    stream=stream)
        tg_all.append(tg + lo)
        ref_all.append(vb.cpu().numpy())
    tg = np.concatenate(tg_all)
    ref = np.concatenate(ref_all)
    w = area.cpu().numpy()[tg]
    n_tau = n if offsets is None else int(np.min(np.diff(off)[np.diff(off) > 0]))
    tau = tau_c * 4.0 * math.pi / n_tau
    vel = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
    table = []
    best = None
    for theta, d, leaf, dual in itertools.product(thetas, degrees, leaf_sizes, traversals):
        p = sts.params(theta, d, leaf, 16, precision, tau)
        sts.sts_set_traversal(ctx, dual)

        def run():
            if offsets is None:
                sts.sts_tree_build(ctx, pos, p, stream=stream)
            else:
                sts.sts_tree_build_batched(ctx, pos, off, p, stream=stream)
            sts.sts_velocity(ctx, zeta, area, p, vel, stream=stream)

        run()
        times = []
        s = stream if stream is not None else torch.cuda.current_stream()
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            run()
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        err = _rel_l2(vel.cpu().numpy()[tg], ref, w)
        table.append((theta, d, leaf, ms, err, bool(dual)))
        if err <= budget and (best is None or ms < best[3]):
            best = (theta, d, leaf, ms, err, bool(dual))
    sts.sts_set_traversal(ctx, False)
    if own:
        ctx_obj.close()
    if best is None:
        raise ValueError(f"no candidate meets the error budget {budget:g}; smallest error "
                         f"{min(t[4] for t in table):.3e}")
    return TuneResult(best[0], best[1], best[2], best[3], best[4], table, best[5])
