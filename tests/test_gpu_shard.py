"""The sharded evaluation on one GPU: the leaf ranges of a partition, each evaluated by
sts_velocity_range (here one after the other, by two contexts that each built the same tree
as two GPUs would), give exactly sts_velocity's result, in the caller's order or as sorted
blocks put back by sts_unpermute."""
import math

import numpy as np
import pytest

from paper_2401_07361_gb300 import shard, sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.fixture(scope="module")
def case():
    n = 20011
    pos = W.uniform_points(n, 41)
    rng = np.random.default_rng(42)
    zeta = rng.standard_normal(n)
    area = W.equal_areas(n)
    return dev(pos), dev(zeta), dev(area), n


# mixed precision with tau = 0 and FP64 have no atomic sums: bit for bit; with tau > 0 the
# close pairs' FP64 corrections are summed by atomics in any order (last-bit differences)
@pytest.mark.parametrize("prec,tau_c,exact", [(sts.STS_FP64, 0.0, True), (sts.STS_MIXED, 0.0, True),
                                              (sts.STS_MIXED, 0.05, False)])
def test_leaf_ranges_union_equals_full_velocity(case, prec, tau_c, exact):
    pos, zeta, area, n = case
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=prec, near_fp64_tau=tau_c * 4 * math.pi / n)
    with sts.Context() as a, sts.Context() as b:
        sts.sts_tree_build(a.h, pos, p)
        full = sts.sts_velocity(a.h, zeta, area, p).cpu().numpy()
        st = sts.sts_stats(a.h)
        work = sts.sts_leaf_work(a.h, 6)
        assert work.sum() == st["pc"] + st["pp"] + n  # PC + PP, self pairs included
        parts = shard.partition(work, 3)
        assert all(hi > lo for lo, hi in parts)
        sts.sts_tree_build(b.h, pos, p)  # a second "GPU": the same tree built again
        ctxs = [a.h, b.h, a.h]
        # rows in the caller's order
        v = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        for c, (lo, hi) in zip(ctxs, parts):
            sts.sts_velocity_range(c, zeta, area, p, lo, hi, vel=v)
        got = v.cpu().numpy()
        # sorted blocks, gathered and put back in order
        blocks = [sts.sts_velocity_range(c, zeta, area, p, lo, hi, out_sorted=True) for c, (lo, hi) in zip(ctxs, parts)]
        slots = [sts.sts_leaf_range(a.h, lo, hi) for lo, hi in parts]
        assert slots[0][0] == 0 and slots[-1][1] == n and all(x[1] == y[0] for x, y in zip(slots, slots[1:]))
        assert [blk.shape[0] for blk in blocks] == [s1 - s0 for s0, s1 in slots]
        got2 = sts.sts_unpermute(a.h, torch.cat(blocks)).cpu().numpy()
        if exact:
            assert np.array_equal(got, full) and np.array_equal(got2, full)
        else:
            scale = np.abs(full).max()
            assert np.abs(got - full).max() <= 1e-13 * scale and np.abs(got2 - full).max() <= 1e-13 * scale


def test_leaf_range_edges(case):
    pos, zeta, area, n = case
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_MIXED, near_fp64_tau=0.0)
    with sts.Context() as c:
        sts.sts_tree_build(c.h, pos, p)
        nl = sts.sts_tree_info(c.h)["leaves"]
        v = torch.full((n, 3), 7.0, dtype=torch.float64, device="cuda")
        sts.sts_velocity_range(c.h, zeta, area, p, 5, 5, vel=v)  # an empty range writes nothing
        assert torch.all(v == 7.0)
        assert sts.sts_leaf_range(c.h, nl, nl) == (n, n)
        for lo, hi in ((-1, 3), (4, 2), (0, nl + 1)):
            with pytest.raises(sts.StsError):
                sts.sts_velocity_range(c.h, zeta, area, p, lo, hi, vel=v)
            with pytest.raises(sts.StsError):
                sts.sts_leaf_range(c.h, lo, hi)
        # the whole range is the full evaluation
        full = sts.sts_velocity(c.h, zeta, area, p).cpu().numpy()
        one = sts.sts_velocity_range(c.h, zeta, area, p, 0, nl).cpu().numpy()
        assert np.array_equal(one, full)
