"""Parity at the full sizes of the other benchmark workloads, each in the launch configuration
``bench.py --workload NAME`` times: tree build and velocity through ``sts_tree_velocity``,
recorded as a CUDA graph and replayed, mixed precision with tau = 0.01 * 4 pi / N (N of the
smallest instance for a forest), theta 0.7, degree 8.

  ico9_jet      N = 2621442 icosahedral vertices (edge ties in the tree build), N_T = 128
  rand10m_sh32  N = 10485762 uniform points, N_T = 256
  ensemble64    64 instances of 10242 to 163842 particles, 3.5e6 in one forest, N_T = 128

The oracle's FP64 tree codes finish at these sizes in tens of seconds, so every target is
compared, for both traversals (target-leaf lists, Sec. 3.4's dual traversal):
  - single instances: the tree and the lists bit for bit, the replayed mixed velocity within
    1e-6 relative l2 (1e-5 max norm) of the oracle's FP64 tree code;
  - the forest: every instance's replayed mixed velocity against the oracle's tree code of
    that instance alone, same bars;
  - the replayed step against an eager call on the same context (equal up to the order of
    the FP64 atomic sums of the close pairs).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CONFIGS = ("ico9_jet", "rand10m_sh32", "ensemble64")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.fixture(scope="module", params=CONFIGS)
def cfg(request):
    wl = W.workload(request.param)
    off = wl.get("offsets")
    n = len(wl["pos"])
    sizes = np.diff(off) if off is not None else np.array([n])
    tau = 0.01 * 4 * math.pi / int(np.min(sizes[sizes > 0]))
    p = sts.params(theta=0.7, degree=8, leaf_size=wl["leaf_size"], max_level=16, precision=sts.STS_MIXED,
                   near_fp64_tau=tau)
    if off is None:
        trees = [O.Tree(wl["pos"], wl["leaf_size"], 16)]
        off = np.array([0, n], dtype=np.int64)
        single = True
    else:
        trees = [O.Tree(wl["pos"][off[b]:off[b + 1]], wl["leaf_size"], 16) for b in range(len(off) - 1)]
        single = False
    return request.param, wl, p, off, trees, single


def _gpu(wl, p, off, single, dual):
    """The replayed step (the first call runs eagerly and records, the second replays), an
    eager call on the same context, and the exports of the tree and lists."""
    st = torch.cuda.Stream()
    n = len(wl["pos"])
    offsets = None if single else off
    with sts.Context() as c:
        sts.sts_set_traversal(c.h, dual)
        x, z, a = dev(wl["pos"]), dev(wl["zeta"]), dev(wl["area"])
        vel = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        sts.sts_set_graph(c.h, True)
        with torch.cuda.stream(st):
            for _ in range(2):
                vel.fill_(float("nan"))
                sts.sts_tree_velocity(c.h, x, z, a, p, vel, offsets=offsets, stream=st)
        st.synchronize()
        vg = vel.cpu().numpy()
        sts.sts_set_graph(c.h, False)
        with torch.cuda.stream(st):
            vel.fill_(float("nan"))
            sts.sts_tree_velocity(c.h, x, z, a, p, vel, offsets=offsets, stream=st)
        st.synchronize()
        ve = vel.cpu().numpy()
        tree = lists = None
        if single:
            tree = sts.sts_tree_export(c.h)
            lists = sts.sts_dual_export(c.h) if dual else sts.sts_lists_export(c.h)
    return vg, ve, tree, lists


@pytest.mark.parametrize("dual", [False, True], ids=["leaf_lists", "dual"])
def test_config_fullsize_parity(cfg, dual):
    name, wl, p, off, trees, single = cfg
    vg, ve, tree, lists = _gpu(wl, p, off, single, dual)
    assert np.all(np.isfinite(vg))
    scale = np.max(np.abs(ve))
    assert np.max(np.abs(vg - ve)) <= 1e-12 * scale, name
    if single:
        tr = trees[0]
        ex = tr.export()
        for k in ("perm", "key", "start", "count", "leaf", "leaves", "parent"):
            assert np.array_equal(ex[k], tree[k]), k
        if dual:
            o = tr.dual_lists(0.7)
            for k in sts.DUAL_KINDS:
                oo, go = np.lexsort((o[k][1], o[k][0])), np.lexsort((lists[k][1], lists[k][0]))
                assert np.array_equal(o[k][0][oo], lists[k][0][go]), k
                assert np.array_equal(o[k][1][oo], lists[k][1][go]), k
        else:
            ol = tr.lists(0.7)
            for k in ("far_off", "far_idx", "near_off", "near_idx"):
                assert np.array_equal(ol[k], lists[k]), k
    worst2 = worstm = 0.0
    for b, tr in enumerate(trees):
        lo, hi = int(off[b]), int(off[b + 1])
        if hi - lo < 2:
            continue
        zb, ab = wl["zeta"][lo:hi], wl["area"][lo:hi]
        ref = tr.velocity_dual(zb, ab, 0.7, 8) if dual else tr.velocity(zb, ab, 0.7, 8)
        e2, em = O.rel_l2(vg[lo:hi], ref, ab), O.rel_max(vg[lo:hi], ref)
        worst2, worstm = max(worst2, e2), max(worstm, em)
    print(f"{name} {'dual' if dual else 'leaf lists'}: mixed vs FP64 oracle rel_l2 {worst2:.3e} rel_max {worstm:.3e}")
    assert worst2 <= 1e-6
    assert worstm <= 1e-5
