"""Parity at the benchmark's full size and launch configuration: N = 655362 uniform points,
Voronoi areas, degree-16 harmonic vorticity, theta = 0.7, degree 8, N_T = 128, mixed
precision with tau = 0.01 * 4 pi / N (the configuration ``bench.py`` times).

The oracle finishes the FP64 tree code at this size in seconds, so the mixed GPU result is
compared with it at every target; the tree and lists are compared bit for bit; the direct
sum is compared on sampled targets.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    wl = W.workload("rand655k_sh16")
    c = sts.Context()
    yield wl, c.h
    c.close()


def test_fullsize_tree_lists_and_mixed_velocity(setup):
    wl, h = setup
    pos, zeta, area = wl["pos"], wl["zeta"], wl["area"]
    n = len(pos)
    tau = 0.01 * 4 * math.pi / n
    p = sts.params(theta=0.7, degree=8, leaf_size=128, max_level=16, precision=sts.STS_MIXED, near_fp64_tau=tau)
    d = lambda a: torch.from_numpy(a).to("cuda")
    sts.sts_tree_build(h, d(pos), p)
    v = sts.sts_velocity(h, d(zeta), d(area), p).cpu().numpy()
    tr = O.Tree(pos, 128, 16)
    ex, gx = tr.export(), sts.sts_tree_export(h)
    for k in ("perm", "key", "start", "count", "leaf", "leaves", "parent"):
        assert np.array_equal(ex[k], gx[k]), k
    ol, gl = tr.lists(0.7), sts.sts_lists_export(h)
    for k in ("far_off", "far_idx", "near_off", "near_idx"):
        assert np.array_equal(ol[k], gl[k]), k
    ref = tr.velocity(zeta, area, 0.7, 8)
    e2, em = O.rel_l2(v, ref, area), O.rel_max(v, ref)
    print(f"mixed vs FP64 oracle tree: rel_l2 {e2:.3e} rel_max {em:.3e}")
    assert e2 <= 1e-6
    assert em <= 1e-5
    p64 = sts.params(theta=0.7, degree=8, leaf_size=128, max_level=16, precision=sts.STS_FP64)
    v64 = sts.sts_velocity(h, d(zeta), d(area), p64).cpu().numpy()
    assert O.rel_l2(v64, ref, area) <= 1e-12


def test_fullsize_direct_sampled_targets(setup):
    wl, h = setup
    pos, zeta, area = wl["pos"], wl["zeta"], wl["area"]
    n = len(pos)
    tg = np.random.default_rng(2).choice(n, 2048, replace=False).astype(np.int64)
    ref = O.direct(pos, zeta, area, targets=tg)
    d = lambda a: torch.from_numpy(a).to("cuda")
    for prec, tol in ((sts.STS_FP64, 1e-12), (sts.STS_MIXED, 1e-6)):
        v = sts.sts_direct_targets(h, d(pos), d(zeta), d(area), d(tg), prec).cpu().numpy()
        assert O.rel_l2(v, ref, area[tg]) <= tol


def test_fullsize_dual_lists_and_mixed_velocity(setup):
    """The dual traversal (PP, PC, CP, CC) at the full size in the launch configuration of
    ``bench.py --dual``: the four pair lists bit for bit, the mixed velocity within 1e-6 of the
    oracle's FP64 dual tree code at every target."""
    wl, h = setup
    pos, zeta, area = wl["pos"], wl["zeta"], wl["area"]
    n = len(pos)
    p = sts.params(theta=0.7, degree=8, leaf_size=128, max_level=16, precision=sts.STS_MIXED,
                   near_fp64_tau=0.01 * 4 * math.pi / n)
    d = lambda a: torch.from_numpy(a).to("cuda")
    sts.sts_tree_build(h, d(pos), p)
    v = sts.sts_velocity_dual(h, d(zeta), d(area), p).cpu().numpy()
    tr = O.Tree(pos, 128, 16)
    o, g = tr.dual_lists(0.7), sts.sts_dual_export(h)
    for k in sts.DUAL_KINDS:
        oo, go = np.lexsort((o[k][1], o[k][0])), np.lexsort((g[k][1], g[k][0]))
        assert np.array_equal(o[k][0][oo], g[k][0][go]) and np.array_equal(o[k][1][oo], g[k][1][go]), k
    ref, st = tr.velocity_dual(zeta, area, 0.7, 8, return_stats=True)
    assert sts.sts_dual_stats(h, 8) == st
    e2, em = O.rel_l2(v, ref, area), O.rel_max(v, ref)
    print(f"dual mixed vs FP64 oracle dual: rel_l2 {e2:.3e} rel_max {em:.3e}")
    assert e2 <= 1e-6
    assert em <= 1e-5
