"""Dual tree traversal (Sec. 3.4, all four interactions PP, PC, CP, CC) on the GPU against the
FP64 CPU oracle, through the C ABI.

Bars: the four pair lists are bit-exact (the same (target, source) node pairs; both sides are
compared after sorting by target, then source), and so are the interaction counts; FP64
velocities within max(1e-12, 0.1 eps cond(V_ref)) relative l2 of the oracle's dual velocity
(10x that in the max-norm); mixed precision within 1e-6 relative l2 of it.

Why the FP64 bar grows with the degree: CP and CC give the velocity U at the target cluster's
proxy points, and the interpolating polynomial's monomial coefficients c solve V_T c = U.  The
oracle solves that system by LU with partial pivoting; the kernel applies the precomputed
V_ref^-1 and the proxies' radial factors.  Both are backward stable, but the coefficients (and
the sum of B_k c_k at a particle, whose terms cancel) carry rounding of order eps cond(V_ref)
relative to the interpolant, which neither side can avoid: cond(V_ref) = 36 at degree 3,
3.5e5 at degree 8, 4.6e8 at degree 12.  Measured: 2.0e-12 on the clustered case at degree 8
(eps cond = 7.8e-11), below 1e-12 everywhere else.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_parity import CASES, _case, _clustered, _fields  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = sts.Context()
    yield c.h
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _sorted_pairs(t, s):
    o = np.lexsort((s, t))
    return t[o], s[o]


def _tau(n):
    return 0.01 * 4 * math.pi / n


def _tol64(degree):
    _, vinv = sts.sts_proxy_reference(degree)
    return max(1e-12, 0.1 * np.finfo(float).eps * np.linalg.cond(np.linalg.inv(vinv)))


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("theta", [0.5, 0.7, 0.9])
def test_dual_lists_bit_exact(ctx, name, theta):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 1)
    p = sts.params(theta=theta, degree=4, leaf_size=leaf, max_level=ml, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p)
    g = sts.sts_dual_export(ctx)
    tr = O.Tree(pos, leaf, ml)
    o = tr.dual_lists(theta)
    for k in sts.DUAL_KINDS:
        gt, gs = _sorted_pairs(*g[k])
        ot, os_ = _sorted_pairs(*o[k])
        assert np.array_equal(gt, ot), k
        assert np.array_equal(gs, os_), k
        assert len(gt) > 0, k  # every case exercises every kind
    # the GPU's own order: by target key (depth-first leaf / cluster order), then source
    ex = sts.sts_tree_export(ctx)
    leaf_rank = np.full(len(ex["level"]), -1)
    leaf_rank[ex["leaves"]] = np.arange(len(ex["leaves"]))
    t, s = g["PP"]
    key = leaf_rank[t]
    assert np.all(np.diff(key) >= 0) and np.all((np.diff(key) > 0) | (np.diff(s) > 0))
    _, st = tr.velocity_dual(zeta, area, theta, 4, return_stats=True)
    assert sts.sts_dual_stats(ctx, 4) == st


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("degree", [3, 8])
def test_dual_velocity_fp64(ctx, name, degree):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 2)
    p = sts.params(theta=0.7, degree=degree, leaf_size=leaf, max_level=ml, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
    ref = O.Tree(pos, leaf, ml).velocity_dual(zeta, area, 0.7, degree)
    tol = _tol64(degree)
    assert O.rel_l2(v, ref, area) <= tol, O.rel_l2(v, ref, area)
    assert O.rel_max(v, ref) <= 10 * tol, O.rel_max(v, ref)


@pytest.mark.parametrize("name", CASES)
def test_dual_velocity_mixed(ctx, name):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 3)
    p = sts.params(theta=0.7, degree=8, leaf_size=leaf, max_level=ml, precision=sts.STS_MIXED,
                   near_fp64_tau=_tau(n))
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
    ref = O.Tree(pos, leaf, ml).velocity_dual(zeta, area, 0.7, 8)
    assert O.rel_l2(v, ref, area) <= 1e-6, O.rel_l2(v, ref, area)
    assert O.rel_max(v, ref) <= 1e-5


@pytest.mark.parametrize("n,leaf", [(2, 1), (3, 1), (5, 2), (17, 4), (64, 64), (65, 64), (129, 16), (700, 128),
                                    (700, 8), (1500, 3)])
def test_dual_small_and_ragged(ctx, n, leaf):
    """Tiny trees (no clusters at all for n <= leaf size), leaves of one particle, odd counts:
    FP64 and mixed against the oracle, and the lists bit for bit."""
    pos = W.uniform_points(n, 180 + n)
    zeta, area = _fields(n, 181)
    tr = O.Tree(pos, leaf)
    ref = tr.velocity_dual(zeta, area, 0.6, 6)
    o = tr.dual_lists(0.6)
    for prec, tol in ((sts.STS_FP64, 1e-12), (sts.STS_MIXED, 1e-6)):
        p = sts.params(theta=0.6, degree=6, leaf_size=leaf, precision=prec, near_fp64_tau=_tau(n))
        sts.sts_tree_build(ctx, dev(pos), p)
        v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
        assert O.rel_l2(v, ref, area) <= tol, (prec, O.rel_l2(v, ref, area))
        g = sts.sts_dual_export(ctx)
        for k in sts.DUAL_KINDS:
            assert all(np.array_equal(a, b) for a, b in zip(_sorted_pairs(*g[k]), _sorted_pairs(*o[k]))), k


def test_dual_empty_and_single(ctx):
    p = sts.params(theta=0.7, degree=4, leaf_size=8, precision=sts.STS_FP64)
    for n in (0, 1):
        pos = W.uniform_points(max(n, 1), 5)[:n]
        sts.sts_tree_build(ctx, dev(pos.reshape(n, 3)), p)
        v = sts.sts_velocity_dual(ctx, dev(np.ones(n)), dev(np.ones(n)), p).cpu().numpy()
        assert v.shape == (n, 3) and np.all(v == 0.0)


def test_dual_batched_instances(ctx):
    """A forest of instances: each target interacts with its own instance only, so every
    instance's dual velocity equals the oracle's on that instance alone."""
    sizes = [3000, 0, 1200, 40]
    pts = [W.uniform_points(m, 300 + i) if m else np.zeros((0, 3)) for i, m in enumerate(sizes)]
    pos = np.vstack(pts)
    n = len(pos)
    zeta, area = _fields(n, 301)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    for prec, tol in ((sts.STS_FP64, 1e-12), (sts.STS_MIXED, 1e-6)):
        p = sts.params(theta=0.7, degree=6, leaf_size=16, precision=prec, near_fp64_tau=_tau(3000))
        sts.sts_tree_build_batched(ctx, dev(pos), off, p)
        v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
        for b in range(len(sizes)):
            a, e = off[b], off[b + 1]
            if e - a < 2:
                continue
            ref = O.Tree(pos[a:e], 16).velocity_dual(zeta[a:e], area[a:e], 0.7, 6)
            assert O.rel_l2(v[a:e], ref, area[a:e]) <= tol, (prec, b)


def test_dual_and_leaf_lists_alternate(ctx):
    """The dual lists replace the target-leaf lists in the context and back: alternating the
    two evaluations on one tree gives each one's own result, bit for bit (FP64)."""
    pos, leaf, ml = _case("rand20000")
    n = len(pos)
    zeta, area = _fields(n, 4)
    p = sts.params(theta=0.7, degree=6, leaf_size=leaf, max_level=ml, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    z, a = dev(zeta), dev(area)
    v1 = sts.sts_velocity(ctx, z, a, p).cpu().numpy()
    d1 = sts.sts_velocity_dual(ctx, z, a, p).cpu().numpy()
    v2 = sts.sts_velocity(ctx, z, a, p).cpu().numpy()
    d2 = sts.sts_velocity_dual(ctx, z, a, p).cpu().numpy()
    assert np.array_equal(v1, v2) and np.array_equal(d1, d2)
    tr = O.Tree(pos, leaf, ml)
    assert O.rel_l2(v1, tr.velocity(zeta, area, 0.7, 6), area) <= 1e-12
    assert O.rel_l2(d1, tr.velocity_dual(zeta, area, 0.7, 6), area) <= 1e-12
    # both approximate the same direct sum at the tree code's accuracy
    ex = O.direct(pos, zeta, area)
    assert O.rel_l2(d1, ex, area) < 1e-3 and O.rel_l2(v1, ex, area) < 1e-3


@pytest.mark.parametrize("degree", [1, 12])
def test_dual_extreme_degrees(ctx, degree):
    """Low and high degrees: the interpolation of CP / CC velocities back to the particles
    uses V_ref^-1 with the proxies' radial factors, against the oracle's solve of V_T."""
    pos = W.uniform_points(3000, 95)
    zeta, area = _fields(3000, 96)
    ref = O.Tree(pos, 16).velocity_dual(zeta, area, 0.7, degree)
    for prec, tol in ((sts.STS_FP64, _tol64(degree)), (sts.STS_MIXED, 1e-6)):
        p = sts.params(theta=0.7, degree=degree, leaf_size=16, precision=prec, near_fp64_tau=_tau(3000))
        sts.sts_tree_build(ctx, dev(pos), p)
        v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
        assert O.rel_l2(v, ref, area) <= tol, (prec, O.rel_l2(v, ref, area))


def test_dual_clustered_close_pairs(ctx):
    """Leaves of 4 inside a 0.01-radius cap (tiny clusters at depth 16) with a large tau: the
    FP64 close-pair path runs for proxy targets too (CP blocks whose distance bound falls
    below tau)."""
    pos = _clustered(4000, 1000, 124)
    n = len(pos)
    zeta, area = _fields(n, 125)
    ref = O.Tree(pos, 4, 16).velocity_dual(zeta, area, 0.6, 6)
    p = sts.params(theta=0.6, degree=6, leaf_size=4, max_level=16, precision=sts.STS_MIXED,
                   near_fp64_tau=1.0 * 4 * math.pi / n)
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
    assert O.rel_l2(v, ref, area) <= 1e-6, O.rel_l2(v, ref, area)


@pytest.mark.parametrize("prec", [sts.STS_FP64, sts.STS_MIXED])
def test_dual_velocity_tangent(ctx, prec):
    """The interpolated CP / CC part enters as x x (the interpolated kernel sum), so the dual
    velocity is tangent to the sphere to rounding, in both precisions."""
    pos, leaf, ml = _case("rand20000")
    zeta, area = _fields(len(pos), 7)
    p = sts.params(theta=0.7, degree=8, leaf_size=leaf, max_level=ml, precision=prec, near_fp64_tau=_tau(len(pos)))
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity_dual(ctx, dev(zeta), dev(area), p).cpu().numpy()
    assert np.max(np.abs(np.sum(pos * v, axis=1))) <= 1e-14 * np.max(np.linalg.norm(v, axis=1))
