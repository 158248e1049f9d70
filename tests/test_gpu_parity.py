"""GPU path vs the FP64 CPU oracle, through the C ABI (``paper_2401_07361_gb300.sts``).

Bars (stated in the method's target): tree, keys, permutation and interaction lists are
bit-exact; FP64 velocities within 1e-12 relative l2 of the oracle; mixed-precision
velocities within 1e-6 relative l2 of the FP64 oracle at the same theta, degree and leaf
size.  Relative l2 is the area-weighted E of Sec. 4.1; the max-norm is
max_i |v_i - v_ref,i| / max_i |v_ref,i|.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TREE_FIELDS = ("perm", "level", "key", "parent", "first_child", "nchild", "start", "count", "leaf", "leaves")


@pytest.fixture(scope="module")
def ctx():
    c = sts.Context()
    yield c.h
    c.close()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda", dtype if dtype is not None else t.dtype)


def _clustered(n_cap, n_uni, seed):
    rng = np.random.default_rng(seed)
    c = np.array([0.3, -0.5, 0.8])
    c /= np.linalg.norm(c)
    p = c + 0.01 * rng.standard_normal((n_cap, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return np.vstack([p, W.uniform_points(n_uni, seed + 1)])


def _case(name):
    if name == "rand3000":
        return W.uniform_points(3000, 21), 16, 16
    if name == "ico4":
        return W.icosahedral_points(4), 32, 16
    if name == "rand20000":
        return W.uniform_points(20000, 22), 64, 16
    if name == "leaf1_depth6":
        return W.uniform_points(5000, 23), 1, 6
    if name == "clustered":
        return _clustered(4000, 1000, 24), 24, 16
    if name == "duplicates":
        p = W.uniform_points(900, 25)
        return np.vstack([p, p[:100]]), 8, 16
    raise KeyError(name)


CASES = ["rand3000", "ico4", "rand20000", "leaf1_depth6", "clustered", "duplicates"]


def _fields(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.uniform(0.5, 1.5, n) * (4 * math.pi / n)


@pytest.mark.parametrize("name", CASES)
def test_tree_bit_exact(ctx, name):
    pos, leaf, ml = _case(name)
    p = sts.params(leaf_size=leaf, max_level=ml)
    sts.sts_tree_build(ctx, dev(pos), p)
    g = sts.sts_tree_export(ctx)
    o = O.Tree(pos, leaf, ml).export()
    for k in TREE_FIELDS:
        assert np.array_equal(g[k], o[k]), k
    assert np.array_equal(g["geom"], o["geom"])  # the FP64 geometry itself, bit for bit


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("theta", [0.5, 0.7, 0.9])
def test_lists_bit_exact(ctx, name, theta):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 1)
    p = sts.params(theta=theta, degree=4, leaf_size=leaf, max_level=ml, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    sts.sts_velocity(ctx, dev(zeta), dev(area), p)
    g = sts.sts_lists_export(ctx)
    tr = O.Tree(pos, leaf, ml)
    o = tr.lists(theta)
    for k in ("far_off", "far_idx", "near_off", "near_idx"):
        assert np.array_equal(g[k], o[k]), k
    _, st = tr.velocity(zeta, area, theta, 4, return_stats=True)
    assert sts.sts_stats(ctx) == st


@pytest.mark.parametrize("case", ["clustered_leaf4_theta0.6", "rand20000_leaf16_theta0.3"])
def test_lists_bit_exact_past_warp_capacity(ctx, case):
    """Leaves whose lists exceed the warp traversal's shared-memory capacity (256 terminals
    for theta >= 0.6, 512 below) go to the per-thread traversal; both must give the oracle's
    lists, and the velocities built on them must match the oracle."""
    if case.startswith("clustered"):
        # leaves of 4 particles inside the 0.01-radius cap are triangles of edge ~1e-3: their
        # FP64 barycentric coordinates carry rounding ~eps / edge, which the two sides take
        # differently (Cramer's rule on one side, a pre-divided frame on the other), and the
        # proxy contraction amplifies it; a dropped or doubled interaction would be O(1e-3)
        pos, leaf, theta, tol = _clustered(4000, 1000, 24), 4, 0.6, 1e-10
    else:
        pos, leaf, theta, tol = W.uniform_points(20000, 22), 16, 0.3, 1e-12
    tr = O.Tree(pos, leaf, 16)
    o = tr.lists(theta)
    terms = np.diff(o["far_off"]) + np.diff(o["near_off"])
    assert terms.max() > (256 if theta >= 0.6 else 512)  # the fallback really runs
    n = len(pos)
    zeta, area = _fields(n, 8)
    p = sts.params(theta=theta, degree=4, leaf_size=leaf, max_level=16, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    g = sts.sts_lists_export(ctx)
    for k in ("far_off", "far_idx", "near_off", "near_idx"):
        assert np.array_equal(g[k], o[k]), k
    assert O.rel_l2(v, tr.velocity(zeta, area, theta, 4), area) <= tol


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("degree", [3, 8])
def test_velocity_fp64_matches_oracle(ctx, name, degree):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 2)
    p = sts.params(theta=0.7, degree=degree, leaf_size=leaf, max_level=ml, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    ref = O.Tree(pos, leaf, ml).velocity(zeta, area, 0.7, degree)
    assert O.rel_l2(v, ref, area) <= 1e-12
    assert O.rel_max(v, ref) <= 1e-11


@pytest.mark.parametrize("name", CASES)
def test_velocity_mixed_within_1e6_of_fp64_oracle(ctx, name):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 3)
    tau = 0.05 * 4 * math.pi / n
    p = sts.params(theta=0.7, degree=8, leaf_size=leaf, max_level=ml, precision=sts.STS_MIXED, near_fp64_tau=tau)
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    ref = O.Tree(pos, leaf, ml).velocity(zeta, area, 0.7, 8)
    assert O.rel_l2(v, ref, area) <= 1e-6
    assert O.rel_max(v, ref) <= 1e-5


@pytest.mark.parametrize("n,leaf", [(2, 1), (3, 1), (5, 2), (17, 4), (64, 64), (65, 64), (129, 16), (700, 128),
                                    (700, 8), (1500, 3)])
def test_small_and_ragged_mixed_and_fp64(ctx, n, leaf):
    """Tiny trees, leaves of one particle, leaves just over a task's 64 targets, odd counts:
    every lane class S = 1..8 and ragged block and task tails, FP64 and mixed against the
    oracle."""
    pos = W.uniform_points(n, 80 + n)
    zeta, area = _fields(n, 81)
    ref = O.Tree(pos, leaf).velocity(zeta, area, 0.6, 6)
    for prec, tol in ((sts.STS_FP64, 1e-12), (sts.STS_MIXED, 1e-6)):
        p = sts.params(theta=0.6, degree=6, leaf_size=leaf, precision=prec, near_fp64_tau=0.01 * 4 * math.pi / n)
        sts.sts_tree_build(ctx, dev(pos), p)
        v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
        assert O.rel_l2(v, ref, area) <= tol, (prec, O.rel_l2(v, ref, area))


@pytest.mark.parametrize("degree", [1, 2, 10, 14, 16])
def test_extreme_degrees(ctx, degree):
    """Degrees 1 to 16 (M = 3 to 153 proxy points, the largest the tables hold) with far
    clusters present, FP64 and mixed against the oracle.  At degree 16 the FP64 tolerance is
    1e-11: cond(V_ref) grows by orders of magnitude per degree, and the contraction carries
    the moments' summation-order rounding (which differs between the two sides) into W."""
    pos = W.uniform_points(3000, 90)
    zeta, area = _fields(3000, 91)
    ref = O.Tree(pos, 16).velocity(zeta, area, 0.7, degree)
    p = sts.params(theta=0.7, degree=degree, leaf_size=16, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    assert sts.sts_stats(ctx)["pc"] > 0
    assert O.rel_l2(v, ref, area) <= (1e-12 if degree <= 14 else 1e-11)
    p = sts.params(theta=0.7, degree=degree, leaf_size=16, precision=sts.STS_MIXED,
                   near_fp64_tau=0.01 * 4 * math.pi / 3000)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    assert O.rel_l2(v, ref, area) <= 1e-6


@pytest.mark.parametrize("name", ["rand3000", "clustered"])
def test_proxy_weights_match_oracle(ctx, name):
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 4)
    p = sts.params(theta=0.7, degree=6, leaf_size=leaf, max_level=ml, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    sts.sts_velocity(ctx, dev(zeta), dev(area), p)
    ids, yt, Wg = sts.sts_clusters_export(ctx, 6)
    tr = O.Tree(pos, leaf, ml)
    oids, oyt, oW = tr.clusters(zeta, area, 6)
    assert np.array_equal(ids, oids)
    assert np.max(np.abs(yt - oyt)) <= 4e-16
    # W_m = rho_m^d sum_k Vinv[k][m] omega_k with omega_k = sum_j w_j B_k(b_j).  The two sides
    # round omega_k differently in two ways: (1) the order of the sum, bounded by
    # (count + 2d + 16) eps sum_j |w_j B_k(b_j)|; (2) the barycentric coordinates b = T^-1 y
    # of Sec. 3.2, whose absolute rounding is ~3 eps |row_i of T^-1| (large for small
    # triangles), moving B_k by at most d sum_i |db_i| since |dB_k/db_i| <= d inside the
    # triangle.  The contraction carries both into W with weights rho_m^d |Vinv[k][m]|
    # (cond(V_ref) ~ 8e3 at d = 6 makes this >> eps |W_m|).
    d = 6
    ex = tr.export()
    vinv = O.vref_inverse(d)
    beta, _ = O.proxy_reference(d)
    aw = np.abs(zeta * area)
    eps = np.finfo(float).eps
    for q, node in enumerate(oids):
        v = ex["geom"][node, :9].reshape(3, 3)
        cnt = ex["count"][node]
        idx = ex["perm"][ex["start"][node]:ex["start"][node] + cnt]
        _, _, om_abs = O.cluster(v.ravel(), d, pos[idx], aw[idx])
        rows = np.array([np.cross(v[1], v[2]), np.cross(v[2], v[0]), np.cross(v[0], v[1])])
        rows /= np.dot(v[0], rows[0])
        db = 3 * eps * np.linalg.norm(rows, axis=1).sum()
        dom = (cnt + 2 * d + 16) * eps * np.abs(om_abs) + 2 * d * db * aw[idx].sum()
        rho = np.linalg.norm(beta @ v, axis=1)
        bound = rho ** d * (np.abs(vinv).T @ dom)
        assert np.all(np.abs(Wg[q] - oW[q]) <= bound), q


@pytest.mark.parametrize("name", ["rand3000", "ico4", "clustered"])
@pytest.mark.parametrize("d", [6, 8, 10, 11])
def test_proxy_weights_tensor_core_match_oracle(ctx, name, d):
    # Mixed precision forms sum_k omega_k Vinv[k][m] on the tensor cores from exact 8-bit digit
    # products (moment k scaled by 2^E_k, E_k = -round(log2(simplex integral of B_k)), then
    # kept to 32 bits of the largest scaled moment; Vinv to every FP64 bit; d = 10 and 11 take
    # two rounds of tensor-memory columns).  W_m = rho_m^d sum_k Vinv[k][m] omega_k then
    # differs from the oracle's FP64 weights only through omega: its FP32 moments (the FP64
    # bound of test_proxy_weights_match_oracle with FP32's epsilon) and that truncation.  A
    # wrong operand layout, digit or scale misses this by orders of magnitude.
    pos, leaf, ml = _case(name)
    n = len(pos)
    zeta, area = _fields(n, 4)
    p = sts.params(theta=0.7, degree=d, leaf_size=leaf, max_level=ml, precision=sts.STS_MIXED,
                   near_fp64_tau=0.0)
    sts.sts_tree_build(ctx, dev(pos), p)
    sts.sts_velocity(ctx, dev(zeta), dev(area), p)
    ids, yt, Wg = sts.sts_clusters_export(ctx, d)
    tr = O.Tree(pos, leaf, ml)
    oids, oyt, oW = tr.clusters(zeta, area, d)
    assert np.array_equal(ids, oids) and len(ids) > 0
    ex = tr.export()
    vinv = np.abs(O.vref_inverse(d))
    beta, _ = O.proxy_reference(d)
    aw = np.abs(zeta * area)
    e32 = float(np.finfo(np.float32).eps)
    fact = math.factorial
    Ek = np.array([-round(math.log2(fact(a) * fact(b) * fact(d - a - b) * 2 / fact(d + 2)))
                   for a in range(d, -1, -1) for b in range(d - a, -1, -1)], dtype=float)
    for q, node in enumerate(oids):
        v = ex["geom"][node, :9].reshape(3, 3)
        cnt = ex["count"][node]
        idx = ex["perm"][ex["start"][node]:ex["start"][node] + cnt]
        _, _, om_abs = O.cluster(v.ravel(), d, pos[idx], aw[idx])
        rows = np.array([np.cross(v[1], v[2]), np.cross(v[2], v[0]), np.cross(v[0], v[1])])
        rows /= np.dot(v[0], rows[0])
        db = 6 * e32 * np.linalg.norm(rows, axis=1).sum()
        dom = (cnt + 2 * d + 16) * e32 * om_abs + 2 * d * db * aw[idx].sum()
        dom = dom + 2.0 ** -31 * np.max((om_abs + dom) * 2.0 ** Ek) * 2.0 ** -Ek
        rho = np.linalg.norm(beta @ v, axis=1)
        bound = rho ** d * (vinv.T @ dom)
        assert np.all(np.abs(Wg[q] - oW[q]) <= bound), (q, np.max(np.abs(Wg[q] - oW[q]) / bound))


@pytest.mark.parametrize("n", [2, 3, 129, 1000, 4099])
@pytest.mark.parametrize("prec", [sts.STS_FP64, sts.STS_MIXED])
def test_direct_matches_oracle(ctx, n, prec):
    pos = W.uniform_points(n, 30 + n)
    zeta, area = _fields(n, 5)
    v = sts.sts_direct(ctx, dev(pos), dev(zeta), dev(area), prec).cpu().numpy()
    ref = O.direct(pos, zeta, area)
    tol = 1e-12 if prec == sts.STS_FP64 else 1e-6
    assert O.rel_l2(v, ref, area) <= tol
    assert O.rel_max(v, ref) <= 10 * tol


def test_direct_duplicates_and_targets(ctx):
    pos = W.uniform_points(700, 40)
    pos = np.vstack([pos, pos[:50]])
    n = len(pos)
    zeta, area = _fields(n, 6)
    tg = np.array([0, 5, 749, 700, 3, 3], np.int64)
    ref = O.direct(pos, zeta, area, targets=tg)
    for prec, tol in ((sts.STS_FP64, 1e-12), (sts.STS_MIXED, 1e-6)):
        v = sts.sts_direct_targets(ctx, dev(pos), dev(zeta), dev(area), dev(tg), prec).cpu().numpy()
        assert np.max(np.abs(v - ref)) <= tol * np.max(np.abs(ref))


def test_edge_cases(ctx):
    p = sts.params(precision=sts.STS_FP64)
    e = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    z0 = torch.zeros(0, dtype=torch.float64, device="cuda")
    sts.sts_tree_build(ctx, e, p)
    assert sts.sts_velocity(ctx, z0, z0, p).shape == (0, 3)
    one = dev(W.uniform_points(1, 1))
    o1 = torch.ones(1, dtype=torch.float64, device="cuda")
    sts.sts_tree_build(ctx, one, p)
    assert torch.all(sts.sts_velocity(ctx, o1, o1, p) == 0)
    assert torch.all(sts.sts_direct(ctx, one, o1, o1) == 0)
    two = W.uniform_points(2, 2)
    z2, a2 = np.array([1.0, -2.0]), np.array([0.3, 0.4])
    sts.sts_tree_build(ctx, dev(two), p)
    v = sts.sts_velocity(ctx, dev(z2), dev(a2), p).cpu().numpy()
    assert np.allclose(v, O.direct(two, z2, a2), rtol=1e-14, atol=0)
    with pytest.raises(sts.StsError):
        sts.sts_velocity(ctx, dev(z2), dev(a2), sts.params(theta=1.0))
    with pytest.raises(sts.StsError):
        sts.sts_tree_build(ctx, dev(two), sts.params(degree=17))
    bad = two.copy()
    bad[1, 0] = np.nan
    with pytest.raises(sts.StsError):
        sts.sts_tree_build(ctx, dev(bad), p)


def test_velocity_requires_tree():
    with sts.Context() as c:
        z = torch.ones(4, dtype=torch.float64, device="cuda")
        with pytest.raises(sts.StsError, match="no tree"):
            sts.sts_velocity(c.h, z, z, sts.params())


def test_rk4_step_matches_oracle(ctx):
    pos = W.uniform_points(3000, 50)
    area = W.equal_areas(3000)
    zeta = W.rh_vorticity(pos, math.pi / 7, 1.0)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_FP64)
    x, z = dev(pos), dev(zeta)
    sts.bve_rk4_step(ctx, x, z, dev(area), 0.01, 2 * math.pi, p)
    vel = lambda xx, zz, aa: O.Tree(xx, 32, 16).velocity(zz, aa, 0.7, 6)
    ox, oz = O.rk4_step(pos, zeta, area, 0.01, 2 * math.pi, vel)
    assert np.max(np.abs(x.cpu().numpy() - ox)) <= 1e-13
    assert np.max(np.abs(z.cpu().numpy() - oz)) <= 1e-12 * np.max(np.abs(oz))
    assert np.max(np.abs(np.linalg.norm(x.cpu().numpy(), axis=1) - 1)) <= 4e-16


def test_repeat_calls_are_deterministic(ctx):
    pos = W.uniform_points(8000, 60)
    zeta, area = _fields(8000, 7)
    p = sts.params(theta=0.7, degree=8, leaf_size=64, precision=sts.STS_MIXED, near_fp64_tau=1e-4)
    sts.sts_tree_build(ctx, dev(pos), p)
    a = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    sts.sts_tree_build(ctx, dev(pos), p)
    b = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    assert np.array_equal(a, b)


def test_tree_bit_exact_on_reused_device_memory():
    """Buffers from cudaMalloc hold whatever the process left there: fill the device memory
    with 0xFF bytes, hand it back, then build in a new context a forest whose sparse faces are
    leaves at the root (their particles never get a child digit written) next to faces that
    split.  The tree must still be the oracle's, bit for bit."""
    junk = torch.full((2**28,), -1, dtype=torch.int64, device="cuda")  # 2 GiB of 0xFF
    torch.cuda.synchronize()
    del junk
    torch.cuda.empty_cache()
    pos = _clustered(3000, 150, 31)  # one dense cap, most faces with a few points
    with sts.Context() as c:
        p = sts.params(leaf_size=32, max_level=16)
        sts.sts_tree_build(c.h, dev(pos), p)
        g = sts.sts_tree_export(c.h)
    o = O.Tree(pos, 32, 16).export()
    assert (o["count"][o["level"] == 0] <= 32).any() and (o["level"] > 0).any()
    for k in TREE_FIELDS:
        assert np.array_equal(g[k], o[k]), k
