"""GPU stream function (the Green's function of Sec. 2 as the kernel) against the FP64
oracle: direct sum and tree code (same lists and proxy weights as the velocity) within
1e-12, interaction counts identical, and psi consistent with the velocity (u = grad psi x x)
through the kinetic-energy identity; the mixed-precision tree code within 1e-6 of the FP64
oracle tree code, with and without the close-pair threshold, and at full size."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    c = sts.Context()
    yield c.h
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _clustered(seed):
    rng = np.random.default_rng(seed)
    c = np.array([0.3, -0.5, 0.8])
    c /= np.linalg.norm(c)
    p = c + 0.01 * rng.standard_normal((2000, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    return np.vstack([p, W.uniform_points(1000, seed + 1)])


def _rel(a, b, w):
    return math.sqrt(np.sum((a - b) ** 2 * w) / np.sum(b**2 * w))


def _abs_sum(pos, zeta, area):
    """(1/4pi) sum_{j != i} |zeta_j A_j log(|x_i - x_j|^2 / 2)| per target: the size of the
    terms, against which FP64 rounding of the potential sum is measured (the sum itself is
    much smaller for zero-mean vorticity: the log terms cancel)."""
    out = np.zeros(len(pos))
    w = np.abs(zeta * area)
    for i0 in range(0, len(pos), 512):
        d = pos[i0:i0 + 512, None, :] - pos[None, :, :]
        h = 0.5 * np.sum(d * d, axis=2)
        with np.errstate(divide="ignore"):
            t = np.where(h > 0, np.abs(np.log(np.where(h > 0, h, 1.0))), 0.0)
        out[i0:i0 + 512] = t @ w / (4 * math.pi)
    return out


def _check_fp64(psi, ref, pos, zeta, area):
    # every target within 1e-12 of its terms' size (summation order and FMA contraction differ
    # between the two sides: up to about n eps, typically sqrt(n) eps); rel l2 within 1e-11
    # (1e-12 for the velocity: the potential's log terms cancel by a factor of about 50 to 100
    # more for zero-mean vorticity)
    assert np.max(np.abs(psi - ref) / _abs_sum(pos, zeta, area)) <= 1e-12
    assert _rel(psi, ref, area) <= 1e-11


@pytest.mark.parametrize("n", [2, 3, 129, 1000, 4099])
def test_direct_potential_matches_oracle(ctx, n):
    pos = W.uniform_points(n, 60 + n)
    rng = np.random.default_rng(n)
    zeta, area = rng.standard_normal(n), rng.uniform(0.5, 1.5, n) * (4 * math.pi / n)
    psi = sts.sts_direct_potential(ctx, dev(pos), dev(zeta), dev(area)).cpu().numpy()
    ref = O.direct_potential(pos, zeta, area)
    _check_fp64(psi, ref, pos, zeta, area)


@pytest.mark.parametrize("case", ["rand3000", "ico4", "clustered", "duplicates"])
@pytest.mark.parametrize("degree", [4, 8])
def test_tree_potential_matches_oracle(ctx, case, degree):
    if case == "rand3000":
        pos, leaf = W.uniform_points(3000, 61), 16
    elif case == "ico4":
        pos, leaf = W.icosahedral_points(4), 32
    elif case == "clustered":
        pos, leaf = _clustered(62), 24
    else:
        p = W.uniform_points(900, 63)
        pos, leaf = np.vstack([p, p[:100]]), 8
    n = len(pos)
    rng = np.random.default_rng(64)
    zeta, area = rng.standard_normal(n), rng.uniform(0.5, 1.5, n) * (4 * math.pi / n)
    p = sts.params(theta=0.7, degree=degree, leaf_size=leaf, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    psi = sts.sts_potential(ctx, dev(zeta), dev(area), p).cpu().numpy()
    st = sts.sts_stats(ctx)
    tr = O.Tree(pos, leaf)
    ref, ost = tr.potential(zeta, area, 0.7, degree, return_stats=True)
    assert st == ost
    _check_fp64(psi, ref, pos, zeta, area)


def test_potential_and_velocity_share_the_tree_and_energy(ctx):
    pos = W.icosahedral_points(5)
    area = W.voronoi_areas(pos)
    zeta = W.rh_vorticity(pos, 0.4, 0.2)
    p = sts.params(theta=0.7, degree=8, leaf_size=64, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), p)
    u = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    psi = sts.sts_potential(ctx, dev(zeta), dev(area), p).cpu().numpy()
    u2 = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    assert np.array_equal(u, u2)  # the potential call leaves the velocity path unchanged
    ep = 0.5 * np.sum(psi * zeta * area)
    eu = 0.5 * np.sum(np.sum(u * u, axis=1) * area)
    assert abs(ep - eu) <= 1e-2 * eu  # both quadratures of the same energy (level 5: 5.4e-3)


def test_potential_arguments(ctx):
    pos = W.uniform_points(100, 65)
    z, a = np.ones(100), np.ones(100)
    with pytest.raises(sts.StsError):
        sts.sts_direct_potential(ctx, dev(pos), dev(z), dev(a), precision=sts.STS_MIXED)
    sts.sts_tree_build(ctx, dev(pos), sts.params(leaf_size=16))
    one = sts.sts_direct_potential(ctx, dev(pos[:1]), dev(z[:1]), dev(a[:1])).cpu().numpy()
    assert one[0] == 0.0


def _check_mixed(psi, ref, pos, zeta, area):
    # the mixed bar (1e-6 rel l2), and every target within 1e-6 of its terms' size
    assert _rel(psi, ref, area) <= 1e-6
    assert np.max(np.abs(psi - ref) / _abs_sum(pos, zeta, area)) <= 1e-6


@pytest.mark.parametrize("case", ["rand3000", "ico4", "clustered", "duplicates"])
@pytest.mark.parametrize("tau_c", [0.0, 0.01])
def test_tree_potential_mixed_matches_oracle(ctx, case, tau_c):
    """Mixed precision (FP32 log2 terms in compensated sums, close pairs in FP64) against the
    FP64 oracle tree code on the same tree; coincident points (the target itself, duplicates)
    add nothing even without a close-pair threshold."""
    if case == "rand3000":
        pos, leaf = W.uniform_points(3000, 61), 16
    elif case == "ico4":
        pos, leaf = W.icosahedral_points(4), 32
    elif case == "clustered":
        pos, leaf = _clustered(62), 24
    else:
        p = W.uniform_points(900, 63)
        pos, leaf = np.vstack([p, p[:100]]), 8
    n = len(pos)
    rng = np.random.default_rng(65)
    zeta = rng.standard_normal(n)
    zeta -= np.mean(zeta)  # zero mean: the log terms cancel, as for a vorticity on the sphere
    area = rng.uniform(0.5, 1.5, n) * (4 * math.pi / n)
    p = sts.params(theta=0.7, degree=8, leaf_size=leaf, precision=sts.STS_MIXED,
                   near_fp64_tau=tau_c * 4 * math.pi / n)
    sts.sts_tree_build(ctx, dev(pos), p)
    psi = sts.sts_potential(ctx, dev(zeta), dev(area), p).cpu().numpy()
    ref = O.Tree(pos, leaf).potential(zeta, area, 0.7, 8)
    _check_mixed(psi, ref, pos, zeta, area)


def test_tree_potential_mixed_fullsize(ctx):
    """rand655k_sh16 (N = 655362, theta 0.7, d 8, N_T 128): the mixed stream function within
    1e-6 (rel l2) of the FP64 tree code on the same tree (which the tests above hold to the
    oracle's tree code within 1e-11)."""
    wl = W.workload("rand655k_sh16")
    pos, zeta, area = wl["pos"], wl["zeta"], wl["area"]
    n = len(pos)
    pm = sts.params(theta=0.7, degree=8, leaf_size=128, precision=sts.STS_MIXED, near_fp64_tau=0.01 * 4 * math.pi / n)
    p64 = sts.params(theta=0.7, degree=8, leaf_size=128, precision=sts.STS_FP64)
    sts.sts_tree_build(ctx, dev(pos), pm)
    psi = sts.sts_potential(ctx, dev(zeta), dev(area), pm).cpu().numpy()
    psi64 = sts.sts_potential(ctx, dev(zeta), dev(area), p64).cpu().numpy()
    assert _rel(psi, psi64, area) <= 1e-6
