"""Batched instances (the ensemble path): a forest of independent instances built and
evaluated together must give every instance exactly what it gets alone, and match the FP64
oracle per instance."""
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


def _instances():
    """Uneven instances: random, icosahedral (edge ties), an empty one, a single particle,
    duplicates, and a tight cluster."""
    rng = np.random.default_rng(7)
    inst = [W.uniform_points(3000, 70), W.icosahedral_points(3), np.zeros((0, 3)), W.uniform_points(1, 71)]
    p = W.uniform_points(400, 72)
    inst.append(np.vstack([p, p[:37]]))
    c = np.array([0.1, 0.9, -0.2])
    c /= np.linalg.norm(c)
    q = c + 0.02 * rng.standard_normal((900, 3))
    inst.append(q / np.linalg.norm(q, axis=1, keepdims=True))
    out = []
    for k, pos in enumerate(inst):
        n = len(pos)
        zeta = rng.standard_normal(n)
        area = rng.uniform(0.5, 1.5, n) * (4 * math.pi / max(n, 1))
        out.append((pos, zeta, area))
    return out


def _concat(inst):
    pos = np.vstack([i[0] for i in inst])
    zeta = np.concatenate([i[1] for i in inst])
    area = np.concatenate([i[2] for i in inst])
    off = np.concatenate([[0], np.cumsum([len(i[0]) for i in inst])]).astype(np.int64)
    return pos, zeta, area, off


@pytest.mark.parametrize("prec,tau", [(sts.STS_FP64, 0.0), (sts.STS_MIXED, 0.0)])
def test_forest_equals_instances_alone_bitwise(ctx, prec, tau):
    inst = _instances()
    pos, zeta, area, off = _concat(inst)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=prec, near_fp64_tau=tau)
    sts.sts_tree_build_batched(ctx, dev(pos), off, p)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    stats = sts.sts_stats(ctx)
    pc = pp = 0
    for b, (ps, z, a) in enumerate(inst):
        sts.sts_tree_build(ctx, dev(ps), p)
        vb = sts.sts_velocity(ctx, dev(z), dev(a), p).cpu().numpy()
        assert np.array_equal(v[off[b]:off[b + 1]], vb), b
        if len(ps) > 1:
            st = sts.sts_stats(ctx)
            pc, pp = pc + st["pc"], pp + st["pp"]
    assert stats == {"pc": pc, "pp": pp}


def test_forest_mixed_with_tau_matches_oracle_per_instance(ctx):
    inst = _instances()
    pos, zeta, area, off = _concat(inst)
    tau = 0.05 * 4 * math.pi / 3000
    p = sts.params(theta=0.7, degree=8, leaf_size=32, precision=sts.STS_MIXED, near_fp64_tau=tau)
    p64 = sts.params(theta=0.7, degree=8, leaf_size=32, precision=sts.STS_FP64)
    sts.sts_tree_build_batched(ctx, dev(pos), off, p)
    v = sts.sts_velocity(ctx, dev(zeta), dev(area), p).cpu().numpy()
    v64 = sts.sts_velocity(ctx, dev(zeta), dev(area), p64).cpu().numpy()
    for b, (ps, z, a) in enumerate(inst):
        if len(ps) < 2:
            assert np.all(v[off[b]:off[b + 1]] == 0)
            continue
        ref = O.Tree(ps, 32).velocity(z, a, 0.7, 8)
        assert O.rel_l2(v64[off[b]:off[b + 1]], ref, a) <= 1e-12, b
        assert O.rel_l2(v[off[b]:off[b + 1]], ref, a) <= 1e-6, b


def test_batched_rk4_equals_instances_alone(ctx):
    inst = [x for x in _instances() if len(x[0]) > 0]
    pos, zeta, area, off = _concat(inst)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_FP64)
    x, z = dev(pos), dev(zeta)
    sts.bve_rk4_step_batched(ctx, x, z, dev(area), off, 0.01, 2 * math.pi, p)
    x, z = x.cpu().numpy(), z.cpu().numpy()
    for b, (ps, zb, a) in enumerate(inst):
        xb, zzb = dev(ps), dev(zb)
        sts.bve_rk4_step(ctx, xb, zzb, dev(a), 0.01, 2 * math.pi, p)
        assert np.array_equal(x[off[b]:off[b + 1]], xb.cpu().numpy()), b
        assert np.array_equal(z[off[b]:off[b + 1]], zzb.cpu().numpy()), b


def test_batched_offsets_are_checked(ctx):
    pos = dev(W.uniform_points(10, 1))
    p = sts.params()
    for bad in ([1, 10], [0, 5, 3, 10], [0, 9]):
        with pytest.raises(sts.StsError):
            sts.sts_tree_build_batched(ctx, pos, bad, p)


def test_autotuner_picks_fastest_within_budget():
    from paper_2401_07361_gb300.autotune import autotune

    pos = W.uniform_points(40962, 90)
    zeta = W.sh_series_vorticity(pos, 8, seed=3)
    area = W.equal_areas(len(pos))
    res = autotune(dev(pos), dev(zeta), dev(area), budget=1e-4, thetas=(0.5, 0.7), degrees=(4, 8),
                   leaf_sizes=(32, 128), samples=1024, repeats=2)
    ok = [t for t in res.table if t[4] <= 1e-4]
    assert res.error <= 1e-4 and ok
    assert res.ms == min(t[3] for t in ok)
    # the chosen parameters reproduce the measured accuracy against the oracle direct sum
    tg = np.random.default_rng(5).choice(len(pos), 256, replace=False)
    ref = O.direct(pos, zeta, area, targets=tg)
    with sts.Context() as c:
        p = res.params(near_fp64_tau=0.05 * 4 * math.pi / len(pos))
        sts.sts_set_traversal(c.h, res.dual)
        sts.sts_tree_build(c.h, dev(pos), p)
        v = sts.sts_velocity(c.h, dev(zeta), dev(area), p).cpu().numpy()
    assert O.rel_l2(v[tg], ref, area[tg]) <= 3e-4
    # both traversals were tried for every (theta, degree, leaf size)
    assert {t[5] for t in res.table} == {False, True} and len(res.table) == 16
