"""RK4 steps recorded as a CUDA graph: replays give exactly the eager results, including
after the particle distribution changes so much that the recording runs out of capacity
(the step is then undone and redone eagerly)."""
import math

import numpy as np
import pytest

from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _state(n, seed):
    pos = W.uniform_points(n, seed)
    zeta = W.rh_vorticity(pos, math.pi / 7, 1.0) + 0.1 * W.sh_series_vorticity(pos, 6, seed=seed)
    area = W.equal_areas(n)
    return pos, zeta, area


def _run(pos, zeta, area, p, steps, graph, stream, offsets=None, dual=False):
    with sts.Context() as c:
        sts.sts_set_graph(c.h, graph)
        sts.sts_set_traversal(c.h, dual)
        x = torch.from_numpy(pos).cuda()
        z = torch.from_numpy(zeta).cuda()
        a = torch.from_numpy(area).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(steps):
                if offsets is None:
                    sts.bve_rk4_step(c.h, x, z, a, 0.01, 2 * math.pi, p, stream=stream)
                else:
                    sts.bve_rk4_step_batched(c.h, x, z, a, offsets, 0.01, 2 * math.pi, p, stream=stream)
        stream.synchronize()
        info = sts.sts_tree_info(c.h, stream=stream)
        return x.cpu().numpy(), z.cpu().numpy(), info


def test_graph_steps_equal_eager_steps():
    pos, zeta, area = _state(6000, 3)
    p = sts.params(theta=0.7, degree=6, leaf_size=64, precision=sts.STS_FP64)
    st = torch.cuda.Stream()
    xe, ze, ie = _run(pos, zeta, area, p, 4, False, st)
    xg, zg, ig = _run(pos, zeta, area, p, 4, True, st)
    assert np.array_equal(xe, xg) and np.array_equal(ze, zg)
    assert ie == ig


def test_graph_batched_mixed_matches_eager():
    sizes = [3000, 1200, 4500]
    parts = [_state(nb, 10 + b) for b, nb in enumerate(sizes)]
    pos = np.vstack([q[0] for q in parts])
    zeta = np.concatenate([q[1] for q in parts])
    area = np.concatenate([q[2] for q in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    p = sts.params(theta=0.7, degree=8, leaf_size=64, precision=sts.STS_MIXED, near_fp64_tau=1e-6)
    st = torch.cuda.Stream()
    xe, ze, _ = _run(pos, zeta, area, p, 3, False, st, off)
    xg, zg, _ = _run(pos, zeta, area, p, 3, True, st, off)
    assert np.max(np.abs(xe - xg)) <= 1e-15
    assert np.max(np.abs(ze - zg)) <= 1e-14 * np.max(np.abs(ze))


def test_graph_overflow_falls_back_to_eager():
    pos, zeta, area = _state(5000, 4)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_FP64)
    st = torch.cuda.Stream()
    with sts.Context() as c:
        sts.sts_set_graph(c.h, True)
        x = torch.from_numpy(pos).cuda()
        z = torch.from_numpy(zeta).cuda()
        a = torch.from_numpy(area).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            sts.bve_rk4_step(c.h, x, z, a, 0.01, 2 * math.pi, p, stream=st)  # eager + record
            # squeeze every particle into a small cap: deeper tree, more nodes than recorded
            ctr = np.array([0.0, 0.0, 1.0])
            q = ctr + 0.02 * np.random.default_rng(5).standard_normal((5000, 3))
            q /= np.linalg.norm(q, axis=1, keepdims=True)
            x.copy_(torch.from_numpy(q).cuda())
            sts.bve_rk4_step(c.h, x, z, a, 0.01, 2 * math.pi, p, stream=st)  # replay overflows -> eager
        st.synchronize()
        xg = x.cpu().numpy()
    with sts.Context() as c:
        x = torch.from_numpy(q).cuda()
        z = torch.from_numpy(zeta).cuda()
        # the first step changed zeta too; redo it eagerly from the same start
        z0 = torch.from_numpy(zeta).cuda()
        x0 = torch.from_numpy(pos).cuda()
        sts.bve_rk4_step(c.h, x0, z0, a, 0.01, 2 * math.pi, p)
        sts.bve_rk4_step(c.h, x, z0, a, 0.01, 2 * math.pi, p)
        torch.cuda.synchronize()
        assert np.array_equal(xg, x.cpu().numpy())


@pytest.mark.parametrize("prec", [sts.STS_FP64, sts.STS_MIXED])
def test_recorded_tree_velocity_equals_eager(prec):
    pos, zeta, area = _state(20000, 8)
    p = sts.params(theta=0.7, degree=8, leaf_size=64, precision=prec)
    st = torch.cuda.Stream()
    d = lambda a: torch.from_numpy(a).cuda()
    x, z, a = d(pos), d(zeta), d(area)
    torch.cuda.synchronize()
    with sts.Context() as c:
        sts.sts_tree_build(c.h, x, p)
        ref = sts.sts_velocity(c.h, z, a, p).cpu().numpy()
    with sts.Context() as c, torch.cuda.stream(st):
        sts.sts_set_graph(c.h, True)
        vel = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(3):  # eager + record, then two replays
            sts.sts_tree_velocity(c.h, x, z, a, p, vel, stream=st)
            outs.append(vel.cpu().numpy())
        info = sts.sts_tree_info(c.h, stream=st)
        lists = sts.sts_lists_export(c.h, stream=st)
    for o in outs:
        assert np.array_equal(o, ref)
    assert info["leaves"] + 1 == len(lists["far_off"]) and info["nfar"] == len(lists["far_idx"])


@pytest.mark.parametrize("prec", [sts.STS_FP64, sts.STS_MIXED])
def test_recorded_dual_tree_velocity_equals_eager(prec):
    """The dual traversal recorded with the build (sts_set_traversal + sts_tree_velocity):
    replays give the eager sts_velocity_dual result bit for bit, and the pair lists exported
    after a replay are the eager ones."""
    pos, zeta, area = _state(20000, 9)
    p = sts.params(theta=0.7, degree=8, leaf_size=64, precision=prec)
    st = torch.cuda.Stream()
    d = lambda a: torch.from_numpy(a).cuda()
    x, z, a = d(pos), d(zeta), d(area)
    torch.cuda.synchronize()
    with sts.Context() as c:
        sts.sts_tree_build(c.h, x, p)
        ref = sts.sts_velocity_dual(c.h, z, a, p).cpu().numpy()
        ref_pairs = sts.sts_dual_export(c.h)
    with sts.Context() as c, torch.cuda.stream(st):
        sts.sts_set_graph(c.h, True)
        sts.sts_set_traversal(c.h, True)
        vel = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(3):  # eager + record, then two replays
            sts.sts_tree_velocity(c.h, x, z, a, p, vel, stream=st)
            outs.append(vel.cpu().numpy())
        pairs = sts.sts_dual_export(c.h, stream=st)
    for o in outs:
        assert np.array_equal(o, ref)
    for k in sts.DUAL_KINDS:
        assert np.array_equal(pairs[k][0], ref_pairs[k][0]) and np.array_equal(pairs[k][1], ref_pairs[k][1]), k


def test_graph_dual_steps_equal_eager_steps():
    pos, zeta, area = _state(6000, 13)
    p = sts.params(theta=0.7, degree=6, leaf_size=64, precision=sts.STS_FP64)
    st = torch.cuda.Stream()
    xe, ze, _ = _run(pos, zeta, area, p, 4, False, st, dual=True)
    xg, zg, _ = _run(pos, zeta, area, p, 4, True, st, dual=True)
    assert np.array_equal(xe, xg) and np.array_equal(ze, zg)
    # the dual traversal is another approximation of the same sum: the two velocities differ by
    # the tree codes' errors (about 1e-4 of |u| at theta 0.7, degree 6), so after 4 steps of
    # dt = 0.01 the positions agree to a few 1e-6
    xl, zl, _ = _run(pos, zeta, area, p, 4, False, st, dual=False)
    assert np.max(np.abs(xl - xe)) < 1e-4


def test_graph_dual_overflow_falls_back_to_eager():
    """A replay whose tree outgrows the recorded dual-traversal capacities (frontier, pairs,
    levels) is undone and redone eagerly: the result equals two eager steps."""
    pos, zeta, area = _state(5000, 14)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_FP64)
    st = torch.cuda.Stream()
    ctr = np.array([0.0, 0.0, 1.0])
    q = ctr + 0.02 * np.random.default_rng(15).standard_normal((5000, 3))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    with sts.Context() as c:
        sts.sts_set_graph(c.h, True)
        sts.sts_set_traversal(c.h, True)
        x = torch.from_numpy(pos).cuda()
        z = torch.from_numpy(zeta).cuda()
        a = torch.from_numpy(area).cuda()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            sts.bve_rk4_step(c.h, x, z, a, 0.01, 2 * math.pi, p, stream=st)  # eager + record
            x.copy_(torch.from_numpy(q).cuda())
            sts.bve_rk4_step(c.h, x, z, a, 0.01, 2 * math.pi, p, stream=st)  # replay overflows -> eager
        st.synchronize()
        xg = x.cpu().numpy()
    with sts.Context() as c:
        sts.sts_set_traversal(c.h, True)
        x = torch.from_numpy(q).cuda()
        z0 = torch.from_numpy(zeta).cuda()
        x0 = torch.from_numpy(pos).cuda()
        a = torch.from_numpy(area).cuda()
        sts.bve_rk4_step(c.h, x0, z0, a, 0.01, 2 * math.pi, p)
        sts.bve_rk4_step(c.h, x, z0, a, 0.01, 2 * math.pi, p)
        torch.cuda.synchronize()
        assert np.array_equal(xg, x.cpu().numpy())


def test_graph_batched_dual_mixed_matches_eager():
    """A forest of instances stepped with the dual traversal, recorded and replayed, equals the
    eager steps (mixed precision: the FP64 close-pair sums are atomics, so to rounding)."""
    sizes = [3000, 1200, 4500]
    parts = [_state(nb, 20 + b) for b, nb in enumerate(sizes)]
    pos = np.vstack([q[0] for q in parts])
    zeta = np.concatenate([q[1] for q in parts])
    area = np.concatenate([q[2] for q in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    p = sts.params(theta=0.7, degree=8, leaf_size=64, precision=sts.STS_MIXED, near_fp64_tau=1e-6)
    st = torch.cuda.Stream()
    xe, ze, _ = _run(pos, zeta, area, p, 3, False, st, off, dual=True)
    xg, zg, _ = _run(pos, zeta, area, p, 3, True, st, off, dual=True)
    assert np.max(np.abs(xe - xg)) <= 1e-15
    assert np.max(np.abs(ze - zg)) <= 1e-14 * np.max(np.abs(ze))
