"""Adaptive mesh refinement (Appendix A) on the GPU against the CPU oracle, through the C ABI.

Bars: the refinement tables (triangle corners, parents, children, levels, midpoint edge ends)
and every pass's triangle states and alive vertices are bit-exact; positions and vorticities
of the vertices are bit-exact (new midpoints are plain IEEE sums, a square root and divisions
on both sides); the particle weights (sums of A / 3, added in any order on the GPU) agree to
1e-14 relative.  The split and merge decisions compare FP64 values computed the same way on
both sides except for the atan2 of the spherical area (each side's own library, ~1 ulp
apart), which can only matter at an exact tie.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TABLES = ("tv", "tparent", "tchild", "tlevel", "vparent")


@pytest.fixture(scope="module")
def ctx():
    c = sts.Context()
    yield c.h
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _start(ctx, level, levels, zeta_fn):
    pos, faces = W.icosahedral_mesh(level)
    area0 = W.equal_areas(len(pos))
    zeta = zeta_fn(pos, area0)
    sts.sts_amr_init(ctx, faces, dev(pos), dev(zeta), levels)
    m = O.Amr(faces, len(pos), levels)
    m.set(pos, zeta)
    return pos, faces, zeta, m


def _compare(ctx, m, what=""):
    g = sts.sts_amr_export(ctx)
    o = m.export()
    for k in ("tstate", "valive", "pos", "zeta"):
        assert np.array_equal(g[k], o[k]), (what, k)
    err = np.max(np.abs(g["area"] - o["area"])) / np.max(o["area"])
    assert err <= 1e-14, (what, err)
    return g


def test_amr_tables_and_base_state_equal_oracle(ctx):
    _, _, _, m = _start(ctx, 2, 3, lambda p, a: W.gaussian_vortex_vorticity(p, a))
    g, o = sts.sts_amr_export(ctx), m.export()
    for k in TABLES:
        assert np.array_equal(g[k], o[k]), k
    info = sts.sts_amr_info(ctx)
    assert (info["n0"], info["nv"], info["t0"], info["nt"]) == (m.n0, m.nv, m.t0, m.nt)
    _compare(ctx, m, "base")
    assert abs(g["area"].sum() - 4 * math.pi) <= 1e-12


def test_amr_full_refinement_and_merge_back(ctx):
    """Every triangle split three times gives the icosahedron refined three more times; three
    passes that meet no criterion merge it back to the base mesh."""
    pos, faces, zeta, m = _start(ctx, 1, 3, lambda p, a: np.cos(3 * p[:, 2]))
    for k in range(4):
        assert sts.sts_amr_step(ctx, 0.0, 0.0) == m.step(0.0, 0.0)
        _compare(ctx, m, f"split {k}")
    assert sts.sts_amr_info(ctx)["particles"] == 10 * 4**4 + 2
    g = sts.sts_amr_export(ctx)
    assert np.max(np.abs(g["pos"][: 10 * 4**4 + 2] - W.icosahedral_points(4))) <= 4e-16
    for k in range(3):
        assert sts.sts_amr_step(ctx, np.inf, np.inf) == m.step(np.inf, np.inf)
        _compare(ctx, m, f"merge {k}")
    assert sts.sts_amr_info(ctx)["particles"] == len(pos)


def test_amr_passes_with_moving_particles_match_oracle(ctx):
    """Gaussian vortex on the level-3 mesh, eps1 / eps2 of the paper's test scaled to the mesh:
    passes alternate with a rigid rotation of the particles and a decay of the vorticity (so
    triangles split, merge and leave hanging vertices), the same state written to both sides
    between passes."""
    pos, faces, zeta, m = _start(ctx, 3, 3, lambda p, a: W.gaussian_vortex_vorticity(p, a))
    ang = 0.05
    R = np.array([[math.cos(ang), -math.sin(ang), 0.0], [math.sin(ang), math.cos(ang), 0.0], [0.0, 0.0, 1.0]])
    seen_split = seen_merge = 0
    for k in range(6):
        eps1, eps2 = 0.01, 1.5
        cg = sts.sts_amr_step(ctx, eps1, eps2)
        co = m.step(eps1, eps2)
        assert cg == co, k
        seen_split += cg[0]
        seen_merge += cg[1]
        g = _compare(ctx, m, f"pass {k}")
        # move: rotate every particle, decay the vorticity, both sides get the same arrays
        p, z, a, ids = sts.sts_amr_gather(ctx)
        ids = ids.cpu().numpy()
        assert np.array_equal(ids, np.flatnonzero(g["valive"]))
        newp = (p.cpu().numpy() @ R.T).copy()
        newz = (0.8 * z.cpu().numpy()).copy()
        sts.sts_amr_scatter(ctx, dev(newp), dev(newz))
        full_p, full_z = np.zeros((m.nv, 3)), np.zeros(m.nv)
        full_p[ids], full_z[ids] = newp, newz
        m.update(full_p, full_z)
        _compare(ctx, m, f"moved {k}")
    assert seen_split > 0 and seen_merge > 0


def test_amr_gaussian_vortex_rk4_steps(ctx):
    """Three RK4 steps of the Gaussian vortex (dt = 0.01 day, the paper's eps1 = 0.0025,
    eps2 = 0.2) on the level-4 mesh with an AMR pass after each: the GPU's passes equal the
    oracle's given the same post-step particles.  The weights tile the sphere up to the
    hanging vertices: a midpoint that only its refined side uses moves with the flow off the
    coarse neighbour's edge, so the two sides overlap or leave a gap of second order in the
    displacement (measured 8e-7 of 4 pi here)."""
    pos, faces, zeta, m = _start(ctx, 4, 3, lambda p, a: W.gaussian_vortex_vorticity(p, a))
    p = sts.params(theta=0.7, degree=6, leaf_size=64, precision=sts.STS_FP64)
    with sts.Context() as tc:
        for k in range(3):
            x, z, a, ids = sts.sts_amr_gather(ctx)
            sts.bve_rk4_step(tc.h, x, z, a, 0.01, 2 * math.pi, p)
            sts.sts_amr_scatter(ctx, x, z)
            ids = ids.cpu().numpy()
            full_p, full_z = np.zeros((m.nv, 3)), np.zeros(m.nv)
            full_p[ids], full_z[ids] = x.cpu().numpy(), z.cpu().numpy()
            m.update(full_p, full_z)
            assert sts.sts_amr_step(ctx, 0.0025, 0.2) == m.step(0.0025, 0.2), k
            g = _compare(ctx, m, f"step {k}")
            assert abs(g["area"].sum() - 4 * math.pi) <= 1e-5
    assert sts.sts_amr_info(ctx)["particles"] > len(pos)
