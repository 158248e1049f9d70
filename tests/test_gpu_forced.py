"""Forced BVE of Sec. 4.4 on the GPU against the FP64 oracle: one RK4 step of the polar
vortex with the wavenumber-1 and -2 forcings, during the ramp and on the plateau, FP64 tree
code within 1e-12 per step and the mixed tree code within 1e-6; no forcing after T_f."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OMEGA = 2 * math.pi


@pytest.fixture(scope="module")
def ctx():
    c = sts.Context()
    yield c.h
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _step(ctx, pos, zeta, area, t, dt, k, p):
    x, z = dev(pos), dev(zeta)
    sts.bve_rk4_step_forced(ctx, x, z, dev(area), t, dt, OMEGA, sts.forcing(k, 0.6 * OMEGA), p)
    return x.cpu().numpy(), z.cpu().numpy()


@pytest.mark.parametrize("k,t", [(1, 1.3), (2, 6.0), (2, 14.2)])
def test_forced_step_matches_oracle(ctx, k, t):
    pos = W.icosahedral_points(4)
    area = W.equal_areas(len(pos))
    zeta = W.polar_vortex_vorticity(pos)
    dt = 1.0 / 48.0
    tr_vel = lambda x, z, a: O.Tree(x, 32).velocity(z, a, 0.7, 6)
    f = lambda x, ts: O.forcing(x, ts, k, 0.6 * OMEGA)
    xr, zr = O.rk4_step(pos, zeta, area, dt, OMEGA, tr_vel, t=t, forcing=f)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_FP64)
    x, z = _step(ctx, pos, zeta, area, t, dt, k, p)
    # the step moves x by dt u and zeta by -2 Omega dt u_z: compare against those increments
    assert np.max(np.abs(x - xr)) <= 1e-12 * np.max(np.abs(xr - pos))
    assert np.max(np.abs(z - zr)) <= 1e-12 * np.max(np.abs(zr - zeta))
    # the forcing changed the step (against the unforced oracle step)
    xu, _ = O.rk4_step(pos, zeta, area, dt, OMEGA, tr_vel)
    assert np.max(np.abs(xr - xu)) > 1e-6 * dt
    pm = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_MIXED, near_fp64_tau=0.01 * 4 * math.pi / len(pos))
    xm, zm = _step(ctx, pos, zeta, area, t, dt, k, pm)
    step = np.linalg.norm(xr - pos, axis=1)
    assert np.sqrt(np.sum(np.linalg.norm(xm - xr, axis=1) ** 2)) <= 1e-6 * np.sqrt(np.sum(step**2))


def test_forced_step_after_tf_equals_unforced(ctx):
    pos = W.icosahedral_points(3)
    area = W.equal_areas(len(pos))
    zeta = W.polar_vortex_vorticity(pos)
    p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_FP64)
    x1, z1 = _step(ctx, pos, zeta, area, 20.0, 0.01, 2, p)
    x2, z2 = dev(pos), dev(zeta)
    sts.bve_rk4_step(ctx, x2, z2, dev(area), 0.01, OMEGA, p)
    assert np.array_equal(x1, x2.cpu().numpy()) and np.array_equal(z1, z2.cpu().numpy())


def test_forced_step_arguments(ctx):
    pos = W.icosahedral_points(2)
    z, a = np.zeros(len(pos)), W.equal_areas(len(pos))
    p = sts.params()
    for bad in (sts.forcing(0, 1.0), sts.forcing(1, 1.0, Tp=0.0), sts.forcing(1, 1.0, Tp=4.0, Tf=5.0),
                sts.forcing(1, 1.0, theta1=2.0)):
        with pytest.raises(sts.StsError):
            sts.bve_rk4_step_forced(ctx, dev(pos), dev(z), dev(a), 1.0, 0.01, OMEGA, bad, p)
