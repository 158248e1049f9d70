"""sts_direct_noalloc: the direct sum for callers that cannot allocate device memory
(inside someone else's graph capture, under another allocator, or in a loop that must not
enter cudaMalloc).  It is called here straight through the C ABI and checked against the
allocating entry point sts_direct on two calls in a row with different inputs: the shared
fixed scratch must not carry anything over.  Both entry points split the sources the same
way and run the same kernels, so the results are compared bit for bit (and, redundantly,
within the tolerances the parity tests use)."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

torch = pytest.importorskip("torch")

STS_ERR_CAPACITY = -3


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    pos = W.uniform_points(n, seed)
    zeta = rng.standard_normal(n)
    area = rng.uniform(0.5, 1.5, n) * (4 * math.pi / n)
    return [torch.from_numpy(a).to("cuda") for a in (pos, zeta, area)]


def _noalloc(lib, pos, zeta, area, prec):
    n = pos.shape[0]
    vel = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.sts_direct_noalloc(C.c_void_p(pos.data_ptr()), C.c_void_p(zeta.data_ptr()),
                                C.c_void_p(area.data_ptr()), n, prec, C.c_void_p(vel.data_ptr()), stream)
    assert rc == 0, lib.sts_last_error()
    torch.cuda.synchronize()
    return vel.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [(sts.STS_FP64, 1e-12), (sts.STS_MIXED, 1e-6)])
def test_noalloc_direct_matches_allocating_direct_twice(prec, tol):
    lib = sts.load()
    with sts.Context() as ctx:
        for n, seed in ((5000, 11), (1777, 12)):
            pos, zeta, area = _inputs(n, seed)
            got = _noalloc(lib, pos, zeta, area, prec)
            ref = sts.sts_direct(ctx.h, pos, zeta, area, prec).cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.array_equal(got, ref), (n, np.max(np.abs(got - ref)))
            a = area.cpu().numpy()
            err = np.sqrt(np.sum(np.sum((got - ref) ** 2, 1) * a) / np.sum(np.sum(ref ** 2, 1) * a))
            assert err <= tol, (n, err)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = sts.load()
    n = 65537
    rc = lib.sts_direct_noalloc(C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), n, sts.STS_FP64,
                                C.c_void_p(16), None)
    assert rc == STS_ERR_CAPACITY
    assert b"65536" in lib.sts_last_error()
