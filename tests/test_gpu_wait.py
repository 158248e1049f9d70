"""The bounded device-side wait of the mixed evaluation's staging: a wait on a barrier that
nothing arrives on gives up, reports STS_ERR_TIMEOUT through the status word, and leaves the
context usable (the failure is made on the device without a fault: nothing arrives)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import sts
from paper_2401_07361_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_wait_gives_up_and_context_stays_usable():
    with sts.Context() as c:
        assert sts.sts_selftest_wait(c.h, 1000) == sts.STS_ERR_TIMEOUT
        assert "gave up" in sts.load().sts_last_error().decode()
        sts.sts_status(c.h)  # the status word was cleared: no error now
        pos = W.uniform_points(500, 3)
        rng = np.random.default_rng(3)
        zeta, area = rng.standard_normal(500), np.full(500, 4 * math.pi / 500)
        dev = lambda a: torch.from_numpy(a).cuda()
        v = sts.sts_direct(c.h, dev(pos), dev(zeta), dev(area), sts.STS_FP64).cpu().numpy()
        assert O.rel_l2(v, O.direct(pos, zeta, area), area) <= 1e-12
        p = sts.params(theta=0.7, degree=6, leaf_size=32, precision=sts.STS_MIXED, near_fp64_tau=1e-4)
        sts.sts_tree_build(c.h, dev(pos), p)
        v = sts.sts_velocity(c.h, dev(zeta), dev(area), p).cpu().numpy()
        sts.sts_status(c.h)  # a normal evaluation never times out
        assert O.rel_l2(v, O.Tree(pos, 32).velocity(zeta, area, 0.7, 6), area) <= 1e-6


def test_wait_selftest_checks_its_argument():
    with sts.Context() as c:
        assert sts.sts_selftest_wait(c.h, 0) == sts.STS_ERR_ARG
        assert sts.sts_selftest_wait(c.h, (1 << 20) + 1) == sts.STS_ERR_ARG
