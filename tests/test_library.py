"""Host-side checks of the CUDA library (no GPU needed): it builds, loads, exports every
entry point that ``include/sts.h`` declares, checks its arguments on the host, and its host
proxy tables (Sec. 3.2 approximate Fekete points, inverse SBB Vandermonde) agree with the
independently written oracle's."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2401_07361_gb300 import build as B
from paper_2401_07361_gb300 import sts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "sts.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b((?:sts|bve)_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = sts.load()
    names = _declared()
    assert "sts_direct" in names and "bve_rk4_step" in names and len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_host_argument_checks_without_gpu():
    lib = sts.load()
    assert lib.sts_create(None) == -1
    assert b"NULL" in lib.sts_last_error()
    assert lib.sts_proxy_reference(0, None, None) == -1
    assert lib.sts_proxy_reference(17, None, None) == -1
    assert lib.sts_tree_build(None, None, 0, None, None) == -1
    lib.sts_destroy(None)


@pytest.mark.parametrize("d", [1, 2, 4, 6, 8, 10, 12, 14, 16])
def test_proxy_points_match_oracle(d):
    beta, vinv = sts.sts_proxy_reference(d)
    obeta, _ = O.proxy_reference(d)
    # the same candidates in the same selection order (the lattice values are exact)
    assert np.array_equal(beta, obeta)
    ov = O.vref_inverse(d)
    scale = np.abs(ov).max()
    assert np.max(np.abs(vinv - ov)) <= 1e-9 * scale * max(1.0, np.linalg.cond(ov) * 1e-6)


def test_build_flags_target_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.NVCC_FLAGS)
    assert "--fmad=false" in B.PER_FILE["sts_tree.cu"]
