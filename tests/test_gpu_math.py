"""Accuracy of the kernels' FP64 helpers against exact references: the
Newton-refined hardware reciprocal (used for the transport denominators and
the column solve's pivots) and the log pressure ratio of the column solve
(atanh series for thin layers, the library logarithm otherwise)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run(what, x, y=None):
    import torch

    from paper_2205_04148_gb300 import build, fv3
    build.build()
    L = fv3.load()
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.as_tensor(y if y is not None else x, device="cuda")
    out = torch.empty_like(xd)
    rc = L.fv3_math_check(what, C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), C.c_void_p(out.data_ptr()),
                          int(x.size), None)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_reciprocal_within_an_ulp():
    rng = np.random.default_rng(1)
    x = 10.0 ** rng.uniform(-6, 14, 200000) * rng.choice([-1.0, 1.0], 200000)
    r = run(0, x)
    exact = 1.0 / x
    ulp = np.spacing(np.abs(exact))
    assert np.abs(r - exact).max() / ulp.max() <= 1.0
    assert (np.abs(r - exact) <= ulp).all()


def test_log_ratio_matches_log1p():
    rng = np.random.default_rng(2)
    pe = 10.0 ** rng.uniform(2, 5, 200000)
    dp = pe * 10.0 ** rng.uniform(-4, 1, 200000)
    got = run(1, pe, dp)
    want = np.log1p(dp / pe)
    # log1p of a correctly rounded quotient: its own error is 1 ulp of dp/pe
    tol = 4 * np.finfo(float).eps * np.abs(want) + np.spacing(dp / pe)
    assert (np.abs(got - want) <= tol).all(), np.max(np.abs(got - want) / tol)
