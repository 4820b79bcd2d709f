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


def test_layer_mean_pressure_matches_quotient():
    """dp / ln(pen / pe) of the column solve: the series branch (|u| <= 1/8)
    and the logarithm branch against the quotient formed from log1p in numpy
    (each side a few roundings from the exact value)"""
    rng = np.random.default_rng(3)
    pe = 10.0 ** rng.uniform(2, 5, 200000)
    dp = pe * 10.0 ** rng.uniform(-4, 1, 200000)
    got = run(2, pe, dp)
    want = dp / np.log1p(dp / pe)
    u = dp / (2 * pe + dp)
    series = u <= 0.125
    assert series.any() and (~series).any()
    eps = np.finfo(float).eps
    # series branch: the rounding of u, the polynomial and the final products;
    # log branch: also the rounding of pen / pe, amplified by 1 / ln(pen / pe)
    tol = np.where(series, 8 * eps, 16 * eps) * np.abs(want)
    assert (np.abs(got - want) <= tol).all(), np.max(np.abs(got - want) / tol)
    # a vanishing layer: pe + dp/2 - dp^2 / (12 pe) + ..., the quadratic term
    # far below an ulp for these sizes
    pe = np.full(1000, 5.0e4)
    dp = 10.0 ** np.linspace(-8, -4, 1000)
    got = run(2, pe, dp)
    assert np.allclose(got, pe + 0.5 * dp, rtol=4e-16, atol=0)

