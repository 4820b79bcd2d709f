"""Accuracy of the kernels' FP64 helpers against exact references: the
Newton-refined hardware reciprocal (used for the transport denominators and
the column solve's pivots), the paired reciprocal of the column solve (1/dz
and 1/(pe + pen) from one reciprocal) and the log pressure ratio of the
column solve (atanh series for thin layers, the library logarithm
otherwise)."""
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


def test_paired_reciprocal_within_two_ulps():
    """1/a as r b with r the reciprocal of a b: the reciprocal's ulp, the
    rounding of a b and of the product r b, over the ranges of the column
    solve (thickness -1e-1 .. -1e4 m, pressure sums 1e1 .. 3e5 Pa) and
    beyond"""
    rng = np.random.default_rng(4)
    a = -(10.0 ** rng.uniform(-1, 4, 200000))
    b = 10.0 ** rng.uniform(1, 5.5, 200000)
    r = run(3, a, b)
    exact = 1.0 / a
    assert (np.abs(r - exact) <= 2 * np.spacing(np.abs(exact))).all()
    a = 10.0 ** rng.uniform(-100, 100, 200000) * rng.choice([-1.0, 1.0], 200000)
    b = 10.0 ** rng.uniform(-100, 100, 200000)
    r = run(3, a, b)
    exact = 1.0 / a
    assert (np.abs(r - exact) <= 2 * np.spacing(np.abs(exact))).all()


def test_float_widening_is_the_conversion():
    """the column solve's integer-pipe widening of its FP32 inputs gives the
    bits of the conversion: normal floats over the whole exponent range,
    subnormal floats, signed zeros and infinities; NaNs stay NaNs"""
    rng = np.random.default_rng(5)
    bits = np.concatenate([rng.integers(0, 2**32, 400000, dtype=np.uint64),
                           np.arange(0, 2**12, dtype=np.uint64),                 # small subnormals
                           np.arange(0x007ff000, 0x00801000, dtype=np.uint64),   # largest subnormals, smallest normals
                           np.arange(0x7f7ff000, 0x7f801000, dtype=np.uint64),   # largest normals, infinity, NaNs
                           np.array([0x80000000, 0x80000001, 0xff800000, 0xffc00001, 0x7fc00000], dtype=np.uint64)])
    f = bits.astype(np.uint32).view(np.float32)
    with np.errstate(invalid="ignore"):   # signalling NaNs are made quiet
        x = f.astype(np.float64)          # exact; the device rounds it back to the same float
    got = run(4, x)
    nan = np.isnan(x)
    assert nan.any() and np.isnan(got[nan]).all()
    assert np.array_equal(got[~nan].view(np.uint64), x[~nan].view(np.uint64))


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

