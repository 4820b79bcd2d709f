"""Pins of the oracle's 1-D PPM face value (Section IX-C fv_tp_2d; reading R4:
Colella-Woodward edge interpolation, monotone limiter, swept-mean face value).

The expected values are closed forms of the exact swept mean, not the PPM
formulas retyped."""
import numpy as np
import pytest


def swept_mean_cells(F, i_face, c):
    """Exact mean of the profile over the part of the upwind cell swept through
    face i_face in one step; F is an antiderivative of the profile, cells are
    [i, i+1] and face i_face sits at x = i_face."""
    if c > 0:
        a, b = i_face - c, i_face
    else:
        a, b = i_face, i_face - c
    return (F(b) - F(a)) / (b - a)


def cell_means(F, lo, hi):
    x = np.arange(lo, hi + 1, dtype=float)
    return F(x[1:]) - F(x[:-1])


@pytest.mark.parametrize("c", [0.05, 0.3, 0.77, 1.0, -0.2, -0.6, -0.999])
def test_linear_exact(orc, c):
    # profile 3 + 0.5 x : antiderivative 3x + x^2/4
    F = lambda x: 3.0 * x + 0.25 * x * x
    q = cell_means(F, 7, 13)          # cells 7..12, face at x = 10
    got = orc.ppm_face(q, c)
    assert abs(got - swept_mean_cells(F, 10, c)) < 1e-13


@pytest.mark.parametrize("c", [0.1, 0.5, 0.9, -0.25, -0.8])
def test_monotone_parabola_exact(orc, c):
    # profile x^2 on x > 0, far from the extremum: no limiting, PPM is exact
    F = lambda x: x ** 3 / 3.0
    q = cell_means(F, 20, 26)
    got = orc.ppm_face(q, c)
    want = swept_mean_cells(F, 23, c)
    assert abs(got - want) < 1e-12 * abs(want)


def test_constant_and_courant_one(orc):
    q = np.full(6, 1234.5678)
    for c in (0.0, 0.3, 1.0, -0.4, -1.0):
        assert orc.ppm_face(q, c) == 1234.5678
    rng = np.random.default_rng(3)
    q = rng.standard_normal(6)
    assert orc.ppm_face(q, 1.0) == q[2]     # upwind cell i-1, whole cell
    assert orc.ppm_face(q, -1.0) == q[3]


def test_mirror_symmetry(orc):
    # reflecting the six cells about the face and flipping the Courant number
    # must give the same face value (the limiter's tie-breaks are symmetric)
    rng = np.random.default_rng(5)
    for _ in range(500):
        q = rng.standard_normal(6)
        c = rng.uniform(-1, 1)
        a = orc.ppm_face(q, c)
        b = orc.ppm_face(q[::-1].copy(), -c)
        assert abs(a - b) <= 4e-16 * max(1.0, abs(a))


def test_extremum_flattened(orc):
    # local maximum in the upwind cell: limiter flattens it -> face value = cell mean
    q = np.array([0.0, 1.0, 5.0, 1.0, 0.0, 0.0])   # cell i-1 = 5 is a peak
    for c in (0.2, 0.7):
        assert orc.ppm_face(q, c) == 5.0


def test_monotone_no_new_extrema(orc):
    # 1-D upwind flux-form update with |c| <= 1 keeps monotone data within bounds
    rng = np.random.default_rng(11)
    n = 64
    for _ in range(20):
        q = np.cumsum(rng.uniform(0, 1, n))   # monotone increasing
        c = rng.uniform(0.05, 1.0)
        qp = np.concatenate([q[-3:] - (q[-1] - q[0] + 1), q, q[:3] + (q[-1] - q[0] + 1)])
        # interior faces only (ignore the wrap seam)
        fv = np.array([orc.ppm_face(qp[i:i + 6], c) for i in range(n + 1)])
        qn = q[3:n - 3] + c * (fv[3:n - 3] - fv[4:n - 2])
        assert np.all(np.diff(qn) >= -1e-12)
        assert qn.min() >= q[2] - 1e-12 and qn.max() <= q[n - 3] + 1e-12


def test_smooth_convergence(orc):
    # sinusoid sampled around a zero crossing (no limiting): the face-value
    # error falls at third order with resolution
    errs = []
    for n in (32, 64, 128):
        x = np.arange(n + 6) - 3
        F = lambda s: -np.cos(2 * np.pi * s / n) * n / (2 * np.pi)
        q = F(x + 1) - F(x)
        c = 0.4
        fv = np.array([orc.ppm_face(q[i:i + 6], c) for i in range(n // 2 - 4, n // 2 + 4)])
        exact = np.array([swept_mean_cells(F, i, c) for i in range(n // 2 - 4, n // 2 + 4)])
        errs.append(np.abs(fv - exact).max())
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4
