"""Pins of the oracle's column solver (Section IX-B riem_solver_c, a
semi-implicit tridiagonal solve; reading R9)."""
import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I


@pytest.mark.parametrize("m", [4, 5, 6, 7, 8])
def test_thomas_vs_dense_lu(orc, m):
    rng = np.random.default_rng(m)
    for _ in range(20):
        off = rng.uniform(0.1, 2.0, m)
        a = np.concatenate([[0.0], -off[:-1]])
        c = np.concatenate([-off[:-1], [0.0]])
        b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 3.0, m)   # SPD, diagonally dominant
        d = rng.standard_normal(m)
        x = orc.thomas(a, b, c, d)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        y = orc.dense_lu(A, d)
        assert np.abs(x - y).max() <= 1e-14 * np.abs(y).max()
        # and a plain residual check of the brute force
        assert np.abs(A @ y - d).max() <= 1e-14 * np.abs(d).max() * 10


def test_thomas_known_solution(orc):
    # tridiag(-1, 2, -1) x = d with x_k = k^2 gives d from the second difference
    m = 8
    x = np.arange(1, m + 1, dtype=float) ** 2
    d = 2 * x - np.concatenate([[0], x[:-1]]) - np.concatenate([x[1:], [0]])
    a = np.concatenate([[0.0], -np.ones(m - 1)])
    c = np.concatenate([-np.ones(m - 1), [0.0]])
    b = np.full(m, 2.0)
    assert np.abs(orc.thomas(a, b, c, d) - x).max() <= 1e-12


def column(nz=8, seed=0):
    rng = np.random.default_rng(seed)
    delp = 1.0e5 / nz * (1 + 0.01 * rng.standard_normal(nz))
    pt = 250 + 30 * rng.uniform(size=nz)
    delz = I.hydrostatic_delz(delp[:, None, None], pt[:, None, None])[:, 0, 0]
    return delp, pt, delz


def test_resting_hydrostatic_column(orc):
    delp, pt, delz = column()
    nz = len(delp)
    pef, gz, sysm, w = orc.riem_column(delp, pt, np.zeros(nz), delz, 10.0)
    pe = 100.0 + np.concatenate([[0.0], np.cumsum(delp)])
    assert np.abs(w).max() < 1e-9
    assert np.abs(pef - pe).max() <= 1e-10 * pe.max()
    gz_h = np.concatenate([np.cumsum((-I.GRAV * delz)[::-1])[::-1], [0.0]])
    assert np.abs(gz - gz_h).max() <= 1e-10 * gz_h.max()


def test_system_symmetric_dominant(orc):
    delp, pt, delz = column(seed=3)
    delz = delz * 1.01   # not hydrostatic: nonzero p'
    _, _, s, _ = orc.riem_column(delp, pt, np.zeros(len(delp)), delz, 10.0)
    a, b, c, r = s
    assert np.array_equal(a[1:], c[:-1])                 # symmetric
    assert np.all(b > np.abs(a) + np.abs(c))             # strictly dominant
    assert a[0] == 0.0 and c[-1] == 0.0


@pytest.mark.parametrize("nz", [4, 6, 8])
def test_column_thomas_matches_dense_lu(orc, nz):
    delp, pt, delz = column(nz, seed=nz)
    rng = np.random.default_rng(nz)
    wc = rng.standard_normal(nz)
    delz = delz * (1 + 0.02 * rng.standard_normal(nz))
    p1, g1, _, w1 = orc.riem_column(delp, pt, wc, delz, 10.0)
    p2, g2, _, w2 = orc.riem_column(delp, pt, wc, delz, 10.0, use_lu=True)
    assert np.abs(w1 - w2).max() <= 1e-13 * np.abs(w2).max()
    assert np.abs(p1 - p2).max() <= 1e-13 * np.abs(p2).max()
    assert np.abs(g1 - g2).max() <= 1e-13 * np.abs(g2).max()


def test_linearity_in_small_perturbation(orc):
    delp, pt, delz = column(8, seed=7)
    nz = len(delp)
    rng = np.random.default_rng(7)
    dw = rng.standard_normal(nz)
    base_p, base_g, _, base_w = orc.riem_column(delp, pt, np.zeros(nz), delz, 10.0)
    r1 = orc.riem_column(delp, pt, 1e-6 * dw, delz, 10.0)
    r2 = orc.riem_column(delp, pt, 2e-6 * dw, delz, 10.0)
    d1 = r1[3] - base_w
    d2 = r2[3] - base_w
    assert np.abs(d2 - 2 * d1).max() <= 1e-10 * np.abs(d2).max()
    # the response of a pure w perturbation is exactly linear in the solve
    assert np.abs(d1).max() > 0


def test_top_and_bottom_conventions(orc):
    delp, pt, delz = column(6, seed=2)
    pef, gz, _, w = orc.riem_column(delp, pt, np.ones(6), delz * 1.05, 10.0)
    assert pef[0] == 100.0 and gz[-1] == 0.0 and w[-1] == 0.0
    assert np.all(np.diff(gz) < 0)          # geopotential decreases downward
