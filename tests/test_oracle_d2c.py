"""Pins of the C-grid winds interpolated from the D-grid winds (reading R7:
mean of the four surrounding values, second order; reading R18: four-point
Lagrange interpolation along and then across, fourth order), and of the
substep with the fourth-order winds."""
import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I


def fields(n):
    # smooth periodic winds sampled at the D-grid points (index units):
    # u at y-faces (x = i + 1/2, y = j), v at x-faces (x = i, y = j + 1/2)
    U = lambda x, y: np.sin(2 * np.pi * x / n + 0.3) * np.cos(4 * np.pi * y / n + 0.1)
    V = lambda x, y: np.cos(2 * np.pi * x / n - 0.2) * np.sin(2 * np.pi * y / n + 0.5)
    jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n), indexing="ij")
    u = U(ii + 0.5, jj)[None]
    jj, ii = np.meshgrid(np.arange(n), np.arange(n + 1), indexing="ij")
    v = V(ii, jj + 0.5)[None]
    # exact values at the C-grid points: uc at x-faces (i, j + 1/2), vc at y-faces (i + 1/2, j)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n + 1), indexing="ij")
    uce = U(ii, jj + 0.5)
    jj, ii = np.meshgrid(np.arange(n + 1), np.arange(n), indexing="ij")
    vce = V(ii + 0.5, jj)
    return u, v, uce, vce


@pytest.mark.parametrize("ordr, ratio", [(2, 4.0), (4, 16.0)])
def test_convergence_order(orc, ordr, ratio):
    err = []
    for n in (16, 32):
        u, v, uce, vce = fields(n)
        uc, vc = orc.d2c(orc.Domain(False, n, 1), 0, u, v, ordr)
        err.append(max(np.abs(uc - uce).max(), np.abs(vc - vce).max()))
    assert 0.8 * ratio <= err[0] / err[1] <= 1.2 * ratio, err


def test_constant_and_linear_exact(orc):
    n = 12
    d = orc.Domain(False, n, 1)
    u = np.full((1, n + 1, n), 3.25)
    v = np.full((1, n, n + 1), -1.5)
    for ordr in (2, 4):
        uc, vc = orc.d2c(d, 0, u, v, ordr)
        assert np.abs(uc - 3.25).max() <= 1e-15 and np.abs(vc + 1.5).max() <= 1e-15


def make(orc, st, cubed, n, nz):
    d = orc.Domain(cubed, n, nz)
    s = orc.State(d)
    s.load(st)
    return d, s


def test_fourth_order_substep_invariants(orc):
    n, nz = 14, 3
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    st = dict(u=np.full((1, nz, n + 1, n), 9.0), v=np.zeros((1, nz, n, n + 1)), w=np.zeros((1, nz, n, n)),
              delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    _, s = make(orc, st, False, n, nz)
    s.substep(orc.params(d2c_ord=4))
    assert np.abs(s.get("u") - 9.0).max() <= 1e-12 * 9.0 and np.abs(s.get("v")).max() <= 1e-12
    # transpose symmetry and mass conservation on a random periodic state
    st = I.periodic_state(16, 3, seed=21)
    tr = dict(u=np.swapaxes(st["v"], 2, 3).copy(), v=np.swapaxes(st["u"], 2, 3).copy())
    for f in ("w", "delp", "pt", "delz"):
        tr[f] = np.swapaxes(st[f], 2, 3).copy()
    _, s = make(orc, st, False, 16, 3)
    _, s2 = make(orc, tr, False, 16, 3)
    m0 = s.mass()
    s.substep(orc.params(d2c_ord=4))
    s2.substep(orc.params(d2c_ord=4))
    assert abs(s.mass() - m0) <= 1e-14 * m0
    for f in ("delp", "pt", "w"):
        a, b = s.get(f), np.swapaxes(s2.get(f), 2, 3)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), f
    a, b = s.get("u"), np.swapaxes(s2.get("v"), 2, 3)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    # and on the cube the fourth-order winds change the result
    st = I.cubed_state(10, 3, seed=22, ntracers=0)
    _, s = make(orc, st, True, 10, 3)
    _, s2 = make(orc, st, True, 10, 3)
    m0 = s.mass()
    s.substep(orc.params(d2c_ord=4))
    s2.substep()
    assert abs(s.mass() - m0) <= 1e-14 * m0
    assert np.abs(s.get("u") - s2.get("u")).max() > 1e-9
