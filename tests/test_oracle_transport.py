"""Pins of the oracle's fv_tp_2d (Section IX-C: 2-D flux-form transport, mass
conserving; reading R5 Lin-Rood splitting) and delnflux (reading R6, del-4
damping).  Periodic 1-tile domain with the uniform metric."""
import numpy as np
import pytest

N = 24
DX = 1.0e5
AREA = DX * DX


@pytest.fixture(scope="module")
def dom(orc):
    return orc.Domain(False, N, 1, dx=DX)


def step(orc, dom, q, crx, cry):
    """one flux-form update with area fluxes consistent with the Courant numbers"""
    xfx = crx * AREA
    yfx = cry * AREA
    Fx, Fy = orc.fv_tp_2d(dom, 0, q[None], crx[None], cry[None], xfx[None], yfx[None])
    div = Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]
    return q + div / AREA, Fx, Fy


def rand_q(seed):
    rng = np.random.default_rng(seed)
    return 1000.0 + 50.0 * rng.standard_normal((N, N))


def test_courant_one_shift_full_period(orc, dom):
    q0 = rand_q(1)
    q = q0.copy()
    crx = np.ones((N, N + 1))
    cry = np.zeros((N + 1, N))
    eps = np.finfo(float).eps
    for s in range(N):
        q, _, _ = step(orc, dom, q, crx, cry)
        assert np.abs(q - np.roll(q0, s + 1, axis=1)).max() <= 4 * eps * (s + 1) * np.abs(q0).max()
    assert np.abs(q - q0).max() <= 4 * eps * N * np.abs(q0).max()


def test_courant_one_diagonal(orc, dom):
    q0 = rand_q(2)
    crx = np.ones((N, N + 1))
    cry = np.ones((N + 1, N))
    q, _, _ = step(orc, dom, q0, crx, cry)
    want = np.roll(np.roll(q0, 1, axis=0), 1, axis=1)
    assert np.abs(q - want).max() <= 64 * np.finfo(float).eps * np.abs(q0).max()


def rand_courant(seed, amp=0.45):
    rng = np.random.default_rng(seed)
    kx = rng.uniform(-amp, amp, (N, N))
    ky = rng.uniform(-amp, amp, (N, N))
    crx = np.concatenate([kx, kx[:, :1]], axis=1)
    cry = np.concatenate([ky, ky[:1, :]], axis=0)
    return crx, cry


def test_constant_preserved(orc, dom):
    crx, cry = rand_courant(3)
    q = np.full((N, N), 287.25)
    # a divergent flow changes the mass; the scalar itself is transported as a
    # mixing ratio: q_new = (q*M + div F) / M_new with M_new from the same fluxes
    ones = np.ones((N, N))
    _, Fx, Fy = step(orc, dom, q, crx, cry)
    _, Mx, My = step(orc, dom, ones, crx, cry)
    divq = Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]
    divm = Mx[:, :-1] - Mx[:, 1:] + My[:-1, :] - My[1:, :]
    qn = (q * AREA + divq) / (AREA + divm)
    assert np.abs(qn - 287.25).max() <= 1e-12 * 287.25


def test_mass_conservation(orc, dom):
    crx, cry = rand_courant(4)
    q = rand_q(4)
    qn, Fx, Fy = step(orc, dom, q, crx, cry)
    assert abs(qn.sum() - q.sum()) <= 1e-14 * np.abs(q).sum()


def test_transpose_symmetry_bitwise(orc, dom):
    crx, cry = rand_courant(5)
    q = rand_q(5)
    _, Fx, Fy = step(orc, dom, q, crx, cry)
    _, Gx, Gy = step(orc, dom, q.T.copy(), cry.T.copy(), crx.T.copy())
    assert np.array_equal(Gx, Fy.T) and np.array_equal(Gy, Fx.T)


def test_reflection_symmetry(orc, dom):
    crx, cry = rand_courant(6)
    q = rand_q(6)
    _, Fx, Fy = step(orc, dom, q, crx, cry)
    qm = q[:, ::-1].copy()
    crxm = -crx[:, ::-1].copy()
    crym = cry[:, ::-1].copy()
    _, Gx, Gy = step(orc, dom, qm, crxm, crym)
    assert np.abs(Gx - (-Fx[:, ::-1])).max() <= 1e-14 * np.abs(Fx).max()
    assert np.abs(Gy - Fy[:, ::-1]).max() <= 1e-14 * np.abs(Fy).max()


def test_linear_field_uniform_flow_exact(orc, dom):
    # uniform flow crx = c on a field linear in y only: x-fluxes carry the row
    # value, y-fluxes vanish; rows keep their values.
    c = 0.3
    q = np.tile(np.arange(N, dtype=float)[:, None] * 2.0 + 10.0, (1, N))
    crx = np.full((N, N + 1), c)
    cry = np.zeros((N + 1, N))
    qn, Fx, Fy = step(orc, dom, q, crx, cry)
    assert np.abs(qn - q).max() <= 1e-13 * np.abs(q).max()
    assert np.allclose(Fx, q[:, :1] * c * AREA, rtol=1e-14, atol=0)


# ------------------------------------------------------------ delnflux ----
def damp_coeff():
    return (0.12 * AREA) ** 2


def apply_damp(orc, dom, q):
    Fx, Fy = orc.delnflux(dom, 0, q[None], damp_coeff())
    return q + (Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]) / AREA, Fx, Fy


def test_checkerboard_amplification(orc, dom):
    i = np.arange(N)
    q = np.where((i[:, None] + i[None, :]) % 2 == 0, 1.0, -1.0)
    qn, _, _ = apply_damp(orc, dom, q)
    # del-4 with coefficient (0.12 dx^2)^2 removes 64 * 0.0144 = 0.9216
    assert np.allclose(qn / q, 1.0 - 0.9216, rtol=1e-12, atol=0)


def test_fourier_mode_amplification(orc, dom):
    # eigenvalue of the 5-point Laplacian for mode (kx, ky): -(4 sin^2(kx/2) +
    # 4 sin^2(ky/2)) / dx^2 ; del-4 damping factor 1 - damp * lambda^2
    kx, ky = 2 * np.pi * 3 / N, 2 * np.pi * 5 / N
    i = np.arange(N)
    q = np.cos(kx * i[None, :] + ky * i[:, None])
    qn, _, _ = apply_damp(orc, dom, q)
    lam = (4 * np.sin(kx / 2) ** 2 + 4 * np.sin(ky / 2) ** 2) / DX ** 2
    fac = 1.0 - damp_coeff() * lam ** 2
    assert np.abs(qn - fac * q).max() <= 1e-12


def test_damping_constant_zero_and_conservative(orc, dom):
    _, Fx, Fy = apply_damp(orc, dom, np.full((N, N), 5.0))
    assert np.all(Fx == 0.0) and np.all(Fy == 0.0)
    q = rand_q(9)
    qn, _, _ = apply_damp(orc, dom, q)
    assert abs(qn.sum() - q.sum()) <= 1e-14 * np.abs(q).sum()
