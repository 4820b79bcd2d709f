"""Pins of the divergence damping (reading R19): second-order damping of the
D-grid winds' divergence at the cell corners with the coefficient
da_min * max(d2_bg, min(0.2, dddmp * dt * |deformation|)), applied through the
corner kinetic energy of the wind update."""
import numpy as np

from paper_2205_04148_gb300 import inputs as I


def flat_state(n, nz, u):
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    return dict(u=u, v=np.zeros((1, nz, n, n + 1)), w=np.zeros((1, nz, n, n)), delp=delp, pt=pt,
                delz=I.hydrostatic_delz(delp, pt))


def run(orc, st, n, nz, cubed=False, **kw):
    d = orc.Domain(cubed, n, nz)
    s = orc.State(d)
    s.load(st)
    s.substep(orc.params(**kw))
    return s


def sine_u(n, nz, k, amp):
    x = (np.arange(n) + 0.5) / n
    return np.broadcast_to(amp * np.sin(2 * np.pi * k * x)[None, None, None, :], (1, nz, n + 1, n)).copy()


def test_background_damping_is_the_discrete_laplacian_eigenvalue(orc):
    # u = A sin(2 pi k x) on the uniform periodic tile: the corner divergence is
    # (u_i - u_{i-1}) / dx and the damping adds d2_bg (u_{i+1} - 2 u_i + u_{i-1})
    # = -4 d2_bg sin^2(pi k / n) u_i to each u, exactly
    n, nz, k, amp, d2 = 32, 2, 3, 5.0, 0.05
    u0 = sine_u(n, nz, k, amp)
    st = flat_state(n, nz, u0)
    du = run(orc, st, n, nz, d2_bg=d2).get("u") - run(orc, st, n, nz).get("u")
    want = -4 * d2 * np.sin(np.pi * k / n) ** 2 * u0
    assert np.abs(du - want).max() <= 1e-11 * np.abs(want).max()


def test_smagorinsky_coefficient_scaling_and_cap(orc):
    n, nz, k = 32, 2, 2
    base = {}
    for amp in (0.01, 0.02):
        st = flat_state(n, nz, sine_u(n, nz, k, amp))
        base[amp] = run(orc, st, n, nz, dddmp=0.5).get("u") - run(orc, st, n, nz).get("u")
    # below the cap the coefficient grows with the deformation: quadratic response
    r = np.abs(base[0.02]).max() / np.abs(base[0.01]).max()
    assert 3.9 <= r <= 4.1, r
    # a huge Smagorinsky coefficient saturates at the cap 0.2 (except where
    # the deformation is within 1e-11 of zero, where the damping itself is tiny)
    st = flat_state(n, nz, sine_u(n, nz, k, 5.0))
    plain = run(orc, st, n, nz).get("u")
    a = run(orc, st, n, nz, dddmp=1e9).get("u")
    b = run(orc, st, n, nz, d2_bg=0.2).get("u")
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b - plain).max()


def test_damping_keeps_invariants(orc):
    n, nz = 16, 3
    st = flat_state(n, nz, np.full((1, nz, n + 1, n), 7.5))
    s = run(orc, st, n, nz, d2_bg=0.1, dddmp=0.2)
    assert np.abs(s.get("u") - 7.5).max() <= 1e-12 * 7.5            # no divergence, no damping
    st = I.periodic_state(16, 3, seed=31)
    tr = dict(u=np.swapaxes(st["v"], 2, 3).copy(), v=np.swapaxes(st["u"], 2, 3).copy())
    for f in ("w", "delp", "pt", "delz"):
        tr[f] = np.swapaxes(st[f], 2, 3).copy()
    s = run(orc, st, 16, 3, d2_bg=0.05, dddmp=0.2)
    s2 = run(orc, tr, 16, 3, d2_bg=0.05, dddmp=0.2)
    a, b = s.get("u"), np.swapaxes(s2.get("v"), 2, 3)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    st = I.cubed_state(10, 3, seed=32, ntracers=0)
    d = orc.Domain(True, 10, 3)
    s = orc.State(d)
    s.load(st)
    m0 = s.mass()
    s.substep(orc.params(d2_bg=0.05, dddmp=0.2))
    assert abs(s.mass() - m0) <= 1e-14 * m0 and np.isfinite(s.get("u")).all()
