"""Invariant pins of the oracle's whole acoustic substep (Section II: the
acoustic substep loop) and remapping step with tracer transport (readings
R7-R13)."""
import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I


def make(orc, st, cubed, n, nz, nq=0):
    d = orc.Domain(cubed, n, nz)
    s = orc.State(d, nq)
    s.load(st)
    return d, s


def tracer_mass(s, d, m):
    q = s.get("q%d" % m)
    dp = s.get("delp")
    A = d.interior("area")[:, None]
    return float(np.sum(q * dp * A))


def test_periodic_mass_conservation(orc):
    st = I.periodic_state(24, 4, seed=1)
    d, s = make(orc, st, False, 24, 4)
    m0 = s.mass()
    for _ in range(3):
        s.substep()
    assert abs(s.mass() - m0) <= 1e-14 * m0


def test_cubed_mass_conservation_substeps(orc):
    st = I.cubed_state(12, 5, seed=2, ntracers=0)
    d, s = make(orc, st, True, 12, 5)
    m0 = s.mass()
    for _ in range(4):
        s.substep()
        assert abs(s.mass() - m0) <= 1e-14 * m0
    assert np.isfinite(s.get("delp")).all()


def test_cubed_run_dyn_tracers(orc):
    st = I.cubed_state(10, 4, seed=3, ntracers=2)
    st["q"][1] = np.full_like(st["q"][1], 0.625)     # constant tracer
    d, s = make(orc, st, True, 10, 4, nq=2)
    m0 = s.mass()
    qm0 = tracer_mass(s, d, 0)
    s.run_dyn(orc.params(n_split=3), n_steps=2)
    assert abs(s.mass() - m0) <= 1e-14 * m0
    assert abs(tracer_mass(s, d, 0) - qm0) <= 1e-13 * qm0
    q1 = s.get("q1")
    assert np.abs(q1 - 0.625).max() <= 1e-13
    q0 = s.get("q0")
    assert q0.min() >= -1e-12 and q0.max() <= 1 + 1e-12   # monotone transport stays in [0, 1]


def test_rest_state_unchanged(orc):
    n, nz = 16, 4
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    st = dict(u=np.zeros((1, nz, n + 1, n)), v=np.zeros((1, nz, n, n + 1)),
              w=np.zeros((1, nz, n, n)), delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    d, s = make(orc, st, False, n, nz)
    s.substep()
    assert np.array_equal(s.get("delp"), delp)
    assert np.array_equal(s.get("u"), st["u"]) and np.array_equal(s.get("v"), st["v"])
    assert np.abs(s.get("pt") - pt).max() <= 1e-13 * 280.0
    assert np.abs(s.get("w")).max() == 0.0


def test_uniform_translation_keeps_winds(orc):
    n, nz = 16, 3
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    st = dict(u=np.full((1, nz, n + 1, n), 12.5), v=np.zeros((1, nz, n, n + 1)),
              w=np.zeros((1, nz, n, n)), delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    d, s = make(orc, st, False, n, nz)
    s.substep()
    assert np.abs(s.get("u") - 12.5).max() <= 1e-12 * 12.5
    assert np.abs(s.get("v")).max() <= 1e-12 * 12.5
    assert np.abs(s.get("delp") - 1000.0).max() <= 1e-12 * 1000.0


def test_horizontally_uniform_dz_and_pgrad(orc):
    # uniform columns: update_dz_c returns delz, p_grad_c adds nothing
    n, nz = 12, 5
    rng = np.random.default_rng(4)
    delp = np.broadcast_to(rng.uniform(900, 1100, nz)[None, :, None, None], (1, nz, n, n)).copy()
    pt = np.broadcast_to(rng.uniform(250, 300, nz)[None, :, None, None], (1, nz, n, n)).copy()
    st = dict(u=np.full((1, nz, n + 1, n), 7.0), v=np.full((1, nz, n, n + 1), -3.0),
              w=np.zeros((1, nz, n, n)), delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    d, s = make(orc, st, False, n, nz)
    s.substep(stop_after=2)
    assert np.abs(s.get("delzc") - st["delz"]).max() <= 1e-12 * np.abs(st["delz"]).max()
    s2 = orc.State(d)
    s2.load(st)
    s2.substep(stop_after=3)
    uc_before = s2.get("uc")
    s2.substep(stop_after=4)   # recomputes c_sw, riem, then adds p_grad_c
    assert np.array_equal(s2.get("uc"), uc_before)


def test_periodic_transpose_symmetry(orc):
    st = I.periodic_state(16, 3, seed=5)
    tr = dict(u=np.swapaxes(st["v"], 2, 3).copy(), v=np.swapaxes(st["u"], 2, 3).copy())
    for f in ("w", "delp", "pt", "delz"):
        tr[f] = np.swapaxes(st[f], 2, 3).copy()
    d, s = make(orc, st, False, 16, 3)
    _, s2 = make(orc, tr, False, 16, 3)
    s.substep()
    s2.substep()
    for f in ("delp", "pt", "w"):
        a, b = s.get(f), np.swapaxes(s2.get(f), 2, 3)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    a, b = s.get("u"), np.swapaxes(s2.get("v"), 2, 3)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_cubed_solid_body_rotation_stays_smooth(orc):
    # 20 substeps of the rigid rotation: no blow-up, winds stay near 20 m/s
    st = I.cubed_state(12, 3, seed=6, ntracers=0)
    d, s = make(orc, st, True, 12, 3)
    for _ in range(20):
        s.substep()
    u = s.get("u")
    assert np.isfinite(u).all() and np.abs(u).max() < 30.0


# --- the closed substep (reading R17: update_dz_d, riem_solver3, D-grid p_grad)
def rest(n, nz, periodic=True):
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    return dict(u=np.zeros((1, nz, n + 1, n)), v=np.zeros((1, nz, n, n + 1)), w=np.zeros((1, nz, n, n)),
                delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))


def test_closed_substep_rest_state(orc):
    n, nz = 12, 5
    st = rest(n, nz)
    d, s = make(orc, st, False, n, nz)
    for _ in range(3):
        s.substep(orc.params(nh_full=1))
    assert np.abs(s.get("u")).max() <= 1e-10 and np.abs(s.get("v")).max() <= 1e-10
    assert np.abs(s.get("w")).max() <= 1e-10
    assert np.abs(s.get("delz") - st["delz"]).max() <= 1e-10 * np.abs(st["delz"]).max()
    assert np.array_equal(s.get("delp"), st["delp"])


def test_closed_substep_horizontally_uniform(orc):
    # a vertical perturbation of w, the same in every column: the pressure
    # gradient adds nothing, every column evolves the same way
    n, nz = 10, 6
    st = rest(n, nz)
    st["w"] = np.broadcast_to(np.sin(np.arange(nz) * 0.9)[None, :, None, None], (1, nz, n, n)).copy()
    st["u"][:] = 4.0
    d, s = make(orc, st, False, n, nz)
    s.substep(orc.params(nh_full=1))
    w, dz = s.get("w"), s.get("delz")
    assert np.abs(w - w[:, :, :1, :1]).max() <= 1e-12
    assert np.abs(dz - dz[:, :, :1, :1]).max() <= 1e-12 * np.abs(dz).max()
    assert np.abs(s.get("u") - 4.0).max() <= 1e-12 * 4.0 and np.abs(s.get("v")).max() <= 1e-12
    assert np.abs(w - st["w"]).max() > 1e-3          # the column solve acted
    # update_dz_d of uniform columns with uniform fluxes returns delz
    _, s2 = make(orc, st, False, n, nz)
    s2.substep(orc.params(nh_full=1), stop_after=6)
    assert np.abs(s2.get("delzd") - st["delz"]).max() <= 1e-12 * np.abs(st["delz"]).max()


def test_closed_substep_conserves_mass_and_stays_bounded(orc):
    st = I.cubed_state(10, 5, seed=12, ntracers=0)
    rng = np.random.default_rng(13)
    st["w"] = 0.5 * rng.standard_normal(st["w"].shape)
    d, s = make(orc, st, True, 10, 5)
    m0 = s.mass()
    for _ in range(30):
        s.substep(orc.params(nh_full=1))
    assert abs(s.mass() - m0) <= 1e-13 * m0
    w = s.get("w")
    assert np.isfinite(w).all() and np.abs(w).max() < 2.0      # implicit vertical waves do not grow
    assert np.isfinite(s.get("delz")).all() and (s.get("delz") < 0).all()
    assert np.abs(s.get("u")).max() < 40.0


def test_closed_substep_transpose_symmetry(orc):
    st = I.periodic_state(14, 3, seed=9)
    rng = np.random.default_rng(10)
    st["w"] = 0.3 * rng.standard_normal(st["w"].shape)
    tr = dict(u=np.swapaxes(st["v"], 2, 3).copy(), v=np.swapaxes(st["u"], 2, 3).copy())
    for f in ("w", "delp", "pt", "delz"):
        tr[f] = np.swapaxes(st[f], 2, 3).copy()
    d, s = make(orc, st, False, 14, 3)
    _, s2 = make(orc, tr, False, 14, 3)
    s.substep(orc.params(nh_full=1))
    s2.substep(orc.params(nh_full=1))
    for f in ("delp", "pt", "w", "delz"):
        a, b = s.get(f), np.swapaxes(s2.get(f), 2, 3)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), f
    a, b = s.get("u"), np.swapaxes(s2.get("v"), 2, 3)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_d_grid_pressure_gradient_closed_form(orc):
    # isothermal hydrostatic air, surface pressure raised by a smooth bump in x:
    # below the top layer the levels follow the surface pressure, so the
    # pressure-gradient acceleration is -R T d ln(ps)/dx; the closed substep's
    # u minus the open substep's u is dt times it, to discretisation error
    n, nz, dx, T, eps, wd = 48, 4, 1.0e5, 280.0, 0.02, 0.15
    x = (np.arange(n) + 0.5) / n
    bump = np.exp(-((x - 0.5) / wd) ** 2)
    delp = np.broadcast_to((1000.0 * (1 + eps * bump))[None, None, None, :], (1, nz, n, n)).copy()
    pt = np.full((1, nz, n, n), T)
    st = dict(u=np.zeros((1, nz, n + 1, n)), v=np.zeros((1, nz, n, n + 1)), w=np.zeros((1, nz, n, n)),
              delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    u = {}
    for nh in (0, 1):
        _, s = make(orc, st, False, n, nz)
        s.substep(orc.params(nh_full=nh))
        u[nh] = s.get("u")
    du = u[1] - u[0]
    dbump = -2 * (x - 0.5) / wd ** 2 * bump / (n * dx)
    want = -20.0 * I.RDGAS * T * eps * dbump / (1 + eps * bump)
    for k in range(1, nz):
        for j in (0, 7, n):
            assert np.abs(du[0, k, j] - want).max() <= 0.05 * np.abs(want).max(), (k, j)
