"""Pins of the oracle's wind updates, pressure gradient, geopotential update
and tracer sub-cycling against results fixed by the continuous equations or
by textbook schemes, not by the oracle's own formulas (readings R7, R8, R10,
R11, R12).

* Vector-invariant balance (c_sw step 5 and the d_sw wind update): a steady
  parallel shear flow u(y) on the f = 0 plane with uniform mass is an exact
  steady solution of the vector-invariant momentum equations, because the
  vorticity flux -zeta u of the v-equation cancels the kinetic-energy gradient
  d(u^2/2)/dy.  The discrete v must therefore vanish as the grid is refined, at
  the scheme's second order.  A flipped sign or a wrong weight of either term
  leaves an O(1) residual; an index shifted by one cell leaves a first-order
  one.
* p_grad_c: isothermal hydrostatic air under a surface-pressure bump feels
  the acceleration -R T d ln(ps)/dx below the top layer (Lin 1997 is exact for
  it up to discretisation).
* update_dz_c: with winds uniform in each layer the flux-form update of the
  interface geopotential is the first-order upwind scheme of the advection
  equation, written here from its textbook form.
* tracer_2d: when the accumulated Courant number exceeds 1 the transport runs
  nsplt = ceil(max |sum c|) passes with the fluxes divided by nsplt (R12);
  those passes are repeated here one by one through the single-plane
  fv_tp_2d export.
"""
import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I

L_DOMAIN = 2.4e6     # periodic domain length (m) held fixed under refinement
U0 = 10.0            # shear-flow amplitude (m/s)
DT = 20.0


def shear_state(n, nz, transpose=False):
    """u(y) = U0 sin(2 pi y / L) on the D-grid (or v(x) when transposed),
    uniform delp and pt, hydrostatic delz"""
    yj = np.arange(n + 1) / n
    prof = U0 * np.sin(2 * np.pi * yj)
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    st = dict(w=np.zeros((1, nz, n, n)), delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    if transpose:
        st["v"] = np.broadcast_to(prof[None, None, None, :], (1, nz, n, n + 1)).copy()
        st["u"] = np.zeros((1, nz, n + 1, n))
    else:
        st["u"] = np.broadcast_to(prof[None, None, :, None], (1, nz, n + 1, n)).copy()
        st["v"] = np.zeros((1, nz, n, n + 1))
    return st


def balance_residuals(orc, transpose, stop_after, field):
    out = []
    for n in (24, 48, 96):
        st = shear_state(n, 2, transpose)
        d = orc.Domain(False, n, 2, dx=L_DOMAIN / n)
        s = orc.State(d)
        s.load(st)
        s.substep(stop_after=stop_after)
        out.append(np.abs(s.get(field)).max())
    return np.array(out)


@pytest.mark.parametrize("transpose", [False, True])
def test_c_sw_wind_update_shear_flow_balance(orc, transpose):
    # c_sw alone (stop 1): the cross-stream C-grid wind starts at zero and
    # receives dt/2 (-zeta u - dK/dy), which cancels in the continuum
    field = "uc" if transpose else "vc"
    r = balance_residuals(orc, transpose, 1, field)
    k = 2 * np.pi / L_DOMAIN
    term = 0.5 * DT * U0 * U0 * k          # size of either term alone
    assert r[0] <= 0.02 * term, r / term
    assert (r[:-1] / r[1:] >= 3.5).all(), r          # second order
    assert (r[:-1] / r[1:] <= 4.5).all(), r


@pytest.mark.parametrize("transpose", [False, True])
def test_d_sw_wind_update_shear_flow_balance(orc, transpose):
    # the whole substep: d_sw's cross-stream wind update dt (-zeta u - dK/dy)
    # with the PPM vorticity flux and the corner kinetic energy
    field = "u" if transpose else "v"
    r = balance_residuals(orc, transpose, -1, field)
    k = 2 * np.pi / L_DOMAIN
    term = DT * U0 * U0 * k
    assert r[0] <= 0.02 * term, r / term
    assert (r[:-1] / r[1:] >= 3.5).all(), r
    assert (r[:-1] / r[1:] <= 4.5).all(), r


def test_shear_flow_along_stream_wind_kept(orc):
    # the along-stream wind of the balanced flow changes only by the del-4
    # damping of the vorticity flux, a fourth-order term: small and
    # converging fast
    errs = []
    for n in (24, 48):
        st = shear_state(n, 2)
        d = orc.Domain(False, n, 2, dx=L_DOMAIN / n)
        s = orc.State(d)
        s.load(st)
        s.substep()
        errs.append(np.abs(s.get("u") - st["u"]).max())
    assert errs[0] <= 1e-3 * U0 and errs[1] <= errs[0] / 8


@pytest.mark.parametrize("axis", ["x", "y"])
def test_p_grad_c_closed_form(orc, axis):
    # uc after p_grad_c (stop 4) minus uc before it (stop 3) is dt/2 times
    # -R T d ln(ps)/dx, evaluated at the C-grid faces; the top layer, bounded
    # by the fixed ptop, is excluded
    n, nz, dx, T, eps, wd = 48, 4, 1.0e5, 280.0, 0.02, 0.15
    xc = (np.arange(n) + 0.5) / n
    bump = np.exp(-((xc - 0.5) / wd) ** 2)
    prof = 1000.0 * (1 + eps * bump)
    shape = (1, nz, n, n)
    delp = np.broadcast_to(prof[None, None, None, :] if axis == "x" else prof[None, None, :, None], shape).copy()
    pt = np.full(shape, T)
    st = dict(u=np.zeros((1, nz, n + 1, n)), v=np.zeros((1, nz, n, n + 1)), w=np.zeros(shape),
              delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt))
    d = orc.Domain(False, n, nz, dx=dx)
    name = "uc" if axis == "x" else "vc"
    got = []
    for stop in (3, 4):
        s = orc.State(d)
        s.load(st)
        s.substep(stop_after=stop)
        got.append(s.get(name))
    dw = got[1] - got[0]
    xf = np.arange(n + 1) / n
    bf = np.exp(-((xf - 0.5) / wd) ** 2)
    dbump = -2 * (xf - 0.5) / wd ** 2 * bf / (n * dx)
    want = -0.5 * DT * I.RDGAS * T * eps * dbump / (1 + eps * bf)
    for k in range(1, nz):
        for row in (0, 17, n - 1):
            val = dw[0, k, row] if axis == "x" else dw[0, k, :, row]
            assert np.abs(val - want).max() <= 0.05 * np.abs(want).max(), (k, row)
    # nothing across the bump's ridge direction
    if axis == "x":
        s = orc.State(d)
        s.load(st)
        s.substep(stop_after=4)
        assert np.abs(s.get("vc")).max() <= 1e-12 * np.abs(want).max()


def test_update_dz_c_upwind_closed_form(orc):
    # winds uniform in each layer (both signs), delz varying in x and y: the
    # interface geopotential gz (0 at the surface, minus g delz summed up) is
    # advected by the first-order upwind scheme with the interface Courant
    # numbers (mean of the two layers', the top interface the top layer's)
    n, nz, dx = 16, 4, 1.0e4
    Uk = np.array([8.0, -5.0, 12.0, -3.0])
    Vk = np.array([-4.0, 6.0, 3.0, -7.0])
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc)
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    dz0 = I.hydrostatic_delz(delp, pt)
    delz = dz0 * (1 + 0.1 * np.sin(2 * np.pi * X) * np.cos(4 * np.pi * Y))[None, None]
    st = dict(u=np.broadcast_to(Uk[None, :, None, None], (1, nz, n + 1, n)).copy(),
              v=np.broadcast_to(Vk[None, :, None, None], (1, nz, n, n + 1)).copy(),
              w=np.zeros((1, nz, n, n)), delp=delp, pt=pt, delz=delz)
    d = orc.Domain(False, n, nz, dx=dx)
    s = orc.State(d)
    s.load(st)
    s.substep(stop_after=2)
    got = s.get("delzc")[0]
    g = I.GRAV
    gz = np.zeros((nz + 1, n, n))
    for k in range(nz - 1, -1, -1):
        gz[k] = gz[k + 1] - g * delz[0, k]
    cx = 0.5 * DT * Uk / dx
    cy = 0.5 * DT * Vk / dx
    cxi = np.concatenate([cx[:1], 0.5 * (cx[:-1] + cx[1:])])
    cyi = np.concatenate([cy[:1], 0.5 * (cy[:-1] + cy[1:])])
    gzn = np.zeros_like(gz)
    for K in range(nz):
        q = gz[K]
        dxm = q - np.roll(q, 1, axis=1)          # q_i - q_{i-1}
        dxp = np.roll(q, -1, axis=1) - q         # q_{i+1} - q_i
        dym = q - np.roll(q, 1, axis=0)
        dyp = np.roll(q, -1, axis=0) - q
        gzn[K] = q - cxi[K] * (dxm if cxi[K] > 0 else dxp) - cyi[K] * (dym if cyi[K] > 0 else dyp)
    want = np.minimum((gzn[1:] - gzn[:-1]) / g, -2.0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # and the update did act
    assert np.abs(got - delz[0]).max() > 1e-3 * np.abs(delz[0] - delz[0].mean((1, 2), keepdims=True)).max()


def translation_state(n, nz, U, V, nq):
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    rng = np.random.default_rng(5)
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc)
    q0 = 0.5 + 0.4 * np.sin(2 * np.pi * X + 0.3) * np.cos(2 * np.pi * Y) + 0.05 * rng.standard_normal((n, n))
    q = [np.broadcast_to(q0, (1, nz, n, n)).copy(), np.full((1, nz, n, n), 0.3)]
    return dict(u=np.full((1, nz, n + 1, n), U), v=np.full((1, nz, n, n + 1), V), w=np.zeros((1, nz, n, n)),
                delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt), q=q[:nq])


@pytest.mark.parametrize("U,V,nsplt", [(25.0, -20.0, 2), (45.0, 30.0, 3)])
def test_tracer_subcycling(orc, U, V, nsplt):
    # dx = 2 km, dt = 20 s, 6 substeps: per-substep Courant numbers 0.25 /
    # 0.45 (< 1), accumulated 1.5 / 2.7 -> nsplt = 2 / 3
    n, nz, dx, ns = 16, 2, 2.0e3, 6
    st = translation_state(n, nz, U, V, 2)
    d = orc.Domain(False, n, nz, dx=dx)
    s = orc.State(d, 2)
    s.load(st)
    m0 = s.mass()
    tm0 = np.sum(st["q"][0] * st["delp"])
    s.run_dyn(orc.params(n_split=ns), 1)
    crx, cry = s.get("crx"), s.get("cry")
    cmax = max(np.abs(crx).max(), np.abs(cry).max())
    assert int(np.ceil(cmax)) == nsplt
    assert max(abs(U), abs(V)) * DT / dx < 1.0
    # the uniform flow is steady: winds, mass and constants kept
    assert abs(s.mass() - m0) <= 1e-14 * m0
    assert np.abs(s.get("q1") - 0.3).max() <= 1e-14
    q = s.get("q0")
    assert abs(np.sum(q * s.get("delp")) - tm0) <= 1e-13 * tm0
    # nsplt passes by hand with the fluxes divided by nsplt (area fluxes; the
    # uniform delp cancels between the mass fluxes and the denominators)
    xfx, yfx = s.get("xfx"), s.get("yfx")
    area = d.interior("area")[0]
    want = st["q"][0][0].copy()
    for k in range(nz):
        qk = want[k].copy()
        for _ in range(nsplt):
            Fx, Fy = orc.fv_tp_2d(d, 0, qk, crx[0, k] / nsplt, cry[0, k] / nsplt, xfx[0, k] / nsplt,
                                  yfx[0, k] / nsplt)
            qk = qk + (Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]) / area
        want[k] = qk
    assert np.abs(q[0] - want).max() <= 1e-13
    # one pass with the whole accumulated fluxes (|c| > 1) is something else
    Fx, Fy = orc.fv_tp_2d(d, 0, st["q"][0][0, 0], crx[0, 0], cry[0, 0], xfx[0, 0], yfx[0, 0])
    one = st["q"][0][0, 0] + (Fx[:, :-1] - Fx[:, 1:] + Fy[:-1, :] - Fy[1:, :]) / area
    assert np.abs(q[0, 0] - one).max() > 1e-3


def test_tracer_subcycling_cube_invariants(orc):
    # a 100 m/s rotation on a sphere of radius R/20 over 30 substeps:
    # accumulated Courant number 1.9 (nsplt 2) with every substep's own below
    # 0.07; a constant tracer stays constant, tracer mass is conserved and the
    # bounded tracer stays within its initial range
    n, nz, ns = 12, 3, 30
    radius = I.RADIUS / 20
    st = I.cubed_state(n, nz, seed=3, ntracers=2, wind=100.0)
    st["q"][1] = np.full_like(st["q"][1], 0.625)
    d = orc.Domain(True, n, nz, radius=radius)
    s = orc.State(d, 2)
    s.load(st)
    area = d.interior("area")[:, None]
    qm0 = float(np.sum(st["q"][0] * st["delp"] * area))
    lo, hi = st["q"][0].min(), st["q"][0].max()
    s.run_dyn(orc.params(n_split=ns), 1)
    cmax = max(np.abs(s.get("crx")).max(), np.abs(s.get("cry")).max())
    assert int(np.ceil(cmax)) == 2
    assert np.abs(s.get("q1") - 0.625).max() <= 1e-14
    q = s.get("q0")
    assert abs(float(np.sum(q * s.get("delp") * area)) - qm0) <= 1e-13 * qm0
    assert q.min() >= lo - 1e-12 and q.max() <= hi + 1e-12
