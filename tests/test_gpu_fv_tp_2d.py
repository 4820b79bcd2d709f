"""The standalone fv_tp_2d entry point (Section IX-C, 2-D flux-form transport;
readings R4-R6) through the C-ABI against the oracle's fv_tp_2d and delnflux,
on every tile and level, in both precisions; the Courant-1 translation and
the mass-flux form on the GPU."""
import numpy as np
import pytest

from gpu_common import TOL64, relerr

pytestmark = pytest.mark.gpu


def inputs(g, seed, amp=0.6):
    """q, crx, cry, xfx, yfx as dense [nt][nz][..] arrays; area fluxes scaled
    by half the mean cell area so every inner-update denominator stays > 0"""
    rng = np.random.default_rng(seed)
    nt, nz, n = g.nt, g.npz, g.member_npx[0]
    a0 = 0.5 * float(np.mean(g.metric("area")))
    q = 1000.0 + 50.0 * rng.standard_normal((nt, nz, n, n))
    crx = rng.uniform(-amp, amp, (nt, nz, n, n + 1))
    cry = rng.uniform(-amp, amp, (nt, nz, n + 1, n))
    return q, crx, cry, crx * a0, cry * a0


def gpu_fluxes(g, q, crx, cry, xfx, yfx, damp=0.0, mass_scale=None):
    from paper_2205_04148_gb300 import fv3
    t = {}
    for name, arr, kind in (("q", q, fv3.KIND_CELL), ("crx", crx, fv3.KIND_XFACE), ("cry", cry, fv3.KIND_YFACE),
                            ("xfx", xfx, fv3.KIND_XFACE), ("yfx", yfx, fv3.KIND_YFACE)):
        t[name] = g.alloc(kind)
        g.put(t[name], kind, arr)
    mfx = mfy = None
    if mass_scale is not None:
        mfx, mfy = g.alloc(fv3.KIND_XFACE), g.alloc(fv3.KIND_YFACE)
        g.put(mfx, fv3.KIND_XFACE, xfx * mass_scale)
        g.put(mfy, fv3.KIND_YFACE, yfx * mass_scale)
    fx, fy = g.fv_tp_2d(t["q"], t["crx"], t["cry"], t["xfx"], t["yfx"], mfx, mfy, damp)
    return g.get(fx, fv3.KIND_XFACE), g.get(fy, fv3.KIND_YFACE)


def oracle_fluxes(orc, cubed, n, q, crx, cry, xfx, yfx, damp=0.0):
    d = orc.Domain(cubed, n, 1)
    nt, nz = q.shape[:2]
    Fx = np.empty((nt, nz, n, n + 1))
    Fy = np.empty((nt, nz, n + 1, n))
    for k in range(nz):
        for t in range(nt):
            fx, fy = orc.fv_tp_2d(d, t, q[:, k], crx[:, k], cry[:, k], xfx[:, k], yfx[:, k])
            if damp:
                dx, dy = orc.delnflux(d, t, q[:, k], damp)
                fx, fy = fx + dx, fy + dy
            Fx[t, k], Fy[t, k] = fx, fy
    return Fx, Fy


@pytest.mark.parametrize("cubed", [False, True])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_fv_tp_2d_matches_oracle(orc, cubed, precision):
    from paper_2205_04148_gb300 import fv3
    n, nz = 20, 3
    g = fv3.Grid(fv3.GRID_CUBED if cubed else fv3.GRID_PERIODIC, n, nz, precision=precision)
    g.set_tiles(32, 8, 2)
    q, crx, cry, xfx, yfx = inputs(g, seed=5 + cubed)
    fx, fy = gpu_fluxes(g, q, crx, cry, xfx, yfx)
    Fx, Fy = oracle_fluxes(orc, cubed, n, q, crx, cry, xfx, yfx)
    tol = TOL64 if precision == 0 else 2e-5
    assert relerr(fx, Fx) <= tol, relerr(fx, Fx)
    assert relerr(fy, Fy) <= tol, relerr(fy, Fy)


def test_fv_tp_2d_damping_matches_oracle(orc):
    from paper_2205_04148_gb300 import fv3
    n, nz = 16, 2
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    q, crx, cry, xfx, yfx = inputs(g, seed=9)
    damp = (0.12 * float(np.min(g.metric("area")))) ** 2
    fx, fy = gpu_fluxes(g, q, crx, cry, xfx, yfx, damp=damp)
    Fx, Fy = oracle_fluxes(orc, True, n, q, crx, cry, xfx, yfx, damp=damp)
    assert relerr(fx, Fx) <= TOL64 and relerr(fy, Fy) <= TOL64
    # the damping flux is a visible part of the total
    fx0, _ = gpu_fluxes(g, q, crx, cry, xfx, yfx)
    assert np.abs(fx - fx0).max() > 1e-6 * np.abs(fx0).max()


def test_fv_tp_2d_mass_flux_form():
    """flux = face value x mass flux: doubling the area fluxes as mass fluxes
    doubles the fluxes exactly"""
    from paper_2205_04148_gb300 import fv3
    g = fv3.Grid(fv3.GRID_CUBED, 12, 2)
    q, crx, cry, xfx, yfx = inputs(g, seed=13)
    fx, fy = gpu_fluxes(g, q, crx, cry, xfx, yfx)
    fx2, fy2 = gpu_fluxes(g, q, crx, cry, xfx, yfx, mass_scale=2.0)
    assert np.array_equal(fx2, 2.0 * fx) and np.array_equal(fy2, 2.0 * fy)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_fv_tp_2d_courant_one_translation(sign):
    """crx = +1 / -1 on the uniform periodic tile: one flux-form update is the
    shift by one cell (east / west) to round-off"""
    from paper_2205_04148_gb300 import fv3
    n, nz = 24, 2
    g = fv3.Grid(fv3.GRID_PERIODIC, n, nz)
    area = 1.0e10
    rng = np.random.default_rng(17)
    q = 1000.0 + 50.0 * rng.standard_normal((1, nz, n, n))
    crx = sign * np.ones((1, nz, n, n + 1))
    cry = np.zeros((1, nz, n + 1, n))
    fx, fy = gpu_fluxes(g, q, crx, cry, crx * area, cry * area)
    qn = q + (fx[..., :-1] - fx[..., 1:] + fy[..., :-1, :] - fy[..., 1:, :]) / area
    assert np.abs(qn - np.roll(q, int(sign), axis=-1)).max() <= 4 * np.finfo(float).eps * np.abs(q).max()


def test_fv_tp_2d_invalid_arguments():
    from paper_2205_04148_gb300 import fv3
    g = fv3.Grid(fv3.GRID_PERIODIC, 16, 2)
    c, x, y = g.alloc(fv3.KIND_CELL), g.alloc(fv3.KIND_XFACE), g.alloc(fv3.KIND_YFACE)
    with pytest.raises(fv3.Fv3Error, match="ARG"):
        g.fv_tp_2d(c, x, y, x, y, mfx=x)
    with pytest.raises(fv3.Fv3Error, match="ALIGN"):
        g.fv_tp_2d(c[1:], x, y, x, y)
    with pytest.raises(fv3.Fv3Error, match="ARG"):
        g.fv_tp_2d(c, x, y, x, y, damp=-1.0)
