"""GPU parity: the CUDA path (called through the C-ABI) against the FP64 oracle,
element by element on the same seeded inputs.  FP64 bound: 1e-12 relative
max-norm per field per substep (the FP64 parity bound of the substep;
GPU and oracle differ only by rounding order, fused multiply-adds and 1-ulp
differences of log / division)."""
import numpy as np
import pytest

from gpu_common import FIELDS, TOL64, pair, relerr, seeded
from paper_2205_04148_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STAGES = {1: ("uc", "vc", "delpc", "ptc", "wc", "fx1", "fy1"), 2: ("delzc",), 3: ("pef", "gz"),
          4: ("uc", "vc")}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2205_04148_gb300 import build
    build.build()


@pytest.mark.parametrize("cubed,n,nz", [(False, 48, 8), (False, 20, 3), (True, 12, 5), (True, 37, 3)])
def test_metric(orc, cubed, n, nz):
    from paper_2205_04148_gb300 import fv3
    g = fv3.Grid(fv3.GRID_CUBED if cubed else fv3.GRID_PERIODIC, n, nz)
    d = orc.Domain(cubed, n, nz)
    for nm in ("area", "rarea", "fA", "dx", "dyc", "cosy", "siny", "dy", "dxc", "cosx", "sinx", "fC", "rareac"):
        a = g.metric(nm)
        b = d.interior(nm)
        if np.abs(b).max() == 0:
            assert np.abs(a).max() == 0, nm
        else:
            assert relerr(a, b) <= 1e-13, (nm, relerr(a, b))


@pytest.mark.parametrize("cubed,n,nz", [(False, 24, 4), (True, 12, 5), (True, 21, 3)])
def test_stages(orc, cubed, n, nz):
    g, gs, d, s, st = pair(orc, cubed, n, nz, seed=3)
    for stop, names in STAGES.items():
        g.stage(gs, stop)
        s2 = orc.State(d)
        s2.load(st)
        s2.substep(stop_after=stop)
        for nm in names:
            e = relerr(g.intermediate(nm), s2.get(nm))
            assert e <= TOL64, (stop, nm, e)


@pytest.mark.parametrize("cubed,n,nz", [(False, 48, 8), (False, 33, 4), (True, 12, 5), (True, 40, 4),
                                        (True, 8, 2)])
def test_full_substep(orc, cubed, n, nz):
    g, gs, d, s, st = pair(orc, cubed, n, nz, seed=5)
    for it in range(2):
        g.substep(gs)
        s.substep()
        for f in FIELDS:
            e = relerr(g.read(gs, f), s.get(f))
            assert e <= TOL64, (it, f, e)


def test_halo_fill_slots(orc):
    """Every halo slot written by fv3_halo_fill equals the oracle's fill."""
    import torch
    from paper_2205_04148_gb300 import fv3
    n, nz = 10, 2
    g, gs, d, s, st = pair(orc, True, n, nz, seed=9)
    g.halo_fill(gs, 31)
    torch.cuda.synchronize()
    s.substep(stop_after=0)   # oracle's fill of the prognostics
    lay = g.layout()
    H = 3
    for f, kind in (("delp", 0), ("u", 2), ("v", 1)):
        raw = gs[f].cpu().numpy()
        nrow = n + 1 + 2 * H if kind == 2 else n + 2 * H
        ncol = n + 1 + 2 * H if kind == 1 else n + 2 * H
        got = np.full((6, nz, nrow, ncol), np.nan)
        for t in range(6):
            for k in range(nz):
                base = lay.offset3 + (t * nz + k) * lay.plane
                for r in range(nrow):
                    row = base + r * lay.pitch + lay.ox - H
                    got[t, k, r] = raw[row:row + ncol]
        want = orc_padded(orc, d, s, f)
        fin = np.isfinite(want)
        assert np.array_equal(np.isnan(got), np.isnan(want)), f
        assert np.array_equal(got[fin], want[fin]), f


def orc_padded(orc, d, s, name):
    """the oracle's padded field (all tiles/levels) through its state IO: fill
    a dense copy into a fresh state and read back the padded buffer"""
    import ctypes as C
    L = d.L
    # use the oracle's own fill on dense data to rebuild its padded arrays
    dense = s.get(name)
    nt, nz = dense.shape[0], dense.shape[1]
    n, H = d.n, 3
    if name == "u":
        shp = (nt, nz, n + 1 + 2 * H, n + 2 * H)
        fx = np.full((nt, nz, n + 2 * H, n + 1 + 2 * H), np.nan)
        fy = np.full(shp, np.nan)
        fy[:, :, H:H + n + 1, H:H + n] = dense
        fx[:, :, H:H + n, H:H + n + 1] = s.get("v")
        _, fy = orc.fill_faces(d, fx, fy, nz, 1, 1)
        return fy.reshape(shp)
    if name == "v":
        shp = (nt, nz, n + 2 * H, n + 1 + 2 * H)
        fx = np.full(shp, np.nan)
        fy = np.full((nt, nz, n + 1 + 2 * H, n + 2 * H), np.nan)
        fx[:, :, H:H + n, H:H + n + 1] = dense
        fy[:, :, H:H + n + 1, H:H + n] = s.get("u")
        fx, _ = orc.fill_faces(d, fx, fy, nz, 1, 1)
        return fx.reshape(shp)
    shp = (nt, nz, n + 2 * H, n + 2 * H)
    c = np.full(shp, np.nan)
    c[:, :, H:H + n, H:H + n] = dense
    return orc.fill_cells(d, c, nz, 3).reshape(shp)


@pytest.mark.parametrize("cubed,n,nz,nq", [(False, 24, 3, 2), (True, 12, 4, 3)])
def test_run_dyn_with_tracers(orc, cubed, n, nz, nq):
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, cubed, n, nz, seed=11, nq=nq)
    prm_g = fv3.params(n_split=3)
    prm_o = orc.params(n_split=3)
    g.run_dyn(gs, prm_g, n_steps=2)
    s.run_dyn(prm_o, n_steps=2)
    for f in FIELDS:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    for m in range(nq):
        e = relerr(g.read(gs, "q%d" % m), s.get("q%d" % m))
        assert e <= TOL64, ("q%d" % m, e)
    assert g.check_status() == 0


SUBCYCLE_RADIUS = I.RADIUS / 20    # a small sphere: C12 cells of about 40 km


@pytest.mark.parametrize("n_split,nsplt", [(30, 2), (45, 3), (60, 4)])
def test_tracer_subcycling_cube(orc, n_split, nsplt):
    """tracer_2d with nsplt > 1 (reading R12): a 100 m/s rotation on a sphere of
    radius R/20 accumulates Courant numbers 1.9 / 2.8 / 3.8 over n_split
    substeps whose own Courant numbers stay below 0.07; the GPU's cmax /
    nsplt kernels and the subcycles in the captured graph against the oracle"""
    from paper_2205_04148_gb300 import fv3
    n, nz, nq = 12, 3, 2
    st = I.cubed_state(n, nz, seed=3, ntracers=nq, wind=100.0)
    st["q"][1] = np.full_like(st["q"][1], 0.625)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz, radius=SUBCYCLE_RADIUS)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    g.run_dyn(gs, fv3.params(n_split=n_split), 1)
    d = orc.Domain(True, n, nz, radius=SUBCYCLE_RADIUS)
    s = orc.State(d, nq)
    s.load(st)
    s.run_dyn(orc.params(n_split=n_split), 1)
    cmax = max(np.abs(s.get("crx")).max(), np.abs(s.get("cry")).max())
    assert int(np.ceil(cmax)) == nsplt
    for f in FIELDS + ("q0", "q1"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    assert np.abs(g.read(gs, "q1") - 0.625).max() <= 1e-14
    assert g.check_status() == 0


@pytest.mark.parametrize("U,V,nsplt", [(25.0, -20.0, 2), (45.0, 30.0, 3)])
def test_tracer_subcycling_translation(orc, U, V, nsplt):
    """uniform translation on a periodic 2 km grid: per-substep Courant numbers
    0.25 / 0.45, accumulated over 6 substeps 1.5 / 2.7"""
    from paper_2205_04148_gb300 import fv3
    n, nz, nq, dx = 16, 2, 2, 2.0e3
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc)
    rng = np.random.default_rng(5)
    q0 = 0.5 + 0.4 * np.sin(2 * np.pi * X + 0.3) * np.cos(2 * np.pi * Y) + 0.05 * rng.standard_normal((n, n))
    delp = np.full((1, nz, n, n), 1000.0)
    pt = np.full((1, nz, n, n), 280.0)
    st = dict(u=np.full((1, nz, n + 1, n), U), v=np.full((1, nz, n, n + 1), V), w=np.zeros((1, nz, n, n)),
              delp=delp, pt=pt, delz=I.hydrostatic_delz(delp, pt),
              q=[np.broadcast_to(q0, (1, nz, n, n)).copy(), np.full((1, nz, n, n), 0.3)])
    g = fv3.Grid(fv3.GRID_PERIODIC, n, nz, dx=dx)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    g.run_dyn(gs, fv3.params(n_split=6), 1)
    d = orc.Domain(False, n, nz, dx=dx)
    s = orc.State(d, nq)
    s.load(st)
    s.run_dyn(orc.params(n_split=6), 1)
    cmax = max(np.abs(s.get("crx")).max(), np.abs(s.get("cry")).max())
    assert int(np.ceil(cmax)) == nsplt
    for f in FIELDS + ("q0", "q1"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    assert g.check_status() == 0


def test_mass_sum(orc):
    g, gs, d, s, st = pair(orc, True, 16, 6, seed=13)
    m_gpu = g.mass(gs)[0]
    m_orc = s.mass()
    assert abs(m_gpu - m_orc) <= 1e-14 * abs(m_orc)
    g.substep(gs)
    s.substep()
    assert abs(g.mass(gs)[0] - s.mass()) <= 1e-14 * abs(m_orc)
    assert abs(g.mass(gs)[0] - m_gpu) <= 1e-14 * abs(m_gpu)   # conserved on the GPU too


def test_batched_members_uneven(orc):
    """Members of different resolution advanced together match their own
    oracle runs."""
    from paper_2205_04148_gb300 import fv3
    sizes = [8, 12, 16]
    nz = 3
    g = fv3.Grid(fv3.GRID_CUBED, 8, nz, n_members=3, member_npx=sizes)
    gs = g.alloc_state(0)
    sts = []
    for m, n in enumerate(sizes):
        st = seeded(True, n, nz, seed=20 + m)
        sts.append(st)
        g.load(gs, st, member=m)
    g.substep(gs)
    for m, n in enumerate(sizes):
        d = orc.Domain(True, n, nz)
        s = orc.State(d)
        s.load(sts[m])
        s.substep()
        for f in FIELDS:
            e = relerr(g.read(gs, f, member=m), s.get(f))
            assert e <= TOL64, (m, f, e)


def test_fp32_bulk_close(orc):
    """FP32-bulk path: error against the FP64 oracle is reported, not bounded
    by the FP64 tolerance; it must stay at FP32 rounding scale after one
    substep."""
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, True, 16, 5, seed=17, precision=fv3.FP32)
    g.substep(gs)
    s.substep()
    for f in ("u", "v", "delp", "pt"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= 2e-4, (f, e)


@pytest.mark.parametrize("cubed", [False, True])
def test_fp32_metric64_close(orc, cubed):
    """FP32 bulk with the metric terms in FP64 (FV3_FP32_M64): at FP32
    rounding scale against the FP64 oracle after one substep and after a
    remapping step with tracers, and not the same arithmetic as the FP32
    metric copies"""
    from paper_2205_04148_gb300 import fv3
    n, nz = (16, 5) if cubed else (24, 4)
    g, gs, d, s, st = pair(orc, cubed, n, nz, seed=19, nq=2, precision=fv3.FP32_M64)
    g.substep(gs)
    s.substep()
    for f in ("u", "v", "delp", "pt"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= 2e-4, (f, e)
    if cubed:   # the cube's metric terms are not exact in float
        g2, gs2, _, _, _ = pair(orc, cubed, n, nz, seed=19, nq=2, precision=fv3.FP32)
        g2.substep(gs2)
        assert any(not np.array_equal(g.read(gs, f), g2.read(gs2, f)) for f in ("u", "v", "delp", "pt"))
    g.load(gs, st)
    s2 = orc.State(d, 2)
    s2.load(st)
    g.run_dyn(gs, fv3.params(n_split=3), 1)
    s2.run_dyn(orc.params(n_split=3), 1)
    for f in FIELDS + ("q0", "q1"):
        e = relerr(g.read(gs, f), s2.get(f))
        assert e <= 2e-4, (f, e)
    assert g.check_status() == 0


def test_courant_guard_reports():
    """A flow with Courant number above 1 is reported by fv3_check_status."""
    from paper_2205_04148_gb300 import fv3
    st = seeded(False, 16, 2, seed=1)
    st["u"] = st["u"] * 0 + 6000.0    # 6 km/s * 20 s / 100 km = 1.2
    g = fv3.Grid(fv3.GRID_PERIODIC, 16, 2)
    gs = g.alloc_state()
    g.load(gs, st)
    g.substep(gs)
    assert g.check_status() == -6
    assert g.check_status() == 0   # cleared


def test_invalid_arguments_rejected():
    from paper_2205_04148_gb300 import fv3
    g = fv3.Grid(fv3.GRID_PERIODIC, 16, 2)
    gs = g.alloc_state()
    bad = dict(gs)
    bad["delp"] = gs["delp"][1:]   # misaligned base
    with pytest.raises(fv3.Fv3Error, match="ALIGN"):
        g.substep(bad)
    with pytest.raises(fv3.Fv3Error, match="ARG"):
        g.substep(gs, fv3.params(dt=-1.0))
    with pytest.raises(fv3.Fv3Error):
        fv3.Grid(fv3.GRID_CUBED, 4, 2)   # npx < 8


@pytest.mark.parametrize("shape", [(32, 8, 5), (32, 16, 4), (64, 8, 1), (16, 16, 3)])
def test_block_shapes(orc, shape):
    """every compiled block shape and level chunk gives the same substep"""
    g, gs, d, s, st = pair(orc, True, 40, 5, seed=23)
    g.set_tiles(*shape)
    assert g.tiles() == shape
    g.substep(gs)
    s.substep()
    for f in FIELDS:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (shape, f, e)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape", [(16, 16), (32, 8), (32, 16), (64, 8)])
def test_whole_and_partial_block_kernels(orc, precision, shape):
    """n = 32 on the cube: 16 x 16, 32 x 8 and 32 x 16 blocks cover every tile
    whole (the full-block instantiations of c_sw, d_sw and tracer_2d run),
    64 x 8 does not (the runtime-extent ones run); a remapping step with
    tracers against the oracle in each case"""
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, True, 32, 3, seed=51, nq=2, precision=precision)
    g.set_tiles(shape[0], shape[1], 2)
    g.run_dyn(gs, fv3.params(n_split=2), 1)
    s.run_dyn(orc.params(n_split=2), 1)
    tol = TOL64 if precision == 0 else 2e-4
    for f in FIELDS + ("q0", "q1"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= tol, (f, e)
    assert g.check_status() == 0


def test_transfer_tuning_keeps_whole_blocks(orc):
    """fv3_autotune_for: tuned on one member for sizes 48, 96 and 128, only
    shapes that cover all three with whole blocks are tried (here 16 x 16),
    and the ensemble run with the result matches the oracle"""
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, True, 24, 4, seed=31)
    (bx, by, kc), best = g.autotune(gs, sizes=[48, 96, 128])
    assert (bx, by) == (16, 16) and best > 0
    g2 = fv3.Grid(fv3.GRID_CUBED, 16, 3, n_members=2, member_npx=[16, 32])
    g2.set_tiles(bx, by, kc)
    gs2 = g2.alloc_state()
    sts = [seeded(True, n, 3, seed=40 + m) for m, n in enumerate((16, 32))]
    for m, stm in enumerate(sts):
        g2.load(gs2, stm, member=m)
    g2.substep(gs2)
    for m, (n, stm) in enumerate(zip((16, 32), sts)):
        so = orc.State(orc.Domain(True, n, 3))
        so.load(stm)
        so.substep()
        for f in FIELDS:
            e = relerr(g2.read(gs2, f, member=m), so.get(f))
            assert e <= TOL64, (m, f, e)


def test_autotune_keeps_parity(orc):
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, True, 24, 6, seed=29, nq=1)
    (bx, by, kc), best = g.autotune(gs)
    assert (bx, by) in ((32, 8), (32, 16), (64, 8), (16, 16)) and 1 <= kc <= 6 and best > 0
    g.load(gs, st)           # autotune ran stages on the state's halos only; reload anyway
    prm_g, prm_o = fv3.params(n_split=2), orc.params(n_split=2)
    g.run_dyn(gs, prm_g, 1)
    s.run_dyn(prm_o, 1)
    for f in FIELDS + ("q0",):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)


@pytest.mark.parametrize("precision", [0, 1])
def test_persistent_launch_matches(orc, precision):
    """Persistent launches (a GPU-filling grid striding over the work list of
    all members) give bitwise the same remapping step as one CTA per item,
    for members of uneven resolution, FP64 and FP32."""
    from paper_2205_04148_gb300 import fv3
    sizes = [8, 16, 12]
    nz, nq = 5, 2
    out = []
    for pers in (False, True):
        g = fv3.Grid(fv3.GRID_CUBED, 8, nz, n_members=3, member_npx=sizes, precision=precision)
        g.set_tiles(32, 8, 2)
        g.set_persistent(pers)
        assert g.persistent() == pers
        gs = g.alloc_state(nq)
        for m, n in enumerate(sizes):
            g.load(gs, seeded(True, n, nz, seed=60 + m, nq=nq), member=m)
        g.run_dyn(gs, fv3.params(n_split=3), 1)
        out.append({(f, m): g.read(gs, f, member=m) for f in FIELDS + ("q1",) for m in range(3)})
        g.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
    # and the FP64 persistent run is the oracle's
    if precision == 0:
        for m, n in enumerate(sizes):
            s = orc.State(orc.Domain(True, n, nz), nq)
            s.load(seeded(True, n, nz, seed=60 + m, nq=nq))
            s.run_dyn(orc.params(n_split=3), 1)
            for f in FIELDS + ("q1",):
                e = relerr(out[1][(f, m)], s.get(f))
                assert e <= TOL64, (m, f, e)


def test_fp32_error_after_100_substeps():
    """FP32-bulk stays close to the FP64 path over 100 substeps (C24 x 8):
    the error grows from FP32 rounding, it does not blow up."""
    from paper_2205_04148_gb300 import fv3
    st = I.cubed_state(24, 8, seed=3, ntracers=0)
    res = {}
    for prec in (fv3.FP64, fv3.FP32):
        g = fv3.Grid(fv3.GRID_CUBED, 24, 8, precision=prec)
        gs = g.alloc_state()
        g.load(gs, st)
        m0 = g.mass(gs)[0]
        for _ in range(100):
            g.substep(gs)
        res[prec] = {f: g.read(gs, f) for f in FIELDS}
        drift = abs(g.mass(gs)[0] - m0) / m0
        assert drift <= (1e-13 if prec == fv3.FP64 else 1e-6), (prec, drift)
        g.close()
    for f in ("u", "v", "delp", "pt"):
        e = relerr(res[fv3.FP32][f], res[fv3.FP64][f])
        print(f, e)
        assert e <= 1e-3, (f, e)


@pytest.mark.parametrize("cubed", [False, True])
def test_fourth_order_c_grid_winds(orc, cubed):
    """c_sw with the fourth-order C-grid winds (reading R18) on the GPU"""
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, cubed, 20, 4, seed=97, nq=1)
    g.run_dyn(gs, fv3.params(n_split=2, d2c_ord=4), 1)
    s.run_dyn(orc.params(n_split=2, d2c_ord=4), 1)
    for f in FIELDS + ("q0",):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    g32, gs32, _, _, _ = pair(orc, cubed, 20, 4, seed=97, nq=1, precision=fv3.FP32)
    g32.run_dyn(gs32, fv3.params(n_split=2, d2c_ord=4), 1)
    for f in ("u", "v", "delp", "pt"):
        e = relerr(g32.read(gs32, f), s.get(f))
        assert e <= 5e-4, (f, e)
    with pytest.raises(fv3.Fv3Error, match="ARG"):
        g.substep(gs, fv3.params(d2c_ord=3))


@pytest.mark.parametrize("cubed", [False, True])
def test_divergence_damping(orc, cubed):
    """divergence damping with the Smagorinsky coefficient (reading R19)"""
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, cubed, 20, 4, seed=99)
    for _ in range(2):
        g.substep(gs, fv3.params(d2_bg=0.04, dddmp=0.3))
        s.substep(orc.params(d2_bg=0.04, dddmp=0.3))
    for f in FIELDS:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    with pytest.raises(fv3.Fv3Error, match="ARG"):
        g.substep(gs, fv3.params(d2_bg=-1.0))
