"""Parity at the benchmark's sizes, in the launch configuration bench.py
times (autotuned block shape and launch mode): the C96 x 80 FP64 substep and
remapping step against the oracle on every element, members of the 24-member
FP32 ensemble against the oracle, and the edge cases of the interface (zero
steps, size limits)."""
import numpy as np
import pytest

from gpu_common import FIELDS, TOL64, relerr, ulp_sensitivity

pytestmark = pytest.mark.gpu


def test_c96x80_fp64_substep_and_step(orc):
    from paper_2205_04148_gb300 import fv3
    from paper_2205_04148_gb300 import inputs as I
    n, nz, nq = 96, 80, 8
    st = I.cubed_state(n, nz, seed=0, ntracers=nq)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    g.autotune(gs)
    g.load(gs, st)
    g.substep(gs)
    s = orc.State(orc.Domain(True, n, nz), nq)
    s.load(st)
    s.substep()
    for f in FIELDS:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    # a whole remapping step with the tracers, from the same start
    g.load(gs, st)
    g.run_dyn(gs, fv3.params(n_split=6), 1)
    s2 = orc.State(orc.Domain(True, n, nz), nq)
    s2.load(st)
    s2.run_dyn(orc.params(n_split=6), 1)
    for f in FIELDS + tuple("q%d" % k for k in range(nq)):
        e = relerr(g.read(gs, f), s2.get(f))
        assert e <= TOL64, (f, e)


def test_batched_ensemble_members(orc):
    """the 8 x C48 + 8 x C96 + 8 x C128 x 80 FP32 ensemble, one substep in
    one launch per stage; one member of each size against the oracle"""
    from paper_2205_04148_gb300 import fv3
    from paper_2205_04148_gb300 import inputs as I
    sizes, nz = [48] * 8 + [96] * 8 + [128] * 8, 80
    base = {n: I.cubed_state(n, nz, seed=0, ntracers=0) for n in (48, 96, 128)}
    g = fv3.Grid(fv3.GRID_CUBED, 128, nz, n_members=24, member_npx=sizes, precision=fv3.FP32)
    gs = g.alloc_state()
    members = {}
    for m, n in enumerate(sizes):
        st = I.perturb_member(base[n], m)
        if m in (3, 11, 19):
            members[m] = st
        g.load(gs, st, member=m)
    g.set_tiles(32, 8, 4)
    g.set_persistent(True)
    g.substep(gs)
    for m, st in members.items():
        n = sizes[m]
        s = orc.State(orc.Domain(True, n, nz))
        s.load(st)
        s.substep()
        for f in ("u", "v", "delp", "pt"):
            e = relerr(g.read(gs, f, member=m), s.get(f))
            assert e <= 2e-4, (m, f, e)


def test_zero_steps_and_limits():
    from paper_2205_04148_gb300 import fv3
    from paper_2205_04148_gb300 import inputs as I
    st = I.cubed_state(8, 3, seed=1, ntracers=1)
    g = fv3.Grid(fv3.GRID_CUBED, 8, 3)
    gs = g.alloc_state(1)
    g.load(gs, st)
    before = {f: g.read(gs, f) for f in FIELDS + ("q0",)}
    g.run_dyn(gs, fv3.params(), 0)
    for f, a in before.items():
        assert np.array_equal(g.read(gs, f), a), f
    with pytest.raises(fv3.Fv3Error, match="SHAPE"):
        fv3.Grid(fv3.GRID_CUBED, 8, 1025)                       # levels beyond the limit
    with pytest.raises(fv3.Fv3Error, match="SHAPE"):
        fv3.Grid(fv3.GRID_CUBED, 64, 2, n_members=200)          # rows beyond one launch's grid


@pytest.mark.parametrize("precision", ["fp32", "fp32_m64"])
def test_c192x80_fp32_substep(orc, precision):
    """The FP32-bulk bench configuration (C192 x 80, 32 x 8 blocks, four levels
    per work item; metric terms in FP32 or in FP64) against the FP64 oracle
    after one substep.  Bound: every
    stored FP32 field is a few tens of roundings (2^-24 ~ 6e-8 each) away from
    the FP64 values it is formed from, so within 1e-6 of the field's maximum
    (measured: <= 2.2e-7); FP64 mass sums of the FP32 delp conserve to FP32
    rounding of the sum of the fluxes."""
    from paper_2205_04148_gb300 import fv3
    from paper_2205_04148_gb300 import inputs as I
    n, nz = 192, 80
    st = I.cubed_state(n, nz, seed=0, ntracers=0)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz, precision=fv3.FP32 if precision == "fp32" else fv3.FP32_M64)
    gs = g.alloc_state()
    g.load(gs, st)
    g.set_tiles(32, 8, 4)
    g.set_persistent(False)
    m0 = g.mass(gs)[0]
    g.substep(gs)
    s = orc.State(orc.Domain(True, n, nz))
    s.load(st)
    s.substep()
    for f in FIELDS + ("delz",):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= 1e-6, (f, e)
    assert abs(g.mass(gs)[0] - m0) <= 1e-6 * m0


def test_c96x80_fp64_all_options_step(orc):
    """One remapping step of the C96 x 80 FP64 state with every physics option
    the bench can switch on (closed substep, vertical remapping, divergence
    damping, fourth-order C-grid winds), in the bench's launch configuration,
    against the oracle on every element of every field.  Bound per field: 1e-12,
    or four times the oracle's own change under a one-ulp perturbation of its
    inputs where that is larger (w after the closed substep, formed by
    cancellation, moves by about 1e-12 under any change of rounding)."""
    from paper_2205_04148_gb300 import fv3
    from paper_2205_04148_gb300 import inputs as I
    n, nz, nq = 96, 80, 2
    opts = dict(nh_full=1, remap=1, d2c_ord=4, d2_bg=0.02, dddmp=0.1)
    st = I.cubed_state(n, nz, seed=0, ntracers=nq)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    g.set_tiles(16, 16, 1)
    g.set_persistent(True)
    g.run_dyn(gs, fv3.params(n_split=6, **opts), 1)
    fields = FIELDS + ("delz", "q0", "q1")
    sens, want = ulp_sensitivity(orc, st, True, n, nz, nq, lambda s: s.run_dyn(orc.params(n_split=6, **opts), 1),
                                 fields)
    for f in fields:
        e = relerr(g.read(gs, f), want[f])
        assert e <= max(TOL64, 4 * sens[f]), (f, e, sens[f])
    assert sens["w"] < 1e-10            # the conditioning stays what it is
