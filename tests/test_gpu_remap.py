"""Vertical remapping on the GPU (reading R16) against the oracle: every field
after a remap, run_dyn with the remap at the end of the step, uneven batched
members, the FP32 form, and conservation on the device."""
import numpy as np
import pytest

from gpu_common import FIELDS, TOL64, relerr, seeded

pytestmark = pytest.mark.gpu

ALL = FIELDS + ("delz",)


def state(cubed, n, nz, seed, nq):
    st = seeded(cubed, n, nz, seed, nq)
    # uneven Lagrangian layers: the reference layers differ from them
    rng = np.random.default_rng(seed + 5)
    st["delp"] = st["delp"] * (1 + 0.2 * rng.uniform(-1, 1, (1,) + st["delp"].shape[1:2] + (1, 1)))
    return st


@pytest.mark.parametrize("cubed", [False, True])
def test_remap_matches_oracle(orc, cubed):
    from paper_2205_04148_gb300 import fv3
    n, nz, nq = 12, 10, 2
    st = state(cubed, n, nz, 71, nq)
    g = fv3.Grid(fv3.GRID_CUBED if cubed else fv3.GRID_PERIODIC, n, nz)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    m0 = g.mass(gs)[0]
    g.remap(gs)
    s = orc.State(orc.Domain(cubed, n, nz), nq)
    s.load(st)
    s.remap()
    for f in ALL + ("q0", "q1"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    assert abs(g.mass(gs)[0] - m0) <= 1e-14 * m0
    # the layers are now the reference ones: a second remap changes nothing
    before = {f: g.read(gs, f) for f in ALL}
    g.remap(gs)
    for f in ALL:
        assert relerr(g.read(gs, f), before[f]) <= 1e-13, f


def test_run_dyn_with_remap(orc):
    from paper_2205_04148_gb300 import fv3
    n, nz, nq = 12, 6, 1
    st = state(True, n, nz, 73, nq)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    g.run_dyn(gs, fv3.params(n_split=2, remap=1), 1)
    s = orc.State(orc.Domain(True, n, nz), nq)
    s.load(st)
    s.run_dyn(orc.params(n_split=2, remap=1), 1)
    for f in ALL + ("q0",):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)


def test_remap_batched_members(orc):
    from paper_2205_04148_gb300 import fv3
    sizes, nz = [8, 12], 5
    g = fv3.Grid(fv3.GRID_CUBED, 8, nz, n_members=2, member_npx=sizes)
    gs = g.alloc_state(0)
    sts = [state(True, n, nz, 80 + m, 0) for m, n in enumerate(sizes)]
    for m, st in enumerate(sts):
        g.load(gs, st, member=m)
    g.remap(gs)
    for m, n in enumerate(sizes):
        s = orc.State(orc.Domain(True, n, nz))
        s.load(sts[m])
        s.remap()
        for f in ALL:
            e = relerr(g.read(gs, f, member=m), s.get(f))
            assert e <= TOL64, (m, f, e)


def test_remap_fp32(orc):
    from paper_2205_04148_gb300 import fv3
    n, nz = 10, 8
    st = state(True, n, nz, 77, 0)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz, precision=fv3.FP32)
    gs = g.alloc_state()
    g.load(gs, st)
    g.remap(gs)
    s = orc.State(orc.Domain(True, n, nz))
    s.load(st)
    s.remap()
    for f in ALL:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= 2e-6, (f, e)
