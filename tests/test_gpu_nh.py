"""The closed acoustic substep on the GPU (reading R17: update_dz_d with the
D-grid area fluxes, riem_solver3 over the whole substep, the D-grid
nonhydrostatic pressure gradient) against the oracle."""
import numpy as np
import pytest

from gpu_common import FIELDS, TOL64, pair, relerr

pytestmark = pytest.mark.gpu

ALL = FIELDS + ("delz",)


@pytest.mark.parametrize("cubed", [False, True])
def test_closed_substep_matches_oracle(orc, cubed):
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, cubed, 16, 6, seed=91)
    for _ in range(2):
        g.substep(gs, fv3.params(nh_full=1))
        s.substep(orc.params(nh_full=1))
    for f in ALL:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    # and the closed substep is not the open one
    s2 = orc.State(d)
    s2.load(st)
    for _ in range(2):
        s2.substep()
    assert relerr(s.get("delz"), s2.get("delz")) > 1e-12


def test_closed_run_dyn_with_tracers_and_remap(orc):
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, True, 12, 5, seed=93, nq=1)
    m0 = g.mass(gs)[0]
    g.run_dyn(gs, fv3.params(n_split=3, nh_full=1, remap=1), 1)
    s.run_dyn(orc.params(n_split=3, nh_full=1, remap=1), 1)
    for f in ALL + ("q0",):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= TOL64, (f, e)
    assert abs(g.mass(gs)[0] - m0) <= 1e-13 * m0


def test_closed_substep_fp32(orc):
    from paper_2205_04148_gb300 import fv3
    g, gs, d, s, st = pair(orc, True, 16, 5, seed=95, precision=fv3.FP32)
    g.substep(gs, fv3.params(nh_full=1))
    s.substep(orc.params(nh_full=1))
    for f in ("u", "v", "delp", "pt", "delz"):
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= 2e-4, (f, e)
