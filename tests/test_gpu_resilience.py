"""Failure detection and resumption without any device fault: non-finite
state values reported through the status word, and a remapping-step run that
is saved to the host, reloaded and continued giving bitwise the same state as
an uninterrupted run (the FP64 path is deterministic)."""
import numpy as np
import pytest

from gpu_common import FIELDS, seeded

pytestmark = pytest.mark.gpu


def test_nonfinite_state_reported():
    from paper_2205_04148_gb300 import fv3
    st = seeded(True, 10, 3, seed=5, nq=1)
    g = fv3.Grid(fv3.GRID_CUBED, 10, 3)
    gs = g.alloc_state(1)
    g.load(gs, st)
    assert g.check_finite(gs) == 0
    for f in ("pt", "u", "q0"):
        bad = {k: (v.copy() if not isinstance(v, list) else [x.copy() for x in v]) for k, v in st.items()}
        if f == "q0":
            bad["q"][0][3, 1, 4, 5] = np.nan
        else:
            bad[f][2, 2, 5, 1] = np.inf
        g.load(gs, bad)
        assert g.check_finite(gs) == -5, f
    g.load(gs, st)
    assert g.check_finite(gs) == 0


def test_resume_from_host_is_bitwise():
    from paper_2205_04148_gb300 import fv3
    n, nz, nq = 12, 4, 2
    st = seeded(True, n, nz, seed=6, nq=nq)
    prm = fv3.params(n_split=3)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    a = g.alloc_state(nq)
    g.load(a, st)
    g.run_dyn(a, prm, 3)
    names = FIELDS + ("delz",) + tuple("q%d" % k for k in range(nq))
    straight = {f: g.read(a, f) for f in names}
    b = g.alloc_state(nq)
    g.load(b, st)
    g.run_dyn(b, prm, 1)
    saved = {f: g.read(b, f) for f in names}           # checkpoint to the host
    g2 = fv3.Grid(fv3.GRID_CUBED, n, nz)                 # a new context, as after a restart
    c = g2.alloc_state(nq)
    ck = {f: saved[f] for f in FIELDS + ("delz",)}
    ck["q"] = [saved["q%d" % k] for k in range(nq)]
    g2.load(c, ck)
    g2.run_dyn(c, prm, 2)
    for f in names:
        assert np.array_equal(g2.read(c, f), straight[f]), f
