"""The oracle against its frozen regression fixtures (tests/golden)."""
import json
import os

import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(f for f in os.listdir(HERE) if f.endswith(".json"))


@pytest.mark.parametrize("fname", FILES)
def test_golden(orc, fname):
    data = json.load(open(os.path.join(HERE, fname)))
    case = data["case"]
    if case["cubed"]:
        st = I.cubed_state(case["n"], case["nz"], seed=case["seed"], ntracers=0)
    else:
        st = I.periodic_state(case["n"], case["nz"], seed=case["seed"])
    d = orc.Domain(case["cubed"], case["n"], case["nz"])
    s = orc.State(d)
    s.load(st)
    s.substep()
    for f, ref in data["result"].items():
        if f == "mass":
            assert abs(s.mass() - ref) <= 1e-14 * abs(ref)
            continue
        a = s.get(f).ravel()
        assert np.allclose(a[ref["idx"]], ref["val"], rtol=1e-12, atol=1e-12 * ref["absmax"])
