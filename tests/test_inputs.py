"""The seeded input generators: batched-ensemble members drawn from a base
state equal the directly generated perturbed states."""
import numpy as np

from paper_2205_04148_gb300 import inputs as I


def test_perturb_member_equals_direct_draw():
    a = I.cubed_state(10, 3, seed=4, ntracers=1, pert_delp=0.01, pert_wind=1.0, member_seed=7)
    base = I.cubed_state(10, 3, seed=4, ntracers=1)
    b = I.perturb_member(base, 7)
    for k in ("u", "v", "w", "delp", "pt", "delz"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["q"][0], b["q"][0])
    # the base state is left as it was, and members differ
    assert np.array_equal(base["delp"], I.cubed_state(10, 3, seed=4, ntracers=1)["delp"])
    c = I.perturb_member(base, 8)
    rel = np.abs(c["delp"] / base["delp"] - 1)
    assert 1e-4 < rel.max() < 0.1
    assert 0.1 < np.abs(c["u"] - base["u"]).max() < 10.0
