"""Shared helpers of the GPU parity tests: build the same seeded state on the
CUDA path (through the C-ABI) and in the FP64 oracle, and compare per field
with the relative max-norm max|gpu - oracle| / max|oracle|."""
import numpy as np

from paper_2205_04148_gb300 import inputs as I

FIELDS = ("u", "v", "w", "delp", "pt")
TOL64 = 1e-12      # FP64 parity bound per field per substep


def relerr(a, b):
    den = float(np.abs(b).max())
    d = float(np.abs(a - b).max())
    return d / den if den > 0 else d


def seeded(cubed, n, nz, seed, nq=0, w_amp=0.5):
    if cubed:
        st = I.cubed_state(n, nz, seed=seed, ntracers=nq)
    else:
        st = I.periodic_state(n, nz, seed=seed)
        rng = np.random.default_rng(seed + 77)
        st["q"] = [rng.uniform(0, 1, st["delp"].shape) for _ in range(nq)]
    # a nonzero vertical velocity exercises the w paths
    rng = np.random.default_rng(seed + 991)
    st["w"] = w_amp * rng.standard_normal(st["w"].shape)
    return st


def pair(orc, cubed, n, nz, seed=0, nq=0, precision=0, members=None):
    """(grid, gpu state, oracle domain, oracle state, dense inputs)"""
    from paper_2205_04148_gb300 import fv3
    st = seeded(cubed, n, nz, seed, nq)
    g = fv3.Grid(fv3.GRID_CUBED if cubed else fv3.GRID_PERIODIC, n, nz, precision=precision)
    gs = g.alloc_state(nq)
    g.load(gs, st)
    d = orc.Domain(cubed, n, nz)
    s = orc.State(d, nq)
    s.load(st)
    return g, gs, d, s, st


def ulp_sensitivity(orc, st, cubed, n, nz, nq, run, fields, seed=1):
    """per field, the relative max-norm change of the oracle's result when pt
    is perturbed by one unit in the last place (random signs): the rounding
    condition of the computation.  A field formed by cancellation (w after
    the closed substep: a small difference of pressure perturbations) moves
    by far more than 1e-16 under any change of rounding, so two correct
    implementations can differ by that much."""
    out = []
    rng = np.random.default_rng(seed)
    for eps in (0.0, 1.0):
        s = orc.State(orc.Domain(cubed, n, nz), nq)
        st2 = dict(st)
        st2["pt"] = st["pt"] * (1 + eps * 2.220446049250313e-16 * rng.choice([-1.0, 1.0], st["pt"].shape))
        s.load(st2)
        run(s)
        out.append({f: s.get(f) for f in fields})
    return {f: relerr(out[1][f], out[0][f]) for f in fields}, out[0]
