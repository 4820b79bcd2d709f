"""Write the oracle regression fixtures in this folder.

The paper (arxiv 2205.04148) prints no numeric value of any FV3 field, so no
fixture here is the paper's.  These files only freeze the oracle's own output
on tiny seeded cases so that an unintended change of its arithmetic shows up;
they call nothing but ``oracle/`` and the seeded input generator.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2205_04148_gb300 import inputs as I  # noqa: E402

CASES = {
    "periodic_n8_nz3_seed7": dict(cubed=False, n=8, nz=3, seed=7),
    "cubed_n6_nz3_seed7": dict(cubed=True, n=6, nz=3, seed=7),
}
FIELDS = ("u", "v", "w", "delp", "pt")


def run(case):
    if case["cubed"]:
        st = I.cubed_state(case["n"], case["nz"], seed=case["seed"], ntracers=0)
    else:
        st = I.periodic_state(case["n"], case["nz"], seed=case["seed"])
    d = O.Domain(case["cubed"], case["n"], case["nz"])
    s = O.State(d)
    s.load(st)
    s.substep()
    out = {}
    for f in FIELDS:
        a = s.get(f)
        flat = a.ravel()
        idx = np.linspace(0, flat.size - 1, 7).astype(int)
        out[f] = {"sum": float(a.sum()), "absmax": float(np.abs(a).max()),
                  "idx": idx.tolist(), "val": [float(x) for x in flat[idx]]}
    out["mass"] = s.mass()
    return out


def main():
    for name, case in CASES.items():
        data = {"case": case, "result": run(case)}
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main()
