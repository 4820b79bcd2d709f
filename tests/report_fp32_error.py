#!/usr/bin/env python3
"""Per-field error of the FP32-bulk path against FP64 after 1 and 100
acoustic substeps (the precision variant: stencil arithmetic and storage in
FP32; the column solve, metric terms and mass sums in FP64).

The same seeded cubed-sphere state (default C192 x 80 levels, solid-body
rotation, Gaussian pt hill) is advanced by

* the FP32-bulk GPU path with FP32 copies of the metric terms (FV3_FP32),
* the FP32-bulk GPU path with the metric terms in FP64 (FV3_FP32_M64),
* the FP64 GPU path (which matches the oracle to 1e-12 per substep), and
* the FP64 oracle (plain C, one thread, on the host cores) -- at every
  reported substep count up to --oracle-substeps,

and for each field (u, v, w, delp, pt, delz) the relative max-norm error
max|x - x_ref| / max|x_ref| and the relative RMS error rms(x - x_ref) /
rms(x_ref - mean x_ref) are reported, together with the time per substep of
both GPU paths (CUDA events, inputs far larger than L2) and the mass drift.

The GPU runs come first; the oracle then runs on the CPU while nothing else
of this script uses the GPU.  Writes one JSON file.

    python tests/report_fp32_error.py --npx 192 --npz 80 --out fp32_error.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FIELDS = ("u", "v", "w", "delp", "pt", "delz")


def errors(x, ref):
    out = {}
    for f in FIELDS:
        a, b = x[f], ref[f]
        d = a - b
        dev = b - b.mean()
        rms_dev = float(np.sqrt((dev * dev).mean()))
        out[f] = {"n_differ": int(np.count_nonzero(d)), "max_abs": float(np.abs(d).max()),
                  "rel_max": float(np.abs(d).max() / max(np.abs(b).max(), 1e-300)),
                  "rel_rms": float(np.sqrt((d * d).mean()) / rms_dev) if rms_dev > 0 else None}
    return out


def gpu_runs(npx, npz, marks, st, reps):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_04148_gb300 import fv3
    torch.cuda.set_device(0)
    res, times, mass = {}, {}, {}
    for label, prec in (("fp32", fv3.FP32), ("fp32_m64", fv3.FP32_M64), ("fp64", fv3.FP64)):
        g = fv3.Grid(fv3.GRID_CUBED, npx, npz, precision=prec)
        gs = g.alloc_state()
        # time per substep (warm state, then reload)
        g.load(gs, st)
        for _ in range(3):
            g.substep(gs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.substep(gs)
        e1.record()
        torch.cuda.synchronize()
        times[label] = e0.elapsed_time(e1) / reps
        g.load(gs, st)
        m0 = g.mass(gs)[0]
        done = 0
        res[label] = {}
        for m in marks:
            for _ in range(m - done):
                g.substep(gs)
            done = m
            res[label][m] = {f: g.read(gs, f) for f in FIELDS}
        mass[label] = float((g.mass(gs)[0] - m0) / m0)
        g.close()
        del gs
        torch.cuda.empty_cache()
    return res, times, mass


def oracle_runs(npx, npz, marks, st, upto):
    from oracle import oracle as O
    d = O.Domain(True, npx, npz)
    s = O.State(d)
    s.load(st)
    out, done, t0 = {}, 0, time.perf_counter()
    for m in marks:
        if m > upto:
            break
        for _ in range(m - done):
            s.substep()
        done = m
        out[m] = {f: s.get(f) for f in FIELDS}
    return out, (time.perf_counter() - t0) / max(1, done)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--npx", type=int, default=192)
    p.add_argument("--npz", type=int, default=80)
    p.add_argument("--marks", default="1,100")
    p.add_argument("--oracle-substeps", type=int, default=100)
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--out", default="fp32_error.json")
    a = p.parse_args()
    marks = sorted(int(x) for x in a.marks.split(","))
    from paper_2205_04148_gb300 import inputs as I
    st = I.cubed_state(a.npx, a.npz, seed=0, ntracers=0)
    gpu, times, mass = gpu_runs(a.npx, a.npz, marks, st, a.reps)
    report = {"config": {"npx": a.npx, "npz": a.npz, "cells": 6 * a.npx * a.npx * a.npz, "marks": marks,
                         "state": "cubed_state(seed=0): solid-body rotation 20 m/s at 30 deg, 5 K pt hill"},
              "ms_per_substep": times, "speedup_fp32_over_fp64": times["fp64"] / times["fp32"],
              "speedup_fp32_m64_over_fp64": times["fp64"] / times["fp32_m64"],
              "mass_drift": mass,
              "fp32_vs_fp64_gpu": {m: errors(gpu["fp32"][m], gpu["fp64"][m]) for m in marks},
              "fp32_m64_vs_fp64_gpu": {m: errors(gpu["fp32_m64"][m], gpu["fp64"][m]) for m in marks}}
    with open(a.out, "w") as fh:
        json.dump(report, fh, indent=1)
    orc, t_orc = oracle_runs(a.npx, a.npz, marks, st, a.oracle_substeps)
    report["oracle_s_per_substep"] = t_orc
    report["fp32_vs_oracle"] = {m: errors(gpu["fp32"][m], orc[m]) for m in orc}
    report["fp32_m64_vs_oracle"] = {m: errors(gpu["fp32_m64"][m], orc[m]) for m in orc}
    report["fp64_gpu_vs_oracle"] = {m: errors(gpu["fp64"][m], orc[m]) for m in orc}
    with open(a.out, "w") as fh:
        json.dump(report, fh, indent=1)
    print(json.dumps(report, indent=1))


if __name__ == "__main__":
    main()
