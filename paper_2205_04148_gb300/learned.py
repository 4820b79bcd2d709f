"""Training and evaluation of the learned face values (reading R14).

The paper has no learned component (it motivates coupling machine-learned
models to the dynamical core, Section III-B).  The learned face value is the
plain PPM face value plus a correction sigma * y from a small network of the
six normalised cells around the face.  The experiment here:

* truth: plain FP64 runs on a fine cubed sphere (C192 by default), coarsened
  4x to the coarse grid (C48): area-weighted delp, delp-weighted pt and
  tracers;
* training samples: coarse six-cell stencils along x and y at interior coarse
  faces of coarsened fine snapshots.  The face value the fine grid resolves
  is the mean of the fine PPM edge values on the r fine faces that make up
  the coarse face (face-length weights for delp; face-length x face-mass
  weights for pt and tracers); the target is its difference from the plain
  coarse PPM face value (for the flow direction of the coarsened fine winds)
  over sigma, the standard deviation of the six cells;
* training: Adam on the mirror-symmetric objective with the library's
  tensor-core gradient kernel (fv3_mlp_grad, fv3_mlp_adam), cosine learning
  rate decay;
* evaluation: coarse runs with plain PPM and with learned face values, and a
  plain run at twice the coarse resolution, from seeds disjoint from the
  training seeds, against the coarsened fine run, with their wall times.

Array handling (views of the library layout, coarse-graining, sampling, the
training targets) uses PyTorch on the device; every substep runs in the
library's kernels.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import fv3
from . import inputs as I

POSITIVE_FIELDS = ("delp", "pt")


def interior(g, t, member=0, nlev=None):
    """[nt][nz][n][n] view of a cell field in the library layout."""
    import torch
    lay = g.layout(member)
    nz = lay.nz if nlev is None else nlev
    return torch.as_strided(t, (lay.ntiles, nz, lay.n, lay.n), (nz * lay.plane, lay.plane, lay.pitch, 1),
                            lay.offset3 + 3 * lay.pitch + lay.ox)


def interior_face(g, t, kind, member=0):
    """[nt][nz][n+1][n] (y-faces, u) or [nt][nz][n][n+1] (x-faces, v) view"""
    import torch
    lay = g.layout(member)
    nj, ni = (lay.n + 1, lay.n) if kind == fv3.KIND_YFACE else (lay.n, lay.n + 1)
    return torch.as_strided(t, (lay.ntiles, lay.nz, nj, ni), (lay.nz * lay.plane, lay.plane, lay.pitch, 1),
                            lay.offset3 + 3 * lay.pitch + lay.ox)


def normalise(st):
    """network inputs x [S, 6] (float) and sigma [S] of six-cell stencils
    st [S, 6] (float64, on the device), formed by the library's kernels
    (fv3_face_stencils, reading R14)"""
    out = fv3.face_stencils(st, plain=False, inputs=True)
    return out["x"], out["sig"]


def plain_face(st, c):
    """plain PPM face value (reading R4) between st[:, 2] and st[:, 3] for
    Courant numbers c [S] (float64, on the device), from the library's kernels"""
    return fv3.face_stencils(st, c)["plain"]


def edge_at(q, fi, dim):
    """fine clamped fourth-order edge values (reading R4, step 1) between
    cells fi - 1 and fi along ``dim`` (-1 = x, -2 = y), from the library's
    kernels; the result has the indices fi in place of ``dim``"""
    import torch
    st = torch.stack([q.index_select(dim, fi + s) for s in range(-2, 2)], -1)   # cells fi-2 .. fi+1
    q6 = torch.cat([st[..., :1], st, st[..., 3:]], -1)       # the edge reads the middle four
    return fv3.face_stencils(q6.reshape(-1, 6), plain=False, edge=True)["edge"].reshape(st.shape[:-1])


def coarsen(fine, area, r, weight=None):
    """r x r block means over the last two axes, area (and weight) weighted"""
    w = area if weight is None else area * weight
    nt, nz, n, _ = fine.shape
    m = n // r
    num = (fine * w).reshape(nt, nz, m, r, m, r).sum((3, 5))
    den = w.expand_as(fine).reshape(nt, nz, m, r, m, r).sum((3, 5))
    return num / den


def coarse_state(fields, area, r):
    dp = fields["delp"]
    out = {"delp": coarsen(dp, area, r)}
    for k, v in fields.items():
        if k != "delp":
            out[k] = coarsen(v, area, r, dp)
    return out


def samples_from_snapshot(fields, winds, area, dxf, dyf, r, rng, per_field, dt=20.0):
    """(x [S,6], t [S]) of normalised coarse stencils and correction targets"""
    import torch
    dp = fields["delp"]
    u, v = winds
    coarse = coarse_state(fields, area, r)
    nt, nz, n, _ = dp.shape
    m = n // r
    dxc = r * float(torch.sqrt(area.mean()))      # coarse cell width for the Courant estimate
    xs, ts = [], []
    I_ = torch.arange(3, m - 2, device=dp.device)
    fi = r * I_
    dpe_x = edge_at(dp, fi, -1)   # fine x-faces fi: [nt, nz, n, nI]
    dpe_y = edge_at(dp, fi, -2)   # fine y-faces fi: [nt, nz, nI, n]
    # normal winds on fine x-faces (from u) and y-faces (from v), coarse-face means
    ucx = 0.25 * (u[..., :-1, fi - 1] + u[..., :-1, fi] + u[..., 1:, fi - 1] + u[..., 1:, fi])   # [nt,nz,n,nI]
    ucx = ucx.reshape(nt, nz, m, r, -1).mean(3)                                                    # [nt,nz,m,nI]
    vcy = 0.25 * (v[..., fi - 1, :-1] + v[..., fi - 1, 1:] + v[..., fi, :-1] + v[..., fi, 1:])     # [nt,nz,nJ,n]
    vcy = vcy.reshape(nt, nz, -1, m, r).mean(4)                                                    # [nt,nz,nJ,m]
    for name, q in fields.items():
        qc = coarse[name]
        for axis in ("x", "y"):
            if axis == "x":
                a = edge_at(q, fi, -1)                          # [nt, nz, n, nI]
                wv = dyf[None, None, :, fi].expand_as(a)
                if name != "delp":
                    wv = wv * dpe_x
                a = (a * wv).reshape(nt, nz, m, r, -1).sum(3) / wv.reshape(nt, nz, m, r, -1).sum(3)
                st = torch.stack([qc[..., :, I_ + s] for s in range(-3, 3)], -1)   # [nt, nz, m, nI, 6]
                c = dt * ucx / dxc
            else:
                a = edge_at(q, fi, -2)                          # [nt, nz, nJ, n]
                wv = dxf[None, None, fi, :].expand_as(a)
                if name != "delp":
                    wv = wv * dpe_y
                a = (a * wv).reshape(nt, nz, -1, m, r).sum(4) / wv.reshape(nt, nz, -1, m, r).sum(4)
                st = torch.stack([qc[..., I_ + s, :] for s in range(-3, 3)], -1)   # [nt, nz, nJ, m, 6]
                c = dt * vcy / dxc
            st = st.reshape(-1, 6)
            a = a.reshape(-1)
            c = c.reshape(-1)
            # half of the faces uniformly, half in proportion to the stencil's
            # relative variation (where the face values, and their errors, matter)
            nsel = min(per_field, st.shape[0])
            uni = torch.as_tensor(rng.choice(st.shape[0], nsel - nsel // 2, replace=False), device=q.device)
            rel = (st.std(1) / st[:, 2:4].abs().mean(1).clamp_min(1e-300)).float()
            gen = torch.Generator(device=q.device)
            gen.manual_seed(int(rng.integers(1 << 62)))
            imp = torch.multinomial(rel + 1e-30, nsel // 2, replacement=False, generator=gen)
            sel = torch.cat([uni, imp])
            st, a, c = st[sel], a[sel], c[sel]
            x, sig = normalise(st)
            ok = sig.double() > 1e-9 * (0.5 * (st[:, 2] + st[:, 3])).abs()
            t = (a - plain_face(st, c)) / sig.double().clamp_min(1e-300)
            ok = ok & (t.abs() < 10.0)
            xs.append(x[ok])
            ts.append(t[ok].float())
    return torch.cat(xs), torch.cat(ts)


def fine_run_samples(npx_fine, r, nz, seeds, snapshots, every, per_field, nq, rng_seed=0):
    import torch
    rng = np.random.default_rng(rng_seed)
    g = fv3.Grid(fv3.GRID_CUBED, npx_fine, nz)
    area = torch.as_tensor(g.metric("area"), device="cuda")[:, None]
    dxf = torch.as_tensor(g.metric("dx")[0], device="cuda")   # y-face lengths of tile 0 (tiles alike)
    dyf = torch.as_tensor(g.metric("dy")[0], device="cuda")   # x-face lengths
    X, T = [], []
    prm = fv3.params(n_split=every)
    for sd in seeds:
        st = I.cubed_state(npx_fine, nz, seed=sd, ntracers=nq)
        gs = g.alloc_state(nq)
        g.load(gs, st)
        for _ in range(snapshots):
            g.run_dyn(gs, prm, 1)
            fields = {"delp": interior(g, gs["delp"]), "pt": interior(g, gs["pt"])}
            for k in range(nq):
                fields["q%d" % k] = interior(g, gs["q"][k])
            winds = (interior_face(g, gs["u"], fv3.KIND_YFACE), interior_face(g, gs["v"], fv3.KIND_XFACE))
            x, t = samples_from_snapshot(fields, winds, area, dxf, dyf, r, rng, per_field)
            X.append(x)
            T.append(t)
    g.close()
    return torch.cat(X), torch.cat(T)


def init_params(seed=0, scale=1.0):
    """Glorot-style random initial parameters (flat float64[1313])."""
    rng = np.random.default_rng(seed)
    w = np.zeros(fv3.MLP_NP)
    w[0:192] = rng.standard_normal(192) * scale * np.sqrt(2.0 / 38)
    w[224:1248] = rng.standard_normal(1024) * scale * np.sqrt(2.0 / 64)
    w[1280:1312] = rng.standard_normal(32) * scale * np.sqrt(2.0 / 33) * 0.1
    return w


def fit(X, T, steps=3000, batch=65536, lr=2e-3, seed=0, log_every=500, holdout=0.05):
    """Adam on mini-batches through the C-ABI training kernels, cosine
    learning-rate decay; the parameters with the lowest loss on a held-out
    part of the samples are returned."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    perm = torch.randperm(X.shape[0], device="cuda", generator=g)
    nh = max(1, int(holdout * X.shape[0]))
    Xh, Th = X[perm[:nh]].contiguous(), T[perm[:nh]].contiguous()
    X, T = X[perm[nh:]], T[perm[nh:]]
    tr = fv3.MlpTrainer(init_params(seed), lr=lr)
    n = X.shape[0]
    hist = []
    best, best_w = float("inf"), tr.w.clone()
    for s in range(1, steps + 1):
        tr.lr = 0.5 * lr * (1 + np.cos(np.pi * (s - 1) / steps))
        idx = torch.randint(0, n, (min(batch, n),), device="cuda", generator=g)
        loss = tr.update(X[idx].contiguous(), T[idx].contiguous())
        if s % log_every == 0 or s == 1 or s == steps:
            yh = fv3.mlp_forward(tr.w, Xh, symmetric=True)
            lh = float(0.5 * ((yh - Th) ** 2).mean())
            hist.append((s, float(loss.item()), lh))
            if lh < best:
                best, best_w = lh, tr.w.clone()
    return best_w, hist


def _coarse_run(npx, nz, seed, nq, init, prm, steps):
    """Run a coarse model from the coarsened fine initial fields ``init``
    (delp, pt, tracers; winds and delz from the generator on the coarse grid);
    return the final interior fields (device tensors) and the wall time."""
    import torch
    stc = I.cubed_state(npx, nz, seed=seed, ntracers=nq)
    stc["delp"] = init["delp"].cpu().numpy()
    stc["pt"] = init["pt"].cpu().numpy()
    stc["delz"] = I.hydrostatic_delz(stc["delp"], stc["pt"])
    stc["q"] = [init["q%d" % k].cpu().numpy() for k in range(nq)]
    g = fv3.Grid(fv3.GRID_CUBED, npx, nz)
    gs = g.alloc_state(nq)
    g.load(gs, stc)
    g.run_dyn(gs, prm, 1)         # warm (graph capture) on a copy of the run
    g.load(gs, stc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.run_dyn(gs, prm, steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {k: interior(g, gs[k]).clone() for k in ("delp", "pt")}
    for k in range(nq):
        out["q%d" % k] = interior(g, gs["q"][k]).clone()
    area = torch.as_tensor(g.metric("area"), device="cuda")[:, None]
    g.close()
    return out, area, dt


def _rel_rms(fields, truth):
    import torch
    errs = {}
    for k in truth:
        dev = truth[k] - truth[k].mean()
        errs[k] = float(torch.sqrt(((fields[k] - truth[k]) ** 2).mean()) / torch.sqrt((dev ** 2).mean()))
    return errs


def coarse_eval(npx, r, nz, seed, substeps, nq, w=None):
    """Fine truth (C{npx*r}) coarsened r x to C{npx}; plain and learned coarse
    runs against it, and (r even) a plain run at twice the coarse resolution
    coarsened 2x -- the plain model given more wall time than the learned
    one.  Relative RMS errors (RMS difference over the truth's RMS deviation
    from its mean) and wall times."""
    import torch
    n_split = 6 if substeps % 6 == 0 or substeps % 5 != 0 else 5
    steps = max(1, substeps // n_split)
    gf = fv3.Grid(fv3.GRID_CUBED, npx * r, nz)
    area = torch.as_tensor(gf.metric("area"), device="cuda")[:, None]
    stf = I.cubed_state(npx * r, nz, seed=seed, ntracers=nq)
    gsf = gf.alloc_state(nq)
    gf.load(gsf, stf)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gf.run_dyn(gsf, fv3.params(n_split=n_split), steps)
    torch.cuda.synchronize()
    t_fine = time.perf_counter() - t0
    fields = {"delp": interior(gf, gsf["delp"]), "pt": interior(gf, gsf["pt"])}
    for k in range(nq):
        fields["q%d" % k] = interior(gf, gsf["q"][k])
    truth = {k: v.clone() for k, v in coarse_state(fields, area, r).items()}
    init = {"delp": torch.as_tensor(stf["delp"], device="cuda"), "pt": torch.as_tensor(stf["pt"], device="cuda")}
    for k in range(nq):
        init["q%d" % k] = torch.as_tensor(stf["q"][k], device="cuda")
    gf.close()
    del gsf, fields
    res = {}
    runs = [("plain", npx, None)]
    if w is not None:
        runs.append(("learned", npx, w))
    if r % 2 == 0:
        runs.append(("plain_2x", 2 * npx, None))
    for label, n, wt in runs:
        prm = fv3.params(n_split=n_split) if wt is None else fv3.params(n_split=n_split, hord=1, mlp=wt)
        out, area_c, dt = _coarse_run(n, nz, seed, nq, coarse_state(init, area, npx * r // n), prm, steps)
        if n != npx:
            out = coarse_state(out, area_c, n // npx)
        err = _rel_rms(out, truth)
        qs = [v for k, v in err.items() if k.startswith("q")]
        res[label] = {"npx": n, "wall_s": dt, "rel_rms_err": err,
                      "tracer_mean_rel_rms_err": float(np.mean(qs)) if qs else None}
    res["t_fine"] = t_fine
    res["substeps"] = steps * n_split
    return res


def experiment(npx=48, r=4, nz=80, train_seeds=(11, 12, 13, 14), snapshots=50, every=10, per_field=4000,
               nq=8, eval_seeds=(1001,), substeps=500, steps=3000, out=None):
    import torch
    t0 = time.perf_counter()
    X, T = fine_run_samples(npx * r, r, nz, train_seeds, snapshots, every, per_field, nq)
    t_data = time.perf_counter() - t0
    w, hist = fit(X, T, steps=steps)
    t_fit = time.perf_counter() - t0 - t_data
    # baseline of the fit: no correction (plain PPM), y = 0
    pred = fv3.mlp_forward(w, X, symmetric=True)
    mse_plain = float((T ** 2).mean())
    mse_net = float(((pred - T) ** 2).mean())
    evals = [coarse_eval(npx, r, nz, sd, substeps, nq, w) for sd in eval_seeds]
    res = {"samples": int(X.shape[0]), "t_data_s": t_data, "t_fit_s": t_fit, "loss_history": hist,
           "sample_mse_plain": mse_plain, "sample_mse_network": mse_net, "eval": evals,
           "config": dict(npx=npx, r=r, nz=nz, train_seeds=list(train_seeds), snapshots=snapshots, every=every,
                          per_field=per_field, nq=nq, eval_seeds=list(eval_seeds), substeps=substeps,
                          steps=steps)}
    if out:
        with open(out, "w") as fh:
            json.dump(res, fh, indent=1)
        np.save(out.replace(".json", "_weights.npy"), w.cpu().numpy())
    return res, w


if __name__ == "__main__":
    import argparse
    p = argparse.ArgumentParser()
    p.add_argument("--npx", type=int, default=48)
    p.add_argument("--r", type=int, default=4)
    p.add_argument("--nz", type=int, default=80)
    p.add_argument("--snapshots", type=int, default=50)
    p.add_argument("--every", type=int, default=10)
    p.add_argument("--per-field", type=int, default=4000)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--substeps", type=int, default=500)
    p.add_argument("--out", default=None)
    a = p.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    res, _ = experiment(npx=a.npx, r=a.r, nz=a.nz, snapshots=a.snapshots, every=a.every, per_field=a.per_field,
                        steps=a.steps, substeps=a.substeps, out=a.out)
    print(json.dumps({k: v for k, v in res.items() if k != "loss_history"}, indent=1))
