"""The FP64 transport's face arithmetic on single stencils (fv3_face_stencils,
fv3_learned_faces; readings R4 and R14) against the oracle: plain PPM face
values and edge values to rounding, the float network inputs within the
float error of the FP64 definition, and the learned face value's plain-PPM
fallback taken on the same faces as the oracle's except where the oracle's
candidate lies within the network's bfloat16 error of a bound."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U24 = 2.0 ** -24


def stencils(seed, n):
    rng = np.random.default_rng(seed)
    st = 300 + rng.standard_normal((n, 6)) * 10.0 ** rng.uniform(-5, 1, (n, 1))
    st[: n // 6] = np.sort(st[: n // 6], axis=1)          # monotone stencils
    st[n // 6: n // 3] = np.sort(st[n // 6: n // 3], axis=1)[:, ::-1]
    st[n // 3: n // 3 + 8] = 0.0                            # zeros and constants
    st[n // 3 + 8: n // 3 + 16] = 12.5
    c = rng.uniform(-0.95, 0.95, n)
    c[:20] = 0.0
    c[20:30] = 1.0
    c[30:40] = -1.0
    return st, c


def cuda(a, dt=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt or torch.float64, device="cuda")


def test_plain_faces_and_edges_match_oracle(orc):
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    st, c = stencils(31, 3000)
    out = fv3.face_stencils(cuda(st), cuda(c), plain=True, edge=True)
    got = out["plain"].cpu().numpy()
    want = np.array([orc.ppm_face(s, cc) for s, cc in zip(st, c)])
    scale = np.abs(st).max(1)
    assert (np.abs(got - want) <= 4e-16 * scale).all()
    e = out["edge"].cpu().numpy()
    ew = np.array([orc.ppm_edge(s[1:5]) for s in st])
    assert (np.abs(e - ew) <= 4e-16 * scale).all()
    # Courant number +1 / -1 gives the upwind cell exactly (the cell before /
    # after the face)
    assert np.array_equal(got[20:30], st[20:30, 2])
    assert np.array_equal(got[30:40], st[30:40, 3])


def test_network_inputs_within_float_error_of_fp64(orc):
    # the kernels normalise in float (offsets from the centre pair's mean,
    # rounded to float); the FP64 definition bounds them: |x| <= sqrt(6),
    # offsets within 2 sqrt(6) sig, so every rounding contributes at most a
    # few float ulps of sig (x) or of sig itself
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    st, c = stencils(32, 3000)
    out = fv3.face_stencils(cuda(st), plain=False, inputs=True)
    x, sig = out["x"].cpu().numpy().astype(np.float64), out["sig"].cpu().numpy().astype(np.float64)
    xo, so = orc.mlp_normalise(st)
    assert (np.abs(sig - so) <= 64 * U24 * so + 1e-300).all()
    assert np.abs(x - xo).max() <= 64 * U24
    # mirror symmetry is exact on the GPU
    outr = fv3.face_stencils(cuda(st[:, ::-1]), plain=False, inputs=True)
    assert np.array_equal(outr["x"].cpu().numpy(), out["x"].cpu().numpy()[:, ::-1])


def test_learned_fallback_on_the_oracles_faces(orc):
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    st, c = stencils(33, 2000)
    w = orc.mlp_init(34, scale=1.0)
    w[1312] = 0.3
    got = fv3.learned_faces(cuda(w, dt=__import__("torch").float32), cuda(st), cuda(c)).cpu().numpy()
    plain = fv3.face_stencils(cuda(st), cuda(c))["plain"].cpu().numpy()
    _, sig = orc.mlp_normalise(st)
    n_acc = n_rej = n_band = 0
    for f in range(len(c)):
        a, acc = orc.learned_candidate(w, st[f], c[f], positive=1, bf16=1)
        p = orc.ppm_face(st[f], c[f])
        lo, hi = min(st[f, 2], st[f, 3]), max(st[f, 2], st[f, 3])
        y = (a - p) / sig[f] if sig[f] > 0 else 0.0
        delta = 2e-2 * (1 + abs(y)) * sig[f] + 4e-16 * abs(st[f]).max()
        gpu_acc = got[f] != plain[f]
        if gpu_acc == acc or got[f] == a == p:
            if acc:
                n_acc += 1
                assert abs(got[f] - a) <= delta, (f, got[f], a)
            else:
                n_rej += 1
                assert got[f] == plain[f] and abs(plain[f] - p) <= 4e-16 * abs(st[f]).max()
        else:
            # the decision differs only where the candidate sits on a bound
            n_band += 1
            assert min(abs(a - lo), abs(a - hi), abs(a)) <= delta, (f, a, lo, hi)
    assert n_acc > 100 and n_rej > 100, (n_acc, n_rej)
    assert n_band <= 0.02 * len(c), n_band
