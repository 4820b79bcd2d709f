"""GPU learned face values (reading R14) against the oracle: tensor-core
inference, the training gradient of the mirror-symmetric network, Adam, and a
learned substep.  Tolerances: bfloat16 operands (8-bit mantissa) and the
hardware tanh make the GPU network agree with the oracle's bfloat16-emulating
evaluation to ~1e-2 and with its FP64 gradient to 2e-2 of the largest entry."""
import numpy as np
import pytest

from gpu_common import FIELDS, relerr, seeded

pytestmark = pytest.mark.gpu


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def test_forward_matches_oracle(orc):
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    rng = np.random.default_rng(0)
    w = orc.mlp_init(1)
    X = rng.standard_normal((1000, 6))
    y_gpu = fv3.mlp_forward(cuda(w), cuda(X), symmetric=False).cpu().numpy()
    y_bf = np.array([orc.mlp_forward_bf16(w, x) for x in X])
    y64 = np.array([orc.mlp_forward(w, x) for x in X])
    assert np.abs(y_gpu - y_bf).max() <= 1e-2 * (1 + np.abs(y_bf).max())
    assert np.abs(y_gpu - y64).max() <= 3e-2 * (1 + np.abs(y64).max())
    ys = fv3.mlp_forward(cuda(w), cuda(X), symmetric=True).cpu().numpy()
    ys64 = orc.mlp_sym_forward(w, X)
    assert np.abs(ys - ys64).max() <= 3e-2 * (1 + np.abs(ys64).max())
    # mirror symmetry of the symmetric evaluation is exact on the GPU
    ysr = fv3.mlp_forward(cuda(w), cuda(X[:, ::-1]), symmetric=True).cpu().numpy()
    assert np.array_equal(ys, ysr)


def test_gradient_matches_oracle(orc):
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    rng = np.random.default_rng(2)
    w = orc.mlp_init(3)
    n = 777
    X = rng.standard_normal((n, 6))
    T = rng.standard_normal(n) * 0.5
    tr = fv3.MlpTrainer(w)
    g, loss = tr.grad(cuda(X), cuda(T), weight=1.0 / n)
    g = g.cpu().numpy()
    l64, g64 = orc.mlp_sym_grad(w, X, T, 1.0 / n)
    assert abs(float(loss.item()) - l64) <= 2e-2 * l64
    for lo, hi in ((0, 192), (192, 224), (224, 1248), (1248, 1280), (1280, 1312), (1312, 1313)):
        err = np.abs(g[lo:hi] - g64[lo:hi]).max() / np.abs(g64[lo:hi]).max()
        assert err <= 2e-2, (lo, hi, err)


def test_fp32_gradient_matches_oracle(orc):
    """the float check path: within 1e-5 of the FP64 gradient, and the
    tensor-core gradient within 2e-2 of it"""
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    rng = np.random.default_rng(7)
    w = orc.mlp_init(8)
    n = 513
    X = rng.standard_normal((n, 6))
    T = rng.standard_normal(n) * 0.5
    tr = fv3.MlpTrainer(w)
    g32, loss32 = tr.grad_fp32(cuda(X), cuda(T), weight=1.0 / n)
    g32 = g32.cpu().numpy()
    l64, g64 = orc.mlp_sym_grad(w, X, T, 1.0 / n)
    assert abs(float(loss32.item()) - l64) <= 1e-5 * l64
    for lo, hi in ((0, 192), (192, 224), (224, 1248), (1248, 1280), (1280, 1312), (1312, 1313)):
        err = np.abs(g32[lo:hi] - g64[lo:hi]).max() / np.abs(g64[lo:hi]).max()
        assert err <= 1e-5, (lo, hi, err)
    gbf, _ = tr.grad(cuda(X), cuda(T), weight=1.0 / n)
    gbf = gbf.cpu().numpy()
    assert np.abs(gbf - g32).max() <= 2e-2 * np.abs(g32).max()


def test_adam_fits_a_smooth_target(orc):
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    rng = np.random.default_rng(4)
    n = 4096
    X = rng.standard_normal((n, 6))
    T = 0.3 * (X[:, 2] + X[:, 3]) + 0.05 * (X[:, 1] + X[:, 4])   # symmetric target
    tr = fv3.MlpTrainer(orc.mlp_init(5, scale=0.5), lr=3e-3)
    xs, ts = cuda(X), cuda(T)
    first = float(tr.update(xs, ts).item())
    for _ in range(300):
        last = float(tr.update(xs, ts).item())
    assert last < 0.1 * first, (first, last)


def test_learned_substep_close_to_oracle(orc):
    """The learned substep (delp and pt through the network) on the GPU against
    the oracle's bfloat16-emulating network: the face values differ by the
    bfloat16 rounding of the network only."""
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    n, nz = 12, 3
    st = seeded(True, n, nz, seed=41)
    w = orc.mlp_init(6, scale=0.3)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    gs = g.alloc_state()
    g.load(gs, st)
    wd = cuda(w)
    g.substep(gs, fv3.params(mlp=wd, hord=1))
    d = orc.Domain(True, n, nz)
    s = orc.State(d)
    s.load(st)
    s.substep(orc.params(mlp=w, mlp_bf16=1, hord=1))
    s_plain = orc.State(d)
    s_plain.load(st)
    s_plain.substep()
    for f in FIELDS:
        e = relerr(g.read(gs, f), s.get(f))
        assert e <= 1e-4, (f, e)
    # and the learned substep is not the plain one
    assert relerr(s.get("pt"), s_plain.get("pt")) > 1e-9
    # mass stays conserved with learned fluxes
    m0 = orc.State(d)
    m0.load(st)
    assert abs(g.mass(gs)[0] - m0.mass()) <= 1e-14 * m0.mass()


def test_zero_network_is_plain_ppm():
    """a network that outputs zero adds no correction: the learned substep is
    the plain one"""
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    n, nz = 12, 3
    st = seeded(True, n, nz, seed=43)
    out = []
    for prm in (fv3.params(), fv3.params(mlp=cuda(np.zeros(fv3.MLP_NP)), hord=1)):
        g = fv3.Grid(fv3.GRID_CUBED, n, nz)
        gs = g.alloc_state()
        g.load(gs, st)
        g.substep(gs, prm)
        out.append({f: g.read(gs, f) for f in FIELDS})
    for f in FIELDS:
        assert relerr(out[1][f], out[0][f]) <= 1e-15, f
