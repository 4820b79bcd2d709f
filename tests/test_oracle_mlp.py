"""Pins of the oracle's learned face value (reading R14: a 6 -> 32 -> 32 -> 1
tanh network on the normalised six cells of the PPM face-value stencil, with
plain PPM as the fallback).  The paper has no learned component; these pins
fix the network, its gradient and the fallback rules."""
import math

import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I


def rand_x(seed, n):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 6))


def test_gradient_matches_central_differences(orc):
    w = orc.mlp_init(1)
    X = rand_x(2, 3)
    T = np.array([0.3, -0.7, 0.1])
    _, g = orc.mlp_grad(w, X, T)
    h = 1e-6
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(192, 20, replace=False), 192 + rng.choice(32, 5, replace=False),
                          224 + rng.choice(1024, 30, replace=False), 1248 + rng.choice(32, 5, replace=False),
                          1280 + np.arange(32), [1312]])
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        lp, _ = orc.mlp_grad(wp, X, T)
        lm, _ = orc.mlp_grad(wm, X, T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_closed_forms(orc):
    rng = np.random.default_rng(4)
    w = np.zeros(orc.MLP_NP)
    w[192:224] = rng.standard_normal(32)        # b1
    w[1248:1280] = rng.standard_normal(32)      # b2
    w[1280:1312] = rng.standard_normal(32)      # W3
    w[1312] = 0.25                              # b3
    x = rng.standard_normal(6)
    want = float(np.tanh(w[1248:1280]) @ w[1280:1312]) + 0.25
    assert abs(orc.mlp_forward(w, x) - want) < 1e-14
    w2 = np.zeros(orc.MLP_NP)
    w2[1312] = -1.5
    assert orc.mlp_forward(w2, x) == -1.5


def test_zero_network_gives_plain_ppm(orc):
    # y = 0 -> no correction: exactly the plain PPM face value, either flow sign
    w = np.zeros(orc.MLP_NP)
    rng = np.random.default_rng(21)
    for _ in range(50):
        q6 = 10 + rng.standard_normal(6)
        c = rng.uniform(-0.9, 0.9)
        assert orc.learned_face(w, q6, c) == orc.ppm_face(q6, c)


def test_constant_output_correction_closed_form(orc):
    # only the output bias: y = beta, correction beta * sigma with sigma the
    # standard deviation of the six cells (sqrt(35/12) for 1..6)
    w = np.zeros(orc.MLP_NP)
    w[1312] = 0.1
    q6 = np.arange(1.0, 7.0)
    for c in (0.3, -0.3):
        plain = orc.ppm_face(q6, c)
        want = plain + 0.1 * math.sqrt(35.0 / 12.0)
        assert 3.0 <= want <= 4.0
        assert abs(orc.learned_face(w, q6, c) - want) <= 1e-6


def test_normalised_inputs(orc):
    # FP64 definition (reading R14): sigma is the population standard
    # deviation, x (sigma + 1e-12 |mean|) the deviations from the mean
    rng = np.random.default_rng(22)
    q = 1000.0 + rng.standard_normal((200, 6)) * 10.0 ** rng.uniform(-6, 2, (200, 1))
    x, sig = orc.mlp_normalise(q)
    mu = q.mean(-1)
    assert np.abs(sig - q.std(-1)).max() <= 1e-9 * sig.min() + 1e-13 * np.abs(mu).max()
    dev = x * (sig + 1e-12 * np.abs(mu))[:, None]
    assert np.abs(dev - (q - mu[:, None])).max() <= 1e-12 * np.abs(mu).max()
    assert (np.abs(x.mean(-1)) <= 1e-14 * np.abs(mu) / sig).all()   # cancellation in q - mean
    xr, sigr = orc.mlp_normalise(q[:, ::-1])
    assert np.array_equal(xr, x[:, ::-1]) and np.array_equal(sigr, sig)
    # a constant stencil: no deviation beyond the rounding of its mean, and
    # eps keeps the inputs near zero
    x0, s0 = orc.mlp_normalise(np.full((1, 6), 3.7))
    assert s0[0] <= 4e-16 * 3.7 and np.abs(x0).max() <= 1e-3


def test_learned_candidate_and_decision(orc):
    # the candidate is plain + sigma y (output-bias network: y = beta) and the
    # fallback keeps it exactly when it lies in the range of the two cells
    w = np.zeros(orc.MLP_NP)
    q6 = np.array([1.0, 2.0, 2.5, 3.5, 4.0, 5.0])
    x, sig = orc.mlp_normalise(q6)
    for beta, keep in ((0.2, True), (0.9, False), (-0.9, False)):
        w[1312] = beta
        a, acc = orc.learned_candidate(w, q6, 0.3)
        assert abs(a - (orc.ppm_face(q6, 0.3) + beta * sig)) <= 1e-14
        assert acc == keep == (2.5 <= a <= 3.5)
        assert orc.learned_face(w, q6, 0.3) == (a if keep else orc.ppm_face(q6, 0.3))


def test_fallbacks(orc):
    q6 = np.array([1.0, 2.0, 2.5, 3.5, 4.0, 5.0])
    plain = orc.ppm_face(q6, 0.3)
    w = np.zeros(orc.MLP_NP)
    w[1312] = 50.0                     # far outside [q_{i-1}, q_i]
    assert orc.learned_face(w, q6, 0.3) == plain
    # positivity: a field near zero whose learned value would be negative
    q6 = np.array([0.0, 0.0, 1e-3, 0.0, 0.0, 0.0])
    w[1312] = -3.0
    assert orc.learned_face(w, q6, -0.2) == orc.ppm_face(q6, -0.2)


def test_bf16_inference_close_to_fp64(orc):
    w = orc.mlp_init(5)
    for x in rand_x(6, 50):
        a = orc.mlp_forward(w, x)
        b = orc.mlp_forward_bf16(w, x)
        assert abs(a - b) <= 3e-2 * (1 + abs(a))


def test_learned_substep_conserves_and_keeps_constants(orc):
    st = I.cubed_state(10, 3, seed=8, ntracers=2)
    st["q"][1] = np.full_like(st["q"][1], 0.4)
    d = orc.Domain(True, 10, 3)
    s = orc.State(d, 2)
    s.load(st)
    m0 = s.mass()
    w = orc.mlp_init(7, scale=0.3)
    prm = orc.params(mlp=w, hord=1, n_split=2)
    s.run_dyn(prm, 1)
    assert abs(s.mass() - m0) <= 1e-14 * m0
    assert np.abs(s.get("q1") - 0.4).max() <= 1e-13
    assert np.isfinite(s.get("pt")).all()
    # the learned run differs from the plain one
    s2 = orc.State(d, 2)
    s2.load(st)
    s2.run_dyn(orc.params(n_split=2), 1)
    assert np.abs(s.get("q0") - s2.get("q0")).max() > 0


def test_symmetric_gradient_matches_central_differences(orc):
    w = orc.mlp_init(11)
    X = rand_x(12, 2)
    T = np.array([0.2, -0.4])
    _, g = orc.mlp_sym_grad(w, X, T)
    h = 1e-6
    for k in list(range(0, 192, 7)) + list(range(224, 1248, 37)) + list(range(1280, 1313)):
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (orc.mlp_sym_grad(wp, X, T)[0] - orc.mlp_sym_grad(wm, X, T)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_learned_face_mirror_symmetric(orc):
    w = orc.mlp_init(13, scale=0.5)
    rng = np.random.default_rng(14)
    for _ in range(100):
        q6 = 10 + rng.standard_normal(6)
        c = rng.uniform(-0.5, 0.5)
        a = orc.learned_face(w, q6, c)
        b = orc.learned_face(w, q6[::-1].copy(), -c)
        assert a == b
