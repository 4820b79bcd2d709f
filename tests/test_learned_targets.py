"""The training-target helpers of the learned face value (reading R14) agree
with the oracle: the plain PPM face value for both flow directions, and the
network inputs formed from a six-cell stencil."""
import numpy as np
import torch

from paper_2205_04148_gb300 import learned


def test_plain_face_matches_oracle(orc):
    rng = np.random.default_rng(31)
    st = 10 + rng.standard_normal((300, 6)) * rng.uniform(0.01, 3, (300, 1))
    st[:50] = np.sort(st[:50], axis=1)            # monotone stencils
    c = rng.uniform(-0.9, 0.9, 300)
    c[:20] = 0.0
    got = learned.plain_face(torch.as_tensor(st), torch.as_tensor(c)).numpy()
    want = np.array([orc.ppm_face(s, cc) for s, cc in zip(st, c)])
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_normalise_matches_oracle(orc):
    rng = np.random.default_rng(32)
    st = 300 + rng.standard_normal((200, 6)) * 10.0 ** rng.uniform(-5, 1, (200, 1))
    x, sig = learned.normalise(torch.as_tensor(st))
    xo, so = orc.mlp_normalise(st)
    # float arithmetic on both sides; vectorised reductions may round a last bit apart
    assert np.abs(sig.numpy() - so).max() <= 2.4e-7 * so.max()
    assert np.abs(x.numpy() - xo).max() <= 1e-6
