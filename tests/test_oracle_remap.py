"""Pins of the oracle's vertical remapping (reading R16: the Lagrangian layers
are remapped to reference layers equally spaced in pressure between the
model top and the surface; piecewise-parabolic reconstruction with the R4
edges and limiter, exact integration over the overlaps)."""
import numpy as np

from paper_2205_04148_gb300 import inputs as I


def rand_interfaces(rng, nz, top=100.0, bottom=1.0e5, spread=0.5):
    """increasing interfaces from top to bottom with random layer thicknesses"""
    dp = 1 + spread * rng.uniform(-1, 1, nz)
    dp *= (bottom - top) / dp.sum()
    pe = np.concatenate([[top], top + np.cumsum(dp)])
    pe[-1] = bottom
    return pe


def test_identity(orc):
    rng = np.random.default_rng(1)
    pe = rand_interfaces(rng, 30)
    q = rng.standard_normal(30)
    assert np.abs(orc.remap_column(pe, pe, q) - q).max() <= 4e-15 * np.abs(q).max()


def test_conservation_and_bounds(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        nz = int(rng.integers(4, 60))
        pe = rand_interfaces(rng, nz)
        pn = rand_interfaces(rng, nz, spread=0.9)
        pn[-1] = pe[-1]
        q = 300 + 20 * rng.standard_normal(nz)
        out = orc.remap_column(pe, pn, q)
        assert abs(np.sum(out * np.diff(pn)) - np.sum(q * np.diff(pe))) <= 1e-14 * np.sum(q * np.diff(pe))
        assert out.min() >= q.min() - 1e-12 and out.max() <= q.max() + 1e-12


def test_constant_preserved(orc):
    rng = np.random.default_rng(3)
    pe = rand_interfaces(rng, 40)
    pn = rand_interfaces(rng, 40)
    pn[-1] = pe[-1]
    out = orc.remap_column(pe, pn, np.full(40, 287.3))
    assert np.abs(out - 287.3).max() <= 1e-12


def test_quadratic_exact_away_from_the_ends(orc):
    # layer means of f(p) = (p - p0)^2 on uniform old layers: the fourth-order
    # edges are exact, the limiter is inactive, so the parabolas are f itself and
    # every new layer inside old layers 2 .. nz-3 gets f's exact mean
    nz, top, bottom, p0 = 40, 100.0, 1.0e5, -5.0e4
    pe = np.linspace(top, bottom, nz + 1)
    rng = np.random.default_rng(4)
    pn = rand_interfaces(rng, nz, spread=0.6)
    pn[-1] = pe[-1]
    F = lambda a, b: ((b - p0) ** 3 - (a - p0) ** 3) / 3.0 / (b - a)
    q = F(pe[:-1], pe[1:])
    out = orc.remap_column(pe, pn, q)
    want = F(pn[:-1], pn[1:])
    inside = (pn[:-1] >= pe[2]) & (pn[1:] <= pe[nz - 2])
    assert inside.sum() > nz // 2
    assert np.abs(out - want)[inside].max() <= 1e-12 * np.abs(want).max()


def test_state_remap(orc):
    n, nz = 10, 6
    st = I.cubed_state(n, nz, seed=3, ntracers=2)
    st["q"][1] = np.full_like(st["q"][1], 0.25)
    d = orc.Domain(True, n, nz)
    s = orc.State(d, 2)
    s.load(st)
    m0 = s.mass()
    dp0 = s.get("delp")
    tr0 = np.sum(s.get("q0") * dp0, axis=1)

    def face_momentum(u, v, dp):
        # interior faces: u on y-faces j = 1..n-1 (cells j-1, j), v on x-faces i = 1..n-1
        mu = np.sum(u[:, :, 1:n, :] * 0.5 * (dp[:, :, :-1, :] + dp[:, :, 1:, :]), axis=1)
        mv = np.sum(v[:, :, :, 1:n] * 0.5 * (dp[:, :, :, :-1] + dp[:, :, :, 1:]), axis=1)
        return mu, mv
    mu0, mv0 = face_momentum(s.get("u"), s.get("v"), dp0)
    s.remap()
    dp1 = s.get("delp")
    mu1, mv1 = face_momentum(s.get("u"), s.get("v"), dp1)
    assert np.abs(mu1 - mu0).max() <= 1e-12 * np.abs(mu0).max()
    assert np.abs(mv1 - mv0).max() <= 1e-12 * np.abs(mv0).max()
    # surface pressure kept, layers equally spaced in pressure
    assert np.abs(dp1.sum(1) - dp0.sum(1)).max() <= 1e-9
    assert np.abs(dp1 - dp1[:, :1]).max() <= 1e-9
    assert abs(s.mass() - m0) <= 1e-14 * m0
    # column tracer mass conserved, constant tracer unchanged
    assert np.abs(np.sum(s.get("q0") * dp1, axis=1) - tr0).max() <= 1e-13 * np.abs(tr0).max()
    assert np.abs(s.get("q1") - 0.25).max() <= 1e-14
    # column height conserved through delz / delp
    assert np.abs(s.get("delz").sum(1) - st["delz"].sum(1)).max() <= 1e-10 * np.abs(st["delz"].sum(1)).max()
    # a second remap is the identity (the layers are already the reference)
    before = {f: s.get(f) for f in ("u", "v", "w", "delp", "pt", "delz", "q0")}
    s.remap()
    for f, a in before.items():
        assert np.abs(s.get(f) - a).max() <= 1e-12 * max(1.0, np.abs(a).max()), f
