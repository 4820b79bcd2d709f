"""Seeded synthetic states for the FV3 acoustic substep.

This module is shared by the CUDA path, the CPU oracle and the benchmark.  It
only synthesises inputs: analytic or random-Fourier fields sampled at the
positions of the grid points.  It holds none of the substep's arithmetic (no
metric terms, no stencils, no halo logic).

Conventions (the C-ABI in ``include/fv3.h`` uses the same ones):

* Dense interior layouts, ``i`` (x) fastest:
  cell fields ``[nt][nz][n][n]``; D-grid ``u`` (x-wind on y-faces)
  ``[nt][nz][n+1][n]``; D-grid ``v`` (y-wind on x-faces) ``[nt][nz][n][n+1]``.
* Levels ``k = 0`` is the model top, ``k = nz-1`` the lowest layer.  ``delz``
  is negative (bottom minus top height), ``ptop = 100 Pa``.
* Cubed-sphere tile ``t`` maps scaled angles ``(sa, sb)`` in ``[-1, 1]`` to
  the unit vector ``normalise(c + tan(sa*pi/4) a + tan(sb*pi/4) b)`` with the
  frames in ``TILE_FRAMES`` (equiangular gnomonic projection, Section II of the
  paper: "gnomonic cubed-sphere grid").  ``tan`` is taken as exactly +-1 at the
  tile edges.  Cell ``(i, j)`` spans corners ``i..i+1`` / ``j..j+1`` with
  ``sa(i) = (2 i - n) / n``.

Random numbers come from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np

GRAV = 9.80665
RDGAS = 287.05
PTOP = 100.0
RADIUS = 6.3712e6
OMEGA = 7.292e-5

# (centre, alpha-direction, beta-direction) per tile; right-handed, a x b = c.
TILE_FRAMES = (
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((0, 1, 0), (-1, 0, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, -1, 0), (0, 0, 1)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
)


# --------------------------------------------------------------------------
# geometry of sample positions (positions only, no metric terms)
# --------------------------------------------------------------------------
def _tan_q(s):
    """tan(s * pi / 4) with exact +-1 at s = +-1."""
    s = np.asarray(s, dtype=np.float64)
    t = np.tan(s * (math.pi / 4.0))
    t = np.where(s == 1.0, 1.0, t)
    t = np.where(s == -1.0, -1.0, t)
    return t


def tile_points(tile: int, sa, sb):
    """Unit vectors of tile ``tile`` at scaled angles ``sa`` (x) and ``sb`` (y)."""
    c, a, b = (np.array(v, dtype=np.float64) for v in TILE_FRAMES[tile])
    ta = _tan_q(sa)[..., None]
    tb = _tan_q(sb)[..., None]
    p = c + ta * a + tb * b
    return p / np.linalg.norm(p, axis=-1, keepdims=True)


def _grid_s(n, idx2):
    """scaled angle of (half-)integer index positions: idx2 = 2 * index."""
    return (np.asarray(idx2, dtype=np.float64) - n) / n


def corner_points(tile, n):
    i = np.arange(n + 1)
    sa = _grid_s(n, 2 * i)
    SA, SB = np.meshgrid(sa, sa)  # [j][i]
    return tile_points(tile, SA, SB)


def centre_points(tile, n):
    i = np.arange(n)
    s = _grid_s(n, 2 * i + 1)
    SA, SB = np.meshgrid(s, s)
    return tile_points(tile, SA, SB)


def _edge_dirs(pa, pb):
    """midpoint (unit) and unit chord direction of the edges pa -> pb."""
    mid = pa + pb
    mid /= np.linalg.norm(mid, axis=-1, keepdims=True)
    d = pb - pa
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return mid, d


# --------------------------------------------------------------------------
# random smooth fields
# --------------------------------------------------------------------------
def _fourier2d(rng, n, kmax, x, y):
    """Random real Fourier series with 0 < |k| <= kmax on the unit-periodic
    square, evaluated at (x, y) in units of the period; unit RMS over the
    evaluation points."""
    f = np.zeros(np.broadcast(x, y).shape)
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            if ky == 0 and kx <= 0:
                continue
            if kx * kx + ky * ky > kmax * kmax:
                continue
            a, b = rng.standard_normal(2)
            ph = 2.0 * math.pi * (kx * x + ky * y)
            f += a * np.cos(ph) + b * np.sin(ph)
    rms = math.sqrt(float(np.mean(f * f)))
    return f / rms if rms > 0 else f


def _fourier3d(rng, kmax, p):
    """Smooth random field on the unit sphere from low-order 3-D Fourier modes
    of the Cartesian coordinates ``p[..., 3]``; zero mean, unit-scale."""
    f = np.zeros(p.shape[:-1])
    for kx in range(0, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kz in range(-kmax, kmax + 1):
                if (kx, ky, kz) <= (0, 0, 0):
                    continue
                if kx * kx + ky * ky + kz * kz > kmax * kmax:
                    continue
                a, b = rng.standard_normal(2)
                ph = 1.3 * (kx * p[..., 0] + ky * p[..., 1] + kz * p[..., 2])
                f += a * np.cos(ph) + b * np.sin(ph)
    return f


def hydrostatic_delz(delp, pt):
    """Layer thickness (negative) of a hydrostatic column: the ideal-gas layer
    thickness between the interface pressures built from ``ptop`` down."""
    pe = PTOP + np.concatenate(
        [np.zeros_like(delp[..., :1, :, :]), np.cumsum(delp, axis=-3)], axis=-3)
    return -(RDGAS / GRAV) * pt * np.log(pe[..., 1:, :, :] / pe[..., :-1, :, :])


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def periodic_state(n=48, nz=8, seed=0, dx=1.0e5):
    """Doubly-periodic uniform tile: delp = 1000 Pa (1 + 0.01 N), pt in
    [250, 300] K from Fourier modes |k| <= 4, u, v with |k| <= 4 and RMS
    10 m/s on the D-grid staggering, w = 0, hydrostatic delz."""
    rng = np.random.default_rng(seed)
    ic = (np.arange(n) + 0.5) / n
    ie = np.arange(n) / n
    delp = np.empty((1, nz, n, n))
    pt = np.empty((1, nz, n, n))
    u = np.empty((1, nz, n + 1, n))
    v = np.empty((1, nz, n, n + 1))
    Xc, Yc = np.meshgrid(ic, ic)
    for k in range(nz):
        delp[0, k] = 1000.0 * (1.0 + 0.01 * _fourier2d(rng, n, 4, Xc, Yc))
        pt[0, k] = np.clip(275.0 + 25.0 * _fourier2d(rng, n, 4, Xc, Yc), 250.0, 300.0)
        # u on y-faces: x = (i+1/2)/n, y = j/n; v on x-faces: x = i/n, y = (j+1/2)/n
        Xu, Yu = np.meshgrid(ic, ie)
        Xv, Yv = np.meshgrid(ie, ic)
        su = rng.integers(1 << 30)
        sv = rng.integers(1 << 30)
        fu = _fourier2d(np.random.default_rng(su), n, 4, Xu, Yu)
        fv = _fourier2d(np.random.default_rng(sv), n, 4, Xv, Yv)
        u[0, k, :n] = 10.0 * fu
        u[0, k, n] = u[0, k, 0]
        v[0, k, :, :n] = 10.0 * fv
        v[0, k, :, n] = v[0, k, :, 0]
    w = np.zeros((1, nz, n, n))
    delz = hydrostatic_delz(delp, pt)
    return dict(u=u, v=v, w=w, delp=delp, pt=pt, delz=delz)


def _perturb(delp, u, v, cen, mid_u, dir_u, mid_v, dir_v, member_seed, pert_delp, pert_wind):
    """In place: delp *= 1 + pert_delp N_m (N_m smooth, unit RMS) and a smooth
    non-divergent wind of amplitude pert_wind m/s added to u, v, all drawn
    from ``member_seed``."""
    mrng = np.random.default_rng(member_seed)
    f = _fourier3d(mrng, 3, cen)
    f /= math.sqrt(float(np.mean(f * f)))
    delp *= (1.0 + pert_delp * f)[:, None]
    if pert_wind:
        # smooth perturbation wind: the gradient-free field axis' x r
        ax2 = mrng.standard_normal(3)
        ax2 /= np.linalg.norm(ax2)

        def vel2(p):
            return np.cross(ax2, p)
        pu = np.sum(vel2(mid_u) * dir_u, axis=-1)
        pv = np.sum(vel2(mid_v) * dir_v, axis=-1)
        u += pert_wind * pu[:, None]
        v += pert_wind * pv[:, None]


def perturb_member(st, member_seed, pert_delp=0.01, pert_wind=1.0):
    """A batched-ensemble member from an unperturbed ``cubed_state`` ``st``:
    the same result as ``cubed_state(..., pert_delp, pert_wind,
    member_seed)`` without redrawing the base state (copies; ``st`` is kept)."""
    nt, nz, n, _ = st["delp"].shape
    cen = np.stack([centre_points(t, n) for t in range(nt)])
    cor = np.stack([corner_points(t, n) for t in range(nt)])
    mid_u, dir_u = _edge_dirs(cor[:, :, :-1], cor[:, :, 1:])
    mid_v, dir_v = _edge_dirs(cor[:, :-1, :], cor[:, 1:, :])
    out = dict(st)
    out["delp"] = st["delp"].copy()
    out["u"] = st["u"].copy()
    out["v"] = st["v"].copy()
    _perturb(out["delp"], out["u"], out["v"], cen, mid_u, dir_u, mid_v, dir_v, member_seed, pert_delp, pert_wind)
    out["delz"] = hydrostatic_delz(out["delp"], st["pt"])
    out["q"] = list(st["q"])
    return out


def cubed_state(n=96, nz=80, seed=0, ntracers=8, wind=20.0, tilt_deg=30.0,
                pert_delp=0.0, pert_wind=0.0, member_seed=None):
    """Six-tile cubed sphere: delp_k = (1e5 - 100)/nz (1 + 0.01 N), a 5 K
    Gaussian pt hill on 280 K centred at (0E, 0N) with radius R/8, solid-body
    rotation of ``wind`` m/s about an axis tilted ``tilt_deg`` from the pole,
    w = 0, hydrostatic delz and ``ntracers`` smooth tracers in [0, 1].

    ``pert_delp`` / ``pert_wind`` add the per-member perturbations of the
    batched ensemble (relative delp noise, absolute wind noise in m/s) drawn
    from ``member_seed``."""
    rng = np.random.default_rng(seed)
    nt = 6
    dp0 = (1.0e5 - PTOP) / nz
    cen = np.stack([centre_points(t, n) for t in range(nt)])  # [t][j][i][3]
    cor = np.stack([corner_points(t, n) for t in range(nt)])  # [t][j+1][i+1][3]

    delp = np.empty((nt, nz, n, n))
    for k in range(nz):
        f = _fourier3d(rng, 3, cen)
        f /= math.sqrt(float(np.mean(f * f)))
        delp[:, k] = dp0 * (1.0 + 0.01 * f)

    hill = np.array([1.0, 0.0, 0.0])
    dist = np.arccos(np.clip(cen @ hill, -1.0, 1.0)) * RADIUS
    r0 = RADIUS / 8.0
    pt2 = 280.0 + 5.0 * np.exp(-(dist / r0) ** 2)
    pt = np.broadcast_to(pt2[:, None], (nt, nz, n, n)).copy()

    tilt = math.radians(tilt_deg)
    axis = np.array([math.sin(tilt), 0.0, math.cos(tilt)])
    ws = wind / RADIUS

    def vel(p):  # p unit vectors [..., 3] -> velocity [..., 3] in m/s
        return ws * RADIUS * np.cross(axis, p)

    # D-grid u on y-faces (edge corner(i,j) -> corner(i+1,j))
    mid_u, dir_u = _edge_dirs(cor[:, :, :-1], cor[:, :, 1:])
    mid_v, dir_v = _edge_dirs(cor[:, :-1, :], cor[:, 1:, :])
    u2 = np.sum(vel(mid_u) * dir_u, axis=-1)  # [t][n+1][n]
    v2 = np.sum(vel(mid_v) * dir_v, axis=-1)  # [t][n][n+1]
    u = np.broadcast_to(u2[:, None], (nt, nz, n + 1, n)).copy()
    v = np.broadcast_to(v2[:, None], (nt, nz, n, n + 1)).copy()

    if member_seed is not None and (pert_delp or pert_wind):
        _perturb(delp, u, v, cen, mid_u, dir_u, mid_v, dir_v, member_seed, pert_delp, pert_wind)

    w = np.zeros((nt, nz, n, n))
    delz = hydrostatic_delz(delp, pt)
    q = []
    for _ in range(ntracers):
        f = _fourier3d(rng, 2, cen)
        lo, hi = float(f.min()), float(f.max())
        q2 = (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)
        q.append(np.broadcast_to(q2[:, None], (nt, nz, n, n)).copy())
    return dict(u=u, v=v, w=w, delp=delp, pt=pt, delz=delz, q=q)


def default_params(dt=20.0, n_split=6):
    """Substep parameters used by every workload (monotone PPM, del-4 damping
    with coefficient 0.12, fully implicit vertical solve)."""
    return dict(dt=dt, n_split=n_split, nord=1, hord=0, d4_bg=0.12, a_imp=1.0,
                dz_min=2.0, ptop=PTOP, grav=GRAV, rdgas=RDGAS, cp_air=1004.6)
