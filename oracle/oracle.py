"""ctypes wrapper of the FP64 CPU oracle (oracle/fv3_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path never imports
this module.  The oracle shares no code with the CUDA library; inputs come
from ``paper_2205_04148_gb300.inputs`` (a module that holds no arithmetic of
the method).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fv3_oracle.c")
LIB = os.path.join(HERE, "libfv3_oracle.so")

_lib = None


def build(force=False):
    """Compile the oracle with gcc (no fused multiply-add, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-o", LIB + ".tmp", SRC, "-lm"])
        os.replace(LIB + ".tmp", LIB)
    return LIB


class OParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_split", C.c_int), ("nord", C.c_int), ("hord", C.c_int),
                ("d4_bg", C.c_double), ("a_imp", C.c_double), ("dz_min", C.c_double),
                ("ptop", C.c_double), ("grav", C.c_double), ("rdgas", C.c_double),
                ("cp_air", C.c_double), ("mlp", C.POINTER(C.c_double)), ("mlp_bf16", C.c_int),
                ("remap", C.c_int), ("nh_full", C.c_int), ("d2c_ord", C.c_int),
                ("d2_bg", C.c_double), ("dddmp", C.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(LIB)
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    L.orc_dom_create.restype = vp
    L.orc_dom_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
    L.orc_dom_free.argtypes = [vp]
    L.orc_dom_info.argtypes = [vp, C.POINTER(C.c_int)]
    L.orc_da_min.restype = C.c_double
    L.orc_da_min.argtypes = [vp]
    L.orc_get_metric.restype = C.c_int
    L.orc_get_metric.argtypes = [vp, C.c_char_p, dp]
    L.orc_ppm_face.restype = C.c_double
    L.orc_ppm_face.argtypes = [dp, C.c_double]
    L.orc_ppm_edge.restype = C.c_double
    L.orc_ppm_edge.argtypes = [dp]
    L.orc_state_create.restype = vp
    L.orc_state_create.argtypes = [vp, C.c_int]
    L.orc_state_free.argtypes = [vp]
    L.orc_state_io.restype = C.c_int
    L.orc_state_io.argtypes = [vp, C.c_char_p, dp, C.c_int]
    L.orc_substep.argtypes = [vp, C.POINTER(OParams), C.c_int, C.c_int]
    L.orc_run_dyn.argtypes = [vp, C.POINTER(OParams), C.c_int]
    L.orc_mass_sum.restype = C.c_double
    L.orc_mass_sum.argtypes = [vp]
    L.orc_thomas.argtypes = [C.c_int, dp, dp, dp, dp, dp]
    L.orc_dense_lu.argtypes = [C.c_int, dp, dp, dp]
    L.orc_riem_column.argtypes = [C.c_int, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double, C.c_double, dp, dp, dp, C.c_int, dp]
    L.orc_fv_tp_2d_dense.argtypes = [vp, C.c_int, dp, dp, dp, dp, dp, dp, dp]
    L.orc_delnflux_dense.argtypes = [vp, C.c_int, dp, C.c_double, dp, dp]
    L.orc_fill_cells.argtypes = [vp, dp, C.c_int, C.c_int]
    L.orc_fill_faces.argtypes = [vp, dp, dp, C.c_int, C.c_int, C.c_int]
    L.orc_copy_corners.argtypes = [vp, dp, C.c_int]
    L.orc_plane_sizes.argtypes = [vp, C.POINTER(C.c_long)]
    L.orc_gpoint.argtypes = [vp, C.c_int, C.c_double, C.c_double, dp]
    L.orc_mlp_forward.restype = C.c_double
    L.orc_mlp_forward.argtypes = [dp, dp, dp, dp]
    L.orc_mlp_backward.restype = C.c_double
    L.orc_mlp_backward.argtypes = [dp, dp, C.c_double, C.c_double, dp]
    L.orc_mlp_forward_bf16.restype = C.c_double
    L.orc_mlp_forward_bf16.argtypes = [dp, dp]
    L.orc_mlp_sym_backward.restype = C.c_double
    L.orc_mlp_sym_backward.argtypes = [dp, dp, C.c_double, C.c_double, dp]
    L.orc_mlp_sym_forward.restype = C.c_double
    L.orc_mlp_sym_forward.argtypes = [dp, dp]
    L.orc_d2c_dense.restype = C.c_int
    L.orc_d2c_dense.argtypes = [C.c_void_p, C.c_int, dp, dp, C.c_int, dp, dp]
    L.orc_remap_column.restype = C.c_double
    L.orc_remap_column.argtypes = [C.c_int, dp, dp, dp, dp]
    L.orc_remap.restype = None
    L.orc_remap.argtypes = [C.c_void_p, C.POINTER(OParams)]
    L.orc_mlp_normalise.restype = C.c_double
    L.orc_mlp_normalise.argtypes = [dp, dp]
    L.orc_learned_candidate.restype = C.c_double
    L.orc_learned_candidate.argtypes = [dp, C.c_int, dp, C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.orc_learned_face.restype = C.c_double
    L.orc_learned_face.argtypes = [dp, C.c_int, dp, C.c_double, C.c_int]
    _lib = L
    return L


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(mlp=None, mlp_bf16=0, **kw):
    """Substep parameters; ``mlp`` (1313 network parameters) with hord=1 selects
    the learned face values."""
    from paper_2205_04148_gb300.inputs import default_params
    p = default_params()
    p.update(kw)
    prm = OParams(p["dt"], p["n_split"], p["nord"], p["hord"], p["d4_bg"], p["a_imp"],
                  p["dz_min"], p["ptop"], p["grav"], p["rdgas"], p["cp_air"], None, int(mlp_bf16),
                  int(p.get("remap", 0)), int(p.get("nh_full", 0)), int(p.get("d2c_ord", 2)),
                  float(p.get("d2_bg", 0.0)), float(p.get("dddmp", 0.0)))
    if mlp is not None:
        w = _c(mlp)
        prm._w = w
        prm.mlp = _p(w)
    return prm


class Domain:
    """A periodic tile (cubed=False) or the six-tile cubed sphere."""

    def __init__(self, cubed, n, nz, dx=1.0e5, radius=6.3712e6, omega=7.292e-5):
        L = _load()
        self.L = L
        self.cubed, self.n, self.nz = bool(cubed), n, nz
        self.nt = 6 if cubed else 1
        self.h = 3
        self.ptr = L.orc_dom_create(int(cubed), n, nz, dx, radius, omega)
        sz = (C.c_long * 6)()
        L.orc_plane_sizes(self.ptr, sz)
        self.pc, self.px, self.py, self.pk, self.wc, self.wx = list(sz)

    def __del__(self):
        try:
            if self.ptr:
                self.L.orc_dom_free(self.ptr)
                self.ptr = None
        except Exception:
            pass

    def neighbours(self):
        out = (C.c_int * (5 + 72))()
        self.L.orc_dom_info(self.ptr, out)
        nb = np.array(out[5:], dtype=np.int64).reshape(6, 4, 3)
        return nb

    @property
    def da_min(self):
        return self.L.orc_da_min(self.ptr)

    def metric(self, name):
        """Padded metric planes of all tiles, shape [nt][rows][cols]."""
        big = np.empty(self.nt * max(self.pc, self.px, self.py, self.pk))
        pl = self.L.orc_get_metric(self.ptr, name.encode(), _p(big))
        if pl < 0:
            raise KeyError(name)
        n, h = self.n, self.h
        shapes = {self.pc: (n + 2 * h, n + 2 * h), self.px: (n + 2 * h, n + 1 + 2 * h),
                  self.pk: (n + 1 + 2 * h, n + 1 + 2 * h)}
        if name in ("dx", "rdx", "dyc", "rdyc", "cosy", "siny"):
            shp = (n + 1 + 2 * h, n + 2 * h)
        else:
            shp = shapes[pl]
        return big[: self.nt * pl].reshape((self.nt,) + shp).copy()

    def interior(self, name):
        """Metric on interior cells / tile faces / corners (no halo)."""
        a = self.metric(name)
        n, h = self.n, self.h
        if name in ("area", "rarea", "fA"):
            return a[:, h:h + n, h:h + n]
        if name in ("dx", "rdx", "dyc", "rdyc", "cosy", "siny"):
            return a[:, h:h + n + 1, h:h + n]
        if name in ("dy", "rdy", "dxc", "rdxc", "cosx", "sinx"):
            return a[:, h:h + n, h:h + n + 1]
        return a[:, h:h + n + 1, h:h + n + 1]

    def point(self, t, X, Y):
        p = np.empty(3)
        self.L.orc_gpoint(self.ptr, t, X, Y, _p(p))
        return p


FIELDS = ("u", "v", "w", "delp", "pt", "delz")


class State:
    def __init__(self, dom: Domain, nq=0):
        self.dom = dom
        self.nq = nq
        self.L = dom.L
        self.ptr = self.L.orc_state_create(dom.ptr, nq)

    def __del__(self):
        try:
            if self.ptr:
                self.L.orc_state_free(self.ptr)
                self.ptr = None
        except Exception:
            pass

    def _shape(self, name):
        d = self.dom
        n, nz, nt = d.n, d.nz, d.nt
        if name in ("u", "vc", "fy1", "mfy", "cry", "yfx", "yfxd"):
            return (nt, nz, n + 1, n)
        if name in ("v", "uc", "fx1", "mfx", "crx", "xfx", "xfxd"):
            return (nt, nz, n, n + 1)
        if name in ("pef", "gz"):
            return (nt, nz + 1, n, n)
        return (nt, nz, n, n)

    def set(self, name, arr):
        a = _c(arr).reshape(self._shape(name))
        rc = self.L.orc_state_io(self.ptr, name.encode(), _p(a), 0)
        if rc:
            raise KeyError(name)

    def get(self, name):
        a = np.empty(self._shape(name))
        rc = self.L.orc_state_io(self.ptr, name.encode(), _p(a), 1)
        if rc:
            raise KeyError(name)
        return a

    def load(self, st):
        for f in FIELDS:
            self.set(f, st[f])
        for m, q in enumerate(st.get("q", [])[: self.nq]):
            self.set("q%d" % m, q)

    def substep(self, prm=None, stop_after=-1, accumulate=0):
        prm = prm or params()
        self.L.orc_substep(self.ptr, C.byref(prm), stop_after, accumulate)

    def remap(self, prm=None):
        """vertical remapping of every column to the reference layers (R16)"""
        prm = prm or params()
        self.L.orc_remap(self.ptr, C.byref(prm))

    def run_dyn(self, prm=None, n_steps=1):
        prm = prm or params()
        self.L.orc_run_dyn(self.ptr, C.byref(prm), n_steps)

    def mass(self):
        return self.L.orc_mass_sum(self.ptr)


def ppm_face(q6, c):
    L = _load()
    q = _c(q6)
    return L.orc_ppm_face(_p(q), float(c))


def ppm_edge(q4):
    """clamped fourth-order edge value between q4[1] and q4[2] (reading R4)"""
    L = _load()
    q = _c(q4)
    return L.orc_ppm_edge(_p(q))


def thomas(a, b, c, d):
    L = _load()
    a, b, c, d = map(_c, (a, b, c, d))
    x = np.empty_like(d)
    L.orc_thomas(len(d), _p(a), _p(b), _p(c), _p(d), _p(x))
    return x


def dense_lu(A, b):
    L = _load()
    A, b = _c(A), _c(b)
    x = np.empty_like(b)
    L.orc_dense_lu(len(b), _p(A), _p(b), _p(x))
    return x


def riem_column(delpc, ptc, wc, delzc, dt, prm=None, use_lu=False):
    """One column of the semi-implicit solve; returns pef, gz, system, w."""
    L = _load()
    from paper_2205_04148_gb300.inputs import default_params
    p = default_params()
    if prm:
        p.update(prm)
    nz = len(delpc)
    delpc, ptc, wc, delzc = map(_c, (delpc, ptc, wc, delzc))
    pef = np.empty(nz + 1)
    gz = np.empty(nz + 1)
    sysm = np.empty(4 * nz)
    w = np.empty(nz + 1)
    L.orc_riem_column(nz, _p(delpc), _p(ptc), _p(wc), _p(delzc), dt, p["ptop"], p["grav"],
                      p["rdgas"], p["cp_air"], p["a_imp"], _p(pef), _p(gz), _p(sysm),
                      int(use_lu), _p(w))
    return pef, gz, sysm.reshape(4, nz), w


def fv_tp_2d(dom: Domain, tile, q, crx, cry, xfx, yfx):
    """Fluxes of level-0 dense inputs on ``tile`` (inputs for all tiles)."""
    L = _load()
    n = dom.n
    q, crx, cry, xfx, yfx = map(_c, (q, crx, cry, xfx, yfx))
    Fx = np.empty((n, n + 1))
    Fy = np.empty((n + 1, n))
    L.orc_fv_tp_2d_dense(dom.ptr, tile, _p(q), _p(crx), _p(cry), _p(xfx), _p(yfx), _p(Fx), _p(Fy))
    return Fx, Fy


def delnflux(dom: Domain, tile, q, damp):
    L = _load()
    n = dom.n
    q = _c(q)
    Fx = np.empty((n, n + 1))
    Fy = np.empty((n + 1, n))
    L.orc_delnflux_dense(dom.ptr, tile, _p(q), float(damp), _p(Fx), _p(Fy))
    return Fx, Fy


def fill_cells(dom: Domain, f, nlev, depth=3):
    L = _load()
    f = _c(f)
    L.orc_fill_cells(dom.ptr, _p(f), nlev, depth)
    return f


def fill_faces(dom: Domain, fx, fy, nlev, kind, corners=0):
    L = _load()
    fx, fy = _c(fx), _c(fy)
    L.orc_fill_faces(dom.ptr, _p(fx), _p(fy), nlev, kind, corners)
    return fx, fy


def copy_corners(dom: Domain, q, direction):
    L = _load()
    q = _c(q)
    L.orc_copy_corners(dom.ptr, _p(q), direction)
    return q


MLP_NP = 1313


def mlp_init(seed=0, scale=1.0):
    """Random network parameters (flat, 1313 values), Glorot-style scale."""
    rng = np.random.default_rng(seed)
    w = np.zeros(MLP_NP)
    w[0:192] = rng.standard_normal(192) * scale * np.sqrt(2.0 / (6 + 32))
    w[224:1248] = rng.standard_normal(1024) * scale * np.sqrt(2.0 / 64)
    w[1280:1312] = rng.standard_normal(32) * scale * np.sqrt(2.0 / 33)
    return w


def mlp_forward(w, x):
    L = _load()
    w, x = _c(w), _c(x)
    h1, h2 = np.empty(32), np.empty(32)
    return L.orc_mlp_forward(_p(w), _p(x), _p(h1), _p(h2))


def mlp_forward_bf16(w, x):
    L = _load()
    w, x = _c(w), _c(x)
    return L.orc_mlp_forward_bf16(_p(w), _p(x))


def mlp_grad(w, X, T, wt=None):
    """Loss sum 0.5 (y - t)^2 wt and its gradient over samples X [F, 6], T [F]."""
    L = _load()
    w = _c(w)
    g = np.zeros(MLP_NP)
    loss = 0.0
    X = _c(X)
    for f in range(len(T)):
        x = np.ascontiguousarray(X[f])
        loss += L.orc_mlp_backward(_p(w), _p(x), float(T[f]), 1.0 if wt is None else float(wt), _p(g))
    return loss, g


def mlp_sym_grad(w, X, T, wt=1.0):
    """Loss sum 0.5 (ys - t)^2 wt of the mirror-symmetric network and its gradient."""
    L = _load()
    w = _c(w)
    g = np.zeros(MLP_NP)
    loss = 0.0
    X = _c(X)
    for f in range(len(T)):
        x = np.ascontiguousarray(X[f])
        loss += L.orc_mlp_sym_backward(_p(w), _p(x), float(T[f]), float(wt), _p(g))
    return loss, g


def mlp_sym_forward(w, X):
    L = _load()
    w, X = _c(w), _c(X)
    return np.array([L.orc_mlp_sym_forward(_p(w), _p(np.ascontiguousarray(x))) for x in X])


def learned_face(w, q6, c, positive=1, bf16=0):
    L = _load()
    w, q6 = _c(w), _c(q6)
    return L.orc_learned_face(_p(w), int(bf16), _p(q6), float(c), int(positive))


def mlp_normalise(q6):
    """network inputs x [..., 6] and sigma [...] of six-cell stencils (reading
    R14, FP64: mean, standard deviation, x = (q - mean) / (sigma + 1e-12
    |mean| + 1e-300), mirror-pair sums)"""
    L = _load()
    q = _c(q6)
    shp = q.shape[:-1]
    q = q.reshape(-1, 6)
    x = np.empty_like(q)
    sig = np.empty(q.shape[0])
    for f in range(q.shape[0]):
        xf = np.empty(6)
        sig[f] = L.orc_mlp_normalise(_p(np.ascontiguousarray(q[f])), _p(xf))
        x[f] = xf
    return x.reshape(shp + (6,)), sig.reshape(shp)


def learned_candidate(w, q6, c, positive=1, bf16=0):
    """(a, accepted): the learned face value candidate plain + sigma y before
    the fallback test, and whether the fallback keeps it (reading R14)"""
    L = _load()
    w, q6 = _c(w), _c(q6)
    acc = C.c_int()
    a = L.orc_learned_candidate(_p(w), int(bf16), _p(q6), float(c), int(positive), C.byref(acc))
    return a, bool(acc.value)


def remap_column(pe, pn, q):
    """conservative piecewise-parabolic remap of layer means q from interfaces
    pe to interfaces pn (reading R16)"""
    L = _load()
    pe, pn, q = _c(pe), _c(pn), _c(q)
    out = np.empty(len(q))
    L.orc_remap_column(len(q), _p(pe), _p(pn), _p(q), _p(out))
    return out


def d2c(dom, tile, u, v, ord=2):
    """C-grid winds (uc on x-faces, vc on y-faces) of tile ``tile`` from dense
    level-0 D-grid winds of all tiles (readings R7, R18)"""
    L = _load()
    n = dom.n
    u, v = _c(u), _c(v)
    uc = np.empty((n, n + 1))
    vc = np.empty((n + 1, n))
    L.orc_d2c_dense(dom.ptr, tile, _p(u), _p(v), int(ord), _p(uc), _p(vc))
    return uc, vc
