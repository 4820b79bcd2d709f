"""Thin ctypes binding of the C-ABI in include/fv3.h (argument marshalling only).

Every step of the substep runs in the CUDA kernels of ``_build/libfv3.so``;
PyTorch only allocates device memory and provides the stream.  The library
must have been built (``__graft_entry__.build()`` or
``python paper_2205_04148_gb300/build.py``): loading fails loudly otherwise,
there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfv3.so")

FV3_OK = 0
STATUS = {0: "FV3_OK", -1: "FV3_ERR_ARG", -2: "FV3_ERR_SHAPE", -3: "FV3_ERR_ALIGN", -4: "FV3_ERR_CUDA",
          -5: "FV3_ERR_NONFINITE", -6: "FV3_ERR_CFL", -7: "FV3_ERR_TIMEOUT", -8: "FV3_ERR_UNSUPPORTED"}
GRID_PERIODIC, GRID_CUBED = 0, 1
FP64, FP32, FP32_M64 = 0, 1, 2
KIND_CELL, KIND_XFACE, KIND_YFACE, KIND_IFACE = 0, 1, 2, 3
DENSE_DEVICE, DENSE_HOST, DENSE_HOST_ASYNC = 0, 1, 2
HALO_WIND, HALO_W, HALO_DELP, HALO_PT, HALO_DELZ, HALO_TRACERS = 1, 2, 4, 8, 16, 32

# exported symbols declared in include/fv3.h
SYMBOLS = ("fv3_init_grid", "fv3_destroy", "fv3_last_error", "fv3_field_elems", "fv3_elem_size",
           "fv3_get_layout", "fv3_import", "fv3_export", "fv3_halo_fill", "fv3_acoustic_substep",
           "fv3_run_dyn", "fv3_mass_sum", "fv3_check_status", "fv3_get_metric", "fv3_stage",
           "fv3_get_intermediate", "fv3_launch_stage", "fv3_kernel_launches", "fv3_calibrate",
           "fv3_set_tiles", "fv3_get_tiles", "fv3_autotune", "fv3_autotune_for", "fv3_riem_solver_c_noalloc",
           "fv3_mlp_forward", "fv3_mlp_work_floats", "fv3_mlp_grad", "fv3_mlp_adam", "fv3_set_persistent",
           "fv3_get_persistent", "fv3_fv_tp_2d", "fv3_math_check", "fv3_vertical_remap",
           "fv3_mlp_grad_fp32", "fv3_mlp_work_floats_fp32", "fv3_check_finite", "fv3_halo_plan",
           "fv3_face_stencils", "fv3_learned_faces", "fv3_halo_gather", "fv3_halo_scatter", "fv3_halo_copy")
PLAN_CELL, PLAN_DGRID, PLAN_CGRID = 0, 2, 3


class HaloEntry(C.Structure):
    _fields_ = [("dst", C.c_int32), ("src", C.c_int32), ("dst_tile", C.c_int32), ("src_tile", C.c_int32),
                ("sign", C.c_int32), ("flags", C.c_int32)]


class GridDesc(C.Structure):
    _fields_ = [("grid_type", C.c_int), ("npx", C.c_int), ("npz", C.c_int), ("n_members", C.c_int),
                ("member_npx", C.POINTER(C.c_int)), ("precision", C.c_int), ("dx", C.c_double),
                ("radius", C.c_double), ("omega", C.c_double)]


class State(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("w", C.c_void_p), ("delp", C.c_void_p),
                ("pt", C.c_void_p), ("delz", C.c_void_p), ("q", C.POINTER(C.c_void_p)), ("nq", C.c_int)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_split", C.c_int), ("nord", C.c_int), ("hord", C.c_int),
                ("d4_bg", C.c_double), ("a_imp", C.c_double), ("dz_min", C.c_double), ("ptop", C.c_double),
                ("grav", C.c_double), ("rdgas", C.c_double), ("cp_air", C.c_double), ("mlp", C.c_void_p),
                ("remap", C.c_int), ("nh_full", C.c_int), ("d2c_ord", C.c_int),
                ("d2_bg", C.c_double), ("dddmp", C.c_double)]


class Layout(C.Structure):
    _fields_ = [("n", C.c_int), ("nz", C.c_int), ("ntiles", C.c_int), ("pitch", C.c_int), ("rows", C.c_int),
                ("ox", C.c_int), ("plane", C.c_longlong), ("offset3", C.c_longlong),
                ("offseti", C.c_longlong)]


_lib = None


class Fv3Error(RuntimeError):
    pass


def load(path=LIB_PATH):
    """Load libfv3.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise Fv3Error("libfv3.so not built (%s): run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp, st, i, d = C.c_void_p, C.c_int, C.c_int, C.c_double
    L.fv3_init_grid.restype = st
    L.fv3_init_grid.argtypes = [C.POINTER(vp), C.POINTER(GridDesc), vp]
    L.fv3_destroy.restype = None
    L.fv3_destroy.argtypes = [vp]
    L.fv3_last_error.restype = C.c_char_p
    L.fv3_last_error.argtypes = [vp]
    L.fv3_field_elems.restype = C.c_size_t
    L.fv3_field_elems.argtypes = [vp, i]
    L.fv3_elem_size.restype = C.c_size_t
    L.fv3_elem_size.argtypes = [vp]
    L.fv3_get_layout.restype = st
    L.fv3_get_layout.argtypes = [vp, i, C.POINTER(Layout)]
    L.fv3_halo_plan.restype = st
    L.fv3_halo_plan.argtypes = [C.POINTER(GridDesc), i, i, C.POINTER(HaloEntry), C.c_size_t,
                                C.POINTER(C.c_size_t), C.POINTER(Layout)]
    for nm in ("fv3_import", "fv3_export"):
        f = getattr(L, nm)
        f.restype = st
        f.argtypes = [vp, i, vp, vp, i, i, i, vp]
    L.fv3_halo_fill.restype = st
    L.fv3_halo_fill.argtypes = [vp, C.POINTER(State), C.c_uint, vp]
    L.fv3_acoustic_substep.restype = st
    L.fv3_acoustic_substep.argtypes = [vp, C.POINTER(State), C.POINTER(Params), vp]
    L.fv3_run_dyn.restype = st
    L.fv3_run_dyn.argtypes = [vp, C.POINTER(State), C.POINTER(Params), i, vp]
    L.fv3_mass_sum.restype = st
    L.fv3_mass_sum.argtypes = [vp, C.POINTER(State), C.POINTER(d), vp]
    L.fv3_check_status.restype = st
    L.fv3_check_status.argtypes = [vp, vp]
    L.fv3_get_metric.restype = st
    L.fv3_get_metric.argtypes = [vp, C.c_char_p, i, C.POINTER(d)]
    L.fv3_stage.restype = st
    L.fv3_stage.argtypes = [vp, C.POINTER(State), C.POINTER(Params), i, vp]
    L.fv3_get_intermediate.restype = st
    L.fv3_get_intermediate.argtypes = [vp, C.c_char_p, i, C.POINTER(d), vp]
    L.fv3_launch_stage.restype = st
    L.fv3_launch_stage.argtypes = [vp, C.POINTER(State), C.POINTER(Params), i, i, vp]
    L.fv3_kernel_launches.restype = C.c_longlong
    L.fv3_kernel_launches.argtypes = [vp]
    L.fv3_calibrate.restype = st
    L.fv3_calibrate.argtypes = [vp, i, vp, C.POINTER(d)]
    L.fv3_set_tiles.restype = st
    L.fv3_set_tiles.argtypes = [vp, i, i, i]
    L.fv3_set_persistent.restype = st
    L.fv3_set_persistent.argtypes = [vp, i]
    L.fv3_get_persistent.restype = st
    L.fv3_get_persistent.argtypes = [vp, C.POINTER(i)]
    L.fv3_vertical_remap.restype = st
    L.fv3_vertical_remap.argtypes = [vp, C.POINTER(State), C.POINTER(Params), vp]
    L.fv3_check_finite.restype = st
    L.fv3_check_finite.argtypes = [vp, C.POINTER(State), vp]
    L.fv3_math_check.restype = st
    L.fv3_math_check.argtypes = [i, vp, vp, vp, i, vp]
    L.fv3_fv_tp_2d.restype = st
    L.fv3_fv_tp_2d.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, d, vp, vp, vp]
    L.fv3_get_tiles.restype = st
    L.fv3_get_tiles.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i)]
    L.fv3_autotune.restype = st
    L.fv3_autotune.argtypes = [vp, C.POINTER(State), C.POINTER(Params), vp, C.POINTER(d)]
    L.fv3_autotune_for.restype = st
    L.fv3_autotune_for.argtypes = [vp, C.POINTER(State), C.POINTER(Params), vp, C.POINTER(d), C.POINTER(i), i]
    L.fv3_mlp_forward.restype = st
    L.fv3_mlp_forward.argtypes = [vp, vp, i, i, vp, vp]
    L.fv3_halo_gather.restype = st
    L.fv3_halo_gather.argtypes = [vp, i, vp, vp, C.c_int64, vp, vp]
    L.fv3_halo_scatter.restype = st
    L.fv3_halo_scatter.argtypes = [vp, i, vp, vp, C.c_int64, vp]
    L.fv3_halo_copy.restype = st
    L.fv3_halo_copy.argtypes = [vp, i, vp, vp, vp, C.c_int64, vp]
    L.fv3_face_stencils.restype = st
    L.fv3_face_stencils.argtypes = [vp, vp, i, vp, vp, vp, vp, vp]
    L.fv3_learned_faces.restype = st
    L.fv3_learned_faces.argtypes = [vp, vp, vp, i, vp, vp]
    L.fv3_mlp_work_floats.restype = C.c_size_t
    L.fv3_mlp_work_floats.argtypes = [i]
    L.fv3_mlp_grad.restype = st
    L.fv3_mlp_grad.argtypes = [vp, vp, vp, i, C.c_float, vp, vp, vp, vp]
    L.fv3_mlp_work_floats_fp32.restype = C.c_size_t
    L.fv3_mlp_work_floats_fp32.argtypes = [i]
    L.fv3_mlp_grad_fp32.restype = st
    L.fv3_mlp_grad_fp32.argtypes = [vp, vp, vp, i, C.c_float, vp, vp, vp, vp]
    L.fv3_mlp_adam.restype = st
    L.fv3_mlp_adam.argtypes = [vp, vp, vp, vp, i, C.c_float, vp]
    L.fv3_riem_solver_c_noalloc.restype = st
    L.fv3_riem_solver_c_noalloc.argtypes = [i, i, vp, vp, vp, vp, vp, vp, C.POINTER(Params), vp]
    _lib = L
    return L


def params(mlp=None, **kw):
    """Substep parameters; ``mlp`` (a device float tensor of 1313 network
    parameters) with hord=1 selects the learned face values."""
    from .inputs import default_params
    p = default_params()
    p.update(kw)
    prm = Params(p["dt"], p["n_split"], p["nord"], p["hord"], p["d4_bg"], p["a_imp"], p["dz_min"],
                 p["ptop"], p["grav"], p["rdgas"], p["cp_air"], None, int(p.get("remap", 0)),
                 int(p.get("nh_full", 0)), int(p.get("d2c_ord", 2)), float(p.get("d2_bg", 0.0)),
                 float(p.get("dddmp", 0.0)))
    if mlp is not None:
        prm.mlp = C.c_void_p(mlp.data_ptr())
        prm._keep = mlp
    return prm


def halo_plan(grid_type, npx, npz, kind=PLAN_CELL, member=0, precision=FP64, n_members=1, member_npx=None,
              dx=1.0e5, radius=6.3712e6, omega=7.292e-5):
    """The halo plan of one member (fv3_halo_plan; host only, no device):
    returns (entries, layout) with entries a dict of int64 numpy arrays dst,
    src, dst_tile, src_tile, sign, flags."""
    L = load()
    mn = (C.c_int * len(member_npx))(*member_npx) if member_npx is not None else None
    desc = GridDesc(grid_type, npx, npz, n_members, C.cast(mn, C.POINTER(C.c_int)) if mn else None, precision,
                    dx, radius, omega)
    total = C.c_size_t()
    lay = Layout()
    n = member_npx[member] if member_npx is not None else npx
    # every halo slot of both arrays of a pair, on six tiles, bounds the plan:
    # one call builds it (the metric behind it is built once)
    cap = 2 * 6 * ((n + 7) * (n + 7) - n * n)
    buf = (HaloEntry * cap)()
    rc = L.fv3_halo_plan(C.byref(desc), member, kind, buf, cap, C.byref(total), C.byref(lay))
    if rc != FV3_OK:
        raise Fv3Error("%s: fv3_halo_plan" % STATUS.get(rc, rc))
    if total.value > cap:   # not expected; ask again with the exact size
        buf = (HaloEntry * total.value)()
        rc = L.fv3_halo_plan(C.byref(desc), member, kind, buf, total.value, C.byref(total), None)
        if rc != FV3_OK:
            raise Fv3Error("%s: fv3_halo_plan" % STATUS.get(rc, rc))
    a = np.frombuffer(buf, dtype=np.int32).reshape(-1, 6)[: total.value].astype(np.int64)
    names = ("dst", "src", "dst_tile", "src_tile", "sign", "flags")
    return {nm: a[:, k].copy() for k, nm in enumerate(names)}, lay


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


class Grid:
    """A context (fv3_init_grid) plus helpers that allocate state tensors in the
    library layout and move dense numpy arrays in and out of them."""

    FIELD_KIND = {"u": KIND_YFACE, "v": KIND_XFACE, "w": KIND_CELL, "delp": KIND_CELL, "pt": KIND_CELL,
                  "delz": KIND_CELL}

    def __init__(self, grid_type, npx, npz, n_members=1, member_npx=None, precision=FP64, dx=1.0e5,
                 radius=6.3712e6, omega=7.292e-5):
        self.L = load()
        self.ptr = C.c_void_p()
        self._mnpx = None
        if member_npx is not None:
            self._mnpx = (C.c_int * len(member_npx))(*member_npx)
        desc = GridDesc(grid_type, npx, npz, n_members,
                        C.cast(self._mnpx, C.POINTER(C.c_int)) if self._mnpx else None,
                        precision, dx, radius, omega)
        self.check(self.L.fv3_init_grid(C.byref(self.ptr), C.byref(desc), None))
        self.precision = precision
        self.n_members = n_members
        self.npz = npz
        self.nt = 6 if grid_type == GRID_CUBED else 1
        self.member_npx = list(member_npx) if member_npx is not None else [npx] * n_members

    def close(self):
        if self.ptr:
            self.L.fv3_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != FV3_OK:
            msg = self.L.fv3_last_error(self.ptr if getattr(self, "ptr", None) else None)
            raise Fv3Error("%s: %s" % (STATUS.get(rc, rc), msg.decode() if msg else ""))

    # ---- layout ----
    def elems(self, kind):
        return int(self.L.fv3_field_elems(self.ptr, kind))

    def layout(self, member=0):
        lay = Layout()
        self.check(self.L.fv3_get_layout(self.ptr, member, C.byref(lay)))
        return lay

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32

    def alloc(self, kind=KIND_CELL):
        import torch
        return torch.zeros(self.elems(kind), dtype=self.torch_dtype, device="cuda")

    def alloc_state(self, nq=0):
        st = {f: self.alloc(k) for f, k in self.FIELD_KIND.items()}
        st["q"] = [self.alloc(KIND_CELL) for _ in range(nq)]
        return st

    def cstate(self, st):
        q = st.get("q", [])
        arr = (C.c_void_p * max(1, len(q)))(*[t.data_ptr() for t in q]) if q else None
        s = State(st["u"].data_ptr(), st["v"].data_ptr(), st["w"].data_ptr(), st["delp"].data_ptr(),
                  st["pt"].data_ptr(), st["delz"].data_ptr(),
                  C.cast(arr, C.POINTER(C.c_void_p)) if arr is not None else None, len(q))
        s._keep = arr
        return s

    # ---- dense <-> library layout ----
    def _dense_shape(self, kind, member):
        n, nt, nz = self.member_npx[member], self.nt, self.npz
        if kind == KIND_XFACE:
            return (nt, nz, n, n + 1)
        if kind == KIND_YFACE:
            return (nt, nz, n + 1, n)
        if kind == KIND_IFACE:
            return (nt, nz + 1, n, n)
        return (nt, nz, n, n)

    def put(self, field, kind, dense, member=0, stream=None):
        a = np.ascontiguousarray(dense, dtype=np.float64).reshape(self._dense_shape(kind, member))
        self.check(self.L.fv3_import(self.ptr, kind, C.c_void_p(field.data_ptr()),
                                     a.ctypes.data_as(C.c_void_p), 1, 1, member, _stream(stream)))
        import torch
        torch.cuda.current_stream().synchronize()

    def get(self, field, kind, member=0, stream=None):
        a = np.empty(self._dense_shape(kind, member))
        self.check(self.L.fv3_export(self.ptr, kind, C.c_void_p(field.data_ptr()),
                                     a.ctypes.data_as(C.c_void_p), 1, 1, member, _stream(stream)))
        return a

    def host_buffer(self, kind, member=0):
        """a page-locked host tensor of the dense shape of `kind`, library dtype"""
        import torch
        return torch.empty(self._dense_shape(kind, member), dtype=self.torch_dtype, pin_memory=True)

    def _host_ok(self, host, kind, member):
        if not (host.is_pinned() and host.is_contiguous() and host.dtype == self.torch_dtype
                and tuple(host.shape) == self._dense_shape(kind, member)):
            raise ValueError("need a contiguous page-locked %s tensor of shape %s"
                             % (self.torch_dtype, self._dense_shape(kind, member)))

    def put_async(self, field, kind, host, member=0, stream=None):
        """enqueue the import of a page-locked dense host tensor"""
        self._host_ok(host, kind, member)
        self.check(self.L.fv3_import(self.ptr, kind, C.c_void_p(field.data_ptr()), C.c_void_p(host.data_ptr()),
                                     DENSE_HOST_ASYNC, int(self.precision == FP64), member, _stream(stream)))

    def get_async(self, field, kind, host, member=0, stream=None):
        """enqueue the export of a field into a page-locked dense host tensor"""
        self._host_ok(host, kind, member)
        self.check(self.L.fv3_export(self.ptr, kind, C.c_void_p(field.data_ptr()), C.c_void_p(host.data_ptr()),
                                     DENSE_HOST_ASYNC, int(self.precision == FP64), member, _stream(stream)))

    def load(self, st, dense, member=0):
        for f, k in self.FIELD_KIND.items():
            self.put(st[f], k, dense[f], member)
        for m, q in enumerate(dense.get("q", [])[: len(st.get("q", []))]):
            self.put(st["q"][m], KIND_CELL, q, member)

    def read(self, st, name, member=0):
        if name.startswith("q") and name[1:].isdigit():
            return self.get(st["q"][int(name[1:])], KIND_CELL, member)
        return self.get(st[name], self.FIELD_KIND[name], member)

    # ---- the substep ----
    def halo_fill(self, st, mask=63, stream=None):
        s = self.cstate(st)
        self.check(self.L.fv3_halo_fill(self.ptr, C.byref(s), mask, _stream(stream)))

    def substep(self, st, prm=None, stream=None):
        s = self.cstate(st)
        prm = prm or params()
        self.check(self.L.fv3_acoustic_substep(self.ptr, C.byref(s), C.byref(prm), _stream(stream)))

    def run_dyn(self, st, prm=None, n_steps=1, stream=None):
        s = self.cstate(st)
        prm = prm or params()
        self.check(self.L.fv3_run_dyn(self.ptr, C.byref(s), C.byref(prm), n_steps, _stream(stream)))

    def remap(self, st, prm=None, stream=None):
        """vertical remapping of every column to the reference layers"""
        s = self.cstate(st)
        prm = prm or params()
        self.check(self.L.fv3_vertical_remap(self.ptr, C.byref(s), C.byref(prm), _stream(stream)))

    def stage(self, st, stop_after, prm=None, stream=None):
        s = self.cstate(st)
        prm = prm or params()
        self.check(self.L.fv3_stage(self.ptr, C.byref(s), C.byref(prm), stop_after, _stream(stream)))

    def intermediate(self, name, member=0, stream=None):
        n, nt, nz = self.member_npx[member], self.nt, self.npz
        shp = {"uc": (nt, nz, n, n + 1), "fx1": (nt, nz, n, n + 1), "mfx": (nt, nz, n, n + 1),
               "crx": (nt, nz, n, n + 1), "xfx": (nt, nz, n, n + 1),
               "vc": (nt, nz, n + 1, n), "fy1": (nt, nz, n + 1, n), "mfy": (nt, nz, n + 1, n),
               "cry": (nt, nz, n + 1, n), "yfx": (nt, nz, n + 1, n),
               "pef": (nt, nz + 1, n, n), "gz": (nt, nz + 1, n, n)}.get(name, (nt, nz, n, n))
        a = np.empty(shp)
        self.check(self.L.fv3_get_intermediate(self.ptr, name.encode(), member,
                                               a.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
        return a

    def metric(self, name, member=0):
        n, nt = self.member_npx[member], self.nt
        if name in ("area", "rarea", "fA"):
            shp = (nt, n, n)
        elif name in ("dx", "rdx", "dyc", "rdyc", "cosy", "siny"):
            shp = (nt, n + 1, n)
        elif name in ("dy", "rdy", "dxc", "rdxc", "cosx", "sinx"):
            shp = (nt, n, n + 1)
        else:
            shp = (nt, n + 1, n + 1)
        a = np.empty(shp)
        self.check(self.L.fv3_get_metric(self.ptr, name.encode(), member, a.ctypes.data_as(C.POINTER(C.c_double))))
        return a

    def mass(self, st, stream=None):
        s = self.cstate(st)
        out = (C.c_double * self.n_members)()
        self.check(self.L.fv3_mass_sum(self.ptr, C.byref(s), out, _stream(stream)))
        return np.array(out[:])

    def set_tiles(self, bx, by, kchunk):
        self.check(self.L.fv3_set_tiles(self.ptr, bx, by, kchunk))

    def set_persistent(self, on=True):
        self.check(self.L.fv3_set_persistent(self.ptr, int(on)))

    def persistent(self):
        on = C.c_int()
        self.check(self.L.fv3_get_persistent(self.ptr, C.byref(on)))
        return bool(on.value)

    def tiles(self):
        bx, by, kc = C.c_int(), C.c_int(), C.c_int()
        self.check(self.L.fv3_get_tiles(self.ptr, C.byref(bx), C.byref(by), C.byref(kc)))
        return bx.value, by.value, kc.value

    def autotune(self, st, prm=None, stream=None, sizes=None):
        """fv3_autotune; with ``sizes`` (tile sizes the result will be
        transferred to) fv3_autotune_for"""
        s = self.cstate(st)
        prm = prm or params()
        best = C.c_double()
        if sizes:
            arr = (C.c_int * len(sizes))(*sizes)
            self.check(self.L.fv3_autotune_for(self.ptr, C.byref(s), C.byref(prm), _stream(stream), C.byref(best),
                                               arr, len(sizes)))
        else:
            self.check(self.L.fv3_autotune(self.ptr, C.byref(s), C.byref(prm), _stream(stream), C.byref(best)))
        return self.tiles(), best.value

    def fv_tp_2d(self, q, crx, cry, xfx, yfx, mfx=None, mfy=None, damp=0.0, fx=None, fy=None, stream=None):
        """fluxes (fx, fy) of q (library-layout tensors of this context);
        fills the halo rings of the inputs"""
        fx = self.alloc(KIND_XFACE) if fx is None else fx
        fy = self.alloc(KIND_YFACE) if fy is None else fy
        ptr = lambda t: None if t is None else t.data_ptr()
        self.check(self.L.fv3_fv_tp_2d(self.ptr, ptr(q), ptr(crx), ptr(cry), ptr(xfx), ptr(yfx), ptr(mfx), ptr(mfy),
                                       float(damp), ptr(fx), ptr(fy), _stream(stream)))
        return fx, fy

    def check_finite(self, st, stream=None):
        """0, or FV3_ERR_NONFINITE if a state field holds NaN or Inf"""
        s = self.cstate(st)
        return self.L.fv3_check_finite(self.ptr, C.byref(s), _stream(stream))

    def check_status(self, stream=None):
        return self.L.fv3_check_status(self.ptr, _stream(stream))


# ---------------------------------------------------------------------------
# learned face values: batch inference and training through the C-ABI
# ---------------------------------------------------------------------------
MLP_NP = 1313


def _chk(rc, what):
    if rc != FV3_OK:
        raise Fv3Error("%s: %s" % (what, STATUS.get(rc, rc)))


def mlp_forward(w, x, symmetric=True, stream=None):
    """w: cuda float32[1313]; x: cuda float32[n, 6] -> cuda float32[n]"""
    import torch
    L = load()
    n = x.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    _chk(L.fv3_mlp_forward(C.c_void_p(w.data_ptr()), C.c_void_p(x.data_ptr()), n, int(symmetric),
                           C.c_void_p(y.data_ptr()), _stream(stream)), "fv3_mlp_forward")
    return y


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def face_stencils(q6, cr=None, plain=True, edge=False, inputs=False, stream=None):
    """Face arithmetic of the FP64 transport on single stencils (fv3_face_stencils).
    q6: cuda float64[n, 6]; cr: cuda float64[n] (needed for ``plain``).
    Returns a dict with the requested ``plain``, ``edge`` (float64[n]) and
    ``x`` (float32[n, 6]), ``sig`` (float32[n])."""
    import torch
    L = load()
    q6 = q6.contiguous()
    n = q6.shape[0]
    out = {}
    dev = q6.device
    if plain:
        out["plain"] = torch.empty(n, dtype=torch.float64, device=dev)
    if edge:
        out["edge"] = torch.empty(n, dtype=torch.float64, device=dev)
    if inputs:
        out["x"] = torch.empty((n, 6), dtype=torch.float32, device=dev)
        out["sig"] = torch.empty(n, dtype=torch.float32, device=dev)
    _chk(L.fv3_face_stencils(_ptr(q6), _ptr(cr.contiguous()) if cr is not None else None, n,
                             _ptr(out.get("plain")), _ptr(out.get("edge")), _ptr(out.get("x")),
                             _ptr(out.get("sig")), _stream(stream)), "fv3_face_stencils")
    return out


def halo_gather(field, src, sign=None, stream=None):
    """message = sign * field.view(-1)[src] on the device (fv3_halo_gather);
    src: cuda int64, sign: cuda int8 or None"""
    import torch
    L = load()
    out = torch.empty(src.numel(), dtype=field.dtype, device=field.device)
    _chk(L.fv3_halo_gather(_ptr(field), field.element_size(), _ptr(src), _ptr(sign), src.numel(), _ptr(out),
                           _stream(stream)), "fv3_halo_gather")
    return out


def halo_scatter(field, dst, values=None, stream=None):
    """field.view(-1)[dst] = values (NaN when values is None) on the device"""
    L = load()
    _chk(L.fv3_halo_scatter(_ptr(field), field.element_size(), _ptr(dst), _ptr(values), dst.numel(),
                            _stream(stream)), "fv3_halo_scatter")


def halo_copy(field, src, dst, sign=None, stream=None):
    """field.view(-1)[dst] = sign * field.view(-1)[src] on the device (dst and
    src disjoint)"""
    L = load()
    _chk(L.fv3_halo_copy(_ptr(field), field.element_size(), _ptr(src), _ptr(dst), _ptr(sign), src.numel(),
                         _stream(stream)), "fv3_halo_copy")


def learned_faces(w, q6, cr, stream=None):
    """learned face values of stencils q6 [n, 6] (cuda float64) at Courant
    numbers cr [n] with network w (cuda float32[1313]) -> cuda float64[n]"""
    import torch
    L = load()
    q6, cr = q6.contiguous(), cr.contiguous()
    v = torch.empty(q6.shape[0], dtype=torch.float64, device=q6.device)
    _chk(L.fv3_learned_faces(_ptr(w), _ptr(q6), _ptr(cr), q6.shape[0], _ptr(v), _stream(stream)),
         "fv3_learned_faces")
    return v


class MlpTrainer:
    """Adam on the face-value network with the C-ABI gradient kernel."""

    def __init__(self, w0, lr=1e-3):
        import torch
        self.w = torch.as_tensor(w0, dtype=torch.float32, device="cuda").contiguous().clone()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.g = torch.zeros_like(self.w)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.lr = lr
        self.step = 0
        self.work = None
        self.L = load()

    def grad(self, x, t, weight=None):
        import torch
        n = x.shape[0]
        need = int(self.L.fv3_mlp_work_floats(n))
        if self.work is None or self.work.numel() < need:
            self.work = torch.empty(need, dtype=torch.float32, device="cuda")
        wt = 1.0 / n if weight is None else weight
        _chk(self.L.fv3_mlp_grad(C.c_void_p(self.w.data_ptr()), C.c_void_p(x.data_ptr()),
                                 C.c_void_p(t.data_ptr()), n, wt, C.c_void_p(self.work.data_ptr()),
                                 C.c_void_p(self.g.data_ptr()), C.c_void_p(self.loss.data_ptr()), _stream(None)),
             "fv3_mlp_grad")
        return self.g, self.loss

    def grad_fp32(self, x, t, weight=None):
        """the same gradient in float arithmetic (the check path, slow)"""
        import torch
        n = x.shape[0]
        work = torch.empty(int(self.L.fv3_mlp_work_floats_fp32(n)), dtype=torch.float32, device="cuda")
        g = torch.empty_like(self.g)
        loss = torch.empty_like(self.loss)
        wt = 1.0 / n if weight is None else weight
        _chk(self.L.fv3_mlp_grad_fp32(C.c_void_p(self.w.data_ptr()), C.c_void_p(x.data_ptr()),
                                      C.c_void_p(t.data_ptr()), n, wt, C.c_void_p(work.data_ptr()),
                                      C.c_void_p(g.data_ptr()), C.c_void_p(loss.data_ptr()), _stream(None)),
             "fv3_mlp_grad_fp32")
        return g, loss

    def update(self, x, t):
        self.grad(x, t)
        self.step += 1
        _chk(self.L.fv3_mlp_adam(C.c_void_p(self.w.data_ptr()), C.c_void_p(self.m.data_ptr()),
                                 C.c_void_p(self.v.data_ptr()), C.c_void_p(self.g.data_ptr()), self.step,
                                 self.lr, _stream(None)), "fv3_mlp_adam")
        return self.loss
