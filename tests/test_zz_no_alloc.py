"""The allocation-free column solve against the library's own riem_solver_c.

fv3_riem_solver_c_noalloc serves callers that cannot allocate device memory
(a fixed pre-reserved budget, or a host framework that owns the device pool):
it takes its inputs and outputs from the caller and keeps its scratch in a
fixed array of the library.  Here it is called through the C-ABI, twice in a
row on two different states, and each result is compared with the pef / gz
that the regular context-based substep computes from the same inputs.  This
file is collected last so that a failure here comes after every other test."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import TOL64, relerr, seeded

pytestmark = pytest.mark.gpu


def to_columns(a):
    """dense [nt][nlev][n][n] -> level-major [nlev][nt*n*n]"""
    nt, nl, n, _ = a.shape
    return np.ascontiguousarray(np.transpose(a, (1, 0, 2, 3)).reshape(nl, nt * n * n))


def test_noalloc_riem_matches_context_path():
    import torch
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    L = fv3.load()
    L.fv3_riem_solver_c_noalloc.restype = C.c_int
    L.fv3_riem_solver_c_noalloc.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 6 + [C.POINTER(fv3.Params),
                                                                                    C.c_void_p]
    n, nz = 12, 8
    prm = fv3.params()
    for seed in (31, 32):   # two calls in a row, different inputs
        st = seeded(True, n, nz, seed)
        g = fv3.Grid(fv3.GRID_CUBED, n, nz)
        gs = g.alloc_state()
        g.load(gs, st)
        g.stage(gs, 3, prm)            # regular path up to riem_solver_c
        ins = [to_columns(g.intermediate(nm)) for nm in ("delpc", "ptc", "wc", "delzc")]
        want_pef = to_columns(g.intermediate("pef"))
        want_gz = to_columns(g.intermediate("gz"))
        ncol = ins[0].shape[1]
        dev = [torch.from_numpy(x).cuda() for x in ins]
        pef = torch.full((nz + 1, ncol), np.nan, dtype=torch.float64, device="cuda")
        gz = torch.full((nz + 1, ncol), np.nan, dtype=torch.float64, device="cuda")
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = L.fv3_riem_solver_c_noalloc(ncol, nz, *[C.c_void_p(t.data_ptr()) for t in dev],
                                         C.c_void_p(pef.data_ptr()), C.c_void_p(gz.data_ptr()), C.byref(prm), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert relerr(pef.cpu().numpy(), want_pef) <= TOL64
        assert relerr(gz.cpu().numpy(), want_gz) <= TOL64
        g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    L = fv3.load()
    L.fv3_riem_solver_c_noalloc.restype = C.c_int
    prm = fv3.params()
    dummy = C.c_void_p(256)   # never dereferenced: the size check comes first
    rc = L.fv3_riem_solver_c_noalloc(200000, 80, dummy, dummy, dummy, dummy, dummy, dummy, C.byref(prm), None)
    assert rc == -2
