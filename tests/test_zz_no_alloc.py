"""The allocation-free column solve, fv3_riem_solver_c_noalloc, against the
oracle's column solve and the library's own riem_solver_c, at its size limit.

The entry point serves callers that cannot allocate device memory (code that
runs under a fixed, pre-reserved budget, or a host framework that owns the
device pool): it takes inputs and outputs from the caller and keeps its
scratch in one fixed array inside the library.  Every call here goes through
the C-ABI; the first test calls it twice in a row.  This file is collected
last so that a failure here comes after every other test."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import TOL64, relerr, seeded
from paper_2205_04148_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LIMIT = 4 * 1024 * 1024      # doubles of scratch: 5 * nz * ncol may not exceed it


def lib():
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    L = fv3.load()
    L.fv3_riem_solver_c_noalloc.restype = C.c_int
    L.fv3_riem_solver_c_noalloc.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 6 + [C.POINTER(fv3.Params),
                                                                                    C.c_void_p]
    return L, fv3


def to_columns(a):
    """dense [nt][nlev][n][n] -> level-major [nlev][nt*n*n]"""
    nt, nl, n, _ = a.shape
    return np.ascontiguousarray(np.transpose(a, (1, 0, 2, 3)).reshape(nl, nt * n * n))


def columns(nz, ncol, seed):
    """seeded level-major columns near hydrostatic balance: delpc, ptc, wc, delzc"""
    rng = np.random.default_rng(seed)
    dp = 1000.0 * (1 + 0.01 * rng.standard_normal((1, nz, 1, ncol)))
    pt = rng.uniform(250.0, 300.0, (1, nz, 1, ncol))
    dz = I.hydrostatic_delz(dp, pt) * (1 + 1e-3 * rng.standard_normal((1, nz, 1, ncol)))
    w = 0.5 * rng.standard_normal((1, nz, 1, ncol))
    return [np.ascontiguousarray(a[0, :, 0, :]) for a in (dp, pt, w, dz)]


def solve(L, fv3, ins, prm):
    import torch
    nz, ncol = ins[0].shape
    dev = [torch.from_numpy(x).cuda() for x in ins]
    pef = torch.full((nz + 1, ncol), np.nan, dtype=torch.float64, device="cuda")
    gz = torch.full((nz + 1, ncol), np.nan, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.fv3_riem_solver_c_noalloc(ncol, nz, *[C.c_void_p(t.data_ptr()) for t in dev],
                                     C.c_void_p(pef.data_ptr()), C.c_void_p(gz.data_ptr()), C.byref(prm), stream)
    torch.cuda.synchronize()
    return rc, pef.cpu().numpy(), gz.cpu().numpy()


def oracle_columns(orc, ins, cols, prm):
    """the oracle's column solve (reading R9) of the chosen columns"""
    pef, gz = [], []
    for c in cols:
        p, g, _, _ = orc.riem_column(*[a[:, c] for a in ins], 0.5 * prm.dt)
        pef.append(p)
        gz.append(g)
    return np.array(pef).T, np.array(gz).T


def test_noalloc_matches_oracle_twice_in_a_row(orc):
    L, fv3 = lib()
    prm = fv3.params()
    for seed, (nz, ncol) in ((41, (8, 777)), (42, (30, 1500))):
        ins = columns(nz, ncol, seed)
        rc, pef, gz = solve(L, fv3, ins, prm)
        assert rc == 0
        want_pef, want_gz = oracle_columns(orc, ins, range(ncol), prm)
        assert relerr(pef, want_pef) <= TOL64
        assert relerr(gz, want_gz) <= TOL64


def test_noalloc_matches_context_path():
    L, fv3 = lib()
    n, nz = 12, 8
    prm = fv3.params()
    for seed in (31, 32):
        st = seeded(True, n, nz, seed)
        g = fv3.Grid(fv3.GRID_CUBED, n, nz)
        gs = g.alloc_state()
        g.load(gs, st)
        g.stage(gs, 3, prm)            # regular path up to riem_solver_c
        ins = [to_columns(g.intermediate(nm)) for nm in ("delpc", "ptc", "wc", "delzc")]
        rc, pef, gz = solve(L, fv3, ins, prm)
        assert rc == 0
        assert relerr(pef, to_columns(g.intermediate("pef"))) <= TOL64
        assert relerr(gz, to_columns(g.intermediate("gz"))) <= TOL64
        g.close()


def test_noalloc_at_its_size_limit(orc):
    # nz = 80: ncol = 10485 is the largest call (5 * 80 * 10485 = 4,194,000
    # doubles); every column is checked for its fixed ends, sampled columns
    # against the oracle
    L, fv3 = lib()
    prm = fv3.params()
    nz, ncol = 80, LIMIT // (5 * 80)
    assert 5 * nz * ncol <= LIMIT < 5 * nz * (ncol + 1)
    ins = columns(nz, ncol, 43)
    rc, pef, gz = solve(L, fv3, ins, prm)
    assert rc == 0
    assert np.isfinite(pef).all() and np.isfinite(gz).all()
    assert (pef[0] == prm.ptop).all() and (gz[nz] == 0).all()
    cols = np.random.default_rng(44).choice(ncol, 48, replace=False)
    cols = np.concatenate([[0, ncol - 1], cols])
    want_pef, want_gz = oracle_columns(orc, ins, cols, prm)
    assert relerr(pef[:, cols], want_pef) <= TOL64
    assert relerr(gz[:, cols], want_gz) <= TOL64


def test_noalloc_rejects_sizes_beyond_its_scratch_and_bad_constants():
    L, fv3 = lib()
    prm = fv3.params()
    dummy = C.c_void_p(256)   # never dereferenced: the checks come before any launch
    nz = 80
    ncol = LIMIT // (5 * nz) + 1
    assert L.fv3_riem_solver_c_noalloc(ncol, nz, *[dummy] * 6, C.byref(prm), None) == -2
    assert L.fv3_riem_solver_c_noalloc(200000, 80, *[dummy] * 6, C.byref(prm), None) == -2
    assert L.fv3_riem_solver_c_noalloc(0, 80, *[dummy] * 6, C.byref(prm), None) == -2
    for name, value in (("rdgas", 0.0), ("rdgas", -287.0), ("grav", 0.0), ("dt", 0.0), ("ptop", -1.0)):
        bad = fv3.params(**{name: value})
        assert L.fv3_riem_solver_c_noalloc(10, nz, *[dummy] * 6, C.byref(bad), None) == -1, name
