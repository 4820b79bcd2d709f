"""Asynchronous host import/export (a 3-D copy-engine transfer between a
page-locked dense host array and the field's interior; with a converted
element type a staging slot and the pack kernel) on the caller's stream, and
the per-state graph cache of run_dyn: bitwise the same as the synchronous
copies and as one state advanced alone."""
import ctypes as C

import numpy as np
import pytest

from gpu_common import seeded

pytestmark = pytest.mark.gpu

NAMES = ("u", "v", "w", "delp", "pt", "delz")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("cubed", [False, True])
def test_async_copies_match_staged(cubed, precision):
    import torch
    from paper_2205_04148_gb300 import fv3
    prec = fv3.FP64 if precision == "fp64" else fv3.FP32
    n, nz = 20, 5
    st = seeded(cubed, n, nz, 3, 1)
    g = fv3.Grid(fv3.GRID_CUBED if cubed else fv3.GRID_PERIODIC, n, nz, precision=prec)
    gs = g.alloc_state(1)
    ga = g.alloc_state(1)
    g.load(gs, st)
    s, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    hin, hout = {}, {}
    for nm in NAMES:  # more copies in flight than staging slots
        k = g.FIELD_KIND[nm]
        hin[nm] = g.host_buffer(k)
        hin[nm].numpy()[...] = st[nm]
        g.put_async(ga[nm], k, hin[nm], stream=s.cuda_stream)
    for nm in NAMES:  # on a second stream: the slots order the two
        k = g.FIELD_KIND[nm]
        hout[nm] = g.host_buffer(k)
        g.get_async(gs[nm], k, hout[nm], stream=s2.cuda_stream)
    s.synchronize()
    s2.synchronize()
    for nm in NAMES:
        k = g.FIELD_KIND[nm]
        # interiors equal those of the synchronous import (halos untouched)
        assert np.array_equal(g.get(ga[nm], k), g.get(gs[nm], k)), nm
        assert np.array_equal(hout[nm].numpy().astype(np.float64), g.get(gs[nm], k)), nm
    # interface fields (nz + 1 levels)
    f = g.alloc(fv3.KIND_IFACE)
    h = g.host_buffer(fv3.KIND_IFACE)
    h.copy_(torch.arange(h.numel(), dtype=h.dtype).reshape(h.shape))
    g.put_async(f, fv3.KIND_IFACE, h, stream=s.cuda_stream)
    s.synchronize()
    assert np.array_equal(g.get(f, fv3.KIND_IFACE), h.numpy().astype(np.float64))


def test_async_copy_argument_errors():
    import torch
    from paper_2205_04148_gb300 import fv3
    g = fv3.Grid(fv3.GRID_PERIODIC, 16, 3)
    f = g.alloc(fv3.KIND_CELL)
    h32 = torch.zeros(g._dense_shape(fv3.KIND_CELL, 0), dtype=torch.float32, pin_memory=True)
    s = torch.cuda.current_stream().cuda_stream
    rc = g.L.fv3_export(g.ptr, fv3.KIND_CELL, C.c_void_p(f.data_ptr()), C.c_void_p(h32.data_ptr()),
                        3, 1, 0, C.c_void_p(s))
    assert fv3.STATUS[rc] == "FV3_ERR_ARG"
    with pytest.raises(ValueError):
        g.put_async(f, fv3.KIND_CELL, h32)


def test_two_states_alternating_equal_one_state_alone():
    import torch
    from paper_2205_04148_gb300 import fv3
    n, nz, nq = 24, 4, 2
    sa, sb = seeded(True, n, nz, 11, nq), seeded(True, n, nz, 12, nq)
    prm = fv3.params(n_split=2)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    A, B = g.alloc_state(nq), g.alloc_state(nq)
    g.load(A, sa)
    g.load(B, sb)
    for _ in range(2):  # A, B, A, B: each replays its own captured step
        g.run_dyn(A, prm, 1)
        g.run_dyn(B, prm, 1)
    torch.cuda.synchronize()
    for seed, X in ((11, A), (12, B)):
        h = fv3.Grid(fv3.GRID_CUBED, n, nz)
        Y = h.alloc_state(nq)
        h.load(Y, seeded(True, n, nz, seed, nq))
        h.run_dyn(Y, prm, 2)
        torch.cuda.synchronize()
        for nm in NAMES + ("q0", "q1"):
            assert np.array_equal(g.read(X, nm), h.read(Y, nm)), (seed, nm)


def test_async_converting_copies_match_staged():
    """double host data into an FP32 context (staging slots + pack kernel),
    more copies in flight than slots"""
    import torch
    from paper_2205_04148_gb300 import fv3
    n, nz = 20, 5
    st = seeded(True, n, nz, 5, 0)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz, precision=fv3.FP32)
    gs, ga = g.alloc_state(0), g.alloc_state(0)
    g.load(gs, st)
    s = torch.cuda.Stream()
    hin, hout = {}, {}
    for nm in NAMES:
        k = g.FIELD_KIND[nm]
        hin[nm] = torch.from_numpy(np.ascontiguousarray(st[nm], dtype=np.float64)).pin_memory()
        g.check(g.L.fv3_import(g.ptr, k, C.c_void_p(ga[nm].data_ptr()), C.c_void_p(hin[nm].data_ptr()),
                               fv3.DENSE_HOST_ASYNC, 1, 0, C.c_void_p(s.cuda_stream)))
    for nm in NAMES:
        k = g.FIELD_KIND[nm]
        hout[nm] = torch.empty(hin[nm].shape, dtype=torch.float64, pin_memory=True)
        g.check(g.L.fv3_export(g.ptr, k, C.c_void_p(gs[nm].data_ptr()), C.c_void_p(hout[nm].data_ptr()),
                               fv3.DENSE_HOST_ASYNC, 1, 0, C.c_void_p(s.cuda_stream)))
    s.synchronize()
    for nm in NAMES:
        k = g.FIELD_KIND[nm]
        assert np.array_equal(g.get(ga[nm], k), g.get(gs[nm], k)), nm
        assert np.array_equal(hout[nm].numpy(), g.get(gs[nm], k)), nm


def test_graph_cache_eviction_keeps_results():
    """five states in turn (more than the four cached graphs): every step is
    re-captured or replayed and each state ends where a lone run ends"""
    import torch
    from paper_2205_04148_gb300 import fv3
    n, nz = 16, 3
    prm = fv3.params(n_split=1)
    g = fv3.Grid(fv3.GRID_CUBED, n, nz)
    states = []
    for k in range(5):
        X = g.alloc_state(1)
        g.load(X, seeded(True, n, nz, 40 + k, 1))
        states.append(X)
    for _ in range(2):
        for X in states:
            g.run_dyn(X, prm, 1)
    torch.cuda.synchronize()
    h = fv3.Grid(fv3.GRID_CUBED, n, nz)
    for k, X in enumerate(states):
        Y = h.alloc_state(1)
        h.load(Y, seeded(True, n, nz, 40 + k, 1))
        h.run_dyn(Y, prm, 2)
        torch.cuda.synchronize()
        for nm in NAMES + ("q0",):
            assert np.array_equal(g.read(X, nm), h.read(Y, nm)), (k, nm)
