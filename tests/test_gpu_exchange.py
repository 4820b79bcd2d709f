"""The host-built halo plan (fv3_halo_plan) is the plan the device applies:
its plane geometry equals the context's layout, and applying it on the CPU to
a field read back from the GPU reproduces fv3_halo_fill slot by slot."""
import numpy as np
import pytest

from gpu_common import seeded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_host_plan_is_the_device_plan(precision):
    import torch

    from paper_2205_04148_gb300 import exchange, fv3
    prec = fv3.FP64 if precision == "fp64" else fv3.FP32
    n, nz = 12, 3
    g = fv3.Grid(fv3.GRID_CUBED, n, nz, n_members=2, member_npx=[12, 16], precision=prec)
    for member in (0, 1):
        lay = g.layout(member)
        for kind in (fv3.PLAN_CELL, fv3.PLAN_DGRID):
            e, hl = fv3.halo_plan(fv3.GRID_CUBED, n, nz, kind=kind, member=member, precision=prec,
                                  n_members=2, member_npx=[12, 16])
            for f in ("n", "nz", "ntiles", "pitch", "rows", "ox", "plane", "offset3", "offseti"):
                assert getattr(hl, f) == getattr(lay, f), (member, kind, f)
    # member 1: fill on the device, then the host plan on a copy of the interiors
    st = seeded(True, 16, nz, 4, 0)
    gs = g.alloc_state()
    g.load(gs, st, member=1)
    lay = g.layout(1)
    P = lay.plane
    def planes(t):
        return t.view(-1)[lay.offset3:lay.offset3 + 6 * nz * P].view(6, nz, P).double().cpu().numpy()
    before = {f: planes(gs[f]).copy() for f in ("delp", "u", "v")}
    g.halo_fill(gs, fv3.HALO_WIND | fv3.HALO_DELP)
    torch.cuda.synchronize()
    after = {f: planes(gs[f]) for f in ("delp", "u", "v")}
    for kind, fields in ((fv3.PLAN_CELL, ("delp",)), (fv3.PLAN_DGRID, ("v", "u"))):
        e, hl = fv3.halo_plan(fv3.GRID_CUBED, 12, nz, kind=kind, member=1, precision=prec, n_members=2,
                              member_npx=[12, 16])
        X = exchange.TileExchange(e, [0] * 6, 0, nz, P, vector=len(fields) == 2)
        buf = torch.from_numpy(np.stack([before[f] for f in fields]))
        X.run(buf)
        dst = np.unique(np.concatenate([e["dst"]]))
        for a, f in enumerate(fields):
            got, want = buf.numpy()[a][:, :, dst], after[f][:, :, dst]
            assert np.array_equal(np.isnan(got), np.isnan(want)), f
            fin = np.isfinite(want)
            assert np.array_equal(got[fin], want[fin]), f


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("owner", [[0, 0, 0, 1, 1, 1], [0, 1, 0, 1, 0, 1], [0, 1, 2, 0, 1, 2]])
def test_device_pack_unpack_reproduces_halo_fill(precision, owner):
    """The device side of the exchange (fv3_halo_gather / fv3_halo_copy /
    fv3_halo_scatter) on one GPU: the ranks' parts of the plan, each on its
    own device buffer, with every message gathered by one rank's kernel and
    scattered by the receiver's (handed over directly, no transport), fill
    the halo slots exactly as fv3_halo_fill does"""
    import torch

    from paper_2205_04148_gb300 import exchange, fv3
    prec = fv3.FP64 if precision == "fp64" else fv3.FP32
    n, nz = 12, 3
    g = fv3.Grid(fv3.GRID_CUBED, n, nz, precision=prec)
    st = seeded(True, n, nz, 6, 0)
    gs = g.alloc_state()
    g.load(gs, st)
    lay = g.layout(0)
    P = lay.plane

    def planes(t):
        return t.view(-1)[lay.offset3:lay.offset3 + 6 * nz * P].view(6, nz, P).clone()

    before = {f: planes(gs[f]) for f in ("delp", "u", "v")}
    g.halo_fill(gs, fv3.HALO_WIND | fv3.HALO_DELP)
    after = {f: planes(gs[f]).cpu().numpy() for f in ("delp", "u", "v")}
    ranks = sorted(set(owner))
    for kind, fields in ((fv3.PLAN_CELL, ("delp",)), (fv3.PLAN_DGRID, ("v", "u"))):
        e, _ = fv3.halo_plan(fv3.GRID_CUBED, n, nz, kind=kind, precision=prec)
        X = {r: exchange.TileExchange(e, owner, r, nz, P, vector=len(fields) == 2) for r in ranks}
        bufs = {r: torch.stack([before[f][X[r].tiles] for f in fields]).contiguous() for r in ranks}
        msgs = {r: X[r].pack(bufs[r]) for r in ranks}
        for r in ranks:
            X[r].local(bufs[r])
        for src in ranks:
            for dst, m in msgs[src].items():
                assert m.is_cuda and m.dtype == bufs[dst].dtype
                X[dst].unpack(bufs[dst], src, m)
        torch.cuda.synchronize()
        dst_slots = np.unique(e["dst"])
        for r in ranks:
            got_all = bufs[r].cpu().numpy()
            for a, f in enumerate(fields):
                got, want = got_all[a][:, :, dst_slots], after[f][X[r].tiles][:, :, dst_slots]
                assert np.array_equal(np.isnan(got), np.isnan(want)), (r, f)
                fin = np.isfinite(want)
                assert np.array_equal(got[fin], want[fin]), (r, f)
