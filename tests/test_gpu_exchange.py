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
