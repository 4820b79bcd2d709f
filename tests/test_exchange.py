"""Halo exchange between ranks holding different tiles (Section V-C: the
halo exchange with the orientation transform between cube faces), on the CPU:
the host-built plan of fv3_halo_plan applied on one rank reproduces the
oracle's halo fill slot by slot; split over two gloo ranks (tiles 0-2 and 3-5,
or interleaved 0, 2, 4 and 1, 3, 5) it gives the same fields; and a rank that never joins makes the other rank's
exchange fail within its timeout instead of hanging."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

N, NZ, H = 8, 2, 3


def _plan(kind):
    from paper_2205_04148_gb300 import fv3
    return fv3.halo_plan(fv3.GRID_CUBED, N, NZ, kind=kind)


def _fields(lay, vector, seed):
    """random interiors in the library's plane layout (halo slots NaN), and
    the same values in the oracle's padded layout"""
    rng = np.random.default_rng(seed)
    A = 2 if vector else 1
    buf = np.full((A, 6, NZ, lay.plane), np.nan)
    # arrays: scalar cells; vector pair: x-faces (n + 1 columns), y-faces (n + 1 rows)
    shapes = [(N, N + 1), (N + 1, N)] if vector else [(N, N)]
    dense = []
    for a, (nj, ni) in enumerate(shapes):
        d = rng.standard_normal((6, NZ, nj, ni))
        dense.append(d)
        for j in range(nj):
            o = (j + H) * lay.pitch + lay.ox
            buf[a, :, :, o:o + ni] = d[:, :, j, :]
    return buf, dense


def _as_oracle(buf, lay, vector):
    """the library-layout planes as the oracle's padded arrays"""
    shapes = [(N + 2 * H, N + 1 + 2 * H), (N + 1 + 2 * H, N + 2 * H)] if vector else [(N + 2 * H, N + 2 * H)]
    out = []
    for a, (rows, cols) in enumerate(shapes):
        o = np.empty((6, NZ, rows, cols))
        for r in range(rows):
            s = r * lay.pitch + lay.ox - H
            o[:, :, r, :] = buf[a, :, :, s:s + cols]
        out.append(o)
    return out


def _oracle_fill(orc, dense, vector):
    d = orc.Domain(True, N, NZ)
    if not vector:
        c = np.full((6, NZ, N + 2 * H, N + 2 * H), np.nan)
        c[:, :, H:H + N, H:H + N] = dense[0]
        return [orc.fill_cells(d, c, NZ, 3).reshape(c.shape)]
    fx = np.full((6, NZ, N + 2 * H, N + 1 + 2 * H), np.nan)
    fy = np.full((6, NZ, N + 1 + 2 * H, N + 2 * H), np.nan)
    fx[:, :, H:H + N, H:H + N + 1] = dense[0]
    fy[:, :, H:H + N + 1, H:H + N] = dense[1]
    fx, fy = orc.fill_faces(d, fx, fy, NZ, 1, 1)
    return [fx.reshape(fx.shape), fy.reshape(fy.shape)]


@pytest.mark.parametrize("vector", [False, True])
def test_plan_on_one_rank_matches_oracle_fill(orc, vector):
    import torch

    from paper_2205_04148_gb300 import exchange, fv3
    entries, lay = _plan(fv3.PLAN_DGRID if vector else fv3.PLAN_CELL)
    buf, dense = _fields(lay, vector, 3)
    X = exchange.TileExchange(entries, [0] * 6, 0, NZ, lay.plane, vector=vector)
    t = torch.from_numpy(buf.copy())
    X.run(t)
    got = _as_oracle(t.numpy(), lay, vector)
    want = _oracle_fill(orc, dense, vector)
    for g, w in zip(got, want):
        # halo slots the oracle fills (finite) and the cube-corner slots (NaN)
        assert np.array_equal(np.isnan(g), np.isnan(w))
        fin = np.isfinite(w)
        assert np.array_equal(g[fin], w[fin])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, kind, vector, out, join=True, owner=(0, 0, 0, 1, 1, 1)):
    import datetime

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=datetime.timedelta(seconds=20))
    from paper_2205_04148_gb300 import exchange, fv3
    entries, lay = fv3.halo_plan(fv3.GRID_CUBED, N, NZ, kind=kind)
    X = exchange.TileExchange(entries, list(owner), rank, NZ, lay.plane, vector=vector)
    buf, _ = _fields(lay, vector, 5)
    mine = torch.from_numpy(np.ascontiguousarray(buf[:, X.tiles]))
    try:
        if join:
            X.run(mine, timeout_s=3.0)
            out.put((rank, "ok", mine.numpy()))
        else:
            out.put((rank, "absent", None))
            dist.barrier()  # stays up until the other rank has given up
    except exchange.ExchangeError as e:
        out.put((rank, "error", str(e)))
        if rank == 0:
            dist.barrier()
    dist.destroy_process_group()


def _spawn(kind, vector, joins, owner=(0, 0, 0, 1, 1, 1)):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, kind, vector, q, joins[r], owner)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = {}
        for _ in range(2):
            r, status, data = q.get(timeout=120)
            res[r] = (status, data)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
    return res


@pytest.mark.parametrize("owner", [(0, 0, 0, 1, 1, 1), (0, 1, 0, 1, 0, 1)])
@pytest.mark.parametrize("kind_name,vector", [("PLAN_CELL", False), ("PLAN_DGRID", True), ("PLAN_CGRID", True)])
def test_two_ranks_equal_one(kind_name, vector, owner):
    import torch

    from paper_2205_04148_gb300 import exchange, fv3
    kind = getattr(fv3, kind_name)
    res = _spawn(kind, vector, (True, True), owner)
    entries, lay = _plan(kind)
    buf, _ = _fields(lay, vector, 5)
    whole = torch.from_numpy(buf.copy())
    exchange.TileExchange(entries, [0] * 6, 0, NZ, lay.plane, vector=vector).run(whole)
    whole = whole.numpy()
    for r in (0, 1):
        tiles = [t for t in range(6) if owner[t] == r]
        status, data = res[r]
        assert status == "ok", data
        assert np.array_equal(np.isnan(data), np.isnan(whole[:, tiles]))
        fin = np.isfinite(whole[:, tiles])
        assert np.array_equal(data[fin], whole[:, tiles][fin])


def test_absent_rank_is_reported():
    from paper_2205_04148_gb300 import fv3
    res = _spawn(fv3.PLAN_CELL, False, (True, False))
    assert res[1][0] == "absent"
    assert res[0][0] == "error" and "rank 1" in res[0][1]
