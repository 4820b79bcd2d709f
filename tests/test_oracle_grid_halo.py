"""Pins of the oracle's cubed-sphere grid (Section II: gnomonic cubed sphere;
reading R1) and halo fill (Section V-C: halo exchange with the orientation
transform between cube faces; readings R2, R3).

Halo positions are checked against a brute-force search of the grid geometry
(matching 3-D corner points between tiles), not against the oracle's own index
map."""
import math

import numpy as np
import pytest

from paper_2205_04148_gb300 import inputs as I

N = 8
H = 3


@pytest.fixture(scope="module")
def cube(orc):
    return orc.Domain(True, N, 1)


def test_total_area(orc):
    for n in (6, 12, 25):
        d = orc.Domain(True, n, 1)
        tot = d.interior("area").sum()
        assert abs(tot / (4 * math.pi * I.RADIUS ** 2) - 1) < 1e-13


def test_area_dihedral_symmetry(cube):
    A = cube.interior("area")
    for t in range(6):
        a = A[t]
        for b in (a[::-1, :], a[:, ::-1], a.T, a[::-1, ::-1], a.T[::-1, :]):
            assert np.abs(b - a).max() <= 1e-12 * a.max()
    assert np.abs(A - A[0]).max() <= 1e-12 * A.max()   # all tiles alike


def test_grid_angle_on_centre_lines(cube):
    cx = cube.interior("cosx")   # [t][n][n+1]
    cy = cube.interior("cosy")   # [t][n+1][n]
    assert np.abs(cx[:, :, N // 2]).max() < 1e-15
    assert np.abs(cy[:, N // 2, :]).max() < 1e-15
    sx = cube.interior("sinx")
    assert np.all(np.abs(cx ** 2 + sx ** 2 - 1) < 1e-15)
    # the coordinate lines are not orthogonal away from the centre lines
    assert np.abs(cx).max() > 0.3


def test_edge_lengths_close_perimeter(cube):
    # a tile edge is the great-circle arc between two adjacent cube corners
    dx = cube.interior("dx")
    edge_angle = math.acos(1.0 / 3.0)   # angle between cube corners (1,1,1), (1,1,-1)
    for t in range(6):
        assert abs(dx[t, 0, :].sum() / I.RADIUS - edge_angle) < 1e-12


def test_neighbour_table_symmetric(cube):
    nb = cube.neighbours()
    for t in range(6):
        for e in range(4):
            t2, e2, rev = nb[t, e]
            assert t2 != t and t2 >= 0
            assert tuple(nb[t2, e2]) == (t, e, rev)


# --------------------------------------------------------- brute force ----
def all_cells():
    cells = {}
    for t in range(6):
        P = I.corner_points(t, N)
        for j in range(N):
            for i in range(N):
                cells[(t, i, j)] = [P[j, i], P[j, i + 1], P[j + 1, i + 1], P[j + 1, i]]
    return cells


def shared(c1, c2, tol=1e-10):
    out = []
    for p in c1:
        for q in c2:
            if np.linalg.norm(p - q) < tol:
                out.append(p)
    return out


EDGES = ("W", "E", "S", "N")


def edge_cell(e, p):
    """inner cell along edge e at position p and the edge's two corners (index space)"""
    if e == "W":
        return (0, p), (0, p), (0, p + 1)
    if e == "E":
        return (N - 1, p), (N, p), (N, p + 1)
    if e == "S":
        return (p, 0), (p, 0), (p + 1, 0)
    return (p, N - 1), (p, N), (p + 1, N)


def strip_chain(cells, t, e, p):
    """Brute force: halo cells at depth 1..4 beyond edge e of tile t at position p."""
    P = I.corner_points(t, N)
    _, c0, c1 = edge_cell(e, p)
    edge = [P[c0[1], c0[0]], P[c1[1], c1[0]]]
    cur = [key for key, cs in cells.items() if key[0] != t and len(shared(cs, edge)) == 2][0]
    t2, i2, j2 = cur
    Q = I.corner_points(t2, N)
    sides = {"W": (Q[j2, i2], Q[j2 + 1, i2]), "E": (Q[j2, i2 + 1], Q[j2 + 1, i2 + 1]),
             "S": (Q[j2, i2], Q[j2, i2 + 1]), "N": (Q[j2 + 1, i2], Q[j2 + 1, i2 + 1])}
    which = [k for k, (a, b) in sides.items() if len(shared([a, b], edge)) == 2][0]
    step = {"W": (1, 0), "E": (-1, 0), "S": (0, 1), "N": (0, -1)}[which]
    return [(t2, i2 + dd * step[0], j2 + dd * step[1]) for dd in range(4)]


def pad_cells(dense):
    out = np.full((dense.shape[0], N + 2 * H, N + 2 * H), np.nan)
    out[:, H:H + N, H:H + N] = dense
    return out


def strip_cell_index(e, p, depth):
    if e == "W":
        return H + p, H - depth
    if e == "E":
        return H + p, H + N - 1 + depth
    if e == "S":
        return H - depth, H + p
    return H + N - 1 + depth, H + p


def test_scalar_halo_matches_geometry(orc, cube):
    cells = all_cells()
    rng = np.random.default_rng(0)
    k = rng.standard_normal(3)
    f = lambda p: np.sin(p @ k) + 0.3 * p[..., 2]
    cen = np.stack([I.centre_points(t, N) for t in range(6)])
    q = pad_cells(f(cen))
    qf = orc.fill_cells(cube, q, 1, 3).reshape(q.shape)
    for t in range(6):
        for e in EDGES:
            for p in range(N):
                chain = strip_chain(cells, t, e, p)
                for depth in range(1, 4):
                    t2, i2, j2 = chain[depth - 1]
                    r, c = strip_cell_index(e, p, depth)
                    assert qf[t, r, c] == q[t2, H + j2, H + i2]
    # corners of the halo stay NaN on the cube (no fourth quadrant)
    assert np.isnan(qf[:, :H, :H]).all() and np.isnan(qf[:, -H:, -H:]).all()


def test_every_strip_is_a_neighbour_copy(orc, cube):
    # all four strips: every halo value equals some interior value of another
    # tile at a cell that shares an edge-chain with the tile (value identity)
    cen = np.stack([I.centre_points(t, N) for t in range(6)])
    vals = np.arange(6 * N * N, dtype=float).reshape(6, N, N)
    q = pad_cells(vals)
    qf = orc.fill_cells(cube, q, 1, 3).reshape(q.shape)
    for t in range(6):
        strips = [qf[t, H:H + N, :H], qf[t, H:H + N, -H:], qf[t, :H, H:H + N], qf[t, -H:, H:H + N]]
        for s in strips:
            ids = s.astype(int).ravel()
            owners = ids // (N * N)
            assert np.all(owners != t)
            assert len(set(ids.tolist())) == ids.size   # no cell used twice in one strip
            # halo cell centres are close to the tile: within 4 cell widths of the edge
            p = cen.reshape(-1, 3)[ids]
            dist_edge = np.min(np.linalg.norm(p[:, None] - cen[t].reshape(-1, 3)[None], axis=-1), axis=1)
            assert dist_edge.max() < 5 * (math.pi / 2 / N)


def halo_face_index(e, p, depth):
    """padded (array, row, col) of the strip face parallel to edge e between
    halo depths `depth` and `depth + 1`"""
    if e == "W":
        return "v", H + p, H - depth
    if e == "E":
        return "v", H + p, H + N + depth
    if e == "S":
        return "u", H - depth, H + p
    return "u", H + N + depth, H + p


def test_vector_halo_rotation(orc, cube):
    """D-grid winds of a rigid rotation: every strip face (all four strips)
    holds the wind component along that face in the tile's own extended
    orientation (+y for W/E strips, +x for S/N strips)."""
    st = I.cubed_state(N, 1, seed=0, ntracers=0)
    vp = np.full((6, N + 2 * H, N + 1 + 2 * H), np.nan)
    up = np.full((6, N + 1 + 2 * H, N + 2 * H), np.nan)
    vp[:, H:H + N, H:H + N + 1] = st["v"][:, 0]
    up[:, H:H + N + 1, H:H + N] = st["u"][:, 0]
    vf, uf = orc.fill_faces(cube, vp, up, 1, 1, 1)
    arrs = {"v": vf.reshape(vp.shape), "u": uf.reshape(up.shape)}
    cells = all_cells()
    tilt = math.radians(30.0)
    axis = np.array([math.sin(tilt), 0.0, math.cos(tilt)])
    vel = lambda q: 20.0 * np.cross(axis, q)
    for t in range(6):
        P = I.corner_points(t, N)
        for e in EDGES:
            for p in range(N):
                chain = strip_chain(cells, t, e, p)
                _, c0, _ = edge_cell(e, p)
                start = P[c0[1], c0[0]]
                for depth in range(1, 3):
                    ends = shared(cells[chain[depth - 1]], cells[chain[depth]])
                    assert len(ends) == 2
                    d0 = [np.linalg.norm(x - start) for x in ends]
                    ps, pe = (ends[0], ends[1]) if d0[0] < d0[1] else (ends[1], ends[0])
                    mid = (ps + pe) / np.linalg.norm(ps + pe)
                    want = vel(mid) @ ((pe - ps) / np.linalg.norm(pe - ps))
                    nm, r, c = halo_face_index(e, p, depth)
                    got = arrs[nm][t, r, c]
                    assert abs(got - want) <= 1e-12 * 20.0, (t, e, p, depth, got, want)


def test_owner_edges_consistent(orc, cube):
    st = I.cubed_state(N, 1, seed=1, ntracers=0)
    vp = np.full((6, N + 2 * H, N + 1 + 2 * H), np.nan)
    up = np.full((6, N + 1 + 2 * H, N + 2 * H), np.nan)
    vp[:, H:H + N, H:H + N + 1] = st["v"][:, 0]
    up[:, H:H + N + 1, H:H + N] = st["u"][:, 0]
    vf, uf = orc.fill_faces(cube, vp, up, 1, 1, 1)
    vf = vf.reshape(vp.shape)
    uf = uf.reshape(up.shape)
    # idempotent: filling again changes nothing
    vg, ug = orc.fill_faces(cube, vf, uf, 1, 1, 1)
    assert np.array_equal(vg.reshape(vp.shape), vf) and np.array_equal(ug.reshape(up.shape), uf)
    # all strips and corner slots finite for the D-grid
    assert np.isfinite(vf).all() and np.isfinite(uf).all()
