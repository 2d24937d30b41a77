"""Pins of the oracle's map export (Fig. 3: Marching Cubes at iso = 0):
facts about the surface that do not come from the oracle itself -- the edges
it may cross, closedness and orientation, exact positions and volumes of
planes and octahedra, Euler characteristic and volume of a ball."""
import numpy as np
import pytest

import synth

def _edge_corners(orc):
    return orc.MC_EDGE_CORNERS


def _grid(orc, state, res=1.0, origin=(0.0, 0.0, 0.0)):
    m, s, h = state
    nz, ny, nx = m.shape
    g = orc.Grid(nx, ny, nz, float(res), tuple(float(o) for o in origin), m.copy(), s.copy(), h.copy())
    return g


def _directed_edges(tri):
    """Directed edges (as pairs of exact vertex tuples) of a triangle soup."""
    out = []
    for t in tri:
        v = [tuple(p) for p in t.tolist()]
        for a, b in ((0, 1), (1, 2), (2, 0)):
            out.append((v[a], v[b]))
    return out


def _signed_volume(tri):
    t = tri.astype(np.float64)
    return float(np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0)


# ------------------------------------------------------------------ the table
def test_table_crosses_exactly_the_sign_changing_edges(orc):
    ec = _edge_corners(orc)
    for cfg in range(256):
        t = orc.mc_config(cfg)
        crossed = {e for e, (a, b) in enumerate(ec) if ((cfg >> a) & 1) != ((cfg >> b) & 1)}
        assert set(t.reshape(-1).tolist()) == crossed, cfg
        # no degenerate triangle
        for tri in t:
            assert len(set(tri.tolist())) == 3


def test_table_surface_ends_on_cube_faces(orc):
    """Inside one cell the triangles form surface pieces whose boundary runs
    over the cube's faces: every boundary edge joins two crossed edges of a
    common face, and every other edge is shared by exactly two triangles in
    opposite directions."""
    ec = _edge_corners(orc)
    faces = [{q for q in range(8) if ((q >> a) & 1) == s} for a in range(3) for s in (0, 1)]
    for cfg in range(256):
        t = orc.mc_config(cfg)
        d = {}
        for tri in t.tolist():
            for a, b in ((0, 1), (1, 2), (2, 0)):
                d[(tri[a], tri[b])] = d.get((tri[a], tri[b]), 0) + 1
        for (a, b), n in d.items():
            assert n == 1, cfg
            if (b, a) in d:
                continue
            ca, cb = set(ec[a]), set(ec[b])
            assert any(ca <= f and cb <= f for f in faces), (cfg, a, b)


def test_table_face_rule_keeps_inside_diagonal_apart(orc):
    """Two diagonal inside corners of a face (corners 0 and 3 of face -z):
    their crossings are joined corner by corner (0 with edges 0 and 4, 3 with
    edges 1 and 5), never across the face."""
    t = orc.mc_config(0b1001)
    pieces = [set(tri) for tri in t.tolist()]
    assert {0, 4, 8} in pieces and {1, 5, 11} in pieces


# ------------------------------------------------------------------ surfaces
def test_plane_is_exact_and_faces_up(orc):
    """Occupied for z <= 2 (distance 1 at z = 2), free above (1 at z = 3):
    the iso-surface is the plane half way, z = 3.0 voxel units, two
    triangles per cell, normals +z, area (nx - 1)(ny - 1) res^2."""
    nx, ny, nz, res = 7, 5, 6, 0.25
    z = np.arange(nz)[:, None, None] * np.ones((nz, ny, nx), int)
    occ = z <= 2
    dist = np.where(occ, 3 - z, z - 2)
    g = _grid(orc, synth.map_state(dist, occ), res=res, origin=(1.0, -2.0, 0.5))
    tri, cell = orc.mesh(g)
    assert len(tri) == 2 * (nx - 1) * (ny - 1)
    np.testing.assert_array_equal(tri[:, :, 2], np.float32(0.5 + res * 3.0))
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    assert (n[:, 2] > 0).all() and np.abs(n[:, :2]).max() == 0
    assert np.isclose(0.5 * np.linalg.norm(n, axis=1).sum(), (nx - 1) * (ny - 1) * res * res)
    assert (np.diff(cell) >= 0).all()


@pytest.mark.parametrize("d_in,d_out", [(1, 1), (1, 3), (2, 1)])
def test_single_voxel_is_an_octahedron(orc, d_in, d_out):
    """One occupied voxel (distance d_in) among free ones (distance d_out):
    8 triangles around it with vertices at t = d_in / (d_in + d_out) voxel
    along each axis, volume (4/3) t^3, normals pointing away from it."""
    n = 5
    dist = np.full((n, n, n), d_out)
    occ = np.zeros((n, n, n), bool)
    occ[2, 2, 2] = True
    dist[2, 2, 2] = d_in
    res = 0.1
    g = _grid(orc, synth.map_state(dist, occ), res=res)
    tri, _ = orc.mesh(g)
    assert len(tri) == 8
    t = d_in / (d_in + d_out)
    c = 2.5 * res
    r = np.abs(tri.astype(np.float64) - c).max(axis=2)
    np.testing.assert_allclose(r, t * res, rtol=1e-6)
    assert np.isclose(_signed_volume(tri), (4.0 / 3.0) * (t * res) ** 3, rtol=1e-5)
    d = _directed_edges(tri)
    assert sorted(d) == sorted((b, a) for a, b in d)


def test_ball_closed_genus_zero_and_volume(orc):
    """Ball of radius 7 voxels: a closed consistently oriented surface
    (every directed edge has its reverse, once), Euler characteristic 2,
    enclosed volume within 8 % of (4/3) pi r^3, every vertex within one
    voxel of the sphere."""
    n, c, r = 24, (11.4, 11.7, 11.2), 7.0
    g = _grid(orc, synth.sphere_state(n, c, r))
    tri, _ = orc.mesh(g)
    d = _directed_edges(tri)
    assert len(set(d)) == len(d)
    assert set(d) == {(b, a) for a, b in d}
    V = len({v for e in d for v in e})
    E = len(d) // 2
    assert V - E + len(tri) == 2
    vol = _signed_volume(tri)
    assert abs(vol - 4.0 / 3.0 * np.pi * r ** 3) < 0.08 * 4.0 / 3.0 * np.pi * r ** 3
    rr = np.linalg.norm(tri.reshape(-1, 3).astype(np.float64) - (np.array(c) + 0.5), axis=1)
    assert np.abs(rr - r).max() < 1.0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_states_are_watertight(orc, seed):
    """Random voxels (every configuration, ambiguous faces included): every
    edge of the surface away from the box's faces is shared by exactly two
    triangles with opposite directions, so cells agree on their shared faces.
    Distances >= 1 keep every vertex strictly inside its edge (a corner at
    distance 0 is exactly on the surface and vertices of several edges
    coincide there)."""
    shape = (9, 10, 11)
    g = _grid(orc, synth.random_state(shape, seed, min_dist=1))
    tri, _ = orc.mesh(g)
    assert len(tri) > 100
    d = _directed_edges(tri)
    assert len(set(d)) == len(d)
    nz, ny, nx = shape
    hi = (nx - 0.5, ny - 0.5, nz - 0.5)

    def on_box_face(a, b):
        return any((a[k] == 0.5 and b[k] == 0.5) or (a[k] == hi[k] and b[k] == hi[k])
                   for k in range(3))
    ds = set(d)
    for a, b in d:
        if (b, a) not in ds:
            assert on_box_face(a, b), (a, b)


def test_iso_between_levels(orc):
    """iso = 0.5 res on the plane state: the crossing moves from the midpoint
    to where the field (-1 at z = 2, +1 at z = 3) reaches 0.5, t = 0.75."""
    nx, ny, nz = 4, 4, 6
    z = np.arange(nz)[:, None, None] * np.ones((nz, ny, nx), int)
    occ = z <= 2
    g = _grid(orc, synth.map_state(np.where(occ, 3 - z, z - 2), occ), res=1.0)
    tri, _ = orc.mesh(g, iso=0.5)
    np.testing.assert_array_equal(tri[:, :, 2], np.float32(2.5 + 0.75))


def test_sub_box_matches_whole_grid_cells(orc):
    """Meshing a box gives exactly the triangles of the whole-grid mesh whose
    cells lie in the box (same vertices: coordinates are global)."""
    st = synth.random_state((8, 9, 10), 11)
    g = _grid(orc, st, res=0.2, origin=(0.3, 0.1, -0.4))
    tri, cell = orc.mesh(g)
    x0, y0, z0, bx, by, bz = 2, 3, 1, 5, 4, 6
    sub, sc = orc.mesh(g, box=(x0, y0, z0, bx, by, bz))
    cx, cy = g.nx - 1, g.ny - 1
    i, j, k = cell % cx, (cell // cx) % cy, cell // (cx * cy)
    sel = (i >= x0) & (i < x0 + bx - 1) & (j >= y0) & (j < y0 + by - 1) & (k >= z0) & (k < z0 + bz - 1)
    np.testing.assert_array_equal(sub, tri[sel])
    bi, bj, bk = i[sel] - x0, j[sel] - y0, k[sel] - z0
    np.testing.assert_array_equal(sc, (bk * (by - 1) + bj) * (bx - 1) + bi)


def test_sdf_field_readout(orc):
    """The field is the readout at every voxel: popcount of the mask, signed
    by the flag, times res (this readout is a reading: parity unpinned)."""
    m, s, h = synth.random_state((3, 4, 5), 4)
    g = _grid(orc, (m, s, h), res=0.05)
    f = orc.sdf_field(g)
    pc = np.array([bin(int(v)).count("1") for v in m.reshape(-1)]).reshape(m.shape)
    want = (np.where(s == 1, 1.0, -1.0) * pc * 0.05).astype(np.float32)
    np.testing.assert_array_equal(f, want)
    np.testing.assert_array_equal(orc.sdf_field(g, (1, 2, 0, 3, 2, 2)), want[0:2, 2:4, 1:4])
