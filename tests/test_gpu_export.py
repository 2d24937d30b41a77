"""GPU parity of the map export (Fig. 3: Marching Cubes at iso = 0, plus the
signed-distance field), through the C ABI, against the oracle.

The field is compared bit for bit; the mesh triangle by triangle (same
order, same float32 vertices, same cell numbers).  Map states come from the
oracle's integration of the room scans or from the seeded state generators;
the full-size terrain map is compared on sampled cells, each meshed alone
by the oracle.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dbt():
    import paper_2509_20081_gb300 as dbt
    return dbt


def _pair(orc, state, res, origin=(0.0, 0.0, 0.0)):
    """The same map state as an oracle grid and a device grid."""
    m, s, h = state
    nz, ny, nx = m.shape
    og = orc.Grid(nx, ny, nz, float(res), tuple(float(o) for o in origin), m, s, h)
    dg = _dbt().Grid(nx, ny, nz, res, origin)
    dg.load(m, s, h)
    return og, dg


def _mesh_gpu(dg, box=None, iso=0.0):
    tri, cell = _dbt().dbt_mesh_extract(dg, box, iso, with_cells=True)
    torch.cuda.synchronize()
    return tri.cpu().numpy(), cell.cpu().numpy()


def _assert_mesh_equal(gpu, ora):
    (gt, gc), (ot, oc) = gpu, ora
    assert gt.shape == ot.shape, (gt.shape, ot.shape)
    np.testing.assert_array_equal(gc, oc)
    if not np.array_equal(gt.view(np.uint32), ot.view(np.uint32)):
        bad = np.argwhere((gt.view(np.uint32) != ot.view(np.uint32)).any(axis=(1, 2)))[:, 0]
        raise AssertionError(f"{len(bad)} triangles differ, first {bad[0]}: gpu {gt[bad[0]]} "
                             f"oracle {ot[bad[0]]}")


@pytest.fixture(scope="module")
def room_state(orc):
    w = synth.room_scan(n_scans=3)
    p = orc.params(**w.params)
    g = orc.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
    for pts, pose in w.scans:
        orc.integrate_scan(g, p, pts, pose)
    return (g.mask, g.sign, g.hits), w.grid.res


def test_sdf_field_room(orc, room_state):
    og, dg = _pair(orc, *room_state)
    f = _dbt().dbt_sdf_field(dg).cpu().numpy()
    np.testing.assert_array_equal(f.view(np.uint32), orc.sdf_field(og).view(np.uint32))
    box = (5, 17, 33, 61, 40, 29)
    f = _dbt().dbt_sdf_field(dg, box).cpu().numpy()
    np.testing.assert_array_equal(f.view(np.uint32), orc.sdf_field(og, box).view(np.uint32))


@pytest.mark.parametrize("iso_vox", [0.0, 0.5, -2.0])
def test_mesh_room(orc, room_state, iso_vox):
    """The room after three scans, whole grid, at iso = 0 (the paper's) and
    two other levels."""
    og, dg = _pair(orc, *room_state)
    iso = iso_vox * room_state[1]
    ora = orc.mesh(og, iso=iso)
    assert len(ora[0]) > 1000
    _assert_mesh_equal(_mesh_gpu(dg, iso=iso), ora)


@pytest.mark.parametrize("shape,box,seed,min_dist", [
    ((9, 10, 11), None, 1, 1),
    ((9, 10, 11), None, 2, 0),                     # distance-0 corners: vertices on corners
    ((33, 17, 65), None, 3, 0),                    # several units, ragged last unit
    ((40, 45, 50), (3, 7, 2, 41, 30, 35), 4, 0),   # a box inside the grid
    ((20, 30, 70), (0, 0, 0, 70, 30, 20), 5, 1),   # box = grid
    ((8, 8, 8), (2, 2, 2, 2, 2, 2), 6, 0),         # a single cell
])
def test_mesh_random_states(orc, shape, box, seed, min_dist):
    st = synth.random_state(shape, seed, min_dist=min_dist)
    og, dg = _pair(orc, st, 0.07, origin=(-1.3, 0.4, 2.2))
    _assert_mesh_equal(_mesh_gpu(dg, box), orc.mesh(og, box))


def test_mesh_sphere_and_plane(orc):
    og, dg = _pair(orc, synth.sphere_state(40, (19.3, 20.1, 18.7), 13.0), 0.05)
    _assert_mesh_equal(_mesh_gpu(dg), orc.mesh(og))


@pytest.mark.parametrize("box", [(0, 0, 0, 1, 9, 9), (3, 3, 3, 0, 4, 4), (0, 0, 0, 9, 9, 9)])
def test_mesh_degenerate_boxes_and_empty_map(orc, box):
    """Boxes with no cells give no triangles; a fresh map (every voxel at
    +32 res) has no surface at iso = 0."""
    dbt = _dbt()
    g = dbt.Grid(9, 9, 9, 0.1)
    tri, cell = dbt.dbt_mesh_extract(g, box, 0.0, with_cells=True)
    assert tri.shape == (0, 3, 3) and cell.shape == (0,)


def test_mesh_truncated_output(orc):
    """max_tri below the total: the count is still the total and exactly the
    first max_tri triangles are written; nothing past them."""
    dbt = _dbt()
    B = dbt.dbtsdf
    st = synth.random_state((12, 13, 14), 8)
    og, dg = _pair(orc, st, 0.1)
    ot, oc = orc.mesh(og)
    need = dbt.dbt_mesh_scratch_size(dg)
    scratch = torch.empty(need, dtype=torch.uint8, device="cuda")
    cap = len(ot) // 3
    tri = torch.full((cap + 10, 3, 3), 7.0, device="cuda")
    cell = torch.full((cap + 10,), -5, dtype=torch.int64, device="cuda")
    n = ctypes.c_int64()
    box = (ctypes.c_int32 * 6)(0, 0, 0, 14, 13, 12)
    B._check(B.lib().dbt_mesh_extract(ctypes.byref(dg.c), box, 0.0, scratch.data_ptr(), need,
                                      tri.data_ptr(), cell.data_ptr(), cap, ctypes.byref(n), None))
    torch.cuda.synchronize()
    assert n.value == len(ot)
    t = tri.cpu().numpy()
    np.testing.assert_array_equal(t[:cap], ot[:cap])
    assert (t[cap:] == 7.0).all()
    c = cell.cpu().numpy()
    np.testing.assert_array_equal(c[:cap], oc[:cap])
    assert (c[cap:] == -5).all()


def test_mesh_argument_errors(orc):
    dbt = _dbt()
    B = dbt.dbtsdf
    g = dbt.Grid(16, 16, 16, 0.1)
    for box in [(0, 0, 0, 17, 16, 16), (-1, 0, 0, 4, 4, 4), (0, 0, 10, 4, 4, 7)]:
        with pytest.raises(B.DbtError) as e:
            dbt.dbt_mesh_extract(g, box)
        assert e.value.status == B.DBT_EINVAL
    with pytest.raises(B.DbtError):
        dbt.dbt_mesh_extract(g, None, float("nan"))
    n = ctypes.c_int64()
    box = (ctypes.c_int32 * 6)(0, 0, 0, 16, 16, 16)
    scratch = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    # scratch too small, unaligned, and triangles without a buffer
    assert B.lib().dbt_mesh_extract(ctypes.byref(g.c), box, 0.0, scratch.data_ptr(), 8, None,
                                    None, 0, ctypes.byref(n), None) == B.DBT_EINVAL
    assert B.lib().dbt_mesh_extract(ctypes.byref(g.c), box, 0.0, scratch.data_ptr() + 8, 1 << 15,
                                    None, None, 0, ctypes.byref(n), None) == B.DBT_EINVAL
    assert B.lib().dbt_mesh_extract(ctypes.byref(g.c), box, 0.0, scratch.data_ptr(), 1 << 16,
                                    None, None, 5, ctypes.byref(n), None) == B.DBT_EINVAL


def test_mesh_full_size_terrain_sampled(orc):
    """A 1600 x 1600 x 320 map (the urban map's size; 819 M cells): the GPU
    meshes all of it; sampled cells (with and without triangles) are meshed
    alone by the oracle and must match the GPU's triangles of that cell."""
    nx, ny, nz, res = 1600, 1600, 320, 0.05
    m, s, _ = synth.terrain_state(nx, ny, nz, 21)
    og = orc.Grid(nx, ny, nz, res, (0.0, 0.0, 0.0), m, s, None)
    dbt = _dbt()
    dg = dbt.Grid(nx, ny, nz, res)
    dg.load(m, s)
    tri, cell = _mesh_gpu(dg)
    assert len(tri) > 5_000_000
    assert (np.diff(cell) >= 0).all()
    rng = synth.Rng(77)
    cx, cy, cz = nx - 1, ny - 1, nz - 1
    with_tri = cell[rng.integers(300, 0, len(cell))]
    anywhere = rng.integers(300, 0, cx * cy * cz)
    for L in np.concatenate([with_tri, anywhere]):
        L = int(L)
        i, j, k = L % cx, (L // cx) % cy, L // (cx * cy)
        ot, _ = orc.mesh(og, box=(i, j, k, 2, 2, 2))
        lo, hi = np.searchsorted(cell, [L, L + 1])
        np.testing.assert_array_equal(tri[lo:hi].view(np.uint32), ot.view(np.uint32),
                                      err_msg=f"cell {L} ({i},{j},{k})")
