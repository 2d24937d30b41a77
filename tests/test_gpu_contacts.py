"""GPU parity of the per-return stage (dbt_scan_contacts) against the oracle.

The device takes the voxel and octahedral-cell floors from binary32 values
with an error bound and falls back to binary64 near a boundary; the oracle
takes them in binary64 (Sec. III-C).  Bit-exact: every return's contact
voxel, bin and discard decision.  Inputs aimed at the decision boundaries
(voxel faces, octahedral cell edges, the z = 0 fold, axis directions) force
the fallback; random poses and the full-size urban scans exercise both.
"""
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


def _params(**kw):
    d = dict(synth.DEFAULT_PARAMS)
    d.update(kw)
    d["dedup_first"] = 0
    return d


def check_contacts(orc, pdict, dims, res, origin, pts, pose):
    """Device contacts of every return == the oracle's kept returns (no
    first-return rule), in order; returns the number inside."""
    dbt = _dbt()
    k = dbt.Kernels(dbt.make_params(**pdict))
    g = dbt.Grid(*dims, res, origin)
    pts = np.ascontiguousarray(pts, np.float32)
    out = dbt.dbt_scan_contacts(g, k, torch.from_numpy(pts).cuda(), pose).cpu().numpy()
    po = orc.params(**pdict)
    og = orc.Grid(dims[0], dims[1], dims[2], res, origin, None, None, None)
    c, b = orc.scan_kept(og, po, pts, pose)
    inside = out[:, 0] >= 0
    assert int(inside.sum()) == len(c)
    np.testing.assert_array_equal(out[inside, :3].astype(np.int64), c)
    np.testing.assert_array_equal(out[inside, 3], b)
    assert np.all(out[~inside] == np.array([-1, 0, 0, 0]))
    return len(c)


def _pose(R, t):
    return synth.make_pose(np.asarray(R, np.float64), np.asarray(t, np.float64))


def test_voxel_faces_and_cell_edges(orc):
    """res = 1/8 (voxel faces exactly representable): returns exactly on
    faces, one binary32 ulp either side, and directions exactly on the
    octahedral cell edges of an 8 x 8 split, on the fold plane z = 0 and on
    the axes."""
    res, dims = 0.125, (64, 64, 64)
    c0 = 4.0                                                   # sensor at the grid centre
    comps = np.array([-0.75, -0.5, -0.25, 0.0, 0.25, 0.5, 0.75, 1.0, -1.0, 0.125, -0.375],
                     np.float64)
    g = np.stack(np.meshgrid(comps, comps, comps, indexing="ij"), -1).reshape(-1, 3)
    g = g[np.any(g != 0, axis=1)]
    pts = []
    for scale in (1.0, 2.0, 2.5, 3.0):                         # exact multiples of 1/8
        p = (g * scale).astype(np.float32)
        pts += [p, np.nextafter(p, np.float32(np.inf)), np.nextafter(p, np.float32(-np.inf))]
    pts = np.concatenate(pts).astype(np.float32)
    for R in (np.eye(3), np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]]),
              np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]])):
        n = check_contacts(orc, _params(kernel_size=11, bins_a=8, bins_b=8), dims, res,
                           (0.0, 0.0, 0.0), pts, _pose(R, (c0, c0, c0)))
        assert n > 0.9 * len(pts)


@pytest.mark.parametrize("na", [8, 6, 5, 16])
def test_octahedral_edges_random_ranges(orc, na):
    """Directions whose octahedral coordinate sits exactly on (or one ulp
    from) a cell edge of an na x na split, at random ranges."""
    rng = synth.Rng(500 + na)
    m = 6000
    k = rng.integers(m, 0, na + 1).astype(np.float64)
    u = 2.0 * k / na - 1.0                                      # edge values of u
    v = rng.uniform(m, -1.0, 1.0)
    s = np.abs(u) + np.abs(v)
    keep = s <= 1.0
    u, v = u[keep], v[keep]
    z = (1.0 - np.abs(u) - np.abs(v)) * np.where(rng.uniform(len(u)) < 0.5, 1.0, -1.0)
    d = np.stack([u, v, z], 1)
    r = rng.uniform(len(d), 0.5, 6.0)
    pts = (d * r[:, None]).astype(np.float32)
    pts = np.concatenate([pts, np.nextafter(pts, np.float32(np.inf))])
    check_contacts(orc, _params(kernel_size=5, bins_a=na, bins_b=na, shadow_radius=2.0),
                   (200, 200, 200), 0.1, (-10.0, -10.0, -10.0), pts,
                   _pose(np.eye(3), (0.0, 0.0, 0.0)))


@pytest.mark.parametrize("seed,res,scheme", [(1, 0.05, 0), (2, 0.1, 0), (3, 0.07, 0),
                                             (4, 0.02, 0), (5, 0.1, 1), (6, 0.3, 1)])
def test_random_poses(orc, seed, res, scheme):
    """Random rotations, translations far from the origin, returns near the
    sensor and far away; azimuth/elevation bins keep the binary64 path."""
    rng = synth.Rng(seed)
    dims = (300, 260, 120)
    origin = (1000.0 - 7.3 * seed, -523.25, 13.0)
    hi = np.array(dims) * res
    t = np.array(origin) + hi * rng.uniform(3, 0.3, 0.7)
    R = synth.random_rotation(rng)
    n = 40000
    dirs = rng.normal(3 * n).reshape(-1, 3)
    rr = np.concatenate([rng.uniform(n // 2, 0.01, 1.0), rng.uniform(n - n // 2, 1.0, 0.6 * hi.min())])
    pts = (dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * rr[:, None]).astype(np.float32)
    a, b = (8, 8) if scheme == 0 else (36, 18)
    inside = check_contacts(orc, _params(kernel_size=11, scheme=scheme, bins_a=a, bins_b=b), dims,
                            res, origin, pts, _pose(R, t))
    assert inside > n // 2


def test_voxel_faces_under_rotation(orc):
    """Map-frame points placed on voxel faces, rotated back into the sensor
    frame (binary32 rounding leaves them within ~1e-6 voxels of a face)."""
    rng = synth.Rng(9)
    res, dims, origin = 0.05, (400, 400, 100), (-10.0, -10.0, -2.5)
    R = synth.random_rotation(rng)
    t = np.array([0.3, -0.7, 0.2])
    n = 30000
    vox = np.stack([rng.integers(n, 20, dims[a] - 20) for a in range(3)], 1).astype(np.float64)
    frac = np.where(rng.uniform(3 * n).reshape(-1, 3) < 0.5, 0.0, rng.uniform(3 * n).reshape(-1, 3))
    w = np.array(origin) + (vox + frac) * res
    pts = ((w - t) @ R).astype(np.float32)
    check_contacts(orc, _params(), dims, res, origin, pts, _pose(R, t))


def test_degenerate_returns(orc):
    pts = np.array([[np.nan, 0, 0], [np.inf, 1, 1], [0, 0, 0], [1e-30, 0, 0], [0, -1e-30, 0],
                    [0, 0, 1e-30], [0, 0, -1e-30], [1e-38, 1e-38, -1e-38], [3.0, 0, 0],
                    [-3.0, 0, 0], [0, 3.0, 0], [0, 0, -3.0], [1e6, 0, 0], [2.0, 2.0, 0.0],
                    [2.0, -2.0, -0.0], [-0.0, 1.0, -1.0]], np.float32)
    check_contacts(orc, _params(), (128, 128, 128), 0.1, (0.0, 0.0, 0.0), pts,
                   _pose(np.eye(3), (6.4, 6.4, 6.4)))


def test_empty_scan_and_errors(orc):
    dbt = _dbt()
    k = dbt.Kernels(dbt.make_params(**_params()))
    g = dbt.Grid(32, 32, 32, 0.1)
    out = dbt.dbt_scan_contacts(g, k, torch.zeros((0, 3), device="cuda"),
                                _pose(np.eye(3), (1.6, 1.6, 1.6)))
    assert tuple(out.shape) == (0, 4)
    bad = np.hstack([np.eye(3) * 2.0, np.zeros((3, 1))])
    with pytest.raises(dbt.DbtError):
        dbt.dbt_scan_contacts(g, k, torch.ones((4, 3), device="cuda"), bad)


def test_urban_scans_full_size(orc):
    """All returns of two full-size urban scans (1600 x 1600 x 320 at 0.05 m)."""
    w = synth.urban_sequence(n_scans=2)
    for pts, pose in w.scans:
        inside = check_contacts(orc, _params(**w.params), (w.grid.nx, w.grid.ny, w.grid.nz),
                                w.grid.res, w.grid.origin, pts, pose)
        assert inside > 30000


def test_floors_follow_the_written_formulas(orc):
    """Returns crafted so that a reciprocal multiply (voxel floor, octahedral
    u) or a fused transform would land in another voxel or cell
    (tests/contact_cases.py): the device gives the written form's answer,
    the oracle's.  All of them take the binary64 path (each lies within an
    ulp of a boundary)."""
    import contact_cases as cc
    for c in cc.all_cases():
        pd = _params(kernel_size=c.kernel_size, shadow_radius=1.0)
        assert check_contacts(orc, pd, c.dims, c.res, c.origin, c.pts, c.pose) == 1
        dbt = _dbt()
        k = dbt.Kernels(dbt.make_params(**pd))
        g = dbt.Grid(*c.dims, c.res, c.origin)
        out = dbt.dbt_scan_contacts(g, k, torch.from_numpy(c.pts).cuda(), c.pose).cpu().numpy()
        got = tuple(int(v) for v in out[0, :3]) if c.kind != "octa" else (int(out[0, 3]),)
        assert got == c.plain and got != c.variant, (c.kind, got, c.plain, c.variant)
