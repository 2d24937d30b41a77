"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Integer work, so the bar is bit-exact: every voxel's mask, sign and hit
counter, and the scan counters.  Small grids are compared whole; the
full-size urban and high-resolution grids are compared on sampled voxels the
oracle folds one by one, plus invariants that hold at any size.
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


def run_gpu(pdict, dims, res, scans, origin=(0.0, 0.0, 0.0), max_points=None, host=False,
            tuning=None):
    dbt = _dbt()
    p = dbt.make_params(**pdict)
    k = dbt.Kernels(p)
    g = dbt.Grid(*dims, res, origin)
    mp = max_points or max([len(s[0]) for s in scans] + [1])
    ws = dbt.Workspace(g, k, mp)
    if tuning:
        ws.set_tuning(k, **tuning)
    stats = []
    for pts, pose in scans:
        if host:
            st = dbt.dbtsdf.dbt_scan_stats()
            h = torch.from_numpy(np.ascontiguousarray(pts)).pin_memory()
            dbt.dbt_integrate_scan_host(g, k, ws, h, pose, st)
            torch.cuda.synchronize()
            stats.append(st.as_dict())
        else:
            x = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
            dbt.dbt_integrate_scan(g, k, ws, x, pose)
            stats.append(dbt.dbt_get_scan_stats(ws))
    out = g.numpy()
    return out, stats, (g, k, ws)


def run_oracle(orc, pdict, dims, res, scans, origin=(0.0, 0.0, 0.0)):
    p = orc.params(**pdict)
    g = orc.Grid.create(*dims, res, origin)
    stats = [orc.integrate_scan(g, p, pts, pose) for pts, pose in scans]
    return g, stats


def assert_same(gpu, ora, gstats, ostats):
    m, s, h = gpu
    for name, a, b in (("mask", m, ora.mask), ("hits", h, ora.hits), ("sign", s, ora.sign)):
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            z, y, x = bad[0]
            raise AssertionError(f"{name} differs at {len(bad)} voxels, first (x,y,z)=({x},{y},{z}):"
                                 f" gpu={a[z, y, x]:#x} oracle={b[z, y, x]:#x}")
    for gs, os_ in zip(gstats, ostats):
        assert gs["error"] == 0
        for key in ("n_input", "n_valid", "n_inside", "n_kept"):
            assert gs[key] == os_[key], (key, gs, os_)


def params(**kw):
    d = dict(synth.DEFAULT_PARAMS)
    d.update(kw)
    return d


# ------------------------------------------------------------------ whole-grid cases
@pytest.fixture(scope="module")
def room3():
    return synth.room_scan(n_scans=3)


def test_room_scan_128(orc, room3):
    """Config 0: 128^3 at 0.10 m, one 16 x 900 scan, K = 11, 64 octahedral bins."""
    scans = room3.scans[:1]
    gpu, gs, _ = run_gpu(room3.params, (128, 128, 128), 0.1, scans)
    ora, os_ = run_oracle(orc, room3.params, (128, 128, 128), 0.1, scans)
    assert os_[0]["n_kept"] > 5000
    assert_same(gpu, ora, gs, os_)


def test_room_sequence_128(orc, room3):
    gpu, gs, _ = run_gpu(room3.params, (128, 128, 128), 0.1, room3.scans)
    ora, os_ = run_oracle(orc, room3.params, (128, 128, 128), 0.1, room3.scans)
    assert_same(gpu, ora, gs, os_)


def test_host_entry_point_matches(orc, room3):
    """dbt_integrate_scan_host (host buffers, copies inside) == device entry point."""
    gpu, gs, _ = run_gpu(room3.params, (128, 128, 128), 0.1, room3.scans[:2], host=True)
    ora, os_ = run_oracle(orc, room3.params, (128, 128, 128), 0.1, room3.scans[:2])
    assert_same(gpu, ora, gs, os_)


def test_host_entry_point_pipelined(orc):
    """Scans handed in from host buffers back to back, no synchronisation in
    between: each copy overlaps the previous scan (two staging buffers, each
    reused three times) and the map equals the oracle's.  The counters of
    every other scan go to pinned memory (stored by the integrate kernel),
    the others to pageable memory (copied)."""
    dbt = _dbt()
    w = synth.urban_sequence(n_scans=6, scale=0.25)
    dims = (w.grid.nx, w.grid.ny, w.grid.nz)
    k = dbt.Kernels(dbt.make_params(**w.params))
    g = dbt.Grid(*dims, w.grid.res, w.grid.origin)
    ws = dbt.Workspace(g, k, max(len(p) for p, _ in w.scans))
    hosts = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p, _ in w.scans]
    h_st = torch.full((len(w.scans), 64), 0xAB, dtype=torch.uint8).pin_memory()
    sts = [dbt.dbtsdf.dbt_scan_stats.from_address(h_st[i].data_ptr()) if i % 2 == 0
           else dbt.dbtsdf.dbt_scan_stats() for i in range(len(w.scans))]
    for h, (_, pose), st in zip(hosts, w.scans, sts):
        dbt.dbt_integrate_scan_host(g, k, ws, h, pose, st)
    torch.cuda.synchronize()
    ora, os_ = run_oracle(orc, w.params, dims, w.grid.res, w.scans, w.grid.origin)
    assert_same(g.numpy(), ora, [st.as_dict() for st in sts], os_)


@pytest.mark.parametrize("variant", [
    dict(dedup_first=0),
    dict(shadow_radius=0.0, dedup_first=0, hit_max=65535),
    dict(dedup_first=0, hit_threshold=5, hit_max=60000),     # counters by compare-and-swap
    dict(shadow_radius=5.0, hit_threshold=1, hit_max=2),
    dict(kernel_size=3, shadow_radius=1.0),
    dict(kernel_size=21, scheme=1, bins_a=40, bins_b=40, shadow_radius=3.0),   # the paper's
    dict(kernel_size=15, scheme=1, bins_a=36, bins_b=18, shadow_radius=6.5),
    dict(kernel_size=17, scheme=0, bins_a=16, bins_b=16, shadow_radius=4.0),
    dict(shadow_radius=5.0, shadow_cos=0.7),                                    # conical shadow
    dict(kernel_size=21, scheme=1, bins_a=40, bins_b=40, shadow_radius=6.0, shadow_cos=0.5),
])
def test_room_variants(orc, room3, variant):
    pd = params(**variant)
    gpu, gs, _ = run_gpu(pd, (128, 128, 128), 0.1, room3.scans[:2])
    ora, os_ = run_oracle(orc, pd, (128, 128, 128), 0.1, room3.scans[:2])
    assert_same(gpu, ora, gs, os_)


@pytest.mark.parametrize("K", [9, 13])
@pytest.mark.parametrize("heavy", [0, 8, 1 << 30])
def test_group_schedules_match_oracle(orc, room3, K, heavy):
    """K = 9 runs heavy bricks on two four-warp groups per CTA, K = 13 on the
    whole CTA; every brick heavy (0), a mix with very heavy bricks (8: more
    than 32 pairs first) and every brick light (2^30)."""
    dbt = _dbt()
    pd = params(kernel_size=K, shadow_radius=3.0)
    k = dbt.Kernels(dbt.make_params(**pd))
    g = dbt.Grid(128, 128, 128, 0.1)
    ws = dbt.Workspace(g, k, max(len(s[0]) for s in room3.scans))
    ws.set_tuning(k, heavy, 0)
    gs = []
    for pts, pose in room3.scans[:2]:
        dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).cuda(), pose)
        gs.append(dbt.dbt_get_scan_stats(ws))
    ora, os_ = run_oracle(orc, pd, (128, 128, 128), 0.1, room3.scans[:2])
    assert_same(g.numpy(), ora, gs, os_)


@pytest.mark.parametrize("depth,K", [(4, 3), (4, 9), (4, 13), (4, 21), (16, 5), (16, 11), (16, 13),
                                     (16, 17)])
def test_brick_depths_match_oracle(orc, room3, depth, K):
    """Bricks 32 x 8 x 4 and 32 x 8 x 16: every brick heavy (0), a mix with
    very heavy bricks (8) and every brick light (2^30), whole grids against
    the oracle.  Depth 4 runs the dense path on the whole CTA from K = 9 on
    (two four-warp groups below), depth 16 keeps the two groups up to K = 11;
    K = 17 is the deepest kernel depth 16 takes."""
    dbt = _dbt()
    pd = params(kernel_size=K, shadow_radius=min(3.0, (K - 1) / 2))
    ora, os_ = run_oracle(orc, pd, (128, 128, 128), 0.1, room3.scans[:2])
    for heavy in (0, 8, 1 << 30):
        gpu, gs, (g, k, ws) = run_gpu(pd, (128, 128, 128), 0.1, room3.scans[:2],
                                      tuning=dict(heavy_pairs=heavy, brick_depth=depth))
        assert ws.tuning()["brick_depth"] == depth
        assert_same(gpu, ora, gs, os_)


def test_brick_depth_16_refused_above_k17():
    dbt = _dbt()
    k = dbt.Kernels(dbt.make_params(**params(kernel_size=19)))
    g = dbt.Grid(64, 64, 64, 0.1)
    ws = dbt.Workspace(g, k, 1000)
    with pytest.raises(dbt.DbtError):
        ws.set_tuning(k, 64, 0, 16)
    with pytest.raises(dbt.DbtError):
        ws.set_tuning(k, 64, 0, 12)
    ws.set_tuning(k, 64, 0, 4)
    assert ws.tuning() == {"heavy_pairs": 64, "integrate_ctas": 0, "brick_depth": 4}
    ws.set_tuning(k, 64, 0, 0)
    assert ws.tuning()["brick_depth"] == 8


@pytest.mark.parametrize("K,tuning", [
    (11, {}),                               # very heavy: whole CTA, dense path
    (11, {"heavy_pairs": 1 << 30}),          # every brick light: one warp
    (15, {}),                               # K > 13: warps' own areas, merged
    (9, {"heavy_pairs": 1 << 30, "brick_depth": 4}),
])
def test_brick_with_more_pairs_than_a_count_round(orc, K, tuning):
    """100,000 returns (first-return rule off) in a 2 x 2 x 2-voxel cube: the
    brick that holds it gets more (return, brick) pairs than one round of
    16-bit counts takes (65,535), so its pairs are integrated in two rounds;
    with hit_max = 65535 some counters receive more increments than that and
    saturate across the rounds."""
    rng = synth.Rng(4242 + K)
    dims, res = (64, 64, 64), 0.1
    lo = np.array([30.0, 30.0, 30.0]) * res
    pts = synth.random_points(rng, 100000, tuple(lo + 0.001), tuple(lo + 2 * res - 0.001))
    pose = synth.make_pose(np.eye(3), (0.0, 0.0, 0.0))
    scans = [(np.ascontiguousarray(pts, np.float32), pose)]
    pd = params(kernel_size=K, dedup_first=0, hit_max=65535, hit_threshold=3,
                shadow_radius=min(3.0, (K - 1) / 2))
    gpu, gs, _ = run_gpu(pd, dims, res, scans, tuning=tuning)
    ora, os_ = run_oracle(orc, pd, dims, res, scans)
    assert os_[0]["n_kept"] == 100000
    assert gs[0]["n_pairs"] > 100000
    assert int(ora.hits.max()) == 65535
    assert_same(gpu, ora, gs, os_)


def _tiny(seed, n, dims, res, dup):
    rng = synth.Rng(seed)
    nx, ny, nz = dims
    hi = np.array([nx, ny, nz]) * res
    pts_w = synth.random_points(rng, n, (0.0, 0.0, 0.0), hi)
    if dup:
        pts_w = np.concatenate([pts_w, pts_w[::dup] + np.float32(0.01 * res)]).astype(np.float32)
    R = synth.random_rotation(rng)
    t = hi / 2 + rng.uniform(3, -res, res)
    pts_s = ((pts_w.astype(np.float64) - t) @ R).astype(np.float32)
    return pts_s, synth.make_pose(R, t)


@pytest.mark.parametrize("dims,K,scheme", [
    ((16, 16, 16), 5, 0), ((33, 17, 9), 3, 0), ((100, 70, 50), 11, 0), ((45, 61, 23), 7, 1),
    ((97, 13, 41), 11, 1), ((40, 40, 40), 21, 0), ((21, 21, 21), 21, 1), ((64, 8, 8), 1, 0),
])
def test_ragged_grids(orc, dims, K, scheme):
    """Grids that are not whole bricks, random poses, duplicates in voxels;
    at every brick depth the kernel size allows (a ragged last brick layer
    in z for depths 4, 8 and 16 alike)."""
    a, b = (8, 8) if scheme == 0 else (40, 40)
    pd = params(kernel_size=K, scheme=scheme, bins_a=a, bins_b=b,
                shadow_radius=min(3.0, (K - 1) / 2))
    scans = [_tiny(100 + i + K, 3000, dims, 0.07, 5) for i in range(3)]
    ora, os_ = run_oracle(orc, pd, dims, 0.07, scans)
    assert sum(s["n_kept"] for s in os_) > 0
    for depth in (8, 4, 16) if K <= 17 else (8, 4):
        gpu, gs, _ = run_gpu(pd, dims, 0.07, scans, origin=(0.0, 0.0, 0.0),
                             tuning=dict(brick_depth=depth))
        assert_same(gpu, ora, gs, os_)


def test_origin_offset_and_negative_coords(orc):
    dims = (48, 40, 36)
    origin = (-2.0, -1.5, -3.25)
    rng = synth.Rng(77)
    pts = synth.random_points(rng, 4000, (-2.5, -2.0, -3.5), (2.0, 1.5, 0.5))
    pose = synth.make_pose(np.eye(3), (0.0, 0.0, 0.0))
    scans = [(pts, pose)]
    pd = params()
    gpu, gs, _ = run_gpu(pd, dims, 0.1, scans, origin=origin)
    ora, os_ = run_oracle(orc, pd, dims, 0.1, scans, origin=origin)
    assert_same(gpu, ora, gs, os_)


# ------------------------------------------------------------------ edge cases
def test_empty_and_degenerate_scans(orc):
    dims = (64, 64, 64)
    pose = synth.make_pose(np.eye(3), (3.2, 3.2, 3.2))
    nanscan = np.full((500, 3), np.nan, np.float32)
    origin_pts = np.zeros((300, 3), np.float32)
    border = np.array([[-3.19, 0, 0], [3.15, 0.0, 0.0], [0, -3.1, 0], [0, 0, 3.1]], np.float32)
    same_voxel = np.tile(np.array([[1.01, 0.51, 0.21]], np.float32), (1000, 1))
    scans = [(np.zeros((0, 3), np.float32), pose), (nanscan, pose), (origin_pts, pose),
             (border, pose), (same_voxel, pose)]
    pd = params()
    gpu, gs, _ = run_gpu(pd, dims, 0.1, scans, max_points=1000)
    ora, os_ = run_oracle(orc, pd, dims, 0.1, scans)
    assert [s["n_kept"] for s in os_] == [0, 0, 0, 0, 1]
    assert_same(gpu, ora, gs, os_)


def test_point_permutation_without_dedup(room3):
    pd = params(dedup_first=0)
    pts, pose = room3.scans[0]
    perm = np.argsort(synth.Rng(4).uniform(len(pts)))
    a, _, _ = run_gpu(pd, (128, 128, 128), 0.1, [(pts, pose)])
    b, _, _ = run_gpu(pd, (128, 128, 128), 0.1, [(pts[perm], pose)])
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_repeatable(room3):
    a, _, _ = run_gpu(room3.params, (128, 128, 128), 0.1, room3.scans)
    b, _, _ = run_gpu(room3.params, (128, 128, 128), 0.1, room3.scans)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_argument_errors(room3):
    dbt = _dbt()
    pd = room3.params
    k = dbt.Kernels(dbt.make_params(**pd))
    g = dbt.Grid(64, 64, 64, 0.1)
    ws = dbt.Workspace(g, k, 100)
    x = torch.zeros((101, 3), device="cuda")
    with pytest.raises(dbt.DbtError):
        dbt.dbt_integrate_scan(g, k, ws, x, np.hstack([np.eye(3), np.zeros((3, 1))]))
    bad = np.hstack([2 * np.eye(3), np.zeros((3, 1))])
    with pytest.raises(dbt.DbtError):
        dbt.dbt_integrate_scan(g, k, ws, x[:10], bad)
    g2 = dbt.Grid(64, 64, 32, 0.1)
    with pytest.raises(dbt.DbtError):
        dbt.dbt_integrate_scan(g2, k, ws, x[:10], np.hstack([np.eye(3), np.zeros((3, 1))]))


# ------------------------------------------------------------------ bins and readout
@pytest.mark.parametrize("scheme,a,b", [(0, 8, 8), (0, 16, 16), (1, 40, 40), (1, 36, 18)])
def test_device_bins_match_oracle(orc, scheme, a, b):
    dbt = _dbt()
    k = dbt.Kernels(dbt.make_params(scheme=scheme, bins_a=a, bins_b=b))
    rng = synth.Rng(31)
    d = rng.normal(3 * 20000).reshape(-1, 3)
    axes = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                     [1, 1, 0], [1, 0, 1], [1, 0, -1], [1, 1, 1], [-1, 1, -1], [3, 1, 0],
                     [1, -3, -4], [0, 0, 0]], np.float64)
    d = np.concatenate([axes, d])
    # directions exactly on octahedral/azimuth edges
    t = np.arange(64) * (2 * np.pi / 64)
    d = np.concatenate([d, np.stack([np.cos(t), np.sin(t), np.zeros(64)], 1)])
    got = dbt.dbt_bin_directions(k, torch.from_numpy(d).cuda()).cpu().numpy()
    po = orc.params(scheme=scheme, bins_a=a, bins_b=b)
    want = np.array([orc.bin_of(po, v) if np.any(v) else -1 for v in d])
    np.testing.assert_array_equal(got, want)


def test_readout_matches_oracle(orc, room3):
    gpu, _, (g, k, ws) = run_gpu(room3.params, (128, 128, 128), 0.1, room3.scans[:1])
    dbt = _dbt()
    rng = synth.Rng(8)
    idx = rng.integers(3 * 2000, -2, 130).reshape(-1, 3).astype(np.int32)
    m, s, h = dbt.dbt_read_voxels(g, torch.from_numpy(idx).cuda())
    sdf = dbt.dbt_read_distance(g, torch.from_numpy(idx).cuda()).cpu().numpy()
    m = m.cpu().numpy().view(np.uint32)
    s = s.cpu().numpy()
    h = h.cpu().numpy().view(np.uint16)
    gm, gsn, gh = gpu
    for j, (x, y, z) in enumerate(idx):
        if 0 <= x < 128 and 0 <= y < 128 and 0 <= z < 128:
            assert (m[j], s[j], h[j]) == (gm[z, y, x], gsn[z, y, x], gh[z, y, x])
            assert sdf[j] == pytest.approx(orc.signed_distance(int(m[j]), int(s[j]), 0.1), rel=1e-6)
        else:
            assert (m[j], s[j], h[j]) == (0xFFFFFFFF, 1, 0)


# ------------------------------------------------------------------ full-size, sampled
def _sampled_check(orc, w, n_scans, n_samples=3000, seed=1):
    """Integrate n_scans on the GPU at full size; compare sampled voxels with
    the oracle's one-by-one fold; check grid-wide invariants on the device."""
    dbt = _dbt()
    gdims = (w.grid.nx, w.grid.ny, w.grid.nz)
    scans = w.scans[:n_scans]
    pd = w.params
    p = dbt.make_params(**pd)
    k = dbt.Kernels(p)
    g = dbt.Grid(*gdims, w.grid.res, w.grid.origin)
    ws = dbt.Workspace(g, k, max(len(s[0]) for s in scans))
    po = orc.params(**pd)
    og = orc.Grid(gdims[0], gdims[1], gdims[2], w.grid.res, w.grid.origin, None, None, None)
    cs, bs = [], []
    kept_total = 0
    for pts, pose in scans:
        dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).cuda(), pose)
        st = dbt.dbt_get_scan_stats(ws)
        c, b = _scan_kept_geometry(orc, po, og, pts, pose)
        assert st["n_kept"] == len(c) and st["error"] == 0
        kept_total += len(c)
        cs.append(c)
        bs.append(b)
    c = np.concatenate(cs)
    b = np.concatenate(bs)
    rng = synth.Rng(seed)
    # half the samples near integrated returns (where state changed), half anywhere
    near = c[rng.integers(n_samples // 2, 0, len(c))] + rng.integers(3 * (n_samples // 2), -6, 7).reshape(-1, 3)
    anywhere = np.stack([rng.integers(n_samples // 2, 0, gdims[a]) for a in range(3)], 1)
    q = np.concatenate([near, anywhere])
    q = q[np.all((q >= 0) & (q < np.array(gdims)), axis=1)]
    m, s, h = dbt.dbt_read_voxels(g, torch.from_numpy(q.astype(np.int32)).cuda())
    om, os_, oh = orc.query_voxels(po, c, b, q)
    np.testing.assert_array_equal(m.cpu().numpy().view(np.uint32), om)
    np.testing.assert_array_equal(h.cpu().numpy().view(np.uint16), oh)
    np.testing.assert_array_equal(s.cpu().numpy(), os_)
    # invariants over the whole grid (on the device)
    mm = g.mask[:, :, :g.nx]
    assert int(((mm & (mm + 1)) != 0).sum()) == 0            # masks stay 2^k - 1
    hits = g.hits[:, :, :g.nx].to(torch.int32) & 0xFFFF
    sign = g.sign[:, :, :g.nx]
    assert bool(((sign == 0) == (hits >= pd["hit_threshold"])).all())
    assert int((g.mask[:, :, g.nx:] != -1).sum()) == 0       # padding untouched
    return kept_total


def _scan_kept_geometry(orc, po, og, pts, pose):
    return orc.scan_kept(og, po, pts, pose)


@pytest.fixture(scope="module")
def urban():
    return synth.urban_sequence(n_scans=8)


def test_urban_full_size_sampled(orc, urban):
    """Config 1 geometry (1600 x 1600 x 320 at 0.05 m, 64 x 1024 scans)."""
    kept = _sampled_check(orc, urban, n_scans=8)
    assert kept > 8 * 30000


def test_highres_full_size_sampled(orc):
    """Config 2 geometry (2000 x 2000 x 400 at 0.02 m, 128 x 2048 scans)."""
    w = synth.urban_sequence(n_scans=2, scale=0.5, res=0.02, beams=128, width=2048, seed_offset=2)
    assert (w.grid.nx, w.grid.ny, w.grid.nz) == (2000, 2000, 400)
    _sampled_check(orc, w, n_scans=2)
