"""Seeded random configurations, whole grids against the oracle.

Each case draws a kernel size (1..21), a bin scheme and resolution, a shadow
radius and shape (hemisphere or cone), a hit threshold and saturation, the
first-return rule on or off, a ragged grid, and a launch tuning (brick depth
4 / 8 / 16, heavy threshold from "every brick heavy" to "none").  Its three
scans mix scattered returns, returns repeated in the same voxels and a dense
cluster of returns in a few voxels (heavy and very heavy bricks).  The
scans are integrated by per-scan launches and, on fresh grids, as one
batch; both must equal the oracle's grid voxel for voxel, with the same
scan counters.
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


def _config(seed):
    """Parameters, grid and tuning of case `seed` (choices only; every
    value the method computes comes from the oracle or the library)."""
    rng = np.random.default_rng(1000 + seed)
    K = int(rng.choice([1, 3, 5, 7, 9, 11, 13, 15, 17, 19, 21]))
    R = (K - 1) // 2
    scheme = int(rng.integers(0, 2))
    if scheme == 0:
        a = b = int(rng.choice([4, 8, 16]))
    else:
        a, b = int(rng.choice([12, 36, 40])), int(rng.choice([9, 18, 40]))
    T = int(rng.integers(1, 6))
    pd = dict(kernel_size=K, scheme=scheme, bins_a=a, bins_b=b,
              shadow_radius=float(rng.uniform(0.0, min(6.5, R))) if R else 0.0,
              shadow_cos=float(rng.choice([0.0, 0.5, 0.7])),
              hit_threshold=T, hit_max=int(rng.choice([T, 7, 255, 65535])) if T <= 7 else 255,
              dedup_first=int(rng.integers(0, 2)))
    tuning = dict(heavy_pairs=int(rng.choice([0, 4, 16, 48, 1 << 30])),
                  brick_depth=int(rng.choice([4, 8, 16] if K <= 17 else [4, 8])))
    dims = tuple(int(x) for x in rng.integers(2 * R + 4, 2 * R + 72, 3))
    return pd, tuning, dims


def _scans(seed, dims, res, R):
    """Three scans: 1,500 scattered returns (every fifth repeated just beside
    itself, so in the same voxel), and 2,500 returns in a 4 x 4 x 2-voxel box
    at the grid's centre, seen from a random pose."""
    rng = synth.Rng(5000 + seed)
    hi = np.array(dims, np.float64) * res
    out = []
    for s in range(3):
        spread = synth.random_points(rng, 1500, (0.0, 0.0, 0.0), tuple(hi))
        spread = np.concatenate([spread, spread[::5] + np.float32(0.01 * res)])
        c = np.floor(hi / res / 2) * res
        cluster = synth.random_points(rng, 2500, tuple(c + 0.001),
                                      tuple(c + np.array([4, 4, 2]) * res - 0.001))
        pts_w = np.concatenate([spread, cluster]).astype(np.float32)
        Rm = synth.random_rotation(rng)
        t = hi / 2 + rng.uniform(3, -res, res)
        pts_s = ((pts_w.astype(np.float64) - t) @ Rm).astype(np.float32)
        out.append((pts_s, synth.make_pose(Rm, t)))
    return out


def _same(gpu, ora, label):
    m, s, h = gpu
    for name, x, y in (("mask", m, ora.mask), ("hits", h, ora.hits), ("sign", s, ora.sign)):
        if not np.array_equal(x, y):
            bad = np.argwhere(x != y)
            z, yy, xx = bad[0]
            raise AssertionError(f"{label}: {name} differs at {len(bad)} voxels, first "
                                 f"(x,y,z)=({xx},{yy},{z}): gpu={x[z, yy, xx]:#x} oracle={y[z, yy, xx]:#x}")


@pytest.mark.parametrize("seed", range(16))
def test_random_configuration_matches_oracle(orc, seed):
    import paper_2509_20081_gb300 as dbt
    pd, tuning, dims = _config(seed)
    res = 0.07
    scans = _scans(seed, dims, res, (pd["kernel_size"] - 1) // 2)
    og = orc.Grid.create(*dims, res, (0.0, 0.0, 0.0))
    po = orc.params(**pd)
    ostats = [orc.integrate_scan(og, po, p, pose) for p, pose in scans]
    label = f"case {seed}: {pd} {tuning} {dims}"

    k = dbt.Kernels(dbt.make_params(**pd))
    g = dbt.Grid(*dims, res)
    ws = dbt.Workspace(g, k, max(len(p) for p, _ in scans))
    ws.set_tuning(k, **tuning)
    xs = [torch.from_numpy(np.ascontiguousarray(p)).cuda() for p, _ in scans]
    for x, (_, pose), os_ in zip(xs, scans, ostats):
        dbt.dbt_integrate_scan(g, k, ws, x, pose)
        st = dbt.dbt_get_scan_stats(ws)
        assert st["error"] == 0, label
        for key in ("n_input", "n_valid", "n_inside", "n_kept"):
            assert st[key] == os_[key], (label, key, st, os_)
    _same(g.numpy(), og, label + " per-scan")

    gb = dbt.Grid(*dims, res)
    b = dbt.Batch([gb], k, sum(len(p) for p, _ in scans), len(scans))
    b.set_tuning(**tuning)
    b.set_items([(0, x, pose) for x, (_, pose) in zip(xs, scans)])
    b.run()
    per, tot = b.stats()
    assert tot["error"] == 0, label
    assert [it["n_kept"] for it in per] == [os_["n_kept"] for os_ in ostats], label
    _same(gb.numpy(), og, label + " batch")
    b.close()
