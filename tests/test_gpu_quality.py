"""GPU parity of the reconstruction-quality metrics (Sec. IV-B) through the
C ABI against the oracle: nearest-neighbour distances (binary32 on the GPU,
binary64 in the oracle: equal within a few float ulps of the coordinates)
and the metrics computed from them, on seeded surface-like point sets; and
the full chain integrate -> mesh -> metrics on a quarter-size urban map,
its distances checked on a sample."""
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


def _tol(extent):
    """Distance tolerance: the coordinates are float32 (ulp <= extent * 2^-23),
    three subtractions, squares and a sum and a root in binary32 against
    binary64: a few ulps of the coordinates."""
    return 8 * extent * 2.0 ** -23


@pytest.mark.parametrize("n_ref,n_q,extent,seed", [(5000, 3000, 10.0, 1), (20000, 20000, 80.0, 2),
                                                    (1, 500, 5.0, 3), (700, 1, 5.0, 4),
                                                    (30000, 4000, 1.0, 5)])
def test_nn_distances_match_oracle(orc, n_ref, n_q, extent, seed):
    rng = synth.Rng(700 + seed)
    ref = synth.point_cloud(rng, n_ref, extent, 0.003 * extent)
    q = synth.point_cloud(rng, n_q, extent, 0.02 * extent)
    d = _dbt().dbt_nn_distances(torch.from_numpy(ref).cuda(), torch.from_numpy(q).cuda()).cpu().numpy()
    want = orc.nn_distances(ref, q)
    np.testing.assert_allclose(d, want, rtol=0, atol=_tol(extent))


def test_nn_degenerate_sets(orc):
    dbt = _dbt()
    q = torch.from_numpy(synth.point_cloud(synth.Rng(5), 100, 3.0, 0.1)).cuda()
    empty = torch.zeros((0, 3), device="cuda")
    assert torch.isinf(dbt.dbt_nn_distances(empty, q)).all()
    assert dbt.dbt_nn_distances(q, empty).numel() == 0
    same = dbt.dbt_nn_distances(q, q)
    assert (same == 0).all()
    # all points on one plane, one line, one point: degenerate boxes
    p = np.zeros((200, 3), np.float32)
    p[:, 0] = np.linspace(0, 1, 200)
    r = np.array([[0.3, 0.0, 0.0], [0.31, 0.0, 0.0]], np.float32)
    d = dbt.dbt_nn_distances(torch.from_numpy(r).cuda(), torch.from_numpy(p).cuda()).cpu().numpy()
    np.testing.assert_allclose(d, orc.nn_distances(r, p), atol=_tol(1.0))


@pytest.mark.parametrize("tol", [0.05, 0.1, 0.2])
def test_quality_metrics_match_oracle(orc, tol):
    rng = synth.Rng(41)
    gt = synth.point_cloud(rng, 20000, 12.0, 0.0)
    pred = synth.point_cloud(synth.Rng(41), 20000, 12.0, 0.0)          # same planes...
    pred = (pred + np.asarray(synth.Rng(9).normal(3 * 20000, 0.05), np.float32).reshape(-1, 3))
    got = _dbt().dbt_quality_metrics(torch.from_numpy(pred).cuda(), torch.from_numpy(gt).cuda(), tol)
    want = orc.quality(pred, gt, tol)
    for k in ("accuracy", "completeness", "chamfer_l1"):
        assert abs(got[k] - want[k]) <= 1e-6 * max(1.0, want[k]), (k, got[k], want[k])
    # fractions: points within a float rounding of the tolerance may fall either way
    dp = orc.nn_distances(gt, pred)
    dg = orc.nn_distances(pred, gt)
    edge_p = np.mean(np.abs(dp - tol) < _tol(12.0))
    edge_g = np.mean(np.abs(dg - tol) < _tol(12.0))
    assert abs(got["precision"] - want["precision"]) <= edge_p + 1e-12
    assert abs(got["recall"] - want["recall"]) <= edge_g + 1e-12
    assert got["n_pred"] == 20000 and got["n_gt"] == 20000
    again = _dbt().dbt_quality_metrics(torch.from_numpy(pred).cuda(), torch.from_numpy(gt).cuda(), tol)
    assert again == got                                                   # deterministic


def test_mesh_centroids(orc):
    dbt = _dbt()
    tri = synth.Rng(3).uniform(9 * 1000, -5, 5).astype(np.float32).reshape(-1, 3, 3)
    c = dbt.dbt_mesh_centroids(torch.from_numpy(tri).cuda()).cpu().numpy()
    want = ((tri[:, 0] + tri[:, 1]) + tri[:, 2]) / np.float32(3.0)
    np.testing.assert_array_equal(c, want.astype(np.float32))


def test_quality_chain_urban_quarter(orc):
    """Integrate a quarter-size urban sequence, mesh it at iso 0, and score
    the mesh centroids against the noise-free surface points of the same
    rays: sampled distances against the oracle, and sane metric values."""
    dbt = _dbt()
    w = synth.urban_sequence(n_scans=6, scale=0.25)
    truth = synth.urban_sequence(n_scans=6, scale=0.25, truth=True)
    k = dbt.Kernels(dbt.make_params(**w.params))
    g = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
    ws = dbt.Workspace(g, k, max(len(p) for p, _ in w.scans))
    for pts, pose in w.scans:
        dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).cuda(), pose)
    tri, _ = dbt.dbt_mesh_extract(g)
    pred = dbt.dbt_mesh_centroids(tri)
    gt = torch.from_numpy(np.concatenate([p for p, _ in truth.scans])).cuda()
    q = dbt.dbt_quality_metrics(pred, gt, 0.1)
    assert q["n_pred"] > 10000 and q["n_gt"] > 100000
    assert 0 < q["accuracy"] < 0.2 and 0 < q["completeness"] < 0.5
    assert 0.5 < q["recall"] <= 1 and 0.5 < q["precision"] <= 1
    # sampled distances against the oracle's brute force
    d = dbt.dbt_nn_distances(gt, pred).cpu().numpy()
    idx = synth.Rng(5).integers(300, 0, len(d))
    p_host = pred.cpu().numpy()[idx]
    want = orc.nn_distances(gt.cpu().numpy(), p_host)
    np.testing.assert_allclose(d[idx], want, atol=_tol(20.0))
