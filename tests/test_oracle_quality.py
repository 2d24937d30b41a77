"""Pins of the oracle's reconstruction-quality metrics (Sec. IV-B: accuracy,
completeness, Chamfer-L1, recall, F-score at a tolerance): closed forms on
lattices, special cases, and nearest-neighbour distances against an
independent library routine (scipy's k-d tree)."""
import numpy as np
import pytest

import synth


def _lattice(n, step=0.1, z=0.0):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([i.ravel() * step, j.ravel() * step, np.full(n * n, z)], 1).astype(np.float32)


def test_identical_sets(orc):
    p = _lattice(20)
    q = orc.quality(p, p, 0.05)
    assert q == {"accuracy": 0.0, "completeness": 0.0, "chamfer_l1": 0.0, "precision": 1.0,
                 "recall": 1.0, "fscore": 1.0}


@pytest.mark.parametrize("delta,t", [(0.02, 0.05), (0.03, 0.025)])
def test_offset_plane_closed_form(orc, delta, t):
    """The same lattice lifted by delta (< half the lattice step): every
    nearest neighbour is the point straight above or below, so accuracy =
    completeness = Chamfer-L1 = delta, and P = R = F = [delta < t]."""
    gt = _lattice(15, step=0.1)
    pred = _lattice(15, step=0.1, z=delta)
    q = orc.quality(pred, gt, t)
    d = float(np.float32(delta))
    for k in ("accuracy", "completeness", "chamfer_l1"):
        assert abs(q[k] - d) < 1e-9
    want = 1.0 if delta < t else 0.0
    assert q["precision"] == q["recall"] == q["fscore"] == want


def test_half_of_the_reference(orc):
    """Predicting every other reference point: accuracy 0 and precision 1;
    each missing point is one lattice step from a kept one, so completeness
    is step / 2 and recall 1/2 below a tolerance of one step."""
    gt = _lattice(10, step=0.2)
    pred = gt[::2]
    q = orc.quality(pred, gt, 0.1)
    assert q["accuracy"] == 0.0 and q["precision"] == 1.0
    assert abs(q["completeness"] - 0.1) < 1e-7
    assert q["recall"] == 0.5
    assert abs(q["fscore"] - 2 * 0.5 / 1.5) < 1e-12


def test_f_is_harmonic_mean_and_empty_sets(orc):
    q = orc.quality_from_distances([0.0, 0.2, 0.3, 0.01], [0.0, 0.5], 0.1)
    assert q["precision"] == 0.5 and q["recall"] == 0.5 and q["fscore"] == 0.5
    assert abs(q["accuracy"] - 0.51 / 4) < 1e-15 and q["completeness"] == 0.25
    z = orc.quality_from_distances([], [], 0.1)
    assert z["fscore"] == 0.0 and z["accuracy"] == 0.0


@pytest.mark.parametrize("seed", [1, 2])
def test_nn_matches_kdtree(orc, seed):
    """The brute-force distances equal a k-d tree's (scipy, an independent
    implementation) on surface-like random sets."""
    kd = pytest.importorskip("scipy.spatial")
    rng = synth.Rng(900 + seed)
    ref = synth.point_cloud(rng, 3000, 10.0, 0.02)
    q = synth.point_cloud(rng, 2000, 10.0, 0.05)
    d = orc.nn_distances(ref, q)
    dk, _ = kd.cKDTree(ref.astype(np.float64)).query(q.astype(np.float64))
    np.testing.assert_allclose(d, dk, rtol=1e-12, atol=1e-12)
