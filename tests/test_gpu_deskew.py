"""GPU parity of the update pre-steps through dbt_integrate_scan_ex:
sequential downsampling (Sec. IV-B) and motion compensation (Sec. III-C),
against the oracle's integrate_scan_ex, whole grids, bit for bit.  The
per-slice poses are the oracle's interpolation (inputs to both sides)."""
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


def _run(orc, pd, dims, res, scans):
    """scans: list of (pts, kw) with kw = dict(pose=..., poses=..., period=..., downsample=...)."""
    dbt = _dbt()
    k = dbt.Kernels(dbt.make_params(**pd))
    g = dbt.Grid(*dims, res)
    ws = dbt.Workspace(g, k, max(len(p) for p, _ in scans))
    og = orc.Grid.create(*dims, res)
    po = orc.params(**pd)
    for pts, kw in scans:
        x = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
        dbt.dbt_integrate_scan_ex(g, k, ws, x, **kw)
        gs = dbt.dbt_get_scan_stats(ws)
        poses = kw.get("poses")
        if poses is None:
            poses = [kw["pose"]]
        os_ = orc.integrate_scan_ex(og, po, pts, poses, period=kw.get("period"),
                                    downsample=kw.get("downsample", 1))
        for key in ("n_input", "n_valid", "n_inside", "n_kept"):
            assert gs[key] == os_[key], (key, gs, os_)
        assert gs["error"] == 0
    m, s, h = g.numpy()
    np.testing.assert_array_equal(m, og.mask)
    np.testing.assert_array_equal(h, og.hits)
    np.testing.assert_array_equal(s, og.sign)
    return os_


@pytest.mark.parametrize("ds", [1, 2, 3, 5])
def test_downsampling_room(orc, ds):
    w = synth.room_scan(n_scans=2)
    scans = [(pts, dict(pose=pose, downsample=ds)) for pts, pose in w.scans]
    st = _run(orc, w.params, (128, 128, 128), 0.1, scans)
    assert st["n_kept"] > 0


@pytest.fixture(scope="module")
def moving():
    """A sensor moving along the urban trajectory at a quarter of the map's
    size: scan k sweeps from pose k to pose k + 1 (beam-major returns, so the
    time runs with the azimuth column: period = width)."""
    return synth.urban_sequence(n_scans=4, scale=0.25, beams=32, width=512)


@pytest.mark.parametrize("mode,n_poses,ds", [(0, 64, 1), (1, 64, 1), (0, 256, 2), (1, 7, 3),
                                             (0, 1, 1)])
def test_motion_compensation_urban_quarter(orc, moving, mode, n_poses, ds):
    w = moving
    scans = []
    for i in range(len(w.scans) - 1):
        pts, T0 = w.scans[i]
        T1 = w.scans[i + 1][1]
        poses = orc.pose_ramp(T0, T1, n_poses, mode)
        scans.append((pts, dict(poses=poses, period=512, downsample=ds)))
    st = _run(orc, w.params, (w.grid.nx, w.grid.ny, w.grid.nz), w.grid.res, scans)
    assert st["n_kept"] > 1000


def test_ex_without_options_is_the_plain_update(orc):
    dbt = _dbt()
    w = synth.room_scan(n_scans=1)
    pts, pose = w.scans[0]
    k = dbt.Kernels(dbt.make_params(**w.params))
    a, b = dbt.Grid(128, 128, 128, 0.1), dbt.Grid(128, 128, 128, 0.1)
    wa, wb = dbt.Workspace(a, k, len(pts)), dbt.Workspace(b, k, len(pts))
    x = torch.from_numpy(pts).cuda()
    dbt.dbt_integrate_scan(a, k, wa, x, pose)
    dbt.dbt_integrate_scan_ex(b, k, wb, x, pose=pose, downsample=1)
    for u, v in zip(a.numpy(), b.numpy()):
        np.testing.assert_array_equal(u, v)


def test_ex_argument_errors(orc):
    dbt = _dbt()
    B = dbt.dbtsdf
    k = dbt.Kernels(dbt.make_params())
    g = dbt.Grid(64, 64, 64, 0.1)
    ws = dbt.Workspace(g, k, 100)
    x = torch.zeros((100, 3), device="cuda")
    T = synth.make_pose(np.eye(3), (3.2, 3.2, 3.2))
    bad = T.copy()
    bad[1, 1] = 3.0
    for kw in [dict(pose=T, downsample=0), dict(poses=[T] * 257, period=10),
               dict(poses=[T, bad], period=10), dict(poses=[T], period=-1)]:
        with pytest.raises(B.DbtError) as e:
            dbt.dbt_integrate_scan_ex(g, k, ws, x, **kw)
        assert e.value.status == B.DBT_EINVAL
