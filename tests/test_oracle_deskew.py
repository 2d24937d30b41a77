"""Pins of the oracle's update pre-steps: sequential downsampling (Sec. IV-B,
DS) and motion compensation (Sec. III-C: each return transformed with the
pose of its time slice; yaw-only or full rotation interpolation)."""
import math

import numpy as np
import pytest

import synth


def _scan(n=3000, seed=5, side=48, res=0.1):
    rng = synth.Rng(seed)
    pts = synth.random_points(rng, n, (-2.0, -2.0, -1.0), (2.0, 2.0, 1.0))
    return pts, side, res


def _pose(R, t):
    return synth.make_pose(R, t)


def _grids_equal(a, b):
    np.testing.assert_array_equal(a.mask, b.mask)
    np.testing.assert_array_equal(a.sign, b.sign)
    np.testing.assert_array_equal(a.hits, b.hits)


@pytest.mark.parametrize("ds", [1, 2, 3, 7])
def test_downsampling_is_every_ds_th_return(orc, ds):
    """DS keeps the returns whose index is a multiple of ds: the same as the
    plain update of that subsequence (first-return rule among the kept)."""
    pts, side, res = _scan()
    pts = np.concatenate([pts, pts[:500]])           # repeated voxels: first-return rule at work
    p = orc.params(kernel_size=7, shadow_radius=2.0)
    pose = _pose(synth.rotation_rpy(0.2, 0.1, -0.4), (2.4, 2.4, 2.4))
    a = orc.Grid.create(side, side, side, res)
    sa = orc.integrate_scan_ex(a, p, pts, [pose], downsample=ds)
    b = orc.Grid.create(side, side, side, res)
    sb = orc.integrate_scan(b, p, pts[::ds], pose)
    _grids_equal(a, b)
    assert sa["n_kept"] == sb["n_kept"] and sa["n_valid"] == sb["n_valid"]


def test_one_pose_per_slice_equals_returns_one_by_one(orc):
    """Without the first-return rule the update is order independent, so a
    motion-compensated scan equals its returns integrated one at a time,
    each with the pose of its slice m(i) = ((i mod period) * M) // period."""
    pts, side, res = _scan(n=1200)
    p = orc.params(kernel_size=5, shadow_radius=2.0, dedup_first=0)
    M, period = 7, 100
    poses = [_pose(synth.rotation_rpy(0.01 * k, -0.02 * k, 0.05 * k), (2.4 + 0.03 * k, 2.4, 2.4))
             for k in range(M)]
    a = orc.Grid.create(side, side, side, res)
    orc.integrate_scan_ex(a, p, pts, poses, period=period)
    b = orc.Grid.create(side, side, side, res)
    for i in range(len(pts)):
        orc.integrate_scan(b, p, pts[i:i + 1], poses[((i % period) * M) // period])
    _grids_equal(a, b)


def test_equal_poses_are_the_single_pose_update(orc):
    pts, side, res = _scan()
    p = orc.params(kernel_size=7, shadow_radius=3.0)
    pose = _pose(synth.rotation_rpy(-0.3, 0.2, 1.0), (2.4, 2.3, 2.5))
    a = orc.Grid.create(side, side, side, res)
    orc.integrate_scan_ex(a, p, pts, [pose] * 5, period=37)
    b = orc.Grid.create(side, side, side, res)
    orc.integrate_scan(b, p, pts, pose)
    _grids_equal(a, b)


# ------------------------------------------------------------------ pose interpolation
def _rot_angle(R):
    return math.acos(max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0)))


POSES = [
    (synth.rotation_rpy(0.0, 0.0, 0.0), synth.rotation_rpy(0.1, -0.2, 0.7)),
    (synth.rotation_rpy(0.3, 0.1, -2.0), synth.rotation_rpy(0.25, 0.12, -1.6)),
    (synth.rotation_rpy(-0.1, 0.05, 3.0), synth.rotation_rpy(-0.1, 0.05, -3.0)),   # yaw wraps
    (synth.rotation_rpy(0.2, 0.2, 0.2), synth.rotation_rpy(0.2, 0.2, 0.2)),        # no motion
]


@pytest.mark.parametrize("k", range(len(POSES)))
@pytest.mark.parametrize("mode", [0, 1])
def test_interp_endpoints_and_rotations(orc, k, mode):
    R0, R1 = POSES[k]
    T0, T1 = _pose(R0, (1.0, -2.0, 0.5)), _pose(R1, (1.4, -1.5, 0.6))
    np.testing.assert_allclose(orc.pose_interp(T0, T1, 0.0, mode), T0.reshape(3, 4), atol=1e-15)
    for tau in (0.0, 0.25, 0.5, 0.9, 1.0):
        Q = orc.pose_interp(T0, T1, tau, mode)
        R = Q[:, :3]
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) > 0
        np.testing.assert_allclose(Q[:, 3], (1.0 + 0.4 * tau, -2.0 + 0.5 * tau, 0.5 + 0.1 * tau),
                                   atol=1e-15)
    if mode == 0:
        np.testing.assert_allclose(orc.pose_interp(T0, T1, 1.0, 0), T1.reshape(3, 4), atol=1e-12)


@pytest.mark.parametrize("k", range(3))
def test_full_interp_constant_angular_rate(orc, k):
    """Full mode: the rotation from R0 grows linearly with tau about one axis
    (geodesic): angle(R0^T R(tau)) = tau angle(R0^T R1), and the half-way
    pose is the same from either end."""
    R0, R1 = POSES[k]
    T0, T1 = _pose(R0, (0, 0, 0)), _pose(R1, (0, 0, 0))
    th = _rot_angle(R0.T @ R1)
    for tau in (0.1, 0.3, 0.5, 0.8):
        R = orc.pose_interp(T0, T1, tau, 0)[:, :3]
        assert abs(_rot_angle(R0.T @ R) - tau * th) < 1e-12
    np.testing.assert_allclose(orc.pose_interp(T0, T1, 0.5, 0), orc.pose_interp(T1, T0, 0.5, 0),
                               atol=1e-12)


@pytest.mark.parametrize("k", range(3))
def test_yaw_interp_turns_about_map_z_only(orc, k):
    """Yaw-only: R(tau) R0^T is a rotation about the map's z axis by
    tau * dpsi, dpsi the wrapped yaw difference (closed form cos / sin)."""
    R0, R1 = POSES[k]
    T0, T1 = _pose(R0, (0, 0, 0)), _pose(R1, (0, 0, 0))
    dpsi = math.atan2(R1[1, 0], R1[0, 0]) - math.atan2(R0[1, 0], R0[0, 0])
    dpsi = (dpsi + math.pi) % (2 * math.pi) - math.pi
    assert abs(dpsi) <= math.pi
    for tau in (0.2, 0.5, 1.0):
        R = orc.pose_interp(T0, T1, tau, 1)[:, :3]
        a = tau * dpsi
        Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
        np.testing.assert_allclose(R @ R0.T, Rz, atol=1e-12)


def test_pure_yaw_motion_both_modes_agree(orc):
    """A sweep that only turns about z: full and yaw-only interpolation give
    the same poses."""
    R0, R1 = synth.rotation_rpy(0, 0, 0.4), synth.rotation_rpy(0, 0, 0.9)
    T0, T1 = _pose(R0, (3, 1, 0)), _pose(R1, (3.5, 1.2, 0))
    for tau in (0.0, 0.3, 0.7, 1.0):
        np.testing.assert_allclose(orc.pose_interp(T0, T1, tau, 0), orc.pose_interp(T0, T1, tau, 1),
                                   atol=1e-12)


def test_half_turn_axis(orc):
    """Near a half turn the axis comes from the symmetric part: a rotation of
    pi about x is reached at tau = 1 and passes through pi/2 about x."""
    T0 = _pose(np.eye(3), (0, 0, 0))
    Rx = np.diag([1.0, -1.0, -1.0])
    T1 = _pose(Rx, (0, 0, 0))
    np.testing.assert_allclose(orc.pose_interp(T0, T1, 1.0, 0)[:, :3], Rx, atol=1e-12)
    R = orc.pose_interp(T0, T1, 0.5, 0)[:, :3]
    np.testing.assert_allclose(np.abs(R), np.array([[1, 0, 0], [0, 0, 1], [0, 1, 0]]), atol=1e-12)
