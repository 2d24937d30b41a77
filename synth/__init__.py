"""Seeded synthetic LiDAR workloads (inputs only; none of the method's arithmetic).

This module is the one source of inputs shared by the oracle tests, the CUDA
parity tests and ``bench.py``.  It builds scenes (box room, urban block),
trajectories and spinning-LiDAR scans by analytic ray casting.  It never
quantises, bins or integrates anything: it only produces float32 returns in
the sensor frame and float64 SE(3) poses.

Random numbers come from a counter-based SplitMix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) with uniform
doubles from the top 53 bits and normals by Box-Muller, so a seed gives the
same scan on every machine and numpy version.

Workloads (the stand-in for the paper's Newer College / Mai City datasets,
which are not available here):
  * ``room_scan``      box room 12.8 m cube, 16 x 900 scan, +-15 deg, 0.5-12 m
  * ``urban_sequence`` urban block (ground, 40 buildings, 200 poles),
                       64 x 1024 scans, +-22.5 deg, 1-60 m, 1 m per scan
  * ``batched_maps``   uneven maps each with a few room scans

Map states for the export path (signed-distance field, Marching Cubes) are
given directly, voxel by voxel, as a distance in whole voxels and an
occupancy flag (``map_state``): a sphere, a stepped terrain with boxes, and
random states.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2509200810
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream: draw k returns mix(seed + (c+1..c+k) * golden)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.seed + idx * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def log_uniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.exp(self.uniform(n, math.log(lo), math.log(hi)))

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi)."""
        return lo + np.floor(self.uniform(n) * (hi - lo)).astype(np.int64)


# ---------------------------------------------------------------- scenes
@dataclass
class Scene:
    """Analytic scene: horizontal planes, inward walls, boxes, vertical cylinders."""
    ground_z: float | None = None                 # infinite floor plane z = ground_z
    walls: tuple | None = None                     # (x0, x1, y0, y1, z_top) inner faces
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))   # x0 y0 z0 x1 y1 z1
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))  # cx cy r z0 z1


def room_scene(rng: Rng, extent: float = 12.8, sensor=(6.4, 6.4, 6.4), n_boxes: int = 6) -> Scene:
    """Box room: floor at 3/8 of the height, 4 walls up to 3/4, no ceiling,
    n_boxes axis-aligned boxes on the floor at least 1/12.8 of the extent
    (1 m at 12.8 m) away from the sensor.  Lengths scale with ``extent``."""
    s = extent / 12.8
    x0, x1 = 0.8 * s, 12.0 * s
    floor = 4.8 * s
    top = 9.6 * s
    boxes = []
    while len(boxes) < n_boxes:
        sx, sy, sz = rng.uniform(3, 0.3 * s, 2.0 * s)
        cx, cy = rng.uniform(2, x0 + 0.2 * s, x1 - 0.2 * s)
        bx0, bx1 = cx - sx / 2, cx + sx / 2
        by0, by1 = cy - sy / 2, cy + sy / 2
        if bx0 < x0 or bx1 > x1 or by0 < x0 or by1 > x1:
            continue
        # horizontal distance from sensor to the box footprint
        dx = max(bx0 - sensor[0], 0.0, sensor[0] - bx1)
        dy = max(by0 - sensor[1], 0.0, sensor[1] - by1)
        if math.hypot(dx, dy) < 1.0 * s:
            continue
        boxes.append((bx0, by0, floor, bx1, by1, floor + sz))
    return Scene(ground_z=floor, walls=(x0, x1, x0, x1, top), boxes=np.array(boxes))


def closed_path(t: np.ndarray, centre, radius: float):
    """Smooth closed curve (Lissajous-like) of the given radius around centre."""
    cx, cy = centre
    x = cx + radius * np.cos(t)
    y = cy + 0.88 * radius * np.sin(t) + 0.12 * radius * np.sin(2.0 * t)
    return x, y


def urban_scene(rng: Rng, extent: float = 80.0, height: float = 16.0, ground: float = 1.0,
                n_buildings: int = 40, n_poles: int = 200, path_radius: float = 25.0,
                corridor: float = 6.0, scale: float = 1.0) -> Scene:
    """Ground plane, box buildings (footprint 4-15 m, height 3-14 m) clear of a
    ``corridor`` around the closed path, and vertical poles (r 0.1-0.4 m,
    height 2-6 m) at least 1 m off the path; every length times ``scale``."""
    centre = (extent / 2.0, extent / 2.0)
    tt = np.linspace(0.0, 2.0 * np.pi, 2000, endpoint=False)
    px, py = closed_path(tt, centre, path_radius)
    margin = 1.0 * scale

    def path_dist_box(x0, y0, x1, y1):
        dx = np.maximum(np.maximum(x0 - px, 0.0), px - x1)
        dy = np.maximum(np.maximum(y0 - py, 0.0), py - y1)
        return float(np.min(np.hypot(dx, dy)))

    boxes = []
    tries = 0
    while len(boxes) < n_buildings and tries < 100000:
        tries += 1
        fx, fy = rng.uniform(2, 4.0 * scale, 15.0 * scale)
        h = float(rng.uniform(1, 3.0 * scale, 14.0 * scale)[0])
        cx, cy = rng.uniform(2, margin + fx / 2, extent - margin - fx / 2)
        x0, x1, y0, y1 = cx - fx / 2, cx + fx / 2, cy - fy / 2, cy + fy / 2
        if x0 < margin or y0 < margin or x1 > extent - margin or y1 > extent - margin:
            continue
        if path_dist_box(x0, y0, x1, y1) < corridor * scale:
            continue
        boxes.append((x0, y0, ground, x1, y1, min(ground + h, height - margin)))
    cyl = []
    tries = 0
    while len(cyl) < n_poles and tries < 100000:
        tries += 1
        r = float(rng.uniform(1, 0.1 * scale, 0.4 * scale)[0])
        h = float(rng.uniform(1, 2.0 * scale, 6.0 * scale)[0])
        cx, cy = rng.uniform(2, margin, extent - margin)
        if float(np.min(np.hypot(px - cx, py - cy))) < r + 1.0 * scale:
            continue
        cyl.append((cx, cy, r, ground, ground + h))
    return Scene(ground_z=ground, walls=None, boxes=np.array(boxes), cylinders=np.array(cyl))


# ---------------------------------------------------------------- ray casting
def _raycast(scene: Scene, origin: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Nearest positive hit distance along unit rays (inf = no hit)."""
    n = dirs.shape[0]
    best = np.full(n, np.inf)
    ox, oy, oz = origin
    dx, dy, dz = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        if scene.ground_z is not None:
            t = (scene.ground_z - oz) / dz
            ok = (dz < 0) & (t > 0)
            best = np.where(ok & (t < best), t, best)
        if scene.walls is not None:
            x0, x1, y0, y1, top = scene.walls
            for (plane, comp, o, sgn) in ((x0, dx, ox, -1), (x1, dx, ox, 1),
                                          (y0, dy, oy, -1), (y1, dy, oy, 1)):
                t = (plane - o) / comp
                ok = (sgn * comp > 0) & (t > 0)
                z = oz + t * dz
                ok &= z <= top
                if scene.ground_z is not None:
                    ok &= z >= scene.ground_z
                best = np.where(ok & (t < best), t, best)
        if scene.boxes.shape[0]:
            inv = 1.0 / np.where(dirs == 0.0, 1e-300, dirs)           # (n, 3)
            lo = (scene.boxes[None, :, 0:3] - origin) * inv[:, None, :]  # (n, B, 3)
            hi = (scene.boxes[None, :, 3:6] - origin) * inv[:, None, :]
            tn = np.max(np.minimum(lo, hi), axis=2)
            tf = np.min(np.maximum(lo, hi), axis=2)
            tn = np.where((tn <= tf) & (tn > 0), tn, np.inf)
            best = np.minimum(best, tn.min(axis=1))
        if scene.cylinders.shape[0]:
            c = scene.cylinders
            a = (dx * dx + dy * dy)[:, None]
            fx = (ox - c[:, 0])[None, :]
            fy = (oy - c[:, 1])[None, :]
            bb = 2.0 * (fx * dx[:, None] + fy * dy[:, None])
            cc = fx * fx + fy * fy - (c[:, 2] * c[:, 2])[None, :]
            disc = bb * bb - 4.0 * a * cc
            t = (-bb - np.sqrt(np.maximum(disc, 0.0))) / (2.0 * a)
            z = oz + t * dz[:, None]
            ok = (disc >= 0) & (a > 0) & (t > 0) & (z >= c[None, :, 3]) & (z <= c[None, :, 4])
            best = np.minimum(best, np.where(ok, t, np.inf).min(axis=1))
            tc = (c[None, :, 4] - oz) / dz[:, None]
            hx = ox + tc * dx[:, None] - c[None, :, 0]
            hy = oy + tc * dy[:, None] - c[None, :, 1]
            okc = (dz[:, None] < 0) & (tc > 0) & (hx * hx + hy * hy <= (c[:, 2] * c[:, 2])[None, :])
            best = np.minimum(best, np.where(okc, tc, np.inf).min(axis=1))
    return best


def _sector_masks(scene: Scene, origin: np.ndarray, nsec: int):
    """Per azimuth sector, the boxes and cylinders whose bounding circle (seen
    from the sensor) overlaps the sector, with a one-sector margin."""
    out = []
    width = 2.0 * np.pi / nsec

    def spans(cx, cy, rad):
        dx, dy = cx - origin[0], cy - origin[1]
        d = np.hypot(dx, dy)
        ang = np.arctan2(dy, dx) % (2.0 * np.pi)
        half = np.where(d > rad, np.arcsin(np.minimum(1.0, rad / np.maximum(d, 1e-12))), np.pi)
        return ang, half + width

    b = scene.boxes
    if b.shape[0]:
        bang, bhalf = spans((b[:, 0] + b[:, 3]) / 2, (b[:, 1] + b[:, 4]) / 2,
                            0.5 * np.hypot(b[:, 3] - b[:, 0], b[:, 4] - b[:, 1]))
    c = scene.cylinders
    if c.shape[0]:
        cang, chalf = spans(c[:, 0], c[:, 1], c[:, 2])
    for k in range(nsec):
        mid = (k + 0.5) * width

        def near(ang, half):
            dd = np.abs((ang - mid + np.pi) % (2.0 * np.pi) - np.pi)
            return dd <= half + width / 2

        bsel = near(bang, bhalf) if b.shape[0] else np.zeros(0, bool)
        csel = near(cang, chalf) if c.shape[0] else np.zeros(0, bool)
        out.append((bsel, csel))
    return out


def rotation_rpy(roll: float, pitch: float, yaw: float) -> np.ndarray:
    """R = Rz(yaw) Ry(pitch) Rx(roll)."""
    cr, sr = math.cos(roll), math.sin(roll)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cy, sy = math.cos(yaw), math.sin(yaw)
    Rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1]])
    Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
    Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return Rz @ Ry @ Rx


def make_pose(R: np.ndarray, t) -> np.ndarray:
    """Row-major 3x4 [R | t] float64."""
    P = np.zeros((3, 4))
    P[:, :3] = R
    P[:, 3] = t
    return P


def lidar_scan(scene: Scene, pose: np.ndarray, beams: int, width: int, fov_deg: float,
               rmin: float, rmax: float, sigma: float, dropout: float, rng: Rng,
               chunk: int = 4096, truth: bool = False) -> np.ndarray:
    """Spinning LiDAR: ``beams`` elevations in [-fov/2, +fov/2], ``width``
    azimuths k 2 pi / width; returns (beams * width, 3) float32 in the sensor
    frame, beam-major; misses, out-of-range and dropped returns are NaN."""
    el = np.deg2rad(np.linspace(-fov_deg / 2.0, fov_deg / 2.0, beams))
    az = np.arange(width) * (2.0 * np.pi / width)
    E, A = np.meshgrid(el, az, indexing="ij")
    ds = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    R = pose[:, :3]
    origin = pose[:, 3]
    dw = ds @ R.T
    n = ds.shape[0]
    t = np.full(n, np.inf)
    # cull boxes and poles per world-azimuth sector: each is tested only on
    # the rays whose azimuth falls within its angular extent seen from the sensor
    nsec = 64
    az_w = np.arctan2(dw[:, 1], dw[:, 0]) % (2.0 * np.pi)
    sec = np.minimum((az_w * (nsec / (2.0 * np.pi))).astype(np.int64), nsec - 1)
    order = np.argsort(sec, kind="stable")
    bounds = np.searchsorted(sec[order], np.arange(nsec + 1))
    prim_sectors = _sector_masks(scene, origin, nsec)
    for k in range(nsec):
        idx = order[bounds[k]:bounds[k + 1]]
        if idx.size == 0:
            continue
        bsel, csel = prim_sectors[k]
        sub = Scene(scene.ground_z, scene.walls, scene.boxes[bsel], scene.cylinders[csel])
        for c0 in range(0, idx.size, chunk):
            j = idx[c0:c0 + chunk]
            t[j] = _raycast(sub, origin, dw[j])
    noise = rng.normal(n, sigma)
    drop = rng.uniform(n) < dropout
    if truth:
        # the exact surface points hit by the same rays, in the map frame
        # (the draws above are still taken, so later scans stay the same)
        ok = np.isfinite(t) & (t >= rmin) & (t <= rmax)
        return (origin + dw[ok] * t[ok, None]).astype(np.float32)
    t = t + noise
    bad = ~np.isfinite(t) | (t < rmin) | (t > rmax) | drop
    with np.errstate(invalid="ignore"):
        pts = ds * t[:, None]
    pts[bad] = np.nan
    return pts.astype(np.float32)


# ---------------------------------------------------------------- workloads
@dataclass
class GridSpec:
    nx: int
    ny: int
    nz: int
    res: float
    origin: tuple = (0.0, 0.0, 0.0)


@dataclass
class Workload:
    name: str
    grid: GridSpec
    scans: list           # list of (points float32 (n,3), pose float64 (3,4))
    params: dict          # kernel_size, scheme, bins_a, bins_b, shadow_radius, ...


DEFAULT_PARAMS = dict(kernel_size=11, scheme=0, bins_a=8, bins_b=8, shadow_radius=3.0,
                      hit_threshold=3, hit_max=255, dedup_first=1)


def room_scan(seed_offset: int = 0, side: int = 128, res: float = 0.10, beams: int = 16,
              width: int = 900, sigma: float = 0.01, n_scans: int = 1) -> Workload:
    """Single-scan room workload: side^3 grid at res, sensor at the centre,
    identity pose, 16 x 900 returns, +-15 deg, 0.5-12 m (scaled with the room)."""
    rng = Rng(BASE_SEED + seed_offset)
    extent = side * res
    c = extent / 2.0
    scene = room_scene(rng, extent=extent, sensor=(c, c, c))
    scans = []
    for k in range(n_scans):
        # later scans (if any) jitter the sensor a little inside the room
        off = np.zeros(3) if k == 0 else rng.uniform(3, -0.05 * extent, 0.05 * extent)
        pose = make_pose(np.eye(3) if k == 0 else rotation_rpy(0.0, 0.0, float(rng.uniform(1, 0, 6.283)[0])),
                         np.array([c, c, c]) + off)
        scale = extent / 12.8
        pts = lidar_scan(scene, pose, beams, width, 30.0, 0.5 * scale, 12.0 * scale, sigma, 0.0, rng)
        scans.append((pts, pose))
    return Workload("room", GridSpec(side, side, side, res), scans, dict(DEFAULT_PARAMS))


def urban_sequence(n_scans: int = 100, seed_offset: int = 1, scale: float = 1.0,
                   res: float = 0.05, beams: int = 64, width: int = 1024,
                   rmax: float = 60.0, truth: bool = False) -> Workload:
    """Urban sequence: grid (80x80x16 m) * scale at res; poses every 1 m * scale
    along a closed path of radius 25 m * scale, yaw along the tangent with
    +-3 deg roll/pitch sinusoids; 2 cm * scale range noise; 2 % dropouts.
    truth: each scan is instead the noise-free surface points its rays hit,
    in the map frame, without dropouts (the reference surface the quality
    metrics compare against)."""
    rng = Rng(BASE_SEED + seed_offset)
    extent, height, ground = 80.0 * scale, 16.0 * scale, 1.0 * scale
    scene = urban_scene(rng, extent=extent, height=height, ground=ground,
                        path_radius=25.0 * scale, scale=scale)
    nx = int(round(extent / res))
    nz = int(round(height / res))
    centre = (extent / 2.0, extent / 2.0)
    # arc-length sampling of the path every 1 m * scale
    tt = np.linspace(0.0, 2.0 * np.pi, 20001)
    x, y = closed_path(tt, centre, 25.0 * scale)
    seg = np.hypot(np.diff(x), np.diff(y))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    scans = []
    for k in range(n_scans):
        sk = (k * 1.0 * scale) % s[-1]
        i = int(np.searchsorted(s, sk))
        i = min(max(i, 1), len(tt) - 1)
        yaw = math.atan2(y[i] - y[i - 1], x[i] - x[i - 1])
        roll = math.radians(3.0) * math.sin(0.31 * k)
        pitch = math.radians(3.0) * math.sin(0.17 * k + 1.0)
        pose = make_pose(rotation_rpy(roll, pitch, yaw), (x[i], y[i], ground + 1.8 * scale))
        pts = lidar_scan(scene, pose, beams, width, 45.0, 1.0 * scale, rmax, 0.02 * scale,
                         0.02, rng, truth=truth)
        scans.append((pts, pose))
    return Workload("urban", GridSpec(nx, nx, nz, res), scans, dict(DEFAULT_PARAMS))


def point_cloud(rng: Rng, n: int, extent: float, sigma: float, planes: int = 6) -> np.ndarray:
    """n points near a few random axis-aligned planes inside [0, extent]^3
    (offsets N(0, sigma)): surface-like sets for the distance metrics."""
    axis = rng.integers(planes, 0, 3)
    level = rng.uniform(planes, 0.1 * extent, 0.9 * extent)
    which = rng.integers(n, 0, planes)
    p = rng.uniform(3 * n, 0.0, extent).reshape(n, 3)
    a = axis[which]
    p[np.arange(n), a] = level[which] + rng.normal(n, sigma)
    return p.astype(np.float32)


def batched_maps(n_maps: int = 32, scans_per_map: int = 8, seed_offset: int = 3,
                 side_lo: int = 64, side_hi: int = 512, n_lo: int = 4096,
                 n_hi: int = 131072) -> list:
    """Uneven independent maps: side log-uniform in [side_lo, side_hi] rounded
    to a multiple of 32, res uniform in [0.05, 0.2] m, the room scene scaled
    to the map, scans of n log-uniform in [n_lo, n_hi] returns as 16 beams x
    n/16 azimuths, per-map seeds."""
    rng = Rng(BASE_SEED + seed_offset)
    sides = np.maximum(32, np.round(rng.log_uniform(n_maps, side_lo, side_hi) / 32.0) * 32).astype(int)
    ress = rng.uniform(n_maps, 0.05, 0.2)
    out = []
    for m in range(n_maps):
        mrng = Rng(BASE_SEED + 1000 * (seed_offset + 1) + m)
        side, res = int(sides[m]), float(ress[m])
        extent = side * res
        c = extent / 2.0
        scene = room_scene(mrng, extent=extent, sensor=(c, c, c))
        scans = []
        for k in range(scans_per_map):
            n = int(mrng.log_uniform(1, n_lo, n_hi)[0])
            width = max(1, n // 16)
            off = mrng.uniform(3, -0.08 * extent, 0.08 * extent)
            pose = make_pose(rotation_rpy(0.0, 0.0, float(mrng.uniform(1, 0.0, 6.283)[0])),
                             np.array([c, c, c]) + off)
            scale = extent / 12.8
            pts = lidar_scan(scene, pose, 16, width, 30.0, 0.5 * scale, 12.0 * scale,
                             0.01 * scale, 0.0, mrng)
            scans.append((pts, pose))
        out.append(Workload(f"map{m}", GridSpec(side, side, side, res), scans, dict(DEFAULT_PARAMS)))
    return out


def random_points(rng: Rng, n: int, lo, hi) -> np.ndarray:
    """Uniform float32 points in the box [lo, hi) (tiny brute-force cases)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    u = rng.uniform(3 * n).reshape(n, 3)
    return (lo + (hi - lo) * u).astype(np.float32)


def random_rotation(rng: Rng) -> np.ndarray:
    """Uniform-ish random rotation from three angles."""
    a = rng.uniform(3, -math.pi, math.pi)
    return rotation_rpy(float(a[0]), float(a[1]) / 2.0, float(a[2]))


def serving_robots(n_robots: int = 16, scans_per_robot: int = 4, duration: float = 60.0,
                   seed_offset: int = 4, side_lo: int = 400, side_hi: int = 1200,
                   z_lo: int = 100, z_hi: int = 200, res: float = 0.05):
    """Robots with resident maps at res (x = y side log-uniform in [side_lo,
    side_hi], z in [z_lo, z_hi]), each with a pool of scans (beams from
    {16, 32, 64, 128} x widths from {900, 1024, 2048}, 14k-262k returns) from
    the urban generator scaled to its map, and Poisson arrival times at a rate
    uniform in [10, 20] Hz over `duration` seconds (scan k of the trace uses
    pool entry k mod scans_per_robot).  Returns (maps, arrivals) with
    arrivals = [(robot, time, pool index)] sorted by time."""
    rng = Rng(BASE_SEED + seed_offset)
    maps, arrivals = [], []
    beams_set, widths = (16, 32, 64, 128), (900, 1024, 2048)
    for r in range(n_robots):
        side = int(round(float(rng.log_uniform(1, side_lo, side_hi)[0])))
        nz = int(rng.integers(1, z_lo, z_hi + 1)[0])
        scale = side * res / 80.0
        while True:
            beams = beams_set[int(rng.integers(1, 0, 4)[0])]
            width = widths[int(rng.integers(1, 0, 3)[0])]
            if 14000 <= beams * width <= 262144:
                break
        w = urban_sequence(n_scans=scans_per_robot, seed_offset=100 + 17 * r + seed_offset,
                           scale=scale, res=res, beams=beams, width=width,
                           rmax=max(10.0, 60.0 * scale))
        w.grid = GridSpec(w.grid.nx, w.grid.ny, min(w.grid.nz, nz) if nz >= 64 else w.grid.nz, res)
        maps.append(w)
        rate = float(rng.uniform(1, 10.0, 20.0)[0])
        t, k = 0.0, 0
        while True:
            t += -math.log(1.0 - float(rng.uniform(1)[0])) / rate
            if t >= duration:
                break
            arrivals.append((r, t, k % scans_per_robot))
            k += 1
    arrivals.sort(key=lambda a: a[1])
    return maps, arrivals


# ---------------------------------------------------------------- map states
def map_state(dist, occupied):
    """A map state as the export path reads it: per voxel a distance mask
    whose `dist` (0..32) low bits are set, sign 0 where `occupied` (else
    1), hits 0.  Returns (mask u32, sign u8, hits u16) of dist's shape."""
    d = np.clip(np.asarray(dist, np.int64), 0, 32).astype(np.uint64)
    mask = ((np.uint64(1) << d) - np.uint64(1)).astype(np.uint32)
    sign = np.where(np.asarray(occupied, bool), 0, 1).astype(np.uint8)
    return mask, sign, np.zeros(mask.shape, np.uint16)


def sphere_state(n: int, centre, radius: float):
    """n^3 voxels; a ball of `radius` voxels around `centre` (voxel units)
    is occupied; distance = | |p - c| - radius | rounded, at least 1."""
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    return map_state(np.maximum(1, np.rint(np.abs(r - radius))), r < radius)


def random_state(shape, seed: int, p_occupied: float = 0.5, min_dist: int = 0, max_dist: int = 32):
    """Independent random voxels: distance uniform in [min_dist, max_dist],
    occupied with probability p_occupied (a stress case: every cell
    configuration, ambiguous faces included)."""
    rng = Rng(BASE_SEED + seed)
    n = int(np.prod(shape))
    dist = rng.integers(n, min_dist, max_dist + 1).reshape(shape)
    occ = (rng.uniform(n) < p_occupied).reshape(shape)
    return map_state(dist, occ)


def terrain_state(nx: int, ny: int, nz: int, seed: int, block: int = 40, n_boxes: int = 60):
    """A stepped terrain: the ground height is constant over block x block
    columns, uniform in [nz/8, nz/2], with n_boxes boxes (sides 8-80 voxels,
    heights up to nz/3) standing on it; occupied = at or below the surface,
    distance = |z - surface| along z (+1 below), capped at 32.  Built slice by
    slice, so full-size maps (1600 x 1600 x 320) take a few seconds."""
    rng = Rng(BASE_SEED + seed)
    gy, gx = -(-ny // block), -(-nx // block)
    h = rng.integers(gy * gx, nz // 8, nz // 2 + 1).reshape(gy, gx)
    top = np.repeat(np.repeat(h, block, 0), block, 1)[:ny, :nx].astype(np.int64)
    for _ in range(n_boxes):
        sx, sy = (int(v) for v in rng.integers(2, 8, 81))
        x0 = int(rng.integers(1, 0, max(1, nx - sx))[0])
        y0 = int(rng.integers(1, 0, max(1, ny - sy))[0])
        hz = int(rng.integers(1, 4, max(5, nz // 3))[0])
        top[y0:y0 + sy, x0:x0 + sx] += hz
    top = np.minimum(top, nz - 2)
    mask = np.empty((nz, ny, nx), np.uint32)
    sign = np.empty((nz, ny, nx), np.uint8)
    for z in range(nz):
        s = z - top
        occ = s <= 0
        m, sg, _ = map_state(np.where(occ, 1 - s, s), occ)
        mask[z] = m
        sign[z] = sg
    return mask, sign, np.zeros((nz, ny, nx), np.uint16)
