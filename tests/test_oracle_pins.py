"""Pins of the oracle to facts outside itself (no GPU).

Each test ties a part of the oracle to something it cannot be circular with:
hand-worked values of the paper's equations (tests/golden/), a closed form
(integer ceil-sqrt, lattice-point counts of OEIS A000605), a library routine
(math.atan2/asin for Eq. 2 away from bin edges), invariants the paper states
(masks only lose bits, Sec. III-A/III-C), or brute force on tiny grids in
the gather form (every voxel: min over returns of ceil |v - c|), which is a
different formulation from the oracle's per-return scatter of Eqs. 4-6.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from conftest import read_golden


# ------------------------------------------------------------------ Eq. 3
def test_eq3_golden_values(orc):
    for ox, oy, oz, r2, c, m in read_golden("eq3_masks.txt"):
        assert int(ox) ** 2 + int(oy) ** 2 + int(oz) ** 2 == int(r2)
        assert orc.distance_mask(int(ox), int(oy), int(oz)) == int(m, 16), (ox, oy, oz)


def _ceil_sqrt(n):
    k = math.isqrt(n)
    return k if k * k == n else k + 1


@pytest.mark.parametrize("K", [1, 3, 11, 21])
def test_eq3_table_closed_form(orc, K):
    """popcount(m) = ceil(|o|) by exact integer arithmetic; m = 2^k - 1."""
    t = orc.mask_table(K)
    R = (K - 1) // 2
    for oz in range(-R, R + 1):
        for oy in range(-R, R + 1):
            for ox in range(-R, R + 1):
                m = int(t[oz + R, oy + R, ox + R])
                k = _ceil_sqrt(ox * ox + oy * oy + oz * oz)
                want = 0xFFFFFFFF if k >= 32 else (1 << k) - 1
                assert m == want
                assert m & (m + 1) == 0       # of the form 2^k - 1


def test_eq1_memory(orc):
    # Eq. 1 with S_voxel = 8 bytes: 128^3 -> 16 MiB; 1600x1600x320 -> 6.5536 GB
    assert orc.grid_bytes_eq1(128, 128, 128) == 16 * 1024 * 1024
    assert orc.grid_bytes_eq1(1600, 1600, 320) == 6_553_600_000


# ------------------------------------------------------------------ bins
def test_octa_golden(orc):
    p = orc.params(scheme=orc.SCHEME_OCTA, bins_a=8, bins_b=8)
    for dx, dy, dz, i, j, b in read_golden("octa_bins.txt"):
        got = orc.bin_of(p, (float(dx), float(dy), float(dz)))
        assert got == int(b) == 8 * int(j) + int(i), (dx, dy, dz, got)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_octa_centre_round_trip(orc, n):
    """The representative direction of each cell falls back into that cell."""
    p = orc.params(scheme=orc.SCHEME_OCTA, bins_a=n, bins_b=n)
    for b in range(n * n):
        assert orc.bin_of(p, orc.bin_dir(p, b)) == b


def test_octa_cells_cover_sphere(orc):
    """Every cell is hit by uniform directions, with area within a factor 3
    of the mean (the octahedral map is area-distorting but bounded)."""
    p = orc.params(scheme=orc.SCHEME_OCTA, bins_a=8, bins_b=8)
    rng = synth.Rng(17)
    d = rng.normal(20000).reshape(-1, 2)
    d = np.column_stack([d, rng.normal(10000)])
    counts = np.bincount([orc.bin_of(p, v) for v in d], minlength=64)
    mean = len(d) / 64
    assert counts.min() > mean / 3 and counts.max() < mean * 3


def test_octa_mirror_symmetry(orc):
    """Mirroring x maps cell column i to n-1-i (away from cell edges)."""
    p = orc.params(scheme=orc.SCHEME_OCTA, bins_a=8, bins_b=8)
    rng = synth.Rng(3)
    for _ in range(2000):
        d = rng.normal(3)
        b1 = orc.bin_of(p, d)
        b2 = orc.bin_of(p, (-d[0], d[1], d[2]))
        s = np.abs(d).sum()
        u = d[0] / s
        if abs(((u + 1) * 4) - round((u + 1) * 4)) < 1e-9 or abs(d[0]) < 1e-9:
            continue
        assert b2 // 8 == b1 // 8 and b2 % 8 == 7 - b1 % 8


def test_azel_golden(orc):
    p = orc.params(scheme=orc.SCHEME_AZEL, bins_a=40, bins_b=40)
    for dx, dy, dz, baz, bel, b in read_golden("azel_axes.txt"):
        got = orc.bin_of(p, (float(dx), float(dy), float(dz)))
        assert got == int(b) == 40 * int(bel) + int(baz), (dx, dy, dz, got)


@pytest.mark.parametrize("baz,bel", [(40, 40), (36, 18), (7, 5)])
def test_azel_matches_atan2_asin(orc, baz, bel):
    """Eq. 2 written with the library's atan2/asin agrees with the edge-count
    form wherever the direction is more than 1e-9 rad from a bin edge."""
    p = orc.params(scheme=orc.SCHEME_AZEL, bins_a=baz, bins_b=bel)
    rng = synth.Rng(11)
    checked = 0
    for _ in range(4000):
        x, y, z = rng.normal(3)
        th = math.atan2(y, x) % (2 * math.pi)
        el = math.asin(z / math.sqrt(x * x + y * y + z * z))
        a = th / (2 * math.pi) * baz
        e = (el + math.pi / 2) / math.pi * bel
        if abs(a - round(a)) < 1e-9 * baz or abs(e - round(e)) < 1e-9 * bel:
            continue
        want = min(int(math.floor(e)), bel - 1) * baz + int(math.floor(a)) % baz
        assert orc.bin_of(p, (x, y, z)) == want
        checked += 1
    assert checked > 3900


# ------------------------------------------------------------------ shadow
def test_ball_counts_oeis(orc):
    """With u_b fixed, S_b and -S_b cover the ball of radius r_s and overlap
    exactly on the plane o . u_b = 0: |S_b| = (N(r) + Z_b) / 2 with N(r) the
    lattice-point count of OEIS A000605."""
    counts = {int(r): int(c) for r, c in read_golden("ball_counts.txt")}
    for r, N in counts.items():
        if r > 5:
            continue
        p = orc.params(kernel_size=11, shadow_radius=float(r))
        S = orc.shadow_table(p)
        for b in range(64):
            u = orc.bin_dir(p, b)
            Z = 0
            for oz in range(-r, r + 1):
                for oy in range(-r, r + 1):
                    for ox in range(-r, r + 1):
                        if ox * ox + oy * oy + oz * oz <= r * r:
                            Z += (ox * u[0] + oy * u[1] + oz * u[2]) == 0
            assert 2 * int(S[b].sum()) == N + Z, (r, b)


def test_shadow_radius_one(orc):
    """r_s = 1: the contact voxel plus the face neighbour along each axis on
    the far side of the surface (sign of that component of u_b), both
    neighbours when the component is zero."""
    p = orc.params(kernel_size=5, shadow_radius=1.0)
    for b in range(64):
        u = orc.bin_dir(p, b)
        want = {(0, 0, 0)}
        for a in range(3):
            for s in (-1, 1):
                if s * u[a] >= 0:
                    o = [0, 0, 0]
                    o[a] = s
                    want.add(tuple(o))
        got = {(ox, oy, oz) for oz in (-1, 0, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1)
               if orc.in_shadow(p, b, ox, oy, oz)}
        assert got == want


def test_shadow_lies_behind_surface(orc):
    """For a ray d the voxel ~3 steps further along d is in the shadow of
    d's bin and the voxel ~3 steps back towards the sensor is not."""
    rng = synth.Rng(5)
    for scheme, a, bb in ((orc.SCHEME_OCTA, 8, 8), (orc.SCHEME_AZEL, 40, 40)):
        p = orc.params(kernel_size=11, scheme=scheme, bins_a=a, bins_b=bb, shadow_radius=3.0)
        for _ in range(300):
            d = rng.normal(3)
            d /= np.linalg.norm(d)
            b = orc.bin_of(p, d)
            o = np.round(2.9 * d).astype(int)
            if (o * o).sum() > 9 or not o.any():
                continue
            u = orc.bin_dir(p, b)
            u = u / np.linalg.norm(u)
            if abs(float(np.dot(o, u))) < 0.5:      # grazing: bin centre may flip it
                continue
            assert orc.in_shadow(p, b, *o)
            assert not orc.in_shadow(p, b, *(-o))


def test_shadow_radius_zero(orc):
    p = orc.params(kernel_size=7, shadow_radius=0.0)
    S = orc.shadow_table(p)
    assert S.sum() == 64 and all(S[b, 3, 3, 3] for b in range(64))


def test_cone_zero_is_hemisphere(orc):
    """shadow_cos = 0 is the hemisphere itself (half-angle 90 degrees)."""
    for scheme, a, b in ((orc.SCHEME_OCTA, 8, 8), (orc.SCHEME_AZEL, 40, 40)):
        h = orc.shadow_table(orc.params(kernel_size=11, scheme=scheme, bins_a=a, bins_b=b,
                                        shadow_radius=4.0))
        c = orc.shadow_table(orc.params(kernel_size=11, scheme=scheme, bins_a=a, bins_b=b,
                                        shadow_radius=4.0, shadow_cos=0.0))
        np.testing.assert_array_equal(h, c)


@pytest.mark.parametrize("num,den", [(1, 2), (3, 4), (1, 1)])
def test_cone_exact_integer_form(orc, num, den):
    """Octahedral bins: the cone o.v >= c |o| |v| with rational c = num/den is
    o.v >= 0 and den^2 (o.v)^2 >= num^2 |o|^2 |v|^2 in integers; brute force
    over every offset and bin (v = the integer cell-centre decode, whose
    direction is pinned by test_octa_centre_round_trip)."""
    K, n, rs = 11, 8, 5.0
    p = orc.params(kernel_size=K, shadow_radius=rs, shadow_cos=num / den)
    S = orc.shadow_table(p)
    R = K // 2
    for b in range(n * n):
        v = np.round(orc.bin_dir(p, b)).astype(np.int64)
        vv = int((v * v).sum())
        for oz in range(-R, R + 1):
            for oy in range(-R, R + 1):
                for ox in range(-R, R + 1):
                    r2 = ox * ox + oy * oy + oz * oz
                    dot = int(ox * v[0] + oy * v[1] + oz * v[2])
                    want = (r2 <= rs * rs and dot >= 0
                            and den * den * dot * dot >= num * num * r2 * vv)
                    assert bool(S[b, oz + R, oy + R, ox + R]) == want, (b, ox, oy, oz)


def test_cone_narrows_to_the_ray(orc):
    """c = 1 keeps only offsets parallel to the bin direction (Cauchy-Schwarz
    equality): at n = 2 the cell of (1, 1, 1) decodes to v = (1, 1, 0), so
    exactly the offsets t v, t >= 0, inside the ball.  The sets shrink as c
    grows and all hold the contact voxel: the conical model concentrates the
    hits on the central voxel (Sec. III-B)."""
    p1 = orc.params(kernel_size=11, bins_a=2, bins_b=2, shadow_radius=5.0, shadow_cos=1.0)
    b = orc.bin_of(p1, (1, 1, 1))
    assert list(np.round(orc.bin_dir(p1, b)).astype(int)) == [1, 1, 0]
    S1 = orc.shadow_table(p1)
    R = 5
    v = np.round(orc.bin_dir(p1, b)).astype(np.int64)
    got = {(ox - R, oy - R, oz - R) for oz, oy, ox in np.argwhere(S1[b])}
    want = {tuple(int(t) * v) for t in range(0, 6)
            if (t * v * t * v).sum() <= 25 and all(abs(t * v) <= R)}
    assert got == want
    prev = None
    for c in (0.0, 0.3, 0.6, 0.9, 1.0):
        S = orc.shadow_table(orc.params(kernel_size=11, shadow_radius=5.0, shadow_cos=c))
        assert all(S[bb, R, R, R] for bb in range(64))
        if prev is not None:
            assert not (S & ~prev).any() and S.sum() < prev.sum()
        prev = S


# ------------------------------------------------------------------ worked example
def test_single_point_worked_example(orc):
    g = orc.Grid.create(5, 5, 5, 1.0)
    p = orc.params(kernel_size=3, shadow_radius=1.0, hit_threshold=1, hit_max=255)
    pose = np.hstack([np.eye(3), np.zeros((3, 1))])
    st = orc.integrate_scan(g, p, np.array([[2.5, 2.5, 2.5]], np.float32), pose)
    assert st["n_kept"] == 1
    assert orc.bin_of(p, (1, 1, 1)) == 45
    for x, y, z, m, s, h in read_golden("single_point_k3.txt"):
        x, y, z = int(x), int(y), int(z)
        assert g.mask[z, y, x] == int(m, 16), (x, y, z)
        assert g.sign[z, y, x] == int(s), (x, y, z)
        assert g.hits[z, y, x] == int(h), (x, y, z)
    # every voxel outside the 3^3 kernel is untouched (Sec. III-A initial state)
    touched = np.zeros((5, 5, 5), bool)
    touched[1:4, 1:4, 1:4] = True
    assert (g.mask[~touched] == 0xFFFFFFFF).all()
    assert (g.hits[~touched] == 0).all() and (g.sign[~touched] == 1).all()


# ------------------------------------------------------------------ brute force
def _brute_force(orc, p, dims, res, origin, scans):
    """Gather form of Sec. III-C: per voxel, min ceil-distance over kept
    returns in range and the count of returns whose shadow covers it."""
    nx, ny, nz = dims
    K = p.kernel_size
    R = (K - 1) // 2
    kept = []
    for pts, pose in scans:
        seen = set()
        for q in pts:
            px, py, pz = float(q[0]), float(q[1]), float(q[2])
            if not (math.isfinite(px) and math.isfinite(py) and math.isfinite(pz)):
                continue
            if px == 0.0 and py == 0.0 and pz == 0.0:
                continue
            # Sec. III-C as written: p_w = R p + t, floor((p_w - o) / res)
            d = [(pose[r][0] * px + pose[r][1] * py) + pose[r][2] * pz for r in range(3)]
            w = [d[r] + pose[r][3] for r in range(3)]
            c = [math.floor((w[a] - origin[a]) / res) for a in range(3)]
            if any(c[a] < R or c[a] > (nx, ny, nz)[a] - 1 - R for a in range(3)):
                continue
            if p.dedup_first:
                if tuple(c) in seen:
                    continue
                seen.add(tuple(c))
            kept.append((c, orc.bin_of(p, d)))
    mask = np.empty((nz, ny, nx), np.uint32)
    hits = np.zeros((nz, ny, nx), np.int64)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                kmin = 99
                cnt = 0
                for c, b in kept:
                    o = (x - c[0], y - c[1], z - c[2])
                    if max(abs(o[0]), abs(o[1]), abs(o[2])) > R:
                        continue
                    kmin = min(kmin, _ceil_sqrt(o[0] ** 2 + o[1] ** 2 + o[2] ** 2))
                    cnt += orc.in_shadow(p, b, *o)
                mask[z, y, x] = 0xFFFFFFFF if kmin >= 32 else (1 << kmin) - 1
                hits[z, y, x] = min(cnt, p.hit_max)
    sign = np.where(hits >= p.hit_threshold, 0, 1).astype(np.uint8)
    return mask, sign, hits.astype(np.uint16), len(kept)


def _tiny_case(seed, n, dims, res, dup_every=0):
    rng = synth.Rng(seed)
    nx, ny, nz = dims
    hi = np.array([nx, ny, nz]) * res
    pts_w = synth.random_points(rng, n, (0.0, 0.0, 0.0), hi)
    if dup_every:
        extra = pts_w[::dup_every] + np.float32(0.01 * res)
        pts_w = np.concatenate([pts_w, extra, pts_w[:3]]).astype(np.float32)
    R = synth.random_rotation(rng)
    t = hi / 2 + rng.uniform(3, -res, res)
    pose = synth.make_pose(R, t)
    # sensor-frame returns: p_s = R^T (p_w - t), then rounded to float32
    pts_s = ((pts_w.astype(np.float64) - t) @ R).astype(np.float32)
    return pts_s, pose


CASES = [
    # seed, n, dims, res, K, r_s, T, Hmax, dedup, scheme
    (1, 30, (14, 13, 12), 0.1, 3, 1.0, 1, 255, 1, 0),
    (2, 40, (16, 16, 16), 0.25, 5, 2.0, 2, 3, 1, 0),
    (3, 25, (18, 15, 16), 0.05, 7, 3.0, 3, 255, 0, 0),
    (4, 50, (16, 16, 16), 0.5, 5, 2.5, 2, 2, 1, 1),
    (5, 20, (13, 17, 15), 0.2, 3, 0.0, 1, 255, 0, 1),
    (6, 35, (16, 16, 16), 0.3, 7, 1.5, 4, 5, 1, 0),
]


@pytest.mark.parametrize("case", CASES)
def test_brute_force_tiny_grids(orc, case):
    seed, n, dims, res, K, rs, T, H, dedup, scheme = case
    a, b = (8, 8) if scheme == 0 else (40, 40)
    p = orc.params(kernel_size=K, scheme=scheme, bins_a=a, bins_b=b, shadow_radius=rs,
                   hit_threshold=T, hit_max=H, dedup_first=dedup)
    scans = [_tiny_case(seed, n, dims, res, dup_every=4),
             _tiny_case(seed + 100, n, dims, res, dup_every=3)]
    g = orc.Grid.create(*dims, res)
    kept = 0
    for pts, pose in scans:
        kept += orc.integrate_scan(g, p, pts, pose)["n_kept"]
    m, s, h, nk = _brute_force(orc, p, dims, res, (0.0, 0.0, 0.0), scans)
    assert kept == nk and nk > 0
    np.testing.assert_array_equal(g.mask, m)
    np.testing.assert_array_equal(g.hits, h)
    np.testing.assert_array_equal(g.sign, s)


def test_first_return_rule_uses_first_bin(orc):
    """Two returns in one voxel with different bins: only the first (lowest
    index) is integrated (Sec. IV-B), so the shadow follows its bin."""
    p = orc.params(kernel_size=5, shadow_radius=2.0, hit_threshold=1)
    pose = synth.make_pose(np.eye(3), (4.5, 4.5, 4.5))
    # both land in voxel (6, 4, 4) of a 1 m grid; x-offsets -0.4/+0.4 from the
    # sensor's x put them in different octahedral columns
    a = np.array([[1.2, -0.4, 0.0]], np.float32)
    b = np.array([[1.2, 0.4, 0.0]], np.float32)
    assert orc.bin_of(p, a[0]) != orc.bin_of(p, b[0])
    g1 = orc.Grid.create(9, 9, 9, 1.0)
    orc.integrate_scan(g1, p, np.concatenate([a, b]), pose)
    g2 = orc.Grid.create(9, 9, 9, 1.0)
    orc.integrate_scan(g2, p, a, pose)
    np.testing.assert_array_equal(g1.hits, g2.hits)
    g3 = orc.Grid.create(9, 9, 9, 1.0)
    orc.integrate_scan(g3, p, np.concatenate([b, a]), pose)
    assert (g3.hits != g1.hits).any()


# ------------------------------------------------------------------ invariants
@pytest.fixture(scope="module")
def room():
    return synth.room_scan(n_scans=3)


def test_masks_only_lose_bits(orc, room):
    g = orc.Grid.create(128, 128, 128, 0.1)
    p = orc.params()
    prev_m, prev_h, prev_s = g.mask.copy(), g.hits.copy(), g.sign.copy()
    for pts, pose in room.scans:
        orc.integrate_scan(g, p, pts, pose)
        assert not (g.mask & ~prev_m).any()          # no bit ever set again
        assert (g.hits >= prev_h).all()              # counters never decrease
        assert (g.sign <= prev_s).all()              # sign only goes free -> occupied
        assert ((g.mask & (g.mask + np.uint32(1))) == 0).all()
        prev_m, prev_h, prev_s = g.mask.copy(), g.hits.copy(), g.sign.copy()
    assert ((g.sign == 0) == (g.hits >= 3)).all()


def test_scan_order_invariance(orc, room):
    p = orc.params()
    g1 = orc.Grid.create(128, 128, 128, 0.1)
    g2 = orc.Grid.create(128, 128, 128, 0.1)
    for pts, pose in room.scans:
        orc.integrate_scan(g1, p, pts, pose)
    for pts, pose in reversed(room.scans):
        orc.integrate_scan(g2, p, pts, pose)
    np.testing.assert_array_equal(g1.mask, g2.mask)
    np.testing.assert_array_equal(g1.hits, g2.hits)
    np.testing.assert_array_equal(g1.sign, g2.sign)


def test_point_order_invariance_without_dedup(orc, room):
    p = orc.params(dedup_first=0)
    pts, pose = room.scans[0]
    perm = np.argsort(synth.Rng(9).uniform(len(pts)))
    g1 = orc.Grid.create(128, 128, 128, 0.1)
    g2 = orc.Grid.create(128, 128, 128, 0.1)
    orc.integrate_scan(g1, p, pts, pose)
    orc.integrate_scan(g2, p, pts[perm], pose)
    np.testing.assert_array_equal(g1.mask, g2.mask)
    np.testing.assert_array_equal(g1.hits, g2.hits)
    np.testing.assert_array_equal(g1.sign, g2.sign)


def test_rs0_hits_count_points_per_voxel(orc, room):
    """r_s = 0, first-return rule off: hits = number of returns per contact
    voxel (saturated), which is the unsigned Fast-TDF count."""
    p = orc.params(shadow_radius=0.0, dedup_first=0, hit_max=65535)
    pts, pose = room.scans[0]
    g = orc.Grid.create(128, 128, 128, 0.1)
    st = orc.integrate_scan(g, p, pts, pose)
    ok = np.all(np.isfinite(pts), axis=1)
    # identity rotation: d = p exactly; c = floor((p + t - 0) * (1 / res))
    c = np.floor((pts[ok].astype(np.float64) + pose[:, 3] - 0.0) * (1.0 / 0.1)).astype(np.int64)
    inside = np.all((c >= 5) & (c <= 122), axis=1)
    c = c[inside]
    want = np.zeros((128, 128, 128), np.int64)
    np.add.at(want, (c[:, 2], c[:, 1], c[:, 0]), 1)
    assert st["n_kept"] == len(c)
    np.testing.assert_array_equal(g.hits.astype(np.int64), want)
    # with the rule on, each contact voxel counts once
    p1 = orc.params(shadow_radius=0.0, dedup_first=1)
    g1 = orc.Grid.create(128, 128, 128, 0.1)
    orc.integrate_scan(g1, p1, pts, pose)
    np.testing.assert_array_equal(g1.hits.astype(np.int64), np.minimum(want, 1))


def test_border_returns_change_nothing(orc):
    """Returns whose K^3 neighbourhood leaves the map are discarded (Sec. III-C)."""
    p = orc.params(kernel_size=11)
    g = orc.Grid.create(32, 32, 32, 0.1)
    pose = synth.make_pose(np.eye(3), (0.0, 0.0, 0.0))
    edge = []
    for a in range(3):
        for v in (0.05, 0.45, 2.75, 3.15):   # voxel 0, 4, 27, 31
            q = [1.6, 1.6, 1.6]
            q[a] = v
            edge.append(q)
    st = orc.integrate_scan(g, p, np.array(edge, np.float32), pose)
    assert st["n_inside"] == 0
    assert (g.mask == 0xFFFFFFFF).all() and (g.hits == 0).all()
    # one step inside (voxel 5 and 26) is kept
    st = orc.integrate_scan(g, p, np.array([[0.55, 1.6, 1.6], [2.65, 1.6, 1.6]], np.float32), pose)
    assert st["n_kept"] == 2


def test_discards_nan_and_origin(orc):
    p = orc.params(kernel_size=3)
    g = orc.Grid.create(8, 8, 8, 1.0)
    pose = synth.make_pose(np.eye(3), (4.0, 4.0, 4.0))
    pts = np.array([[np.nan, 0, 0], [0, 0, 0], [np.inf, 1, 1], [0.5, 0.5, 0.5]], np.float32)
    st = orc.integrate_scan(g, p, pts, pose)
    assert st["n_valid"] == 1 and st["n_kept"] == 1


def test_query_voxels_agree_with_full_integration(orc, room):
    """The sampled per-voxel fold equals the full scatter integration."""
    p = orc.params()
    g = orc.Grid.create(128, 128, 128, 0.1)
    cs, bs = [], []
    for pts, pose in room.scans:
        orc.integrate_scan(g, p, pts, pose)
        c, b = orc.scan_kept(g, p, pts, pose)
        cs.append(c)
        bs.append(b)
    c = np.concatenate(cs)
    b = np.concatenate(bs)
    rng = synth.Rng(21)
    changed = np.argwhere(g.hits > 0)
    sel = changed[np.floor(rng.uniform(300) * len(changed)).astype(int)]
    q = np.concatenate([sel[:, ::-1], rng.integers(300, 0, 128).reshape(-1, 3)])
    m, s, h = orc.query_voxels(p, c, b, q)
    np.testing.assert_array_equal(m, g.mask[q[:, 2], q[:, 1], q[:, 0]])
    np.testing.assert_array_equal(h, g.hits[q[:, 2], q[:, 1], q[:, 0]])
    np.testing.assert_array_equal(s, g.sign[q[:, 2], q[:, 1], q[:, 0]])


def test_signed_distance_readout(orc):
    assert orc.signed_distance(0x7, 1, 0.1) == pytest.approx(0.3)
    assert orc.signed_distance(0x1F, 0, 0.05) == pytest.approx(-0.25)
    assert orc.signed_distance(0x0, 0, 0.05) == 0.0


# ------------------------------------------------------------------ arithmetic of the floors
def test_contact_floors_follow_the_written_formulas(orc):
    """Sec. III-C: p_w = R p + t and voxel floor((p_w - o) / res), evaluated
    as written (unfused products and sums, a true division; the octahedral
    u = d_x / s likewise).  On returns crafted so that a reciprocal multiply
    or a fused transform would give another voxel or cell (rational
    emulation in tests/contact_cases.py), the oracle gives the written
    form's answer, which where it is decided is also the floor of the exact
    real value."""
    import contact_cases as cc
    cases = cc.all_cases()
    assert {c.kind for c in cases} == {"division", "transform", "octa"}
    for c in cases:
        assert c.plain != c.variant
        p = orc.params(kernel_size=c.kernel_size)
        g = orc.Grid(c.dims[0], c.dims[1], c.dims[2], c.res, c.origin, None, None, None)
        cont, bins = orc.scan_kept(g, p, c.pts, c.pose)
        assert len(cont) == 1, c
        got = tuple(int(v) for v in cont[0]) if c.kind != "octa" else (int(bins[0]),)
        assert got == c.plain, (c.kind, got, c.plain, c.variant)
        if c.exact is not None:
            assert got == c.exact
