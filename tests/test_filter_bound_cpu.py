"""The binary32 filter of the per-return stage, checked in exact arithmetic.

The device takes the voxel floor from fa . p + fb (+ B) and the octahedral
cell from binary32 directions, each with an error bound, and falls back to
binary64 when a value lies within its bound of an integer (Sec. III-C's
floors; the filter is an evaluation strategy, not part of the method).
Here that arithmetic is replayed step by step with every binary32 operation
rounded exactly (rationals), on realistic and adversarial inputs, and two
facts are checked against the exact real values and the oracle:
  1. every bound holds: |value - exact| <= bound;
  2. whenever the filter decides, its decision equals the binary64 one (the
     voxel floor as the oracle computes it, the oracle's bin).
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import synth

U32_REL = 3.5e-7          # FILTER_REL
U32_ABS = 1e-37           # FILTER_ABS


def r32(x: Fr, up: bool = False) -> float:
    """x rounded to binary32 (to nearest even, or toward +inf), as a float."""
    if x == 0:
        return 0.0
    neg = x < 0
    a = -x if neg else x
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    q = Fr(2) ** max(e - 23, -149)
    m = a / q
    n = m.numerator // m.denominator
    r = m - n
    if up:
        if r > 0 and not neg:
            n += 1
    elif r > Fr(1, 2) or (r == Fr(1, 2) and n % 2 == 1):
        n += 1
    v = float(n * q)
    return -v if neg else v


def f32(v) -> float:
    return float(np.float32(v))


def add(a, b):
    return r32(Fr(a) + Fr(b))


def sub(a, b):
    return r32(Fr(a) - Fr(b))


def mul(a, b):
    return r32(Fr(a) * Fr(b))


def fma(a, b, c):
    return r32(Fr(a) * Fr(b) + Fr(c))


def div(a, b, up=False):
    return r32(Fr(a) / Fr(b), up)


def r64(x: Fr) -> float:
    return float(x)                   # correctly rounded


def row64(r, p):
    """Sec. III-C's row (r0 x + r1 y) + r2 z in binary64, as the oracle and
    the device's binary64 path evaluate it (no fused multiply-add)."""
    return r64(Fr(r64(Fr(r64(Fr(r[0]) * Fr(p[0]))) + Fr(r64(Fr(r[1]) * Fr(p[1]))))) +
               Fr(r64(Fr(r[2]) * Fr(p[2]))))


def pose_filter(R, t, org, inv_res):
    """The host preparation (binary64 like the library's host code)."""
    fa, fr, fb, fbi, fe0 = [], [], [], [], []
    for r in range(3):
        b = (t[r] - org[r]) * inv_res
        B = math.floor(abs(Fr(b)) + Fr(1, 2))          # std::round: halves away from zero
        B = float(-B if b < 0 else B)
        fbi.append(int(B))
        fb.append(f32(b - B))
        fe0.append(f32((abs(t[r]) + abs(org[r])) * inv_res * 2.0 ** -46 + 2.0 ** -22))
        fa.append([f32(R[r][j] * inv_res) for j in range(3)])
        fr.append([f32(R[r][j]) for j in range(3)])
    return fa, fr, fb, fbi, fe0


def floor_certain(v, e):
    f = float(math.floor(v))
    return (sub(v, f) > e and sub(add(f, 1.0), v) > e), int(f)


def voxel_checks(R, t, org, res, p):
    """Returns (decided, floors) and asserts the bounds; p binary32 values.
    The filter's data use the host's 1 / res; the value it must decide is
    the binary64 floor((p_w - o) / res) with a true division."""
    inv_res = 1.0 / res
    fa, fr, fb, fbi, fe0 = pose_filter(R, t, org, inv_res)
    out = []
    decided = True
    for r in range(3):
        a = fa[r]
        c = fma(a[2], p[2], fma(a[1], p[1], fma(a[0], p[0], fb[r])))
        S = add(add(add(abs(mul(a[0], p[0])), abs(mul(a[1], p[1]))), abs(mul(a[2], p[2]))), abs(fb[r]))
        e = fma(S, f32(U32_REL), add(fe0[r], f32(U32_ABS)))
        exact = (sum(Fr(R[r][j]) * Fr(p[j]) for j in range(3)) + Fr(t[r]) - Fr(org[r])) / Fr(res)
        assert abs(Fr(c) + fbi[r] - exact) <= Fr(e), (r, c, e)
        ok, q = floor_certain(c, e)
        # the binary64 value the oracle and the fallback compute
        d = row64(R[r], p)
        c64 = r64(Fr(r64(Fr(r64(Fr(d) + Fr(t[r]))) - Fr(org[r]))) / Fr(res))
        if ok:
            assert q + fbi[r] == math.floor(c64), (r, c, e, c64)
        decided = decided and ok
        out.append(q + fbi[r])
    return decided, out


def octa_bin_f32(d, e, n):
    """bin_octa_f32 of the device, step by step; -1 when it defers."""
    ax, ay, az = abs(d[0]), abs(d[1]), abs(d[2])
    s = add(add(ax, ay), az)
    es = add(mul(add(add(e[0], e[1]), e[2]), f32(1.001)), mul(s, f32(2.5e-7)))
    if not (s > mul(4.0, es)) or not (az > e[2]):
        return -1
    u, v = div(d[0], s), div(d[1], s)
    eu = add(mul(div(add(e[0], es), s, up=True), f32(1.01)), f32(1.2e-7))
    ev = add(mul(div(add(e[1], es), s, up=True), f32(1.01)), f32(1.2e-7))
    if d[2] < 0.0:
        if not (ax > e[0] and ay > e[1]):
            return -1
        fu, fv = sub(1.0, abs(v)), sub(1.0, abs(u))
        eu, ev = add(ev, f32(1.2e-7)), add(eu, f32(1.2e-7))
        u = -fu if d[0] < 0.0 else fu
        v = -fv if d[1] < 0.0 else fv
    h = mul(0.5, float(n))
    au, av = mul(add(u, 1.0), h), mul(add(v, 1.0), h)
    bu = add(add(mul(mul(add(eu, f32(2.4e-7)), h), f32(1.01)), mul(abs(au), f32(1.2e-7))), f32(1e-6))
    bv = add(add(mul(mul(add(ev, f32(2.4e-7)), h), f32(1.01)), mul(abs(av), f32(1.2e-7))), f32(1e-6))
    oku, i = floor_certain(au, bu)
    okv, j = floor_certain(av, bv)
    if not (oku and okv):
        return -1
    return min(max(j, 0), n - 1) * n + min(max(i, 0), n - 1)


def direction_checks(orc, po, R, p, n):
    fr = [[f32(R[r][j]) for j in range(3)] for r in range(3)]
    d32, e32 = [], []
    for r in range(3):
        a = fr[r]
        d32.append(fma(a[2], p[2], fma(a[1], p[1], mul(a[0], p[0]))))
        S = add(add(abs(mul(a[0], p[0])), abs(mul(a[1], p[1]))), abs(mul(a[2], p[2])))
        e32.append(fma(S, f32(U32_REL), f32(U32_ABS)))
        exact = sum(Fr(R[r][j]) * Fr(p[j]) for j in range(3))
        assert abs(Fr(d32[r]) - exact) <= Fr(e32[r])
    b = octa_bin_f32(d32, e32, n)
    if b >= 0:
        d64 = [row64(R[r], p) for r in range(3)]
        assert b == orc.bin_of(po, np.array(d64)), (p, d32, b)
    return b >= 0


def _rotation(rng):
    return synth.random_rotation(rng).tolist()


@pytest.mark.parametrize("seed,res", [(1, 0.05), (2, 0.1), (3, 0.02), (4, 0.3)])
def test_voxel_bound_random(seed, res):
    rng = synth.Rng(seed)
    R = _rotation(rng)
    t = (rng.uniform(3, -120.0, 120.0)).tolist()
    org = (rng.uniform(3, -1000.0, 1000.0)).tolist()
    decided = 0
    for k in range(300):
        dr = rng.normal(3)
        rr = float(rng.uniform(1, 0.01, 80.0)[0])
        p = [f32(x) for x in (dr / np.linalg.norm(dr) * rr)]
        ok, _ = voxel_checks(R, t, org, res, p)
        decided += ok
    assert decided > 280          # the filter decides nearly every return


def test_voxel_bound_on_faces():
    """Map-frame points on voxel faces (and a few ulps off), rotated back
    into the sensor frame in binary32: every bound holds, every decision is
    binary64's, and the filter defers on most of them."""
    rng = synth.Rng(11)
    R = _rotation(rng)
    t = [0.3, -0.7, 0.2]
    org = [-10.0, -10.0, -2.5]
    res = 0.05
    Rn = np.array(R)
    deferred = 0
    for k in range(200):
        vox = rng.integers(3, 20, 380).astype(np.float64)
        w = np.array(org) + vox * res + rng.normal(3) * 1e-9
        p = [f32(x) for x in (Rn.T @ (w - np.array(t)))]
        ok, _ = voxel_checks(R, t, org, res, p)
        deferred += not ok
    assert deferred > 100


def test_octahedral_bound(orc):
    po = orc.params(scheme=0, bins_a=8, bins_b=8)
    rng = synth.Rng(21)
    decided = 0
    edge_deferred = 0
    for k in range(300):
        R = _rotation(rng)
        dr = rng.normal(3)
        p = [f32(x) for x in dr / np.linalg.norm(dr) * float(rng.uniform(1, 0.5, 60.0)[0])]
        decided += direction_checks(orc, po, R, p, 8)
    # exact cell edges and the fold plane at R = I: the filter must defer
    I = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]
    for p in ([-0.5, 0.25, 0.25], [0.25, 0.5, -0.25], [1.0, 0.0, 0.0], [0.3, 0.2, 0.0],
              [0.0, 0.7, -0.3], [-0.75, 0.125, 0.125]):
        edge_deferred += not direction_checks(orc, po, I, [f32(x) for x in p], 8)
    assert decided > 280 and edge_deferred == 6
