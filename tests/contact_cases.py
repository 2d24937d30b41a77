"""Returns aimed where two evaluation orders of the per-return floors differ.

Sec. III-C writes the per-return steps as formulas: p_w = R p + t and the
voxel index floor((p_w - o) / res); the octahedral cell (Cigolle et al.)
divides the direction by its 1-norm.  The oracle evaluates them as written
in binary64: unfused products and sums, true divisions.  Two plausible
variants round differently:
  - a reciprocal multiply, (p_w - o) * fl(1 / res) or d_x * fl(1 / s);
  - a fused transform, fma(r2, z, fma(r1, y, r0 * x)).
Each case below is a return for which the written form and a variant give
different voxels or cells, so a test on it fails if either side drifts to the
variant.  Every binary64 operation is emulated here with exact rationals
rounded once (``float(Fraction)`` rounds to nearest), independently of the
oracle's C and of the CUDA library.  Test infrastructure only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction as F

import numpy as np

import synth


def r64(x: F) -> float:
    return float(x)


def mul(a, b):
    return r64(F(a) * F(b))


def add(a, b):
    return r64(F(a) + F(b))


def sub(a, b):
    return r64(F(a) - F(b))


def div(a, b):
    return r64(F(a) / F(b))


def fma(a, b, c):
    return r64(F(a) * F(b) + F(c))


def row_plain(r, p):
    """(r0 x + r1 y) + r2 z, each operation rounded."""
    return add(add(mul(r[0], p[0]), mul(r[1], p[1])), mul(r[2], p[2]))


def row_fused(r, p):
    return fma(r[2], p[2], fma(r[1], p[1], mul(r[0], p[0])))


def octa_cell(u: float, n: int) -> int:
    return math.floor(mul(mul(add(u, 1.0), 0.5), float(n)))


@dataclass
class Case:
    """One return under one pose on one grid; ``plain`` is the written
    form's contact (x, y, z) or octahedral cell, ``variant`` the other
    order's."""
    kind: str
    pts: np.ndarray          # (1, 3) float32
    pose: np.ndarray         # (3, 4) float64
    res: float
    origin: tuple
    dims: tuple
    kernel_size: int
    plain: tuple
    variant: tuple
    exact: tuple | None      # floor of the exact real value where it is decided


def division_case() -> Case:
    """x = fl(0.3), res = 0.1: fl(x / 0.1) = 2.9999999999999996 (floor 2, as
    the exact quotient 2.99999999999999972...), but fl(1 / 0.1) = 10 and
    fl(x * 10) = 3.  The return lands there on all three axes: R = I,
    p = (0.25, 0.25, 0.25), t = fl(0.3) - 0.25 (exact by Sterbenz), so that
    p_w = fl(0.3) exactly."""
    x = 0.3
    t = sub(x, 0.25)
    assert add(0.25, t) == x
    plain = math.floor(div(x, 0.1))
    variant = math.floor(mul(x, div(1.0, 0.1)))
    exact = math.floor(F(x) / F(0.1))
    assert plain == exact == 2 and variant == 3
    pose = np.hstack([np.eye(3), np.full((3, 1), t)])
    return Case("division", np.full((1, 3), 0.25, np.float32), pose, 0.1, (0.0, 0.0, 0.0),
                (8, 8, 8), 3, (plain,) * 3, (variant,) * 3, (exact,) * 3)


def transform_cases(n: int = 6, seed: int = 77) -> list[Case]:
    """Random rotations and binary32 returns whose map-frame x differs
    between the unfused and the fused row, with t chosen so that one of the
    two lands exactly on the voxel face x = 1.5 (res = 0.5, origin 0, so the
    division is exact) and the other one ulp below it."""
    rng = synth.Rng(seed)
    out = []
    while len(out) < n:
        R = synth.random_rotation(rng)
        d = rng.normal(3)
        p = (d / np.linalg.norm(d) * rng.uniform(1, 1.1, 1.6)[0]).astype(np.float32)
        pd = [float(v) for v in p]
        a, b = row_plain(R[0], pd), row_fused(R[0], pd)
        if a == b or not (0.8 < a < 2.9):
            continue
        # t so that the larger of the two sums to exactly 1.5 (Sterbenz: exact)
        t0 = sub(1.5, max(a, b))
        if add(max(a, b), t0) != 1.5:
            continue
        wa, wb = add(a, t0), add(b, t0)
        ca, cb = math.floor(div(wa, 0.5)), math.floor(div(wb, 0.5))
        if ca == cb:
            continue
        # y and z: well inside their voxels for both forms
        t = [t0]
        for r in (1, 2):
            ya = row_plain(R[r], pd)
            t.append(sub(4.25, ya))
        cy = [math.floor(div(add(row_plain(R[r], pd), t[r]), 0.5)) for r in (1, 2)]
        cyv = [math.floor(div(add(row_fused(R[r], pd), t[r]), 0.5)) for r in (1, 2)]
        if cy != cyv:
            continue
        pose = np.hstack([R, np.array(t)[:, None]])
        out.append(Case("transform", p[None, :], pose, 0.5, (0.0, 0.0, 0.0), (16, 16, 16), 3,
                        (ca, cy[0], cy[1]), (cb, cyv[0], cyv[1]), None))
    return out


def octa_cases(n: int = 6, cells: int = 8, seed: int = 5) -> list[Case]:
    """Directions whose octahedral u sits on a cell edge of a cells x cells
    split, for which u = d_x / s and u = d_x * fl(1 / s) fall in different
    cells; R = I (so d = p exactly), upper half (no fold).  The written
    form's cell is also the floor of the exact real u's cell coordinate."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        k = int(rng.integers(1, cells))
        ue = -1.0 + 2.0 * k / cells
        dy = np.float32(rng.uniform(0.05, 2.0))
        dz = np.float32(rng.uniform(0.05, 2.0))
        a = float(dy) + float(dz)
        dx0 = np.float32(ue * a / (1.0 - ue) if ue >= 0 else ue * a / (1.0 + ue))
        for dx in (dx0, np.nextafter(dx0, np.float32(1e9)), np.nextafter(dx0, np.float32(-1e9))):
            x, y, z = float(dx), float(dy), float(dz)
            s = add(add(abs(x), abs(y)), abs(z))
            up, ur = div(x, s), mul(x, div(1.0, s))
            cp, cr = octa_cell(up, cells), octa_cell(ur, cells)
            if cp == cr:
                continue
            exact = math.floor((F(x) / F(s) + 1) / 2 * cells)
            if exact != cp:
                continue
            v = div(y, s)
            j = min(max(octa_cell(v, cells), 0), cells - 1)
            if octa_cell(mul(y, div(1.0, s)), cells) != octa_cell(v, cells):
                continue
            plain = j * cells + min(max(cp, 0), cells - 1)
            variant = j * cells + min(max(cr, 0), cells - 1)
            if plain == variant:
                continue
            pose = np.hstack([np.eye(3), np.full((3, 1), 16.0)])
            out.append(Case("octa", np.array([[x, y, z]], np.float32), pose, 0.5,
                            (0.0, 0.0, 0.0), (64, 64, 64), 3, (plain,), (variant,), (plain,)))
            break
    return out


def all_cases() -> list[Case]:
    return [division_case()] + transform_cases() + octa_cases()
