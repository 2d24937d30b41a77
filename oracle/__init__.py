"""DB-TSDF oracle: test infrastructure, never product code.

A ctypes wrapper around ``dbtsdf_oracle.c``, the plain single-threaded C
restatement of DB-TSDF scan integration (arXiv 2509.20081, Sec. III).  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library under ``paper_2509_20081_gb300/``.

Each wrapper names the passage of the paper its C function follows.  The
grid used here is dense, x fastest, without row padding: index
``(z * ny + y) * nx + x``; arrays are shaped ``(nz, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dbtsdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SCHEME_OCTA = 0
SCHEME_AZEL = 1


_SRC_OMP = os.path.join(_HERE, "dbtsdf_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _compile(lib_path: str, srcs: list, extra: list, force: bool) -> str:
    if (not force and os.path.exists(lib_path)
            and all(os.path.getmtime(lib_path) >= os.path.getmtime(s) for s in srcs)):
        return lib_path
    tmp = lib_path + f".{os.getpid()}.tmp"
    subprocess.run(["gcc"] + _CFLAGS + extra + ["-o", tmp, srcs[0], "-lm"], check=True)
    os.replace(tmp, lib_path)
    return lib_path


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no fused multiply-add)."""
    return _compile(_LIB, [_SRC], [], force)


def build_omp(force: bool = False) -> str | None:
    """Compile the points-parallel variant (OpenMP; it includes the oracle's
    source).  None when the compiler has no OpenMP runtime."""
    try:
        return _compile(_LIB_OMP, [_SRC_OMP, _SRC], ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        return None


class Params(ctypes.Structure):
    _fields_ = [("kernel_size", ctypes.c_int),
                ("scheme", ctypes.c_int),
                ("bins_a", ctypes.c_int),
                ("bins_b", ctypes.c_int),
                ("shadow_radius", ctypes.c_double),
                ("hit_threshold", ctypes.c_int),
                ("hit_max", ctypes.c_int),
                ("dedup_first", ctypes.c_int),
                ("shadow_cos", ctypes.c_double)]


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("res", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("mask", ctypes.c_void_p), ("sign", ctypes.c_void_p),
                ("hits", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("n_input", ctypes.c_int64), ("n_valid", ctypes.c_int64),
                ("n_inside", ctypes.c_int64), ("n_kept", ctypes.c_int64),
                ("n_mask_writes", ctypes.c_int64), ("n_shadow_incs", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def load(path: str):
    """Load an oracle shared object and declare its signatures."""
    L = ctypes.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def _declare(L):
    """ctypes signatures of the oracle's C functions."""
    P = ctypes.POINTER
    L.orc_distance_mask.restype = ctypes.c_uint32
    L.orc_distance_mask.argtypes = [ctypes.c_int] * 3
    L.orc_bin_octa.restype = ctypes.c_int
    L.orc_bin_octa.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int]
    L.orc_bin_azel.restype = ctypes.c_int
    L.orc_bin_azel.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int] * 2
    L.orc_bin_az.restype = ctypes.c_int
    L.orc_bin_az.argtypes = [ctypes.c_double] * 2 + [ctypes.c_int]
    L.orc_bin_el.restype = ctypes.c_int
    L.orc_bin_el.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int]
    L.orc_bin.restype = ctypes.c_int
    L.orc_bin.argtypes = [P(Params)] + [ctypes.c_double] * 3
    L.orc_bin_dir.restype = None
    L.orc_bin_dir.argtypes = [P(Params), ctypes.c_int, P(ctypes.c_double)]
    L.orc_in_shadow.restype = ctypes.c_int
    L.orc_in_shadow.argtypes = [P(Params)] + [ctypes.c_int] * 4
    L.orc_grid_init.restype = None
    L.orc_grid_init.argtypes = [P(_Grid)]
    L.orc_grid_bytes_eq1.restype = ctypes.c_int64
    L.orc_grid_bytes_eq1.argtypes = [ctypes.c_int64] * 3
    L.orc_integrate_scan.restype = ctypes.c_int64
    L.orc_integrate_scan.argtypes = [P(_Grid), P(Params), ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p, P(Stats)]
    L.orc_integrate_scan_ex.restype = ctypes.c_int64
    L.orc_integrate_scan_ex.argtypes = [P(_Grid), P(Params), ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                        P(Stats)]
    L.orc_pose_interp.restype = None
    L.orc_pose_interp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_void_p]
    L.orc_scan_kept.restype = ctypes.c_int64
    L.orc_scan_kept.argtypes = [P(Params), P(_Grid), ctypes.c_void_p, ctypes.c_int64,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_query_voxels.restype = None
    L.orc_query_voxels.argtypes = [P(Params), ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.orc_signed_distance.restype = ctypes.c_double
    L.orc_signed_distance.argtypes = [ctypes.c_uint32, ctypes.c_uint8, ctypes.c_double]
    L.orc_mc_config.restype = ctypes.c_int
    L.orc_mc_config.argtypes = [ctypes.c_int, ctypes.c_void_p]
    L.orc_sdf_field.restype = None
    L.orc_sdf_field.argtypes = [P(_Grid), ctypes.c_void_p, ctypes.c_void_p]
    L.orc_nn_distances.restype = None
    L.orc_nn_distances.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_void_p]
    L.orc_quality_from_distances.restype = None
    L.orc_quality_from_distances.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_int64, ctypes.c_double, ctypes.c_void_p]
    L.orc_mesh.restype = ctypes.c_int64
    L.orc_mesh.argtypes = [P(_Grid), ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                           ctypes.c_int64, ctypes.c_void_p]


def params(kernel_size=11, scheme=SCHEME_OCTA, bins_a=8, bins_b=8, shadow_radius=3.0,
           hit_threshold=3, hit_max=255, dedup_first=1, shadow_cos=0.0) -> Params:
    return Params(kernel_size, scheme, bins_a, bins_b, float(shadow_radius),
                  hit_threshold, hit_max, dedup_first, float(shadow_cos))


# ---------------------------------------------------------------- tables
def distance_mask(x: int, y: int, z: int) -> int:
    """Eq. 3 for one kernel offset."""
    return int(lib().orc_distance_mask(x, y, z))


def mask_table(kernel_size: int) -> np.ndarray:
    """Eq. 3 over the whole K^3 kernel, shaped (K, K, K) as [oz][oy][ox]."""
    R = (kernel_size - 1) // 2
    t = np.empty((kernel_size,) * 3, dtype=np.uint32)
    for oz in range(-R, R + 1):
        for oy in range(-R, R + 1):
            for ox in range(-R, R + 1):
                t[oz + R, oy + R, ox + R] = lib().orc_distance_mask(ox, oy, oz)
    return t


def bin_of(p: Params, d) -> int:
    """Eq. 2 (az/el) or the octahedral cell of direction d."""
    return int(lib().orc_bin(ctypes.byref(p), float(d[0]), float(d[1]), float(d[2])))


def bin_dir(p: Params, b: int) -> np.ndarray:
    """Representative direction of bin b (positive multiple of u_b)."""
    out = (ctypes.c_double * 3)()
    lib().orc_bin_dir(ctypes.byref(p), b, out)
    return np.array(out[:], dtype=np.float64)


def in_shadow(p: Params, b: int, ox: int, oy: int, oz: int) -> bool:
    """Sec. III-B hemispherical shadow membership of offset o for bin b."""
    return bool(lib().orc_in_shadow(ctypes.byref(p), b, ox, oy, oz))


def shadow_table(p: Params) -> np.ndarray:
    """Boolean (bins, K, K, K) [b][oz][oy][ox]: o in S_b."""
    K = p.kernel_size
    R = (K - 1) // 2
    nb = p.bins_a * p.bins_b
    t = np.zeros((nb, K, K, K), dtype=bool)
    rs = int(np.floor(p.shadow_radius))
    L = lib()
    for b in range(nb):
        for oz in range(-min(rs, R), min(rs, R) + 1):
            for oy in range(-min(rs, R), min(rs, R) + 1):
                for ox in range(-min(rs, R), min(rs, R) + 1):
                    t[b, oz + R, oy + R, ox + R] = L.orc_in_shadow(ctypes.byref(p), b, ox, oy, oz)
    return t


# ---------------------------------------------------------------- grid
@dataclass
class Grid:
    """Dense oracle grid (nz, ny, nx), x fastest, no padding."""
    nx: int
    ny: int
    nz: int
    res: float
    origin: tuple
    mask: np.ndarray
    sign: np.ndarray
    hits: np.ndarray

    @classmethod
    def create(cls, nx, ny, nz, res, origin=(0.0, 0.0, 0.0)):
        g = cls(nx, ny, nz, float(res), tuple(float(o) for o in origin),
                np.empty((nz, ny, nx), np.uint32), np.empty((nz, ny, nx), np.uint8),
                np.empty((nz, ny, nx), np.uint16))
        lib().orc_grid_init(ctypes.byref(g._c()))
        return g

    def _c(self) -> _Grid:
        ptr = (lambda a: None if a is None else a.ctypes.data)
        return _Grid(self.nx, self.ny, self.nz, self.res, (ctypes.c_double * 3)(*self.origin),
                     ptr(self.mask), ptr(self.sign), ptr(self.hits))

    def copy(self):
        return Grid(self.nx, self.ny, self.nz, self.res, self.origin,
                    self.mask.copy(), self.sign.copy(), self.hits.copy())


def integrate_scan_ex(g: Grid, p: Params, xyz, poses, period: int | None = None,
                      downsample: int = 1) -> dict:
    """Sec. III-C update with sequential downsampling (every downsample-th
    return) and motion compensation: return i uses poses[m(i)],
    m(i) = ((i mod period) * len(poses)) // period (period defaults to n)."""
    pts = _as_points(xyz)
    ps = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 12))
    per = int(period) if period else max(1, pts.shape[0])
    st = Stats()
    r = lib().orc_integrate_scan_ex(ctypes.byref(g._c()), ctypes.byref(p), pts.ctypes.data,
                                    pts.shape[0], ps.ctypes.data, ps.shape[0], per,
                                    int(downsample), ctypes.byref(st))
    if r < 0:
        raise RuntimeError("oracle integrate_scan_ex failed")
    return st.as_dict()


POSE_FULL = 0
POSE_YAW = 1


def pose_interp(T0, T1, tau: float, mode: int = POSE_FULL) -> np.ndarray:
    """Motion-compensation pose at time fraction tau (3 x 4)."""
    a = _as_pose(T0)
    b = _as_pose(T1)
    out = np.empty(12, np.float64)
    lib().orc_pose_interp(a.ctypes.data, b.ctypes.data, float(tau), int(mode), out.ctypes.data)
    return out.reshape(3, 4)


def pose_ramp(T0, T1, n_poses: int, mode: int = POSE_FULL) -> np.ndarray:
    """Poses at the slice centres tau_m = (m + 0.5) / n_poses, (n_poses, 3, 4)."""
    return np.stack([pose_interp(T0, T1, (m + 0.5) / n_poses, mode) for m in range(n_poses)])


def _as_points(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    return a


def _as_pose(pose) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
    return a


def integrate_scan(g: Grid, p: Params, xyz, pose) -> dict:
    """Sec. III-C update of grid g with one scan (returns in array order)."""
    pts = _as_points(xyz)
    ps = _as_pose(pose)
    st = Stats()
    gc = g._c()
    r = lib().orc_integrate_scan(ctypes.byref(gc), ctypes.byref(p), pts.ctypes.data,
                                 pts.shape[0], ps.ctypes.data, ctypes.byref(st))
    if r < 0:
        raise RuntimeError("oracle integrate_scan failed")
    return st.as_dict()


_lib_omp = None


def lib_omp():
    """The points-parallel variant's library (built on first use)."""
    global _lib_omp
    if _lib_omp is None:
        path = build_omp()
        if path is None:
            raise RuntimeError("the OpenMP variant of the oracle could not be built (no OpenMP runtime)")
        L = load(path)
        P = ctypes.POINTER
        L.orc_integrate_scan_omp.restype = ctypes.c_int64
        L.orc_integrate_scan_omp.argtypes = [P(_Grid), P(Params), ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_int, P(Stats)]
        L.orc_omp_max_threads.restype = ctypes.c_int
        L.orc_omp_max_threads.argtypes = []
        _lib_omp = L
    return _lib_omp


def integrate_scan_omp(g: Grid, p: Params, xyz, pose, threads: int | None = None) -> dict:
    """The same Sec. III-C update as integrate_scan, with the returns' contacts
    and Eq. 4-6 updates spread over `threads` host threads (per-voxel atomics;
    the first-return rule still in array order).  Bit-identical map; the
    n_mask_writes counter depends on the threads' order."""
    pts = _as_points(xyz)
    ps = _as_pose(pose)
    L = lib_omp()
    nt = int(threads) if threads else int(L.orc_omp_max_threads())
    st = Stats()
    r = L.orc_integrate_scan_omp(ctypes.byref(g._c()), ctypes.byref(p), pts.ctypes.data,
                                 pts.shape[0], ps.ctypes.data, nt, ctypes.byref(st))
    if r < 0:
        raise RuntimeError("oracle integrate_scan_omp failed")
    return st.as_dict()


def omp_threads() -> int:
    """Threads the OpenMP runtime uses by default (all host cores)."""
    return int(lib_omp().orc_omp_max_threads())


def scan_kept(g: Grid, p: Params, xyz, pose):
    """Kept returns of one scan: (contacts (m,3) int64, bins (m,) int32)."""
    pts = _as_points(xyz)
    ps = _as_pose(pose)
    n = pts.shape[0]
    c = np.empty((max(n, 1), 3), np.int64)
    b = np.empty(max(n, 1), np.int32)
    gc = g._c()
    m = lib().orc_scan_kept(ctypes.byref(p), ctypes.byref(gc), pts.ctypes.data, n,
                            ps.ctypes.data, c.ctypes.data, b.ctypes.data)
    if m < 0:
        raise RuntimeError("oracle scan_kept failed")
    return c[:m].copy(), b[:m].copy()


def query_voxels(p: Params, contacts: np.ndarray, bins: np.ndarray, q: np.ndarray,
                 mask=None, sign=None, hits=None):
    """State of each query voxel after folding the kept returns (in order).

    ``contacts``/``bins`` are concatenated ``scan_kept`` outputs of the scans
    in order.  Starting state defaults to the Sec. III-A initial state."""
    c = np.ascontiguousarray(contacts, dtype=np.int64).reshape(-1, 3)
    b = np.ascontiguousarray(bins, dtype=np.int32).reshape(-1)
    qq = np.ascontiguousarray(q, dtype=np.int64).reshape(-1, 3)
    nq = qq.shape[0]
    m = np.full(nq, 0xFFFFFFFF, np.uint32) if mask is None else np.array(mask, np.uint32)
    s = np.ones(nq, np.uint8) if sign is None else np.array(sign, np.uint8)
    h = np.zeros(nq, np.uint16) if hits is None else np.array(hits, np.uint16)
    lib().orc_query_voxels(ctypes.byref(p), c.shape[0], c.ctypes.data, b.ctypes.data, nq,
                           qq.ctypes.data, m.ctypes.data, s.ctypes.data, h.ctypes.data)
    return m, s, h


def signed_distance(mask: int, sign: int, res: float) -> float:
    """Proposed readout (parity unpinned): (+/-) popcount(mask) * res."""
    return float(lib().orc_signed_distance(mask, sign, res))


def grid_bytes_eq1(nx, ny, nz) -> int:
    """Eq. 1 with S_voxel = 8 bytes."""
    return int(lib().orc_grid_bytes_eq1(nx, ny, nz))


# ---------------------------------------------------------------- export
MC_EDGE_CORNERS = ((0, 1), (2, 3), (4, 5), (6, 7), (0, 2), (1, 3), (4, 6), (5, 7),
                   (0, 4), (1, 5), (2, 6), (3, 7))


def mc_config(cfg: int) -> np.ndarray:
    """Triangles (as edge ids, shape (t, 3)) of Marching-Cubes configuration
    cfg, bit q = corner q inside (Fig. 3 export; table derived in the C)."""
    buf = np.zeros(3 * 12, np.int32)
    n = int(lib().orc_mc_config(int(cfg), buf.ctypes.data))
    return buf[:3 * n].reshape(n, 3).copy()


def _box(g: Grid, box) -> np.ndarray:
    if box is None:
        box = (0, 0, 0, g.nx, g.ny, g.nz)
    b = np.ascontiguousarray(np.asarray(box, dtype=np.int64).reshape(6))
    if (b[:3] < 0).any() or (b[3:] < 0).any() or (b[:3] + b[3:] > (g.nx, g.ny, g.nz)).any():
        raise ValueError("box outside the grid")
    return b


def sdf_field(g: Grid, box=None) -> np.ndarray:
    """Signed distance (proposed readout) of every voxel of the box
    (x0, y0, z0, bx, by, bz), shaped (bz, by, bx), float32."""
    b = _box(g, box)
    out = np.empty((int(b[5]), int(b[4]), int(b[3])), np.float32)
    lib().orc_sdf_field(ctypes.byref(g._c()), b.ctypes.data, out.ctypes.data)
    return out


def mesh(g: Grid, box=None, iso: float = 0.0):
    """Marching Cubes at iso over the box's cells (Fig. 3: export as a mesh
    at iso = 0).  Returns (triangles (t, 3, 3) float32 map-frame vertices,
    cell number of each triangle (t,) int64), cells x-fastest."""
    b = _box(g, box)
    gc = g._c()
    n = int(lib().orc_mesh(ctypes.byref(gc), b.ctypes.data, float(iso), None, 0, None))
    tri = np.empty((n, 3, 3), np.float32)
    cell = np.empty(n, np.int64)
    if n:
        lib().orc_mesh(ctypes.byref(gc), b.ctypes.data, float(iso), tri.ctypes.data, n,
                       cell.ctypes.data)
    return tri, cell


# ---------------------------------------------------------------- quality
QUALITY_KEYS = ("accuracy", "completeness", "chamfer_l1", "precision", "recall", "fscore")


def _pts(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1, 3))


def nn_distances(ref, query) -> np.ndarray:
    """Distance of each query point to its nearest reference point (Sec.
    IV-B metrics), brute force in binary64."""
    r, q = _pts(ref), _pts(query)
    out = np.empty(q.shape[0], np.float64)
    lib().orc_nn_distances(r.ctypes.data, r.shape[0], q.ctypes.data, q.shape[0], out.ctypes.data)
    return out


def quality_from_distances(d_pred, d_gt, tolerance: float) -> dict:
    a = np.ascontiguousarray(np.asarray(d_pred, np.float64))
    b = np.ascontiguousarray(np.asarray(d_gt, np.float64))
    out = np.empty(6, np.float64)
    lib().orc_quality_from_distances(a.ctypes.data, a.size, b.ctypes.data, b.size,
                                     float(tolerance), out.ctypes.data)
    return dict(zip(QUALITY_KEYS, out.tolist()))


def quality(pred, gt, tolerance: float) -> dict:
    """Accuracy, completeness, Chamfer-L1, precision, recall and F-score of a
    predicted point set against the reference points (Sec. IV-B)."""
    return quality_from_distances(nn_distances(gt, pred), nn_distances(pred, gt), tolerance)
