"""Thin ctypes binding of libdbtsdf.so (include/dbtsdf.h).

Functions carry the C names and only marshal arguments; every step of the
integration runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the library is missing or
the process has no CUDA device, calls fail with an exception.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

DBT_OK, DBT_EINVAL, DBT_ENOMEM, DBT_ECUDA, DBT_ETIMEOUT, DBT_ESTATE = range(6)
DBT_BINS_OCTA, DBT_BINS_AZEL = 0, 1
_STATUS = {0: "DBT_OK", 1: "DBT_EINVAL", 2: "DBT_ENOMEM", 3: "DBT_ECUDA",
           4: "DBT_ETIMEOUT", 5: "DBT_ESTATE"}
HEADER = os.path.join(_build.INCLUDE, "dbtsdf.h")


class DbtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class dbt_params(ctypes.Structure):
    _fields_ = [("kernel_size", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("bins_a", ctypes.c_int32), ("bins_b", ctypes.c_int32),
                ("shadow_radius", ctypes.c_double), ("hit_threshold", ctypes.c_int32),
                ("hit_max", ctypes.c_int32), ("dedup_first", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("shadow_cos", ctypes.c_double)]


class dbt_scan_options(ctypes.Structure):
    _fields_ = [("downsample", ctypes.c_int32), ("n_poses", ctypes.c_int32),
                ("period", ctypes.c_int64), ("poses", ctypes.c_void_p)]


DBT_MOTION_FULL = 0
DBT_MOTION_YAW = 1


class dbt_tuning(ctypes.Structure):
    _fields_ = [("heavy_pairs", ctypes.c_int32), ("integrate_ctas", ctypes.c_int32),
                ("brick_depth", ctypes.c_int32)]

    def as_dict(self):
        return {"heavy_pairs": int(self.heavy_pairs), "integrate_ctas": int(self.integrate_ctas),
                "brick_depth": int(self.brick_depth)}


class dbt_quality(ctypes.Structure):
    _fields_ = [("accuracy", ctypes.c_double), ("completeness", ctypes.c_double),
                ("chamfer_l1", ctypes.c_double), ("precision", ctypes.c_double),
                ("recall", ctypes.c_double), ("fscore", ctypes.c_double),
                ("n_pred", ctypes.c_int64), ("n_gt", ctypes.c_int64)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if t is ctypes.c_double else int(getattr(self, k)))
                for k, t in self._fields_}


class dbt_grid(ctypes.Structure):
    _fields_ = [("mask", ctypes.c_void_p), ("sign", ctypes.c_void_p), ("hits", ctypes.c_void_p),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("pitch_x", ctypes.c_int32), ("res", ctypes.c_double),
                ("origin", ctypes.c_double * 3)]


class dbt_scan_stats(ctypes.Structure):
    _fields_ = [("n_input", ctypes.c_int64), ("n_valid", ctypes.c_int64),
                ("n_inside", ctypes.c_int64), ("n_kept", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("n_bricks", ctypes.c_int64),
                ("error", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class dbt_batch_item(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n", ctypes.c_int64),
                ("d_xyz", ctypes.c_void_p), ("pose", ctypes.c_double * 12)]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_SIGS = {
    "dbt_grid_layout": [ctypes.c_int32] * 3 + [_P(ctypes.c_int32)] + [_P(ctypes.c_size_t)] * 3,
    "dbt_grid_init": [_P(dbt_grid), _vp],
    "dbt_kernels_build": [_P(dbt_params), _P(_vp)],
    "dbt_kernels_destroy": [_vp],
    "dbt_kernels_export": [_vp, _vp, _vp],
    "dbt_tables_host": [_P(dbt_params), _vp, _vp],
    "dbt_bin_directions": [_vp, _vp, ctypes.c_int64, _vp, _vp],
    "dbt_scan_contacts": [_P(dbt_grid), _vp, _vp, ctypes.c_int64, _P(ctypes.c_double), _vp, _vp],
    "dbt_workspace_size": [_P(dbt_grid), _vp, ctypes.c_int64, _P(ctypes.c_size_t)],
    "dbt_workspace_create": [_P(dbt_grid), _vp, ctypes.c_int64, _vp, ctypes.c_size_t, _vp,
                             _P(_vp)],
    "dbt_workspace_reset": [_vp, _vp],
    "dbt_workspace_destroy": [_vp],
    "dbt_integrate_scan": [_P(dbt_grid), _vp, _vp, _vp, ctypes.c_int64,
                           _P(ctypes.c_double), _vp],
    "dbt_integrate_scan_host": [_P(dbt_grid), _vp, _vp, _vp, ctypes.c_int64,
                                _P(ctypes.c_double), _P(dbt_scan_stats), _vp],
    "dbt_get_scan_stats": [_vp, _P(dbt_scan_stats), _vp],
    "dbt_read_voxels": [_P(dbt_grid), _vp, ctypes.c_int64, _vp, _vp, _vp, _vp],
    "dbt_read_distance": [_P(dbt_grid), _vp, ctypes.c_int64, _vp, _vp],
    "dbt_sync": [_vp, _vp],
    "dbt_workspace_set_timing": [_vp, _vp, _vp],
    "dbt_batch_size": [_P(dbt_grid), ctypes.c_int32, _vp, ctypes.c_int64, ctypes.c_int32,
                       _P(ctypes.c_size_t)],
    "dbt_batch_create": [_P(dbt_grid), ctypes.c_int32, _vp, ctypes.c_int64, ctypes.c_int32, _vp,
                         ctypes.c_size_t, _vp, _P(_vp)],
    "dbt_batch_set_items": [_vp, _P(dbt_batch_item), ctypes.c_int32, _vp],
    "dbt_batch_run": [_vp, _vp],
    "dbt_batch_stats": [_vp, _P(dbt_scan_stats), ctypes.c_int32, _P(dbt_scan_stats), _vp],
    "dbt_batch_destroy": [_vp],
    "dbt_integrate_scan_noalloc": [_P(dbt_grid), _vp, _vp, ctypes.c_int64, _P(ctypes.c_double),
                                   _P(dbt_scan_stats), _vp],
    "dbt_op_rates": [ctypes.c_int32, _P(ctypes.c_double), _P(ctypes.c_double)],
    "dbt_noalloc_check": [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_int64],
    "dbt_scan_footprint": [_P(dbt_grid), _vp, _vp, _vp, ctypes.c_int64, _P(ctypes.c_double),
                           _vp, ctypes.c_size_t, _P(ctypes.c_int64), _vp],
    "dbt_integrate_scan_ex": [_P(dbt_grid), _vp, _vp, _vp, ctypes.c_int64, _P(ctypes.c_double),
                              _P(dbt_scan_options), _vp],
    "dbt_pose_ramp": [_P(ctypes.c_double), _P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                      _P(ctypes.c_double)],
    "dbt_workspace_set_tuning": [_vp, _vp, _P(dbt_tuning)],
    "dbt_workspace_get_tuning": [_vp, _P(dbt_tuning)],
    "dbt_batch_set_tuning": [_vp, _P(dbt_tuning)],
    "dbt_batch_get_tuning": [_vp, _P(dbt_tuning)],
    "dbt_batch_autotune": [_vp, ctypes.c_int32, _vp, _P(dbt_tuning)],
    "dbt_workspace_autotune": [_P(dbt_grid), _vp, _vp, _vp, ctypes.c_int64, _P(ctypes.c_double),
                               ctypes.c_int32, _vp, _P(dbt_tuning)],
    "dbt_sdf_field": [_P(dbt_grid), _P(ctypes.c_int32), _vp, _vp],
    "dbt_mesh_scratch_size": [_P(dbt_grid), _P(ctypes.c_int32), _P(ctypes.c_size_t)],
    "dbt_mesh_extract": [_P(dbt_grid), _P(ctypes.c_int32), ctypes.c_double, _vp, ctypes.c_size_t,
                         _vp, _vp, ctypes.c_int64, _P(ctypes.c_int64), _vp],
    "dbt_mesh_table": [_vp, _vp],
    "dbt_mesh_centroids": [_vp, ctypes.c_int64, _vp, _vp],
    "dbt_nn_scratch_size": [ctypes.c_int64, _P(ctypes.c_size_t)],
    "dbt_nn_distances": [_vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp, ctypes.c_size_t, _vp, _vp],
    "dbt_quality_scratch_size": [ctypes.c_int64, ctypes.c_int64, _P(ctypes.c_size_t)],
    "dbt_quality_metrics": [_vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_double, _vp,
                            ctypes.c_size_t, _P(dbt_quality), _vp],
}

_lib = None


def lib(path: str | None = None):
    """Load libdbtsdf.so (building it in-tree if it is missing or stale)."""
    global _lib
    if _lib is None:
        p = path or _build.build()
        L = ctypes.CDLL(p)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.dbt_last_error.restype = ctypes.c_char_p
        L.dbt_last_error.argtypes = []
        L.dbt_version.restype = ctypes.c_char_p
        L.dbt_version.argtypes = []
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions include/dbtsdf.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(dbt_\w+)\s*\(", text, re.M)


def _check(status: int):
    if status != DBT_OK:
        raise DbtError(status, lib().dbt_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C names
def dbt_version() -> str:
    return lib().dbt_version().decode()


def dbt_grid_layout(nx: int, ny: int, nz: int):
    pitch = ctypes.c_int32()
    mb, sb, hb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().dbt_grid_layout(nx, ny, nz, ctypes.byref(pitch), ctypes.byref(mb),
                                 ctypes.byref(sb), ctypes.byref(hb)))
    return pitch.value, mb.value, sb.value, hb.value


def dbt_grid_init(grid: "Grid", stream=None):
    _check(lib().dbt_grid_init(ctypes.byref(grid.c), _stream_ptr(stream)))


def make_params(kernel_size=11, scheme=DBT_BINS_OCTA, bins_a=8, bins_b=8, shadow_radius=3.0,
                hit_threshold=3, hit_max=255, dedup_first=1, shadow_cos=0.0) -> dbt_params:
    return dbt_params(kernel_size, scheme, bins_a, bins_b, float(shadow_radius), hit_threshold,
                      hit_max, dedup_first, 0, float(shadow_cos))


def dbt_tables_host(params: dbt_params):
    """Host-built tables: (K^3 masks [oz][oy][ox], bins x K^3 shadow bytes)."""
    K = params.kernel_size
    nb = params.bins_a * params.bins_b
    m = np.empty(K ** 3, np.uint32)
    s = np.empty(nb * K ** 3, np.uint8)
    _check(lib().dbt_tables_host(ctypes.byref(params), m.ctypes.data, s.ctypes.data))
    return m.reshape(K, K, K), s.reshape(nb, K, K, K)


class Kernels:
    """dbt_kernels_build / dbt_kernels_destroy."""

    def __init__(self, params: dbt_params):
        self.params = params
        h = _vp()
        _check(lib().dbt_kernels_build(ctypes.byref(params), ctypes.byref(h)))
        self.h = h

    def export(self):
        K = self.params.kernel_size
        nb = self.params.bins_a * self.params.bins_b
        m = np.empty(K ** 3, np.uint32)
        s = np.empty(nb * K ** 3, np.uint8)
        _check(lib().dbt_kernels_export(self.h, m.ctypes.data, s.ctypes.data))
        return m.reshape(K, K, K), s.reshape(nb, K, K, K)

    def close(self):
        if self.h:
            _check(lib().dbt_kernels_destroy(self.h))
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dbt_bin_directions(kernels: Kernels, dirs, stream=None):
    """Device binning of float64 (n, 3) directions (torch tensor on CUDA)."""
    import torch
    d = dirs.to(torch.float64).contiguous()
    out = torch.empty(d.shape[0], dtype=torch.int32, device=d.device)
    _check(lib().dbt_bin_directions(kernels.h, d.data_ptr(), d.shape[0], out.data_ptr(),
                                    _stream_ptr(stream)))
    return out


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class Grid:
    """Dense SoA grid in torch device memory: mask u32, sign u8, hits u16,
    each shaped (nz, ny, pitch_x)."""

    def __init__(self, nx, ny, nz, res, origin=(0.0, 0.0, 0.0), device="cuda", init=True,
                 stream=None):
        import torch
        pitch, mb, sb, hb = dbt_grid_layout(nx, ny, nz)
        self.nx, self.ny, self.nz, self.pitch = nx, ny, nz, pitch
        self.res = float(res)
        self.origin = tuple(float(o) for o in origin)
        self.mask = torch.empty((nz, ny, pitch), dtype=torch.int32, device=device)
        self.sign = torch.empty((nz, ny, pitch), dtype=torch.uint8, device=device)
        self.hits = torch.empty((nz, ny, pitch), dtype=torch.int16, device=device)
        for t in (self.mask, self.sign, self.hits):
            if t.data_ptr() % 256:
                raise DbtError(DBT_EINVAL, "torch returned a non-256-byte-aligned buffer")
        self.c = dbt_grid(self.mask.data_ptr(), self.sign.data_ptr(), self.hits.data_ptr(),
                          nx, ny, nz, pitch, self.res, (ctypes.c_double * 3)(*self.origin))
        if init:
            dbt_grid_init(self, stream)

    def load(self, mask, sign, hits=None, stream=None):
        """Sets the state from host arrays shaped (nz, ny, nx) (mask u32, sign
        u8, hits u16; hits None = 0), e.g. a map saved with numpy()."""
        import torch
        shp = (self.nz, self.ny, self.nx)
        for a in (mask, sign) + (() if hits is None else (hits,)):
            if tuple(np.shape(a)) != shp:
                raise ValueError(f"state arrays must be shaped {shp}")
        with torch.cuda.stream(stream) if stream is not None else _nullctx():
            self.mask[:, :, :self.nx].copy_(
                torch.from_numpy(np.ascontiguousarray(mask, np.uint32).view(np.int32)))
            self.sign[:, :, :self.nx].copy_(torch.from_numpy(np.ascontiguousarray(sign, np.uint8)))
            if hits is None:
                self.hits[:, :, :self.nx].zero_()
            else:
                self.hits[:, :, :self.nx].copy_(
                    torch.from_numpy(np.ascontiguousarray(hits, np.uint16).view(np.int16)))

    def numpy(self):
        """Host copies without padding: (mask u32, sign u8, hits u16), (nz, ny, nx)."""
        m = self.mask[:, :, :self.nx].cpu().numpy().view(np.uint32)
        s = self.sign[:, :, :self.nx].cpu().numpy()
        h = self.hits[:, :, :self.nx].cpu().numpy().view(np.uint16)
        return m, s, h


class Workspace:
    """Caller-owned device scratch (a torch uint8 tensor) + the library handle."""

    def __init__(self, grid: Grid, kernels: Kernels, max_points: int, stream=None):
        import torch
        nbytes = ctypes.c_size_t()
        _check(lib().dbt_workspace_size(ctypes.byref(grid.c), kernels.h, max_points,
                                        ctypes.byref(nbytes)))
        self.nbytes = nbytes.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=grid.mask.device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = self.buf.data_ptr() + off
        h = _vp()
        _check(lib().dbt_workspace_create(ctypes.byref(grid.c), kernels.h, max_points, self.ptr,
                                          self.nbytes, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.max_points = max_points

    def reset(self, stream=None):
        _check(lib().dbt_workspace_reset(self.h, _stream_ptr(stream)))

    def set_tuning(self, kernels: "Kernels", heavy_pairs: int = 64, integrate_ctas: int = 0,
                   brick_depth: int = 0):
        """dbt_workspace_set_tuning (launch choices only; results do not change)."""
        t = dbt_tuning(int(heavy_pairs), int(integrate_ctas), int(brick_depth))
        _check(lib().dbt_workspace_set_tuning(self.h, kernels.h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = dbt_tuning()
        _check(lib().dbt_workspace_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def close(self):
        if self.h:
            lib().dbt_workspace_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _pose_arg(pose):
    a = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
    return a, a.ctypes.data_as(_P(ctypes.c_double))


def dbt_integrate_scan(grid: Grid, kernels: Kernels, ws: Workspace, xyz, pose, stream=None):
    """Integrate one scan; xyz is a CUDA float32 tensor (n, 3), pose (3, 4)."""
    n = int(xyz.shape[0])
    if n and (not xyz.is_cuda or not xyz.is_contiguous()):
        raise DbtError(DBT_EINVAL, "xyz must be a contiguous CUDA float32 tensor")
    keep, pp = _pose_arg(pose)
    _check(lib().dbt_integrate_scan(ctypes.byref(grid.c), kernels.h, ws.h,
                                    xyz.data_ptr() if n else None, n, pp, _stream_ptr(stream)))


def dbt_scan_contacts(grid: Grid, kernels: Kernels, xyz, pose, stream=None):
    """Contact voxel and bin of every return, without integrating: a CUDA
    int32 (n, 4) tensor of (x, y, z, bin), x = -1 for returns that are not
    valid or fall within R voxels of the grid boundary."""
    import torch
    n = int(xyz.shape[0])
    if n and (not xyz.is_cuda or not xyz.is_contiguous() or xyz.dtype != torch.float32):
        raise DbtError(DBT_EINVAL, "xyz must be a contiguous CUDA float32 tensor")
    out = torch.empty((n, 4), dtype=torch.int32, device=xyz.device if n else "cuda")
    keep, pp = _pose_arg(pose)
    _check(lib().dbt_scan_contacts(ctypes.byref(grid.c), kernels.h, xyz.data_ptr() if n else None,
                                   n, pp, out.data_ptr() if n else None, _stream_ptr(stream)))
    return out


def dbt_integrate_scan_ex(grid: Grid, kernels: Kernels, ws: Workspace, xyz, pose=None,
                          downsample: int = 1, poses=None, period: int | None = None,
                          stream=None):
    """Integrate one scan with sequential downsampling (every downsample-th
    return) and/or motion compensation (poses: (M, 3, 4), return i uses
    poses[((i mod period) * M) // period]; period defaults to n)."""
    n = int(xyz.shape[0])
    if n and (not xyz.is_cuda or not xyz.is_contiguous()):
        raise DbtError(DBT_EINVAL, "xyz must be a contiguous CUDA float32 tensor")
    opt = dbt_scan_options(int(downsample), 0, 1, None)
    keep_p = None
    if poses is not None:
        keep_p = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 12))
        opt.n_poses = keep_p.shape[0]
        opt.period = int(period) if period else max(1, n)
        opt.poses = keep_p.ctypes.data
        pp = None
    else:
        keep, pp = _pose_arg(pose)
    _check(lib().dbt_integrate_scan_ex(ctypes.byref(grid.c), kernels.h, ws.h,
                                       xyz.data_ptr() if n else None, n, pp, ctypes.byref(opt),
                                       _stream_ptr(stream)))


def dbt_workspace_autotune(grid: Grid, kernels: Kernels, ws: Workspace, xyz, pose,
                           n_trials: int = 3, stream=None) -> dict:
    """Times the candidate tunings on one scan integrated into grid (a
    scratch grid: it is integrated repeatedly) and sets the fastest on ws."""
    n = int(xyz.shape[0])
    keep, pp = _pose_arg(pose)
    t = dbt_tuning()
    _check(lib().dbt_workspace_autotune(ctypes.byref(grid.c), kernels.h, ws.h,
                                        xyz.data_ptr() if n else None, n, pp, int(n_trials),
                                        _stream_ptr(stream), ctypes.byref(t)))
    return t.as_dict()


def dbt_pose_ramp(start, end, n_poses: int, mode: int = DBT_MOTION_FULL) -> np.ndarray:
    """Motion-compensation poses at tau_m = (m + 0.5) / n_poses, (n_poses, 3, 4)."""
    a = np.ascontiguousarray(np.asarray(start, np.float64).reshape(12))
    b = np.ascontiguousarray(np.asarray(end, np.float64).reshape(12))
    out = np.empty(12 * int(n_poses), np.float64)
    P = ctypes.POINTER(ctypes.c_double)
    _check(lib().dbt_pose_ramp(a.ctypes.data_as(P), b.ctypes.data_as(P), int(n_poses), int(mode),
                               out.ctypes.data_as(P)))
    return out.reshape(-1, 3, 4)


def dbt_integrate_scan_host(grid: Grid, kernels: Kernels, ws: Workspace, xyz_host, pose,
                            stats: dbt_scan_stats | None = None, stream=None):
    """Integrate one scan from host memory (a pinned CPU float32 tensor or a
    numpy array); the scan counters land in ``stats`` when the stream gets there
    (stored by the integrate kernel when ``stats`` lies in pinned memory)."""
    n = int(xyz_host.shape[0])
    ptr = xyz_host.data_ptr() if hasattr(xyz_host, "data_ptr") else xyz_host.ctypes.data
    keep, pp = _pose_arg(pose)
    _check(lib().dbt_integrate_scan_host(ctypes.byref(grid.c), kernels.h, ws.h, ptr if n else None,
                                         n, pp, ctypes.byref(stats) if stats is not None else None,
                                         _stream_ptr(stream)))


def dbt_get_scan_stats(ws: Workspace, stream=None, check: bool = True) -> dict:
    st = dbt_scan_stats()
    r = lib().dbt_get_scan_stats(ws.h, ctypes.byref(st), _stream_ptr(stream))
    if check:
        _check(r)
    return st.as_dict()


def dbt_read_voxels(grid: Grid, idx, stream=None):
    """idx: CUDA int32 (n, 3) voxel coordinates -> (mask, sign, hits) tensors."""
    import torch
    i = idx.to(torch.int32).contiguous()
    n = i.shape[0]
    m = torch.empty(n, dtype=torch.int32, device=i.device)
    s = torch.empty(n, dtype=torch.uint8, device=i.device)
    h = torch.empty(n, dtype=torch.int16, device=i.device)
    _check(lib().dbt_read_voxels(ctypes.byref(grid.c), i.data_ptr(), n, m.data_ptr(),
                                 s.data_ptr(), h.data_ptr(), _stream_ptr(stream)))
    return m, s, h


def dbt_read_distance(grid: Grid, idx, stream=None):
    import torch
    i = idx.to(torch.int32).contiguous()
    out = torch.empty(i.shape[0], dtype=torch.float32, device=i.device)
    _check(lib().dbt_read_distance(ctypes.byref(grid.c), i.data_ptr(), i.shape[0],
                                   out.data_ptr(), _stream_ptr(stream)))
    return out


def _box(grid: Grid, box):
    b = (0, 0, 0, grid.nx, grid.ny, grid.nz) if box is None else tuple(int(v) for v in box)
    if len(b) != 6:
        raise ValueError("box is (x0, y0, z0, bx, by, bz)")
    return (ctypes.c_int32 * 6)(*b)


def dbt_sdf_field(grid: Grid, box=None, stream=None):
    """Signed distance of every voxel of the box, a (bz, by, bx) float32
    tensor on the grid's device."""
    import torch
    b = _box(grid, box)
    out = torch.empty((b[5], b[4], b[3]), dtype=torch.float32, device=grid.mask.device)
    _check(lib().dbt_sdf_field(ctypes.byref(grid.c), b, out.data_ptr() if out.numel() else None,
                               _stream_ptr(stream)))
    return out


def dbt_mesh_scratch_size(grid: Grid, box=None) -> int:
    n = ctypes.c_size_t()
    _check(lib().dbt_mesh_scratch_size(ctypes.byref(grid.c), _box(grid, box), ctypes.byref(n)))
    return int(n.value)


def dbt_mesh_extract(grid: Grid, box=None, iso: float = 0.0, with_cells: bool = False,
                     scratch=None, stream=None):
    """Marching Cubes at iso over the box (two passes: count, then emit into
    a buffer of exactly that size).  Returns (triangles (t, 3, 3) float32,
    cell numbers (t,) int64 or None) on the grid's device."""
    import torch
    dev = grid.mask.device
    b = _box(grid, box)
    need = dbt_mesh_scratch_size(grid, box)
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(need, dtype=torch.uint8, device=dev)
    n = ctypes.c_int64()
    sp = _stream_ptr(stream)
    _check(lib().dbt_mesh_extract(ctypes.byref(grid.c), b, float(iso), scratch.data_ptr(), need,
                                  None, None, 0, ctypes.byref(n), sp))
    t = int(n.value)
    tri = torch.empty((t, 3, 3), dtype=torch.float32, device=dev)
    cell = torch.empty(t, dtype=torch.int64, device=dev) if with_cells else None
    if t:
        m = ctypes.c_int64()
        _check(lib().dbt_mesh_extract(ctypes.byref(grid.c), b, float(iso), scratch.data_ptr(),
                                      need, tri.data_ptr(),
                                      cell.data_ptr() if cell is not None else None, t,
                                      ctypes.byref(m), sp))
        if int(m.value) != t:
            raise RuntimeError("grid changed between the mesh passes")
    return tri, cell


def dbt_mesh_table():
    """(ntri (256,) uint8, edges (256, 5, 3) uint8) of the library's table."""
    nt = np.zeros(256, np.uint8)
    ed = np.zeros(256 * 15, np.uint8)
    _check(lib().dbt_mesh_table(nt.ctypes.data, ed.ctypes.data))
    return nt, ed.reshape(256, 5, 3)


def dbt_sync(stream=None, ws: Workspace | None = None):
    _check(lib().dbt_sync(_stream_ptr(stream), ws.h if ws is not None else None))


def dbt_workspace_set_timing(ws: Workspace, ev_begin=None, ev_end=None):
    """Record torch.cuda.Event pair around each later scan's integrate kernel."""
    _check(lib().dbt_workspace_set_timing(ws.h, ev_begin.cuda_event if ev_begin else None,
                                          ev_end.cuda_event if ev_end else None))


def footprint_bytes(grid: Grid) -> int:
    words = (grid.pitch * grid.ny * grid.nz + 31) // 32
    return 2 * words * 4 + 16


def dbt_scan_footprint(grid: Grid, kernels: Kernels, ws: Workspace, xyz, pose, bits, stream=None):
    """(U, U_s) of one scan: distinct voxels under kept returns' kernels and
    shadows.  ``bits`` is a CUDA uint8 tensor of footprint_bytes(grid)."""
    n = int(xyz.shape[0])
    keep, pp = _pose_arg(pose)
    out = (ctypes.c_int64 * 2)()
    _check(lib().dbt_scan_footprint(ctypes.byref(grid.c), kernels.h, ws.h,
                                    xyz.data_ptr() if n else None, n, pp, bits.data_ptr(),
                                    bits.numel(), out, _stream_ptr(stream)))
    return int(out[0]), int(out[1])


def dbt_integrate_scan_noalloc(grid: Grid, kernels: Kernels, xyz, pose,
                               stats: dbt_scan_stats | None = None, stream=None):
    """Integrate one scan without any workspace: the library's fixed scratch
    is used (at most 65,536 returns; see include/dbtsdf.h)."""
    n = int(xyz.shape[0])
    keep, pp = _pose_arg(pose)
    _check(lib().dbt_integrate_scan_noalloc(ctypes.byref(grid.c), kernels.h,
                                            xyz.data_ptr() if n else None, n, pp,
                                            ctypes.byref(stats) if stats is not None else None,
                                            _stream_ptr(stream)))


def dbt_op_rates(iters: int = 1 << 14) -> tuple[float, float]:
    """(voxel-ANDs/s, counter increments/s): the measured peak rates of the
    integration's elementary shared-memory updates on the current device."""
    a, c = ctypes.c_double(), ctypes.c_double()
    _check(lib().dbt_op_rates(iters, ctypes.byref(a), ctypes.byref(c)))
    return a.value, c.value


def dbt_noalloc_check(nx: int, ny: int, nz: int, kernel_size: int, n: int) -> None:
    """Raises DbtError (DBT_EINVAL) when dbt_integrate_scan_noalloc cannot
    take n returns on an nx x ny x nz grid at this kernel size.  Host only."""
    _check(lib().dbt_noalloc_check(nx, ny, nz, kernel_size, n))


class Batch:
    """dbt_batch_*: many scans of several grids integrated by one launch
    sequence (dbt_batch_run), which is also capturable in a CUDA graph."""

    def __init__(self, grids: list, kernels: Kernels, max_points: int, max_items: int, stream=None):
        import torch
        self.grids = list(grids)
        arr = (dbt_grid * len(grids))(*[g.c for g in grids])
        self._arr = arr
        nbytes = ctypes.c_size_t()
        _check(lib().dbt_batch_size(arr, len(grids), kernels.h, max_points, max_items,
                                    ctypes.byref(nbytes)))
        self.nbytes = nbytes.value
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=grids[0].mask.device)
        ptr = self.buf.data_ptr() + (-self.buf.data_ptr()) % 256
        h = _vp()
        _check(lib().dbt_batch_create(arr, len(grids), kernels.h, max_points, max_items, ptr,
                                      self.nbytes, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.kernels = kernels
        self.n_items = 0
        self._keep = []

    def set_items(self, items, stream=None):
        """items: list of (grid index, CUDA float32 (n, 3) tensor, pose (3, 4))."""
        arr = (dbt_batch_item * max(1, len(items)))()
        keep = []
        for i, (gi, xyz, pose) in enumerate(items):
            n = int(xyz.shape[0])
            p = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(12))
            arr[i].grid = gi
            arr[i].reserved = 0
            arr[i].n = n
            arr[i].d_xyz = xyz.data_ptr() if n else None
            arr[i].pose[:] = p.tolist()
            keep.append(xyz)
        _check(lib().dbt_batch_set_items(self.h, arr, len(items), _stream_ptr(stream)))
        self._keep = keep
        self.n_items = len(items)

    def run(self, stream=None):
        _check(lib().dbt_batch_run(self.h, _stream_ptr(stream)))

    def set_tuning(self, heavy_pairs: int = 64, integrate_ctas: int = 0, brick_depth: int = 0):
        """dbt_batch_set_tuning (launch choices only; results do not change)."""
        t = dbt_tuning(int(heavy_pairs), int(integrate_ctas), int(brick_depth))
        _check(lib().dbt_batch_set_tuning(self.h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = dbt_tuning()
        _check(lib().dbt_batch_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def autotune(self, n_trials: int = 3, stream=None) -> dict:
        """dbt_batch_autotune: times the candidate tunings on the current
        items (integrating them repeatedly: use scratch grids) and keeps the
        fastest."""
        t = dbt_tuning()
        _check(lib().dbt_batch_autotune(self.h, int(n_trials), _stream_ptr(stream), ctypes.byref(t)))
        return t.as_dict()

    def stats(self, stream=None, check=True):
        per = (dbt_scan_stats * max(1, self.n_items))()
        tot = dbt_scan_stats()
        r = lib().dbt_batch_stats(self.h, per, self.n_items, ctypes.byref(tot), _stream_ptr(stream))
        if check:
            _check(r)
        return [per[i].as_dict() for i in range(self.n_items)], tot.as_dict()

    def close(self):
        if self.h:
            lib().dbt_batch_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ quality
def _pts_arg(x):
    n = int(x.shape[0])
    if n and (not x.is_cuda or not x.is_contiguous() or x.dim() != 2 or x.shape[1] != 3):
        raise DbtError(DBT_EINVAL, "points must be a contiguous CUDA float32 (n, 3) tensor")
    return n, (x.data_ptr() if n else None)


def dbt_mesh_centroids(tri, stream=None):
    """Centroids (t, 3) of a (t, 3, 3) float32 triangle tensor."""
    import torch
    t = tri.reshape(-1, 9)
    n = int(t.shape[0])
    out = torch.empty((n, 3), dtype=torch.float32, device=tri.device)
    _check(lib().dbt_mesh_centroids(t.data_ptr() if n else None, n,
                                    out.data_ptr() if n else None, _stream_ptr(stream)))
    return out


def dbt_nn_distances(ref, query, stream=None):
    """Exact nearest-neighbour distance of each query point to ref (float32)."""
    import torch
    nr, pr = _pts_arg(ref)
    nq, pq = _pts_arg(query)
    nbytes = ctypes.c_size_t()
    _check(lib().dbt_nn_scratch_size(nr, ctypes.byref(nbytes)))
    dev = query.device if nq else ref.device
    scratch = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    out = torch.empty(nq, dtype=torch.float32, device=dev)
    _check(lib().dbt_nn_distances(pr, nr, pq, nq, scratch.data_ptr(), nbytes.value,
                                  out.data_ptr() if nq else None, _stream_ptr(stream)))
    return out


def dbt_quality_metrics(pred, gt, tolerance: float, stream=None) -> dict:
    """Accuracy, completeness, Chamfer-L1, precision, recall, F-score (Sec. IV-B)."""
    import torch
    npd, pp = _pts_arg(pred)
    ngt, pg = _pts_arg(gt)
    nbytes = ctypes.c_size_t()
    _check(lib().dbt_quality_scratch_size(npd, ngt, ctypes.byref(nbytes)))
    dev = pred.device if npd else gt.device
    scratch = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
    q = dbt_quality()
    _check(lib().dbt_quality_metrics(pp, npd, pg, ngt, float(tolerance), scratch.data_ptr(),
                                     nbytes.value, ctypes.byref(q), _stream_ptr(stream)))
    return q.as_dict()
