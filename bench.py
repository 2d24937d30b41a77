#!/usr/bin/env python
"""DB-TSDF scan-integration benchmark (one JSON line on stdout).

Default workload: the urban sequence -- 100 scans of a 64-beam spinning
LiDAR (64 x 1024 = 65,536 float32 returns, +-22.5 deg, 1-60 m, 2 cm noise,
2 % dropouts) along a closed trajectory (1 m per scan, float64 SE(3) poses)
through a synthetic urban block (ground, 40 buildings, 200 poles), into a
dense 1600 x 1600 x 320 grid at 0.05 m (80 x 80 x 16 m), K = 11, 64
octahedral bins, r_s = 3, T = 3, H_max = 255.  Synthetic data stands in for
the paper's Newer College / Mai City sequences.

A step is one scan through the whole path (transform, voxel, bin, first
return rule, brick binning, integration of Eqs. 4-6).  W warm-up scans run
on the grid, which is then re-initialised, and K scans are timed in
trajectory order from an empty map (scan k = trajectory scan k mod 100), as
in online mapping.  The 5.7 GB grid exceeds the 129 MB L2; consecutive scans
share map regions as a moving robot's do, and no L2 flush is inserted.

value: kept returns integrated per second (the returns that reach Eqs.
4-6: valid, neighbourhood inside the map, first of their voxel), with the
scans resident in HBM; raw_points_per_s counts every return handed in.
e2e: the same through the host-buffer entry point dbt_integrate_scan_host
(pinned host scans copied in, scan counters copied out, inside the timed
region).  roofline: the brick integration kernel against two ceilings --
bytes, 12 N + 8 U + 6 U_s + 96 per scan (points in, read and write every
covered mask, counter and sign of every shadow voxel, the pose; U and U_s
counted exactly per scan before timing) over the measured HBM copy
bandwidth, and ops, N_kept K^3 voxel-ANDs plus the shadow increments (Eq. 7)
over the measured peak rates of the kernel's own shared-memory updates
(dbt_op_rates) -- frac = the larger ceiling time over the kernel's CUDA-event
time.  Extra keys: per-scan latency over all 100 workload scans, the batched
graph-replayed form, the high-resolution workload (2000 x 2000 x 400 at 0.02
m, 262,144 returns per scan), the paper's parameters (K = 21, 40 x 40 az/el
bins) on the room and urban scans, 32 uneven maps in one graph against 256
plain launches, and the serving loop (continuous batching against FIFO at
equal offered loads).

--impl reference times the oracle (plain single-threaded C) on the same
workload and metric, on a bounded sample of returns per step.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "LiDAR points integrated/sec (ms/scan)"
UNIT = "points/s"
INTEGRATE_SRC = os.path.join(ROOT, "paper_2509_20081_gb300", "csrc", "integrate.cu")

# ncu dram__bytes_read.sum + dram__bytes_write.sum of k_integrate, per kept
# return, from the capture summarised under profiles/ (valid only for the
# integrate.cu source with this sha256 prefix; otherwise traffic is null).
NCU_TRAFFIC = {"integrate_sha": "80ab203c51b11876", "bytes_per_kept_return": 855.8,
               "source": "profiles/k_integrate_urban_half.md (urban_half, 39.9 k kept returns "
                         "per scan, 34.2 MB DRAM read+write per launch), scaled by kept returns"}

# Kernels one scan (or one batch run) launches: voxelize, alloc, fill, integrate.
KERNELS_PER_SCAN = 4
INTEGRATE_TIMING_EVERY = 10

WORKLOADS = {
    "urban": dict(n_scans=100, scale=1.0, res=0.05, beams=64, width=1024, seed_offset=1),
    "urban_half": dict(n_scans=20, scale=0.5, res=0.05, beams=64, width=1024, seed_offset=1),
    "highres": dict(n_scans=50, scale=0.5, res=0.02, beams=128, width=2048, seed_offset=2),
}


def load_workload(name: str) -> synth.Workload:
    """Generate (or reuse from a per-machine cache) the workload's scans."""
    if name == "room":
        return synth.room_scan()
    kw = WORKLOADS[name]
    key = hashlib.sha256((name + json.dumps(kw, sort_keys=True) +
                          open(os.path.join(ROOT, "synth", "__init__.py")).read()).encode()).hexdigest()[:16]
    cache = os.path.join(tempfile.gettempdir(), f"dbtsdf_{name}_{key}.npz")
    w0 = None
    if os.path.exists(cache):
        try:
            z = np.load(cache)
            g = synth.GridSpec(*[int(v) for v in z["dims"]], float(z["res"]))
            scans = [(z["pts"][i], z["poses"][i]) for i in range(z["pts"].shape[0])]
            return synth.Workload(name, g, scans, dict(synth.DEFAULT_PARAMS))
        except Exception:
            pass
    w0 = synth.urban_sequence(**kw)
    tmp = cache + f".{os.getpid()}.npz"
    np.savez(tmp, pts=np.stack([s[0] for s in w0.scans]), poses=np.stack([s[1] for s in w0.scans]),
             dims=np.array([w0.grid.nx, w0.grid.ny, w0.grid.nz]), res=np.array(w0.grid.res))
    os.replace(tmp, cache)
    return w0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during the run.

    NVML (libnvidia-ml, read-only queries) is polled from a thread every
    ~0.25 ms, so that even a few-millisecond timed region gets samples;
    without NVML, nvidia-smi is run at its fastest period (20 ms).
    mark() stamps a region; stats(region) summarises its samples."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReason* bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index: int, pci_bus_id: str | None = None, period_s: float = 0.00025):
        import threading
        self.samples = []            # (time, sm_mhz, reasons bitmask)
        self.max_mhz = None
        self.marks = {}
        self.proc = None
        self.path = None
        self.thread = None
        self.stop_flag = threading.Event()
        self.source = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            ok = False
            if pci_bus_id:
                ok = nv.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(h)) == 0
            if not ok and nv.nvmlDeviceGetHandleByIndex_v2(gpu_index, ctypes.byref(h)) != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:     # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons

            def poll():
                c = ctypes.c_uint()
                r = ctypes.c_ulonglong()
                while not self.stop_flag.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c)) == 0:
                        rr = r.value if reasons_fn(h, ctypes.byref(r)) == 0 else 0
                        self.samples.append((time.perf_counter(), float(c.value), rr))
                    time.sleep(period_s)
            self.thread = threading.Thread(target=poll, daemon=True)
            self.thread.start()
            self.source = "nvml"
        except (OSError, AttributeError):
            self._start_smi(gpu_index)

    def _start_smi(self, gpu_index):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi"
        except Exception:
            self.proc = None

    def wait_first(self, timeout_s: float = 5.0):
        """Blocks until the first sample exists, so that samples cover what follows."""
        t_end = time.time() + timeout_s
        while time.time() < t_end:
            if self.samples or (self.path and os.path.exists(self.path) and os.path.getsize(self.path) > 0):
                return
            if self.thread is None and self.proc is None:
                return
            time.sleep(0.001)

    def mark(self, name: str, begin: bool):
        self.marks.setdefault(name, [None, None])[0 if begin else 1] = time.perf_counter()

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=2)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            now = time.perf_counter()
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    bits = sum(b for b, k in ((0x8, 5), (0x40, 6), (0x20, 7), (0x4, 8))
                               if f[k].lower() == "active")
                    self.samples.append((now, float(f[1]), bits))
                    if f[2].replace(".", "").isdigit():
                        self.max_mhz = max(self.max_mhz or 0.0, float(f[2]))
            os.unlink(self.path)

    def stats(self, region: str | None = None):
        rows = self.samples
        if region is not None and self.source == "nvml" and region in self.marks:
            t0, t1 = self.marks[region]
            rows = [r for r in rows if t0 is not None and t1 is not None and t0 <= r[0] <= t1]
        if not rows:
            return None
        bits = 0
        for r in rows:
            bits |= r[2]
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(v for b, v in self.REASONS.items() if bits & b),
                "samples": len(rows), "source": self.source}


def pci_bus_id(torch, dev) -> str | None:
    p = torch.cuda.get_device_properties(dev)
    try:
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except AttributeError:
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def integrate_sha() -> str:
    return hashlib.sha256(open(INTEGRATE_SRC, "rb").read()).hexdigest()[:16]


# ------------------------------------------------------------------ CPU baseline
def cpu_baseline(w: synth.Workload, budget_s: float = 15.0, max_scans: int | None = None):
    """Oracle (single-threaded C) on the first scans of the workload until
    ~budget_s of CPU work; returns (points/s, scans run, seconds)."""
    import oracle
    g = oracle.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    p = oracle.params(**w.params)
    t0 = time.perf_counter()
    done = 0
    pts_total = 0
    kept_total = 0
    for pts, pose in w.scans:
        st = oracle.integrate_scan(g, p, pts, pose)
        done += 1
        pts_total += len(pts)
        kept_total += st["n_kept"]
        if time.perf_counter() - t0 > budget_s or (max_scans and done >= max_scans):
            break
    dt = time.perf_counter() - t0
    return pts_total / dt, done, dt, kept_total / dt


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu, else the ISA)."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_baseline_parallel(w: synth.Workload, budget_s: float = 15.0) -> dict:
    """The oracle's points-parallel variant (OpenMP over the returns, atomic
    per-voxel updates, as the paper runs on its host cores) on all host
    cores, on the first scans of the workload until ~budget_s."""
    import oracle
    if oracle.build_omp() is None:
        return {"unavailable": "the C compiler has no OpenMP runtime"}
    threads = oracle.omp_threads()
    g = oracle.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    p = oracle.params(**w.params)
    t0 = time.perf_counter()
    done = 0
    pts_total = 0
    kept_total = 0
    for pts, pose in w.scans:
        st = oracle.integrate_scan_omp(g, p, pts, pose, threads=threads)
        done += 1
        pts_total += len(pts)
        kept_total += st["n_kept"]
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": kept_total / dt, "raw_points_per_s": pts_total / dt, "unit": UNIT,
            "cores": threads, "kind": "oracle_openmp",
            "sample": f"first {done} scans of the workload, full grid, {dt:.1f} s on "
                      f"{threads} threads", "cpu": cpu_model(), "host_cores": os.cpu_count()}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = load_workload(args.workload)
    import oracle
    p = oracle.params(**w.params)
    g = oracle.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    stride = args.ref_stride
    times = []
    pts_done = 0
    kept_done = 0
    for s in range(args.warmup + args.steps):
        pts, pose = w.scans[s % len(w.scans)]
        sample = np.ascontiguousarray(pts[::stride])
        t0 = time.perf_counter()
        st = oracle.integrate_scan(g, p, sample, pose)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            pts_done += len(sample)
            kept_done += st["n_kept"]
    total = sum(times)
    value = kept_done / total
    sample_desc = (f"every {stride}th return of each scan ({pts_done // max(1, args.steps)} "
                   f"returns/step, {kept_done // max(1, args.steps)} kept) of the "
                   f"{args.workload} workload, grid at full size")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(args, w),
            "points_counted": "kept returns (valid, K^3 neighbourhood inside the map, first of "
                              "their voxel)",
            "raw_points_per_s": pts_done / total,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample_desc, "cpu": cpu_model(), "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, w):
    return {"workload": f"{args.workload}: {len(w.scans)} scans x {len(w.scans[0][0])} returns, "
                        f"grid {w.grid.nx}x{w.grid.ny}x{w.grid.nz} at {w.grid.res} m",
            "kernel": w.params["kernel_size"], "bins": "octahedral 8x8",
            "shadow_radius": w.params["shadow_radius"], "T": w.params["hit_threshold"],
            "H_max": w.params["hit_max"], "points_per_scan": len(w.scans[0][0]),
            "parallelism": f"replicas x{args.gpus}",
            "l2": "grid larger than L2 (no flush); consecutive scans overlap as on a trajectory"}


# ------------------------------------------------------------------ our arm
class Ctx:
    """What every leg of our arm shares: the modules, the device, the
    measured peaks and the clock sampler."""

    def __init__(self, args, rank, world):
        import torch

        import paper_2509_20081_gb300 as dbt
        from paper_2509_20081_gb300 import dbtsdf as B
        self.torch, self.dbt, self.B = torch, dbt, B
        self.args, self.rank, self.world = args, rank, world
        self.dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(self.dev)
        self.stream = torch.cuda.current_stream()
        self.peak, self.peak_kind = measured_peaks()
        self._op_rates = None
        self.clocks = ClockSampler(self.dev.index, pci_bus_id(torch, self.dev)) if rank == 0 else None
        if self.clocks:
            self.clocks.wait_first()

    def op_rates(self):
        if self._op_rates is None:
            self._op_rates = self.B.dbt_op_rates(1 << 14)
        return self._op_rates

    def barrier(self):
        if self.world > 1:
            self.torch.distributed.barrier()


def shadow_sizes(B, params) -> np.ndarray:
    """|S_b| per bin, from the library's host-built tables (Sec. III-B)."""
    _, sh = B.dbt_tables_host(params)
    return sh.reshape(sh.shape[0], -1).astype(np.int64).sum(1)


def scan_work(ctx, g, k, ws, params, x, pose, bits, s_sizes) -> dict:
    """Exact work of one scan, outside any timed region: N returns handed
    in, U and U_s (distinct voxels under the kept returns' K^3 neighbourhoods
    and shadow sets, dbt_scan_footprint), the kept returns (first of their
    contact voxel among those inside, from dbt_scan_contacts) and their
    shadow increments sum |S_b|."""
    dbt, B = ctx.dbt, ctx.B
    u, us = B.dbt_scan_footprint(g, k, ws, x, pose, bits)
    c = dbt.dbt_scan_contacts(g, k, x, pose).cpu().numpy()
    v = c[:, 0] >= 0
    key = (c[v, 2].astype(np.int64) * g.c.ny + c[v, 1]) * g.c.pitch_x + c[v, 0]
    bins = c[v, 3]
    if params.dedup_first:
        _, first = np.unique(key, return_index=True)
        bins = bins[first]
    return {"n": int(x.shape[0]), "u": int(u), "us": int(us), "kept": int(len(bins)),
            "shadow": int(s_sizes[bins].sum())}


def alg_bytes(wk: dict) -> int:
    """Bytes one scan must move at least (12 N + 8 U + 6 U_s + 96): its
    returns in, each covered mask read and written, counter (2 + 2) and sign
    (1 + 1) of each shadow voxel, the binary64 pose."""
    return 12 * wk["n"] + 8 * wk["u"] + 6 * wk["us"] + 96


def roofline(ctx, works: list, ms_int: float, K: int, traffic) -> dict:
    """The integrate kernel against its byte and op ceilings; frac = the
    larger ceiling time over the measured time."""
    and_rate, cnt_rate = ctx.op_rates()
    ab = statistics.mean(alg_bytes(w) for w in works)
    n_and = statistics.mean(w["kept"] * K ** 3 for w in works)
    n_cnt = statistics.mean(w["shadow"] for w in works)
    t = ms_int * 1e-3
    t_hbm = ab / (ctx.peak * 1e9)
    t_op = n_and / and_rate + n_cnt / cnt_rate
    op_side = {"voxel_ands": n_and, "counter_incs": n_cnt, "and_per_s": and_rate,
               "count_per_s": cnt_rate, "t_ms": t_op * 1e3, "frac": t_op / t,
               "source": "dbt_op_rates micro-benchmark on this GPU (Eq. 4 as byte-wise minima of "
                         "packed codes, Eq. 5 16-bit increments, shared memory, 4 CTAs/SM)"}
    hbm_side = {"alg_bytes": ab, "t_ms": t_hbm * 1e3, "frac": t_hbm / t,
                "achieved_gbs": ab / t / 1e9, "peak_gbs": ctx.peak}
    base = {"kernel": "k_integrate", "ms_per_launch": ms_int, "traffic": traffic,
            "alg_bytes_per_launch": ab, "peak_source": f"{ctx.peak_kind} hbm_gbs",
            "hbm_side": hbm_side, "op_side": op_side}
    if t_hbm >= t_op:
        base.update({"bound": "hbm", "achieved": ab / t / 1e9, "peak": ctx.peak, "unit": "GB/s",
                     "frac": t_hbm / t})
    else:
        ops = n_and + n_cnt
        base.update({"bound": "alu", "achieved": ops / t / 1e12, "peak": ops / t_op / 1e12,
                     "unit": "T updates/s", "frac": t_op / t})
    return base


def plain_leg(ctx, w, pdict, steps: int, warmup: int, autotune: bool, e2e: bool = False,
              region: str | None = None, latency_scans: int | None = None, traffic_fn=None):
    """Per-scan launches of w's scans on a fresh map: the timed region (K
    scans back to back, the integrate kernel of every tenth bracketed by
    events), per-scan latency over the workload's scans (an event between
    scans), optionally the host-buffer entry point."""
    torch, dbt, B = ctx.torch, ctx.dbt, ctx.B
    stream = ctx.stream
    nsc = len(w.scans)
    p = dbt.make_params(**pdict)
    k = dbt.Kernels(p)
    g = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    ws = dbt.Workspace(g, k, max(len(s[0]) for s in w.scans))
    d_scans = [torch.from_numpy(np.ascontiguousarray(s[0])).to(ctx.dev) for s in w.scans]
    poses = [s[1] for s in w.scans]
    bits = torch.empty(B.footprint_bytes(g), dtype=torch.uint8, device=ctx.dev)
    ss = shadow_sizes(B, p)
    works = [scan_work(ctx, g, k, ws, p, d_scans[i], poses[i], bits, ss) for i in range(nsc)]
    del bits
    torch.cuda.empty_cache()
    tuning = (B.dbt_workspace_autotune(g, k, ws, d_scans[0], poses[0], n_trials=3) if autotune
              else ws.tuning())
    for s_ in range(warmup):
        dbt.dbt_integrate_scan(g, k, ws, d_scans[s_ % nsc], poses[s_ % nsc])
    dbt.dbt_grid_init(g)
    ws.reset()
    timed_steps = list(range(0, steps, INTEGRATE_TIMING_EVERY))
    evb = {s_: torch.cuda.Event(enable_timing=True) for s_ in timed_steps}
    eve = {s_: torch.cuda.Event(enable_timing=True) for s_ in timed_steps}
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    for e in list(evb.values()) + list(eve.values()):   # torch creates the CUDA event on first record
        e.record(stream)
    ctx.barrier()
    torch.cuda.synchronize()
    if ctx.clocks and region:
        ctx.clocks.mark(region, True)
    t0.record(stream)
    for s_ in range(steps):
        if s_ in evb:
            B.dbt_workspace_set_timing(ws, evb[s_], eve[s_])
        dbt.dbt_integrate_scan(g, k, ws, d_scans[s_ % nsc], poses[s_ % nsc])
        if s_ in evb:
            B.dbt_workspace_set_timing(ws, None, None)
    t1.record(stream)
    torch.cuda.synchronize()
    if ctx.clocks and region:
        ctx.clocks.mark(region, False)
    ctx.barrier()
    ms = t0.elapsed_time(t1)
    st = dbt.dbt_get_scan_stats(ws)
    assert st["error"] == 0, st
    t_int = [evb[s_].elapsed_time(eve[s_]) for s_ in timed_steps]

    # per-scan latency over the workload's scans on a fresh map: an event
    # between scans, and around each integrate kernel
    nl = latency_scans or nsc
    dbt.dbt_grid_init(g)
    ws.reset()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(nl + 1)]
    ib = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    ie = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    for e in ib + ie:                # created by torch on its first record
        e.record(stream)
    torch.cuda.synchronize()
    for s_ in range(nl):
        evs[s_].record(stream)
        B.dbt_workspace_set_timing(ws, ib[s_], ie[s_])
        dbt.dbt_integrate_scan(g, k, ws, d_scans[s_ % nsc], poses[s_ % nsc])
    evs[nl].record(stream)
    torch.cuda.synchronize()
    B.dbt_workspace_set_timing(ws, None, None)
    t_scan = sorted(evs[s_].elapsed_time(evs[s_ + 1]) for s_ in range(nl))
    t_int_all = [ib[s_].elapsed_time(ie[s_]) for s_ in range(nl)]

    kept_timed = sum(works[s_ % nsc]["kept"] for s_ in range(steps))
    raw_timed = sum(works[s_ % nsc]["n"] for s_ in range(steps))
    ms_int = statistics.mean(t_int)
    tw = [works[s_ % nsc] for s_ in timed_steps]
    traffic = traffic_fn(statistics.mean(x["kept"] for x in tw)) if traffic_fn else None
    out = {"value": ctx.world * kept_timed / (ms * 1e-3), "unit": UNIT,
           "raw_points_per_s": ctx.world * raw_timed / (ms * 1e-3),
           "ms_per_step": ms / steps, "steps": steps,
           "kept_per_scan": kept_timed / steps, "returns_per_scan": raw_timed / steps,
           "latency_ms": {"p50": pct(t_scan, 50), "p99": pct(t_scan, 99), "max": t_scan[-1],
                          "scans": nl,
                          "what": "device time per scan, plain per-scan launches, over the "
                                  "workload's scans from an empty map (an event between scans)"},
           "tuning": tuning,
           "roofline": roofline(ctx, tw, ms_int, pdict["kernel_size"], traffic),
           "integrate_ms_all_scans": {"mean": statistics.mean(t_int_all), "max": max(t_int_all),
                                      "share_of_scan": statistics.mean(t_int_all) /
                                      statistics.mean(t_scan)}}
    out["roofline"].update({"timed_launches": f"{len(t_int)} of {steps} (every "
                                              f"{INTEGRATE_TIMING_EVERY}th scan of the timed region)",
                            "share_of_step": ms_int / (ms / steps)})
    if e2e:
        dbt.dbt_grid_init(g)
        ws.reset()
        h_scans = [torch.from_numpy(np.ascontiguousarray(s[0])).pin_memory() for s in w.scans]
        h_stats = torch.zeros((steps, 64), dtype=torch.uint8).pin_memory()
        st_ptrs = [B.dbt_scan_stats.from_address(h_stats[s_].data_ptr()) for s_ in range(steps)]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ctx.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for s_ in range(steps):
            B.dbt_integrate_scan_host(g, k, ws, h_scans[s_ % nsc], poses[s_ % nsc], st_ptrs[s_])
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.barrier()
        ms_e2e = e0.elapsed_time(e1)
        assert all(sp.error == 0 and sp.n_input == int(h_scans[s_ % nsc].shape[0])
                   and sp.n_kept == works[s_ % nsc]["kept"]
                   for s_, sp in enumerate(st_ptrs)), "scan counters of the host entry point"
        npts = len(w.scans[0][0])
        out["e2e_ms"] = ms_e2e
        out["e2e"] = {"value": ctx.world * kept_timed / (ms_e2e * 1e-3), "unit": UNIT,
                      "h2d_bytes_per_step": npts * 12,
                      "d2h_bytes_per_step": ctypes.sizeof(B.dbt_scan_stats),
                      "ms_per_step": ms_e2e / steps,
                      "raw_points_per_s": ctx.world * raw_timed / (ms_e2e * 1e-3)}
    out["_state"] = (k, g, d_scans, poses, works)
    return out


def run_ours(args, rank, world):
    ctx = Ctx(args, rank, world)
    torch = ctx.torch
    w = load_workload(args.workload)
    pdict = dict(w.params)

    def traffic_fn(kept):
        if NCU_TRAFFIC["integrate_sha"] == integrate_sha() and NCU_TRAFFIC["bytes_per_kept_return"]:
            return NCU_TRAFFIC["bytes_per_kept_return"] * kept
        return None

    main = plain_leg(ctx, w, pdict, args.steps, args.warmup, not args.no_autotune, e2e=True,
                     region="timed", traffic_fn=traffic_fn)
    k, g, d_scans, poses, works = main.pop("_state")
    batched = run_batched(ctx, w, k, g, d_scans, poses, args.steps, works)
    del k, g, d_scans, poses
    torch.cuda.empty_cache()
    ms, ms_e2e = max_over_ranks([main["ms_per_step"] * args.steps, main["e2e_ms"]], ctx.dev, world)
    extra = {}
    if not args.no_extra_legs and args.workload == "urban":
        extra = extra_legs(ctx, args)
    if ctx.clocks:
        ctx.clocks.stop()
    if rank != 0:
        return 0
    rf = main["roofline"]
    rf["traffic_source"] = (NCU_TRAFFIC["source"] if rf["traffic"] is not None
                            else "no ncu capture of this integrate.cu yet")
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": workload_config(args, w),
        "points_counted": "kept returns (valid, K^3 neighbourhood inside the map, first of their "
                          "voxel): the returns Eqs. 4-6 integrate",
        "raw_points_per_s": main["raw_points_per_s"],
        "kept_per_scan": main["kept_per_scan"], "returns_per_scan": main["returns_per_scan"],
        "e2e": main["e2e"],
        "latency_ms": main["latency_ms"],
        "batched": batched,
        "tuning": main["tuning"],
        "gpu_launches": KERNELS_PER_SCAN * args.steps,
        "roofline": rf,
        "integrate_ms_all_scans": main["integrate_ms_all_scans"],
        "clocks": ctx.clocks.stats("timed") if ctx.clocks else None,
        "clocks_whole_run": ctx.clocks.stats() if ctx.clocks else None,
    }
    line.update(extra)
    if not args.no_cpu_baseline and world == 1:
        v, nsc_run, secs, kept_per_s = cpu_baseline(w, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": kept_per_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "raw_points_per_s": v,
                                "sample": f"first {nsc_run} scans of the workload, full grid, "
                                          f"{secs:.1f} s of single-thread CPU",
                                "cpu": cpu_model(), "host_cores": os.cpu_count()}
        line["cpu_parallel_baseline"] = cpu_baseline_parallel(w, budget_s=args.cpu_budget)
    print(json.dumps(line), flush=True)
    return 0


def extra_legs(ctx, args) -> dict:
    """The other workloads of the line, each measured the same way (kept
    returns/s, latency, roofline), after the headline's timed region."""
    torch = ctx.torch
    out = {}
    # high resolution: 2000 x 2000 x 400 at 0.02 m, 50 scans of 262,144 returns
    wh = load_workload("highres")
    leg = plain_leg(ctx, wh, dict(wh.params), len(wh.scans), 3, autotune=not args.no_autotune)
    k, g, d_scans, poses, works = leg.pop("_state")
    leg["batched"] = run_batched(ctx, wh, k, g, d_scans, poses, len(wh.scans), works)
    leg["config"] = workload_config_of("highres", wh)
    out["highres"] = leg
    del k, g, d_scans, poses, wh
    torch.cuda.empty_cache()
    # the paper's parameters (Sec. III-B: K = 21, 40 x 40 azimuth / elevation bins)
    paper = dict(synth.DEFAULT_PARAMS, kernel_size=21, scheme=1, bins_a=40, bins_b=40)
    pp = {}
    wr = synth.room_scan(n_scans=20)
    leg = plain_leg(ctx, wr, paper, 20, 3, autotune=not args.no_autotune)
    leg.pop("_state")
    leg["config"] = workload_config_of("room", wr, paper)
    pp["room"] = leg
    wu = load_workload("urban")
    wu = synth.Workload(wu.name, wu.grid, wu.scans[:20], wu.params)
    leg = plain_leg(ctx, wu, paper, 20, 3, autotune=not args.no_autotune)
    leg.pop("_state")
    leg["config"] = workload_config_of("urban", wu, paper)
    pp["urban"] = leg
    out["paper_params"] = pp
    del wr, wu
    torch.cuda.empty_cache()
    out["maps"] = maps_leg(ctx, steps=3, warmup=3, autotune=not ctx.args.no_autotune)
    torch.cuda.empty_cache()
    out["serving"] = serving_leg(ctx, duration=args.serving_duration,
                                 speeds=[float(x) for x in args.serving_speeds.split(",")])
    torch.cuda.empty_cache()
    return out


def workload_config_of(name, w, pdict=None) -> dict:
    pdict = pdict or w.params
    bins = (f"octahedral {pdict['bins_a']}x{pdict['bins_b']}" if pdict["scheme"] == 0
            else f"az/el {pdict['bins_a']}x{pdict['bins_b']}")
    return {"workload": f"{name}: {len(w.scans)} scans x {len(w.scans[0][0])} returns, "
                        f"grid {w.grid.nx}x{w.grid.ny}x{w.grid.nz} at {w.grid.res} m",
            "kernel": pdict["kernel_size"], "bins": bins, "shadow_radius": pdict["shadow_radius"]}


def max_over_ranks(vals, dev, world):
    """Element-wise maximum of per-rank timings (every rank gets the result)."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def pct(sorted_vals, q):
    i = min(len(sorted_vals) - 1, max(0, int(round(q / 100.0 * (len(sorted_vals) - 1)))))
    return sorted_vals[i]


def run_batched(ctx, w, k, g, d_scans, poses, steps, works):
    """The same scans as graph-replayed batches of args.batch consecutive
    scans (one dbt_batch_run per batch, captured once, replayed in order)."""
    torch, dbt = ctx.torch, ctx.dbt
    args, stream, world = ctx.args, ctx.stream, ctx.world
    S = max(1, args.batch)
    nsc = len(w.scans)
    groups = [list(range(i, min(i + S, steps))) for i in range(0, steps, S)]
    batches, graphs = [], []
    cap = torch.cuda.Stream()
    for grp in groups:
        items = [(0, d_scans[s % nsc], poses[s % nsc]) for s in grp]
        b = dbt.Batch([g], k, sum(int(x.shape[0]) for _, x, _ in items), len(items))
        b.set_items(items)
        batches.append(b)
    torch.cuda.synchronize()
    with torch.cuda.stream(cap):
        batches[0].run(stream=cap)                  # configures the kernels before capture
        tuning = (batches[0].tuning() if args.no_autotune
                  else batches[0].autotune(n_trials=2, stream=cap))   # g is re-initialised below
    for b in batches:
        b.set_tuning(**tuning)
    torch.cuda.synchronize()
    for b in batches:
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=cap):
            b.run(stream=cap)
        graphs.append(gr)
    for _ in range(max(1, args.warmup // S)):
        graphs[0].replay()
    dbt.dbt_grid_init(g)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(graphs) + 1)]
    ctx.barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i, gr in enumerate(graphs):
        gr.replay()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    ctx.barrier()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(len(graphs)))
    ms = ev[0].elapsed_time(ev[-1])
    kept = sum(works[s % nsc]["kept"] for s in range(steps))
    raw = sum(works[s % nsc]["n"] for s in range(steps))
    out = {"value": world * kept / (ms * 1e-3), "unit": UNIT,
           "raw_points_per_s": world * raw / (ms * 1e-3), "scans_per_batch": S,
           "ms_per_scan": ms / steps, "batch_ms_p50": pct(per, 50), "batch_ms_p99": pct(per, 99),
           "scan_latency_ms_p99": pct(per, 99),
           "latency_note": "a scan's result is ready when its batch completes: its latency is "
                           "the batch's (plus waiting for the batch to fill, not counted here)",
           "launch": "one CUDA graph per batch (dbt_batch_run captured), replayed in order",
           "tuning": tuning}
    for b in batches:
        b.close()
    return out


def maps_leg(ctx, steps: int, warmup: int, autotune: bool, n_maps: int = 32) -> dict:
    """Uneven independent maps (side 64-512 voxels at 0.05-0.2 m), 8 scans
    of 4,096-131,072 returns each: a step integrates all scans of all maps,
    either as one graph-replayed batch or as one plain launch sequence per
    scan.  Both from freshly initialised maps, same scans, same device."""
    torch, dbt = ctx.torch, ctx.dbt
    dev, stream = ctx.dev, ctx.stream
    maps = synth.batched_maps(n_maps=n_maps, scans_per_map=8)
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    grids = [dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res) for w in maps]
    items = [(m, torch.from_numpy(pts).to(dev), pose) for m, w in enumerate(maps)
             for pts, pose in w.scans]
    npts = sum(int(x.shape[0]) for _, x, _ in items)
    # plain: one workspace per map, one dbt_integrate_scan per scan
    wss = [dbt.Workspace(grids[m], k, max(int(x.shape[0]) for mm, x, _ in items if mm == m))
           for m in range(len(maps))]

    def plain_pass():
        for m, x, pose in items:
            dbt.dbt_integrate_scan(grids[m], k, wss[m], x, pose)

    # each map's workspace tuned on its first scan (the grids are
    # re-initialised before the timed passes)
    plain_tunings = []
    for m in range(len(maps)):
        x, pose = next((x, pose) for mm, x, pose in items if mm == m)
        plain_tunings.append(ctx.B.dbt_workspace_autotune(grids[m], k, wss[m], x, pose, n_trials=2)
                             if autotune else wss[m].tuning())
    depths = sorted({t["brick_depth"] for t in plain_tunings})
    plain_tuning = {"brick_depth_maps": {str(d): sum(t["brick_depth"] == d for t in plain_tunings)
                                         for d in depths},
                    "what": "per map workspace, autotuned on its first scan" if autotune
                            else "default tuning"}

    b = dbt.Batch(grids, k, npts, len(items))
    b.set_items(items)
    cap = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(cap):
        b.run(stream=cap)
        tuning = b.autotune(n_trials=2, stream=cap) if autotune else b.tuning()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        b.run(stream=cap)

    def timed(fn):
        for _ in range(warmup):
            fn()
        for gg in grids:
            dbt.dbt_grid_init(gg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.barrier()
        return e0.elapsed_time(e1) / steps

    ms_batch = timed(graph.replay)
    ms_plain = timed(plain_pass)
    # kept returns of one step (every scan counted once, from its own counters)
    for gg in grids:
        dbt.dbt_grid_init(gg)
    kept = 0
    for m, x, pose in items:
        dbt.dbt_integrate_scan(grids[m], k, wss[m], x, pose)
        kept += dbt.dbt_get_scan_stats(wss[m])["n_kept"]
    ms_batch, ms_plain = max_over_ranks([ms_batch, ms_plain], dev, ctx.world)
    b.close()
    vox = sum(w.grid.nx * w.grid.ny * w.grid.nz for w in maps)
    return {"value": ctx.world * kept / (ms_batch * 1e-3), "unit": UNIT,
            "config": {"workload": f"maps: {len(maps)} maps ({vox / 1e6:.0f} M voxels), "
                                   f"{len(items)} scans, {npts} returns ({kept} kept) per step"},
            "batched": {"value": ctx.world * kept / (ms_batch * 1e-3), "ms_per_step": ms_batch,
                        "raw_points_per_s": ctx.world * npts / (ms_batch * 1e-3),
                        "launch": "one CUDA graph of dbt_batch_run over all scans",
                        "tuning": tuning},
            "plain": {"value": ctx.world * kept / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                      "raw_points_per_s": ctx.world * npts / (ms_plain * 1e-3),
                      "launch": f"{len(items)} dbt_integrate_scan calls "
                                f"({KERNELS_PER_SCAN} kernels each)",
                      "tuning": plain_tuning},
            "batched_over_plain": ms_plain / ms_batch, "steps": steps}


def run_maps(args, rank, world):
    ctx = Ctx(args, rank, world)
    leg = maps_leg(ctx, args.steps, args.warmup, not args.no_autotune, n_maps=args.maps)
    if ctx.clocks:
        ctx.clocks.stop()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": leg["batched"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": dict(leg["config"], parallelism=f"replicas x{args.gpus}",
                           l2="grids larger than L2 in total; no flush"),
            "batched": leg["batched"], "plain": leg["plain"],
            "gpu_launches": KERNELS_PER_SCAN * args.steps,
            "clocks": ctx.clocks.stats() if ctx.clocks else None}
    print(json.dumps(line), flush=True)
    return 0


def run_mesh(args, rank, world):
    """Map export (Fig. 3: Marching Cubes at iso = 0) at the urban map's size:
    a 1600 x 1600 x 320 stepped-terrain map state (819 M cells; --mesh-side
    scales it).  A step is
    one dbt_mesh_extract of the whole map (count pass, scan, emit pass);
    value = cells meshed per second.  Roofline: the count pass, 5 bytes read
    per voxel (mask + sign)."""
    import torch

    import paper_2509_20081_gb300 as dbt
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    nx = ny = args.mesh_side
    nz, res = args.mesh_side // 5, 0.05
    m, s, _ = synth.terrain_state(nx, ny, nz, 21)
    g = dbt.Grid(nx, ny, nz, res)
    g.load(m, s)
    B = dbt.dbtsdf
    box = (B.ctypes.c_int32 * 6)(0, 0, 0, nx, ny, nz)
    need = dbt.dbt_mesh_scratch_size(g)
    scratch = torch.empty(need, dtype=torch.uint8, device=dev)
    n = B.ctypes.c_int64()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def extract(tri_ptr, cap):
        B._check(B.lib().dbt_mesh_extract(B.ctypes.byref(g.c), box, 0.0, scratch.data_ptr(), need,
                                          tri_ptr, None, cap, B.ctypes.byref(n), sp))
    extract(None, 0)
    ntri = int(n.value)
    tri = torch.empty((ntri, 3, 3), dtype=torch.float32, device=dev)
    host = torch.empty((ntri, 3, 3), dtype=torch.float32).pin_memory()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return sum(a.elapsed_time(b) for a, b in ev) / args.steps

    clk = ClockSampler(dev.index or 0, pci_bus_id(torch, dev))
    clk.wait_first()
    ms_count = timed(lambda: extract(None, 0))
    ms_full = timed(lambda: extract(tri.data_ptr(), ntri))
    clk.stop()
    sample = clk.stats()

    def e2e():
        extract(tri.data_ptr(), ntri)
        host.copy_(tri, non_blocking=True)
    ms_e2e = timed(e2e)
    ms_full, ms_count, ms_e2e = max_over_ranks([ms_full, ms_count, ms_e2e], dev, world)
    if rank != 0:
        return 0
    cells = (nx - 1) * (ny - 1) * (nz - 1)
    vox = nx * ny * nz
    peak, src = measured_peaks()
    achieved = 5.0 * vox / (ms_count * 1e-3) / 1e9
    line = {"metric": "map cells meshed/sec (Marching Cubes, iso = 0)",
            "value": world * cells / (ms_full * 1e-3), "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_full,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"mesh: stepped terrain map {nx}x{ny}x{nz} at {res} m "
                                   f"({cells / 1e6:.0f} M cells, {ntri} triangles)",
                       "parallelism": f"replicas x{args.gpus}",
                       "l2": "map (5.7 GB) larger than L2; no flush"},
            "count_ms": ms_count, "emit_ms": ms_full - ms_count, "triangles": ntri,
            "e2e": {"value": world * cells / (ms_e2e * 1e-3), "unit": "cells/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 36 * ntri + 8,
                    "what": "extract + copy of the triangles to pinned host memory"},
            "gpu_launches": 6 * args.steps,
            "roofline": {"bound": "hbm", "kernel": "count pass (k_mc_count + scans)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "alg_bytes_per_launch": 5.0 * vox, "peak_source": src},
            "clocks": sample}
    if not args.no_cpu_baseline:
        import oracle
        og = oracle.Grid(nx, ny, nz, res, (0.0, 0.0, 0.0), m, s, None)
        t0 = time.perf_counter()
        done = 0
        z0 = 0
        while time.perf_counter() - t0 < args.cpu_budget and z0 + 2 <= nz:
            oracle.mesh(og, box=(0, 0, z0, nx, ny, 2))
            done += (nx - 1) * (ny - 1)
            z0 += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {z0} cell layers of the map, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def run_quality(args, rank, world):
    """Reconstruction quality (Sec. IV-B) of the urban map: the 100 urban
    scans integrated, the map meshed at iso = 0, the mesh centroids scored
    against the noise-free surface points of the same rays at a 10 cm
    tolerance (the paper's).  value: points scored per second by
    dbt_quality_metrics (both directions, predicted + reference points)."""
    import torch

    import paper_2509_20081_gb300 as dbt
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = load_workload("urban")
    kw = dict(WORKLOADS["urban"])
    truth = synth.urban_sequence(truth=True, **kw)
    k = dbt.Kernels(dbt.make_params(**w.params))
    g = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
    ws = dbt.Workspace(g, k, max(len(p) for p, _ in w.scans))
    for pts, pose in w.scans:
        dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).to(dev), pose)
    tri, _ = dbt.dbt_mesh_extract(g)
    pred = dbt.dbt_mesh_centroids(tri)
    # reference: the surface points inside the volume a return can update
    # (its K^3 neighbourhood inside the map, Sec. III-C); rays also hit
    # ground and walls beyond the map, which no map of this extent holds
    allgt = np.concatenate([p for p, _ in truth.scans])
    R = (w.params["kernel_size"] - 1) // 2
    lo = np.array(w.grid.origin) + R * w.grid.res
    hi = np.array(w.grid.origin) + (np.array([w.grid.nx, w.grid.ny, w.grid.nz]) - R) * w.grid.res
    keep = np.all((allgt >= lo) & (allgt < hi), axis=1)
    gt = torch.from_numpy(np.ascontiguousarray(allgt[keep])).to(dev)
    del tri
    tol = 0.10
    q = None
    for _ in range(args.warmup):
        q = dbt.dbt_quality_metrics(pred, gt, tol)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        q = dbt.dbt_quality_metrics(pred, gt, tol)
        b.record()
    torch.cuda.synchronize()
    ms = max_over_ranks([sum(a.elapsed_time(b) for a, b in ev) / args.steps], dev, world)[0]
    if rank != 0:
        return 0
    n = int(pred.shape[0]) + int(gt.shape[0])
    line = {"metric": "quality-metric points scored/sec (Sec. IV-B, both directions)",
            "value": world * n / (ms * 1e-3), "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"quality: urban map after {len(w.scans)} scans, "
                                   f"{int(pred.shape[0])} mesh centroids vs {int(gt.shape[0])} "
                                   f"noise-free surface points inside the updatable volume "
                                   f"(of {allgt.shape[0]}), tolerance {tol} m",
                       "parallelism": f"replicas x{args.gpus}"},
            "quality": {k2: v for k2, v in q.items()},
            "gpu_launches": 16 * args.steps}
    if not args.no_cpu_baseline:
        import oracle
        rng = synth.Rng(11)
        idx = rng.integers(200, 0, int(pred.shape[0]))
        sample = pred.cpu().numpy()[idx]
        ref = gt.cpu().numpy()
        t0 = time.perf_counter()
        oracle.nn_distances(ref, sample)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(idx) / dt, "unit": "points/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(idx)} predicted points against all "
                                          f"{ref.shape[0]} reference points, brute force, "
                                          f"{dt:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def serving_leg(ctx, duration: float, speeds: list, slo_ms: float = 100.0,
                hbm_budget_gb: float = 120.0) -> dict:
    """16 robots with resident maps, Poisson scan arrivals (10-20 Hz each)
    over `duration` simulated seconds, replayed at each speed-up (offered
    load = the trace's returns / (duration / speed-up)): continuous batching
    (2 streams, rounds of all pending scans of maps not in flight) against
    plain FIFO (one scan per round, one stream), the same trace for both.
    Latency = completion - arrival on the simulated clock."""
    torch, dbt = ctx.torch, ctx.dbt
    from paper_2509_20081_gb300 import serve
    maps, arrivals = synth.serving_robots(duration=duration)
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    robots = {r: (w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, (0.0, 0.0, 0.0))
              for r, w in enumerate(maps)}
    pools = [[torch.from_numpy(p).to(ctx.dev) for p, _ in w.scans] for w in maps]
    npts = sum(int(pools[r][i].shape[0]) for r, _, i in arrivals)
    budget = int(hbm_budget_gb * (1 << 30))
    results = {}
    for mode, kw in (("batched", dict(n_streams=2, max_round_points=4 << 20, max_round_items=1024)),
                     ("plain", dict(n_streams=1, max_round_points=262144, max_round_items=1))):
        srv = serve.Server(k, robots, budget_bytes=budget, **kw)
        admitted = len(srv.grids)
        res = []
        for sp in speeds:
            srv.reset()
            trace = [serve.Scan(r, t, pools[r][i], maps[r].scans[i][1]) for r, t, i in arrivals
                     if r in srv.grids]
            t0 = time.perf_counter()
            done = srv.replay(trace, speed=sp)
            wall = time.perf_counter() - t0
            st = serve.latency_stats(done)
            st.update({"speedup": sp, "wall_s": wall, "rounds": srv.rounds,
                       "points_per_s": sum(s.n for s in done) / wall,
                       "offered_points_per_s": sum(s.n for s in trace) / (duration / sp)})
            res.append(st)
        results[mode] = {"admitted_maps": admitted, "runs": res}
        srv.close()
        del srv
        torch.cuda.empty_cache()

    def sustained(runs):
        ok = [r for r in runs if r.get("p99_ms", 1e9) <= slo_ms]
        return max(ok, key=lambda r: r["speedup"]) if ok else None

    at_load = []
    for rb, rp in zip(results["batched"]["runs"], results["plain"]["runs"]):
        at_load.append({"speedup": rb["speedup"], "offered_points_per_s": rb["offered_points_per_s"],
                        "batched_p50_ms": rb.get("p50_ms"), "batched_p99_ms": rb.get("p99_ms"),
                        "plain_p50_ms": rp.get("p50_ms"), "plain_p99_ms": rp.get("p99_ms"),
                        "batched_points_per_s": rb["points_per_s"],
                        "plain_points_per_s": rp["points_per_s"]})
    return {"config": {"workload": f"serving: {len(maps)} robots, {len(arrivals)} scans "
                                   f"({npts} returns) over {duration} s simulated, Poisson "
                                   f"10-20 Hz per robot", "slo_p99_ms": slo_ms,
                       "hbm_budget_gb": hbm_budget_gb,
                       "points_counted": "returns handed in (raw)"},
            "at_equal_load": at_load,
            "sustained": {"batched": sustained(results["batched"]["runs"]),
                          "plain": sustained(results["plain"]["runs"])},
            "runs": results}


def run_serving(args, rank, world):
    ctx = Ctx(args, rank, world)
    leg = serving_leg(ctx, args.duration, [float(x) for x in args.speeds.split(",")],
                      slo_ms=args.slo_ms, hbm_budget_gb=args.hbm_budget_gb)
    if ctx.clocks:
        ctx.clocks.stop()
    if rank != 0:
        return 0
    best_b = leg["sustained"]["batched"]
    line = {"metric": METRIC, "value": best_b["points_per_s"] if best_b else 0.0, "unit": UNIT,
            "n_gpus": world, "steps": 0, "warmup": 0, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": dict(leg["config"], parallelism=f"replicas x{args.gpus}"),
            "at_equal_load": leg["at_equal_load"], "sustained": leg["sustained"],
            "serving": leg["runs"], "clocks": ctx.clocks.stats() if ctx.clocks else None}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload",
                    choices=["urban", "urban_half", "highres", "maps", "serving", "mesh", "quality"],
                    default="urban")
    ap.add_argument("--maps", type=int, default=32, help="maps workload: number of maps")
    ap.add_argument("--mesh-side", type=int, default=1600,
                    help="mesh workload: map side in voxels (height side / 5), e.g. 800 for a "
                         "profiler-sized case")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: simulated seconds")
    ap.add_argument("--speeds", default="1,8,16,24,32,48,64",
                    help="serving: replay speed-ups")
    ap.add_argument("--slo-ms", type=float, default=100.0, help="serving: p99 latency bound")
    ap.add_argument("--hbm-budget-gb", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="urban: only the headline legs (no highres, paper-parameter, maps, "
                         "serving keys)")
    ap.add_argument("--serving-duration", type=float, default=20.0,
                    help="serving key of the default line: simulated seconds")
    ap.add_argument("--serving-speeds", default="16,48",
                    help="serving key of the default line: replay speed-ups (equal loads for both "
                         "modes)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch tuning (short runs, profiler captures)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--batch", type=int, default=10, help="scans per batch in the batched leg")
    ap.add_argument("--ref-stride", type=int, default=16,
                    help="reference arm: integrate every n-th return of each scan")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        if args.workload == "maps":
            return run_maps(args, rank, world)
        if args.workload == "serving":
            return run_serving(args, rank, world)
        if args.workload == "mesh":
            return run_mesh(args, rank, world)
        if args.workload == "quality":
            return run_quality(args, rank, world)
        return run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
