"""Continuous-batching request loop over resident maps.

Several robots each own a map that stays resident on the device.  Their
scans arrive over time (e.g. Poisson); the loop integrates them in rounds:
every round takes all pending scans of maps that are not already on the GPU
(up to a point budget) and launches them as one dbt_batch_run.  Rounds run
on a small pool of streams, so a round whose maps are free starts while
another round is still executing; a map is never in two rounds at once,
which keeps its bricks owned by one launch.  Because a batch is exact for
any grouping of a map's scans (see dbt_batch_*), every map ends in the same
state as integrating its scans one by one, alone.

Maps are admitted against a device-memory budget (grid bytes plus the
rounds' scratch); a robot whose map does not fit waits until memory is
released.  Latency of a scan = completion of its round - its arrival.
All integration work runs in libdbtsdf's kernels; this module only
schedules.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

from . import dbtsdf as B


@dataclass
class Scan:
    robot: int
    arrival: float          # seconds, simulated clock
    xyz: object             # CUDA float32 (n, 3) tensor
    pose: np.ndarray        # (3, 4) float64
    n: int = 0
    done: float = -1.0      # completion, simulated clock


class Admission:
    """Device-memory budget for resident maps (host-side bookkeeping)."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.used = 0
        self.held = {}

    def try_reserve(self, key, nbytes: int) -> bool:
        if key in self.held:
            return True
        if self.used + nbytes > self.budget:
            return False
        self.held[key] = int(nbytes)
        self.used += int(nbytes)
        return True

    def release(self, key):
        self.used -= self.held.pop(key, 0)


def grid_bytes(nx: int, ny: int, nz: int) -> int:
    pitch, mb, sb, hb = B.dbt_grid_layout(nx, ny, nz)
    return mb + sb + hb


def check_scan_size(n: int, max_round_points: int) -> None:
    """A scan larger than a round's point budget could never be scheduled
    (it would wait forever and hold its robot's later scans behind it), so
    it is refused when submitted."""
    if n > max_round_points:
        raise ValueError(f"scan of {n} returns exceeds the round budget of "
                         f"{max_round_points} returns (max_round_points)")


def select_round(order, busy_maps, pending, max_round_points: int, max_round_items: int):
    """Scans of the next round: for each map in order that is not in a round
    already, the longest prefix of its pending scans (scans of one map stay
    in arrival order) that keeps the round within max_round_points returns
    and max_round_items scans.  Returns [(map, number of scans taken)]."""
    takes, pts, n_items = [], 0, 0
    for rid in order:
        if rid in busy_maps or not pending[rid]:
            continue
        k = 0
        for sc in pending[rid]:
            if pts + sc.n > max_round_points or n_items + k >= max_round_items:
                break
            k += 1
            pts += sc.n
        if k:
            takes.append((rid, k))
            n_items += k
    return takes


@dataclass
class _Slot:
    stream: object
    batch: object = None
    event: object = None
    scans: list = field(default_factory=list)
    maps: set = field(default_factory=set)
    t_launch: float = 0.0


class Server:
    """Continuous batching of scans over resident maps.

    robots: {robot id: (nx, ny, nz, res, origin)}.  Maps are admitted in
    robot order while the budget allows, counting the rounds' scratch too;
    the others wait and are admitted when a robot retires and its map is
    freed.  max_round_points / max_round_items cap one round.
    """

    def __init__(self, kernels: B.Kernels, robots: dict, budget_bytes: int, n_streams: int = 2,
                 max_round_points: int = 4 << 20, max_round_items: int = 1024, device="cuda"):
        import torch
        self.torch = torch
        self.k = kernels
        self.adm = Admission(budget_bytes)
        self.device = device
        self.n_streams = n_streams
        self.max_round_points = max_round_points
        self.max_round_items = max_round_items
        self.specs = dict(robots)
        self.grids = {}
        self.waiting = list(robots)
        self.slots = []
        self.pending = {}
        self.busy_maps = set()
        self.completed = []
        self.rounds = 0
        self.round_sizes = []
        self.retiring = set()
        self._admit()

    def _scratch_bytes(self, rids) -> int:
        if not rids:
            return 0
        grids = (B.dbt_grid * len(rids))()
        for i, rid in enumerate(rids):
            nx, ny, nz, res, origin = self.specs[rid]
            pitch = B.dbt_grid_layout(nx, ny, nz)[0]
            grids[i] = B.dbt_grid(256, 512, 768, nx, ny, nz, pitch, res,
                                  (B.ctypes.c_double * 3)(*origin))
        nbytes = B.ctypes.c_size_t()
        B._check(B.lib().dbt_batch_size(grids, len(rids), self.k.h, self.max_round_points,
                                        self.max_round_items, B.ctypes.byref(nbytes)))
        return self.n_streams * (nbytes.value + 256)

    def _admit(self):
        """Admit waiting robots that fit, then (re)build the round buffers;
        only called while no round is in flight."""
        current = sorted(self.grids)
        self.adm.release("scratch")
        admitted = list(current)
        for rid in list(self.waiting):
            nx, ny, nz, _, _ = self.specs[rid]
            need = grid_bytes(nx, ny, nz)
            scratch = self._scratch_bytes(sorted(admitted + [rid]))
            if self.adm.used + need + scratch <= self.adm.budget:
                self.adm.try_reserve(("map", rid), need)
                admitted.append(rid)
                self.waiting.remove(rid)
        self.adm.try_reserve("scratch", self._scratch_bytes(sorted(admitted)))
        for rid in admitted:
            if rid not in self.grids:
                nx, ny, nz, res, origin = self.specs[rid]
                self.grids[rid] = B.Grid(nx, ny, nz, res, origin, device=self.device)
                self.pending[rid] = []
        self.order = sorted(self.grids)
        self.index = {rid: i for i, rid in enumerate(self.order)}
        for s in self.slots:
            s.batch.close()
        self.slots = []
        if self.grids:
            glist = [self.grids[r] for r in self.order]
            for _ in range(self.n_streams):
                b = B.Batch(glist, self.k, self.max_round_points, self.max_round_items)
                self.slots.append(_Slot(stream=self.torch.cuda.Stream(device=self.device), batch=b))

    def retire(self, rid):
        """Robot rid leaves once its pending scans are integrated; its map
        is then freed and waiting robots may be admitted."""
        self.retiring.add(rid)

    def _retire_done(self):
        gone = [r for r in self.retiring if r in self.grids and not self.pending[r]
                and r not in self.busy_maps]
        if not gone or any(s.event is not None for s in self.slots):
            return
        for r in gone:
            self.retiring.discard(r)
            del self.grids[r]
            del self.pending[r]
            self.adm.release(("map", r))
        self._admit()

    # -------------------------------------------------------------- scheduling
    def submit(self, scan: Scan):
        if scan.robot not in self.grids:
            raise KeyError(f"robot {scan.robot} has no admitted map")
        scan.n = int(scan.xyz.shape[0])
        check_scan_size(scan.n, self.max_round_points)
        self.pending[scan.robot].append(scan)

    def _launch(self, slot: _Slot, now: float):
        takes = select_round(self.order, self.busy_maps, self.pending, self.max_round_points,
                             self.max_round_items)
        items, scans, maps = [], [], set()
        for rid, k in takes:
            take = self.pending[rid][:k]
            del self.pending[rid][:k]
            maps.add(rid)
            for sc in take:
                items.append((self.index[rid], sc.xyz, sc.pose))
                scans.append(sc)
        if not items:
            return False
        torch = self.torch
        with torch.cuda.stream(slot.stream):
            slot.batch.set_items(items, stream=slot.stream)
            slot.batch.run(stream=slot.stream)
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        slot.scans, slot.maps, slot.t_launch = scans, maps, now
        self.busy_maps |= maps
        self.rounds += 1
        self.round_sizes.append(len(items))
        return True

    def poll(self, now: float):
        """Retire finished rounds (completion stamped `now`) and launch new ones."""
        for slot in self.slots:
            if slot.event is not None and slot.event.query():
                for sc in slot.scans:
                    sc.done = now
                    self.completed.append(sc)
                self.busy_maps -= slot.maps
                slot.event, slot.scans, slot.maps = None, [], set()
        if self.retiring:
            self._retire_done()
        for slot in self.slots:
            if slot.event is None:
                if not self._launch(slot, now):
                    break

    def idle(self) -> bool:
        return all(s.event is None for s in self.slots) and not any(self.pending.values())

    def map_state(self, rid):
        return self.grids[rid]

    def reset(self):
        """Fresh maps (Sec. III-A state) and empty statistics; no round may be in flight."""
        self.torch.cuda.synchronize()
        for g in self.grids.values():
            B.dbt_grid_init(g)
        for rid in self.pending:
            self.pending[rid] = []
        self.completed, self.rounds, self.round_sizes = [], 0, []
        self.torch.cuda.synchronize()

    def drain(self, clock):
        while not self.idle():
            self.poll(clock())

    # -------------------------------------------------------------- replay
    def replay(self, arrivals: list, speed: float = 1.0):
        """arrivals: list of Scan (any order).  The simulated clock runs
        `speed` times faster than the wall clock; scans are submitted when the
        clock passes their arrival.  Returns the completed scans."""
        heap = [(sc.arrival, i, sc) for i, sc in enumerate(arrivals)]
        heapq.heapify(heap)
        t0 = time.perf_counter()

        def clock():
            return (time.perf_counter() - t0) * speed

        while heap or not self.idle():
            now = clock()
            while heap and heap[0][0] <= now:
                self.submit(heapq.heappop(heap)[2])
            self.poll(now)
        self.torch.cuda.synchronize()
        return self.completed

    def close(self):
        for s in self.slots:
            if s.batch is not None:
                s.batch.close()


def latency_stats(scans) -> dict:
    lat = np.array([s.done - s.arrival for s in scans if s.done >= 0.0])
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3)}
