"""Oracle replays in worker processes, for the full-size parity tests.

Test infrastructure only.  The workers are started with the spawn method
(the parent already holds a CUDA context, and a child forked from it
could hang), each loads the oracle and integrates one map's scans in order,
and returns digests of its final state: SHA-256 of the mask, sign and hits
bytes of every slab of z-planes.  The GPU side computes the same digests
from its read-back map, so large maps are compared element for element
without moving gigabytes between processes; a mismatch names the slab.
"""
from __future__ import annotations

import hashlib
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

SLAB = 16          # z-planes per digest


def slab_digests(mask: np.ndarray, sign: np.ndarray, hits: np.ndarray, z0: int = 0) -> dict:
    """{slab index: hex digest} of arrays shaped (nz, ny, nx), x fastest;
    z0 is the first plane's index in the whole map (a multiple of SLAB)."""
    out = {}
    for z in range(0, mask.shape[0], SLAB):
        h = hashlib.sha256()
        for a, t in ((mask, np.uint32), (sign, np.uint8), (hits, np.uint16)):
            h.update(np.ascontiguousarray(a[z:z + SLAB], t).tobytes())
        out[(z0 + z) // SLAB] = h.hexdigest()
    return out


def gpu_digests(grid) -> dict:
    """The same digests of a device map (paper_2509_20081_gb300 Grid), read
    back slab by slab without its row padding."""
    out = {}
    for z in range(0, grid.nz, SLAB):
        m = grid.mask[z:z + SLAB, :, :grid.nx].cpu().numpy().view(np.uint32)
        s = grid.sign[z:z + SLAB, :, :grid.nx].cpu().numpy()
        h = grid.hits[z:z + SLAB, :, :grid.nx].cpu().numpy().view(np.uint16)
        out.update(slab_digests(m, s, h, z0=z))
    return out


def _replay(job):
    """Worker: (dims, res, origin, params dict, [(pts, pose)]) -> (digests, kept)."""
    import oracle
    (nx, ny, nz), res, origin, pdict, scans = job
    g = oracle.Grid.create(nx, ny, nz, res, origin)
    p = oracle.params(**pdict)
    kept = 0
    for pts, pose in scans:
        kept += oracle.integrate_scan(g, p, pts, pose)["n_kept"]
    return slab_digests(g.mask, g.sign, g.hits), kept


def replay_all(jobs: list) -> list:
    """Runs every job (see _replay) on up to all host cores; results in order."""
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_replay, jobs))


def first_mismatch(a: dict, b: dict):
    """Lowest slab whose digests differ (or that one side lacks), else None."""
    bad = sorted(k for k in set(a) | set(b) if a.get(k) != b.get(k))
    return bad[0] if bad else None
