"""Whole-map parity at the workloads' full sizes, against the oracle.

Every voxel's mask, sign and hit counter (bit-exact, the state is integer)
after integrating, in the launch forms the benchmark times:
  - urban sequence (1600 x 1600 x 320 at 0.05 m, scans of 65,536 returns):
    the first 8 scans by per-scan launches (32 x 8 x 8 bricks), and the same
    8 as one batch at another launch tuning (32 x 8 x 4 bricks);
  - high resolution (2000 x 2000 x 400 at 0.02 m, 262,144 returns per scan):
    4 scans by per-scan launches (32 x 8 x 16 bricks);
  - 32 uneven maps (64^3 to 512^3) x 8 scans, all in one dbt_batch_run
    (32 x 8 x 4 bricks);
  - serving (16 robots, Poisson arrivals over 60 s simulated): every map
    after the first 5 s of the trace went through the continuous-batching
    loop, then the two robots with the smallest streams for the full 60 s.
The oracle runs sequentially, scan by scan in arrival order; the big maps
are compared slab by slab (urban, highres) or by per-slab digests computed
on both sides (maps, serving; tests/oracle_pool.py).
"""
import numpy as np
import pytest

import synth
from oracle_pool import SLAB, first_mismatch, gpu_digests, replay_all

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare_slabs(g, og):
    """Device grid g (padded rows) == oracle grid og, slab by slab."""
    for z in range(0, g.nz, SLAB):
        m = g.mask[z:z + SLAB, :, :g.nx].cpu().numpy().view(np.uint32)
        s = g.sign[z:z + SLAB, :, :g.nx].cpu().numpy()
        h = g.hits[z:z + SLAB, :, :g.nx].cpu().numpy().view(np.uint16)
        for name, a, b in (("mask", m, og.mask[z:z + SLAB]), ("sign", s, og.sign[z:z + SLAB]),
                           ("hits", h, og.hits[z:z + SLAB])):
            if not np.array_equal(a, b):
                bad = int((a != b).sum())
                raise AssertionError(f"{name} differs in {bad} voxels of planes {z}..{z + SLAB - 1}")


def _oracle_sequence(orc, w, scans):
    og = orc.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    po = orc.params(**w.params)
    kept = [orc.integrate_scan(og, po, pts, pose)["n_kept"] for pts, pose in scans]
    return og, kept


def test_urban_full_size_eight_scans(orc):
    import paper_2509_20081_gb300 as dbt
    w = synth.urban_sequence(n_scans=8)
    assert (w.grid.nx, w.grid.ny, w.grid.nz) == (1600, 1600, 320)
    k = dbt.Kernels(dbt.make_params(**w.params))
    g = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    ws = dbt.Workspace(g, k, 65536)
    xs = [torch.from_numpy(p).cuda() for p, _ in w.scans]
    kept = []
    for x, (_, pose) in zip(xs, w.scans):
        dbt.dbt_integrate_scan(g, k, ws, x, pose)
        kept.append(dbt.dbt_get_scan_stats(ws)["n_kept"])
    og, okept = _oracle_sequence(orc, w, w.scans)
    assert kept == okept and min(kept) > 30000
    _compare_slabs(g, og)
    del og
    # the same scans as one batch, another tuning: equal to the per-scan map
    gb = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    b = dbt.Batch([gb], k, 8 * 65536, 8)
    b.set_tuning(heavy_pairs=96, integrate_ctas=304, brick_depth=4)
    b.set_items([(0, x, pose) for x, (_, pose) in zip(xs, w.scans)])
    b.run()
    torch.cuda.synchronize()
    for a, c in ((g.mask, gb.mask), (g.sign, gb.sign), (g.hits, gb.hits)):
        assert torch.equal(a[:, :, :g.nx], c[:, :, :g.nx])
    b.close()


def test_highres_full_size_four_scans(orc):
    import paper_2509_20081_gb300 as dbt
    w = synth.urban_sequence(n_scans=4, scale=0.5, res=0.02, beams=128, width=2048, seed_offset=2)
    assert (w.grid.nx, w.grid.ny, w.grid.nz) == (2000, 2000, 400)
    k = dbt.Kernels(dbt.make_params(**w.params))
    g = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, w.grid.origin)
    ws = dbt.Workspace(g, k, 262144)
    ws.set_tuning(k, brick_depth=16)
    kept = []
    for pts, pose in w.scans:
        dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).cuda(), pose)
        kept.append(dbt.dbt_get_scan_stats(ws)["n_kept"])
    og, okept = _oracle_sequence(orc, w, w.scans)
    assert kept == okept and min(kept) > 100000
    _compare_slabs(g, og)


def test_maps_all_32_in_one_batch():
    import paper_2509_20081_gb300 as dbt
    maps = synth.batched_maps(n_maps=32, scans_per_map=8)
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    grids = [dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res) for w in maps]
    items = [(m, torch.from_numpy(p).cuda(), pose) for m, w in enumerate(maps) for p, pose in w.scans]
    b = dbt.Batch(grids, k, sum(int(x.shape[0]) for _, x, _ in items), len(items))
    b.set_tuning(brick_depth=4)
    b.set_items(items)
    b.run()
    per, tot = b.stats()
    torch.cuda.synchronize()
    jobs = [((w.grid.nx, w.grid.ny, w.grid.nz), w.grid.res, (0.0, 0.0, 0.0), w.params, w.scans)
            for w in maps]
    res = replay_all(jobs)
    assert sum(kk for _, kk in res) == sum(int(it["n_kept"]) for it in per)
    for m, (dig, _) in enumerate(res):
        bad = first_mismatch(gpu_digests(grids[m]), dig)
        assert bad is None, f"map {m}: planes {bad * SLAB}..{bad * SLAB + SLAB - 1} differ"
    b.close()


def test_serving_replay_every_map_5s_and_two_full_streams():
    import paper_2509_20081_gb300 as dbt
    from paper_2509_20081_gb300 import serve
    maps, arrivals = synth.serving_robots(duration=60.0)
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    robots = {r: (w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, (0.0, 0.0, 0.0))
              for r, w in enumerate(maps)}
    srv = serve.Server(k, robots, budget_bytes=120 << 30, n_streams=2)
    assert len(srv.grids) == len(maps)
    pools = [[torch.from_numpy(p).cuda() for p, _ in w.scans] for w in maps]
    stream_size = {r: sum(len(maps[r].scans[i][0]) for rr, _, i in arrivals if rr == r)
                   for r in range(len(maps))}
    full = sorted(stream_size, key=lambda r: stream_size[r])[:2]

    def scans_of(sel):
        return [serve.Scan(r, t, pools[r][i], maps[r].scans[i][1]) for r, t, i in arrivals if sel(r, t)]

    # phase 1: every robot's scans of the first 5 s (rounds mix all maps)
    first = scans_of(lambda r, t: t < 5.0)
    done = srv.replay(first, speed=50.0)
    assert len(done) == len(first) and srv.rounds < len(first)
    jobs = []
    for r, w in enumerate(maps):
        sc = [w.scans[i] for rr, t, i in arrivals if rr == r and t < 5.0]
        jobs.append(((w.grid.nx, w.grid.ny, w.grid.nz), w.grid.res, (0.0, 0.0, 0.0), w.params, sc))
    for r in full:                                    # the two full streams, from an empty map
        w = maps[r]
        sc = [w.scans[i] for rr, t, i in arrivals if rr == r]
        jobs.append(((w.grid.nx, w.grid.ny, w.grid.nz), w.grid.res, (0.0, 0.0, 0.0), w.params, sc))
    # the oracle replays run on the host while the GPU side goes on
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(1) as tp:
        fut = tp.submit(replay_all, jobs)
        dig5 = {r: gpu_digests(srv.map_state(r)) for r in range(len(maps))}
        # phase 2: the rest of the two smallest robots' streams
        srv.completed = []
        rest = scans_of(lambda r, t: r in full and t >= 5.0)
        done = srv.replay(rest, speed=50.0)
        assert len(done) == len(rest)
        dig_full = {r: gpu_digests(srv.map_state(r)) for r in full}
        res = fut.result()
    for r in range(len(maps)):
        bad = first_mismatch(dig5[r], res[r][0])
        assert bad is None, f"robot {r} after 5 s: planes {bad * SLAB}.. differ"
    for j, r in enumerate(full):
        bad = first_mismatch(dig_full[r], res[len(maps) + j][0])
        assert bad is None, f"robot {r} full stream: planes {bad * SLAB}.. differ"
    srv.close()
