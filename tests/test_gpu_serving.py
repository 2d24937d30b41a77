"""Continuous batching: results are the same alone and in the mix."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _robots(n=4, scans=6):
    maps = synth.batched_maps(n_maps=n, scans_per_map=scans, side_lo=64, side_hi=160,
                              n_lo=3000, n_hi=30000, seed_offset=7)
    arrivals = []
    for rid, w in enumerate(maps):
        for k, (pts, pose) in enumerate(w.scans):
            # every robot's k-th scan arrives at the same instant, so rounds mix robots
            arrivals.append((rid, 0.004 * k, pts, pose))
    return maps, arrivals


def _alone(dbt, k, w, scans):
    g = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
    ws = dbt.Workspace(g, k, max(len(p) for p, _ in scans))
    for pts, pose in scans:
        dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).cuda(), pose)
    return g


def test_serving_mix_equals_alone(orc):
    import paper_2509_20081_gb300 as dbt
    from paper_2509_20081_gb300 import serve
    maps, arrivals = _robots()
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    robots = {rid: (w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, (0.0, 0.0, 0.0))
              for rid, w in enumerate(maps)}
    srv = serve.Server(k, robots, budget_bytes=8 << 30, n_streams=2, max_round_points=200000,
                       max_round_items=64)
    scans = [serve.Scan(rid, t, torch.from_numpy(p).cuda(), pose) for rid, t, p, pose in arrivals]
    done = srv.replay(scans, speed=1.0)
    assert len(done) == len(scans) and all(s.done >= s.arrival for s in done)
    assert srv.rounds < len(scans)                 # scans were batched together
    assert max(srv.round_sizes) > 1
    for rid, w in enumerate(maps):
        alone = _alone(dbt, k, w, w.scans)
        mixed = srv.map_state(rid)
        for a, b in ((alone.mask, mixed.mask), (alone.sign, mixed.sign), (alone.hits, mixed.hits)):
            assert torch.equal(a, b)
    # two robots' served maps against the oracle's sequential replay of their streams
    po = orc.params(**maps[0].params)
    for rid in (0, 1):
        w = maps[rid]
        og = orc.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
        for pts, pose in w.scans:
            orc.integrate_scan(og, po, pts, pose)
        m, sg, h = srv.map_state(rid).numpy()
        np.testing.assert_array_equal(m, og.mask)
        np.testing.assert_array_equal(sg, og.sign)
        np.testing.assert_array_equal(h, og.hits)
    st = serve.latency_stats(done)
    assert st["n"] == len(scans) and st["p99_ms"] >= st["p50_ms"] >= 0.0
    srv.close()


def test_serving_admission_and_retire():
    """With room for one map, the second robot waits until the first retires."""
    import paper_2509_20081_gb300 as dbt
    from paper_2509_20081_gb300 import serve
    maps, arrivals = _robots(n=2, scans=3)
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    robots = {rid: (w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res, (0.0, 0.0, 0.0))
              for rid, w in enumerate(maps)}
    need0 = serve.grid_bytes(*robots[0][:3])
    need1 = serve.grid_bytes(*robots[1][:3])
    srv = serve.Server(k, robots, budget_bytes=1 << 40, n_streams=1,
                       max_round_points=100000, max_round_items=16)
    scr = max(srv._scratch_bytes([0]), srv._scratch_bytes([1]))
    # both maps never fit at once; either one alone does
    budget = max(need0, need1) + scr + min(need0, need1) // 2
    srv.close()
    srv = serve.Server(k, robots, budget_bytes=budget, n_streams=1, max_round_points=100000,
                       max_round_items=16)
    assert sorted(srv.grids) == [0] and srv.waiting == [1]
    for rid, t, p, pose in arrivals:
        if rid == 0:
            srv.submit(serve.Scan(0, t, torch.from_numpy(p).cuda(), pose))
    srv.retire(0)
    srv.drain(lambda: 0.0)
    srv.poll(0.0)
    assert sorted(srv.grids) == [1] and srv.waiting == []
    for rid, t, p, pose in arrivals:
        if rid == 1:
            srv.submit(serve.Scan(1, t, torch.from_numpy(p).cuda(), pose))
    srv.drain(lambda: 0.0)
    alone = _alone(dbt, k, maps[1], maps[1].scans)
    assert torch.equal(alone.mask, srv.map_state(1).mask)
    assert torch.equal(alone.hits, srv.map_state(1).hits)
    srv.close()
