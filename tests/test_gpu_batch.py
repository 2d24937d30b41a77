"""Batched integration (many scans of many uneven maps in one launch
sequence) against one-by-one integration and the oracle, bit-exact."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def maps():
    # uneven maps of the batched workload's generator, small enough for the oracle
    return synth.batched_maps(n_maps=5, scans_per_map=3, side_lo=40, side_hi=160,
                              n_lo=2000, n_hi=20000)


def _items(ws_maps):
    items = []
    for m, w in enumerate(ws_maps):
        for pts, pose in w.scans:
            items.append((m, torch.from_numpy(pts).cuda(), pose))
    return items


def _interleaved(items):
    # scans of different maps interleaved, each map's scans kept in order
    by = {}
    for it in items:
        by.setdefault(it[0], []).append(it)
    out = []
    while any(by.values()):
        for m in sorted(by):
            if by[m]:
                out.append(by[m].pop(0))
    return out


def test_batch_equals_one_by_one_and_oracle(orc, maps):
    import paper_2509_20081_gb300 as dbt
    p = dbt.make_params(**maps[0].params)
    k = dbt.Kernels(p)
    grids_b = [dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res) for w in maps]
    grids_s = [dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res) for w in maps]
    items = _interleaved(_items(maps))
    total = sum(int(x.shape[0]) for _, x, _ in items)
    b = dbt.Batch(grids_b, k, total, len(items))
    b.set_items(items)
    b.run()
    per, tot = b.stats()
    assert tot["error"] == 0 and tot["n_input"] == total
    kept_single = []
    for gi, x, pose in items:
        g = grids_s[gi]
        ws = dbt.Workspace(g, k, max(1, int(x.shape[0])))
        dbt.dbt_integrate_scan(g, k, ws, x, pose)
        kept_single.append(dbt.dbt_get_scan_stats(ws)["n_kept"])
    assert [s["n_kept"] for s in per] == kept_single
    po = orc.params(**maps[0].params)
    for m, w in enumerate(maps):
        for a, c in zip(grids_b[m].numpy(), grids_s[m].numpy()):
            np.testing.assert_array_equal(a, c)
        og = orc.Grid.create(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
        for pts, pose in w.scans:
            orc.integrate_scan(og, po, pts, pose)
        mm, ss, hh = grids_b[m].numpy()
        np.testing.assert_array_equal(mm, og.mask)
        np.testing.assert_array_equal(hh, og.hits)
        np.testing.assert_array_equal(ss, og.sign)


def test_batch_sequence_one_map(orc):
    """Eight consecutive urban scans of one map in one batch == one by one."""
    import paper_2509_20081_gb300 as dbt
    w = synth.urban_sequence(n_scans=8, scale=0.5)
    k = dbt.Kernels(dbt.make_params(**w.params))
    ga = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
    gb = dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res)
    xs = [torch.from_numpy(s[0]).cuda() for s in w.scans]
    b = dbt.Batch([gb], k, sum(int(x.shape[0]) for x in xs), len(xs))
    b.set_items([(0, x, s[1]) for x, s in zip(xs, w.scans)])
    b.run()
    per, tot = b.stats()
    ws = dbt.Workspace(ga, k, 65536)
    for x, s in zip(xs, w.scans):
        dbt.dbt_integrate_scan(ga, k, ws, x, s[1])
    for a, c in ((ga.mask, gb.mask), (ga.sign, gb.sign), (ga.hits, gb.hits)):
        assert torch.equal(a, c)
    assert tot["n_kept"] == sum(s["n_kept"] for s in per) > 100000


def test_batch_graph_replay(maps):
    """dbt_batch_run captured in a CUDA graph and replayed gives the same state
    as a direct run (twice applied: the second pass is idempotent on masks,
    and counts add)."""
    import paper_2509_20081_gb300 as dbt
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    items = _items(maps)
    total = sum(int(x.shape[0]) for _, x, _ in items)
    ga = [dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res) for w in maps]
    gb = [dbt.Grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.res) for w in maps]
    ba = dbt.Batch(ga, k, total, len(items))
    ba.set_items(items)
    bb = dbt.Batch(gb, k, total, len(items))
    bb.set_items(items)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        bb.run(stream=s)            # warm-up outside capture (kernel configuration)
    torch.cuda.synchronize()
    for g in gb:
        dbt.dbt_grid_init(g)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        bb.run(stream=s)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    ba.run()
    ba.run()
    torch.cuda.synchronize()
    for a, c in zip(ga, gb):
        for x, y in ((a.mask, c.mask), (a.sign, c.sign), (a.hits, c.hits)):
            assert torch.equal(x, y)


def test_batch_argument_errors(maps):
    import paper_2509_20081_gb300 as dbt
    k = dbt.Kernels(dbt.make_params(**maps[0].params))
    g = [dbt.Grid(32, 32, 32, 0.1)]
    b = dbt.Batch(g, k, 100, 2)
    x = torch.zeros((60, 3), device="cuda")
    pose = np.hstack([np.eye(3), np.zeros((3, 1))])
    with pytest.raises(dbt.DbtError):
        b.set_items([(0, x, pose), (0, x, pose)])         # 120 > max_points
    with pytest.raises(dbt.DbtError):
        b.set_items([(1, x, pose)])                       # no grid 1
    with pytest.raises(dbt.DbtError):
        b.set_items([(0, x, pose)] * 3)                   # more than max_items


# ------------------------------------------------------------------ tuning
def test_every_tuning_gives_the_same_maps(orc):
    """The heavy-brick threshold and the integrate grid are launch choices:
    every candidate leaves bit-identical maps (single scans and batches)."""
    import paper_2509_20081_gb300 as dbt
    w = synth.urban_sequence(n_scans=3, scale=0.25)
    k = dbt.Kernels(dbt.make_params(**w.params))
    dims = (w.grid.nx, w.grid.ny, w.grid.nz)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ref = None
    for heavy, ctas, depth in [(48, 0, 8), (0, 0, 8), (16, sms, 4), (1 << 30, 2 * sms, 8),
                               (96, 1, 16), (24, 4 * sms, 8), (0, 0, 4), (8, 0, 16),
                               (1 << 30, 0, 4), (64, 3 * sms, 16)]:
        g = dbt.Grid(*dims, w.grid.res)
        ws = dbt.Workspace(g, k, max(len(p) for p, _ in w.scans))
        ws.set_tuning(k, heavy, ctas, depth)
        assert ws.tuning() == {"heavy_pairs": heavy, "integrate_ctas": ctas, "brick_depth": depth}
        for pts, pose in w.scans:
            dbt.dbt_integrate_scan(g, k, ws, torch.from_numpy(pts).cuda(), pose)
        st = dbt.dbt_get_scan_stats(ws)
        assert st["error"] == 0
        out = g.numpy()
        if ref is None:
            ref = out
        else:
            for a, b in zip(out, ref):
                np.testing.assert_array_equal(a, b)
        gb = dbt.Grid(*dims, w.grid.res)
        b = dbt.Batch([gb], k, sum(len(p) for p, _ in w.scans), len(w.scans))
        b.set_tuning(heavy, ctas, depth)
        b.set_items([(0, torch.from_numpy(p).cuda(), pose) for p, pose in w.scans])
        b.run()
        for a, r in zip(gb.numpy(), ref):
            np.testing.assert_array_equal(a, r)
        b.close()


def test_autotune_picks_a_candidate_and_keeps_results(orc):
    import paper_2509_20081_gb300 as dbt
    w = synth.urban_sequence(n_scans=2, scale=0.25)
    k = dbt.Kernels(dbt.make_params(**w.params))
    dims = (w.grid.nx, w.grid.ny, w.grid.nz)
    items = [(0, torch.from_numpy(p).cuda(), pose) for p, pose in w.scans]
    scratch = dbt.Grid(*dims, w.grid.res)
    b = dbt.Batch([scratch], k, sum(len(p) for p, _ in w.scans), len(items))
    b.set_items(items)
    best = b.autotune(n_trials=2)
    assert best["heavy_pairs"] in (16, 24, 32, 40, 48, 64, 96, 128, 192, 256)
    assert best["brick_depth"] in (4, 8, 16)
    assert best == b.tuning()
    b.close()
    g = dbt.Grid(*dims, w.grid.res)
    b = dbt.Batch([g], k, sum(len(p) for p, _ in w.scans), len(items))
    b.set_tuning(**best)
    b.set_items(items)
    b.run()
    og = orc.Grid.create(*dims, w.grid.res)
    po = orc.params(**w.params)
    for p, pose in w.scans:
        orc.integrate_scan(og, po, p, pose)
    m, s, h = g.numpy()
    np.testing.assert_array_equal(m, og.mask)
    np.testing.assert_array_equal(h, og.hits)
    np.testing.assert_array_equal(s, og.sign)
    ws_grid = dbt.Grid(*dims, w.grid.res)
    ws = dbt.Workspace(ws_grid, k, len(w.scans[0][0]))
    t = dbt.dbtsdf.dbt_workspace_autotune(ws_grid, k, ws, items[0][1], w.scans[0][1], n_trials=1)
    assert t == ws.tuning()


def test_tuning_refuses_bad_values():
    import paper_2509_20081_gb300 as dbt
    B = dbt.dbtsdf
    k = dbt.Kernels(dbt.make_params())
    g = dbt.Grid(64, 64, 64, 0.1)
    ws = dbt.Workspace(g, k, 100)
    for heavy, ctas in [(-1, 0), (48, -2), (48, 10 ** 7)]:
        with pytest.raises(B.DbtError) as e:
            ws.set_tuning(k, heavy, ctas)
        assert e.value.status == B.DBT_EINVAL
