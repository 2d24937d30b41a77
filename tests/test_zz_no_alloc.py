"""dbt_integrate_scan_noalloc against dbt_integrate_scan.

Some callers of this library cannot call cudaMalloc while they run (a
real-time mapping loop that allocates nothing after start-up, or a plugin
whose host framework owns all device memory), so they cannot hand over a
workspace.  For them the library offers dbt_integrate_scan_noalloc, which
works in a fixed scratch array compiled into the library.  These tests call
it through the C ABI and check that two scans in a row leave exactly the same
grid state and scan counters as the workspace entry point (the state is
integer, so the comparison is bit-exact, as everywhere in the GPU tests),
and that inputs beyond its stated limits are refused.  The file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _both(w, n_scans):
    import paper_2509_20081_gb300 as dbt
    from paper_2509_20081_gb300 import dbtsdf as B
    k = dbt.Kernels(dbt.make_params(**w.params))
    dims = (w.grid.nx, w.grid.ny, w.grid.nz)
    ga = dbt.Grid(*dims, w.grid.res, w.grid.origin)
    gb = dbt.Grid(*dims, w.grid.res, w.grid.origin)
    ws = dbt.Workspace(ga, k, max(len(s[0]) for s in w.scans[:n_scans]))
    pinned = torch.full((n_scans, 64), 0xAB, dtype=torch.uint8).pin_memory()
    for i, (pts, pose) in enumerate(w.scans[:n_scans]):
        x = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
        dbt.dbt_integrate_scan(ga, k, ws, x, pose)
        sa = dbt.dbt_get_scan_stats(ws)
        # counters into pageable memory (copied) and pinned memory (stored by the kernel)
        st = B.dbt_scan_stats() if i % 2 == 0 else B.dbt_scan_stats.from_address(pinned[i].data_ptr())
        B.dbt_integrate_scan_noalloc(gb, k, x, pose, st)
        torch.cuda.synchronize()
        sb = st.as_dict()
        assert sb["error"] == 0 and sa["error"] == 0
        for key in ("n_input", "n_valid", "n_inside", "n_kept", "n_pairs", "n_bricks"):
            assert sa[key] == sb[key], (key, sa, sb)
        for a, b in ((ga.mask, gb.mask), (ga.sign, gb.sign), (ga.hits, gb.hits)):
            assert torch.equal(a, b)
    return sa


def test_noalloc_room_two_scans_match():
    st = _both(synth.room_scan(n_scans=2), 2)
    assert st["n_kept"] > 0


def test_noalloc_urban_at_limit_two_scans_match():
    """1600 x 1600 x 320 grid, scans of exactly 65,536 returns (the limit)."""
    w = synth.urban_sequence(n_scans=2)
    assert len(w.scans[0][0]) == 65536
    st = _both(w, 2)
    assert st["n_kept"] > 30000


def test_noalloc_refuses_oversize():
    """A scan past the 65,536-return limit is refused before anything is
    enqueued (real buffers only; the oversize-grid refusal is checked on the
    host by tests/test_noalloc_cpu.py through dbt_noalloc_check, the check
    this entry point applies first)."""
    import paper_2509_20081_gb300 as dbt
    from paper_2509_20081_gb300 import dbtsdf as B
    k = dbt.Kernels(dbt.make_params())
    g = dbt.Grid(64, 64, 64, 0.1)
    x = torch.zeros((65537, 3), device="cuda")
    pose = np.hstack([np.eye(3), np.zeros((3, 1))])
    with pytest.raises(dbt.DbtError) as e:
        B.dbt_integrate_scan_noalloc(g, k, x, pose)
    assert e.value.status == B.DBT_EINVAL and "65536" in str(e.value)
    torch.cuda.synchronize()
    m, s, h = g.numpy()
    assert (m == 0xFFFFFFFF).all() and (s == 1).all() and (h == 0).all()
