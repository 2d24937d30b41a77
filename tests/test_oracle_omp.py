"""The points-parallel (OpenMP) variant of the oracle against the oracle.

The variant is the CPU baseline that runs like the paper's implementation
(per-return updates spread over the host cores, Sec. IV); it must leave
exactly the map the sequential oracle leaves (the per-voxel updates are
atomic, and AND, the saturating count and the one-way sign do not depend on
their order).  Whole-grid comparison of mask, sign and hits, and of every
counter that does not depend on the order, for several thread counts and
parameter sets.
"""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def omp(orc):
    if orc.build_omp() is None:
        pytest.skip("no OpenMP runtime for the C compiler")
    orc.lib_omp()
    return orc


@pytest.fixture(scope="module")
def room():
    return synth.room_scan(n_scans=3)


ORDER_FREE = ("n_input", "n_valid", "n_inside", "n_kept", "n_shadow_incs")


def _run(orc, pdict, dims, res, origin, scans, threads):
    p = orc.params(**pdict)
    ga = orc.Grid.create(*dims, res, origin)
    gb = orc.Grid.create(*dims, res, origin)
    for pts, pose in scans:
        sa = orc.integrate_scan(ga, p, pts, pose)
        sb = orc.integrate_scan_omp(gb, p, pts, pose, threads=threads)
        assert {k: sa[k] for k in ORDER_FREE} == {k: sb[k] for k in ORDER_FREE}
        if threads == 1:
            assert sa["n_mask_writes"] == sb["n_mask_writes"]
    for a, b in ((ga.mask, gb.mask), (ga.sign, gb.sign), (ga.hits, gb.hits)):
        np.testing.assert_array_equal(a, b)
    return sa


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_room_sequence(omp, room, threads):
    st = _run(omp, room.params, (128, 128, 128), 0.1, (0.0, 0.0, 0.0), room.scans, threads)
    assert st["n_kept"] > 5000


@pytest.mark.parametrize("variant", [
    dict(dedup_first=0),
    dict(shadow_radius=5.0, hit_threshold=1, hit_max=2),
    dict(kernel_size=3, shadow_radius=1.0),
    dict(kernel_size=21, scheme=1, bins_a=40, bins_b=40, shadow_radius=6.0, shadow_cos=0.5),
])
def test_room_variants(omp, room, variant):
    pd = dict(room.params)
    pd.update(variant)
    _run(omp, pd, (128, 128, 128), 0.1, (0.0, 0.0, 0.0), room.scans[:1], 6)


def test_urban_quarter(omp):
    """Two scans of the urban generator at a quarter of its size (400 x 400 x
    80 at 0.05 m), every return."""
    w = synth.urban_sequence(n_scans=2, scale=0.25)
    st = _run(omp, w.params, (w.grid.nx, w.grid.ny, w.grid.nz), w.grid.res, w.grid.origin,
              w.scans, 8)
    assert st["n_kept"] > 1000


def test_bad_arguments(omp):
    p = omp.params(kernel_size=4)
    g = omp.Grid.create(32, 32, 32, 0.1)
    with pytest.raises(RuntimeError):
        omp.integrate_scan_omp(g, p, np.zeros((4, 3), np.float32), np.eye(3, 4), threads=2)
