"""Host-side logic of the serving loop (no GPU): memory admission."""
from paper_2509_20081_gb300.serve import Admission, grid_bytes


def test_admission_budget():
    a = Admission(1000)
    assert a.try_reserve("m1", 600)
    assert not a.try_reserve("m2", 500)          # would exceed the budget
    assert a.try_reserve("m1", 600) and a.used == 600   # idempotent
    a.release("m1")
    assert a.used == 0 and a.try_reserve("m2", 500) and a.try_reserve("m3", 500)
    assert not a.try_reserve("m4", 1)


def test_grid_bytes_matches_layout():
    # 7 bytes per voxel over the padded row pitch (Eq. 1 with S_voxel = 7)
    assert grid_bytes(1200, 1200, 200) == 1216 * 1200 * 200 * 7
    assert grid_bytes(400, 400, 100) == 416 * 400 * 100 * 7
