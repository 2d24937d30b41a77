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


class _S:
    def __init__(self, n):
        self.n = n


def test_oversize_scan_is_refused():
    """A scan past the round budget could never be scheduled; submit refuses it."""
    import pytest
    from paper_2509_20081_gb300.serve import check_scan_size
    check_scan_size(100, 100)
    with pytest.raises(ValueError):
        check_scan_size(101, 100)


def test_round_selection_with_a_tiny_budget():
    """Rounds take whole scans in arrival order per map, skip maps already on
    the GPU, and stop at the point and item budgets; repeated rounds drain
    every pending scan (no scan that fits the budget waits forever)."""
    from paper_2509_20081_gb300.serve import select_round
    pending = {0: [_S(4), _S(4), _S(3)], 1: [_S(5)], 2: [_S(2), _S(2)]}
    assert select_round([0, 1, 2], set(), pending, 10, 8) == [(0, 2), (2, 1)]
    assert select_round([0, 1, 2], {0}, pending, 10, 8) == [(1, 1), (2, 2)]
    assert select_round([0, 1, 2], set(), pending, 100, 3) == [(0, 3)]
    # drain with budget 5: every scan is taken eventually
    left = {r: list(v) for r, v in pending.items()}
    rounds = 0
    while any(left.values()):
        takes = select_round([0, 1, 2], set(), left, 5, 8)
        assert takes, left
        for r, k in takes:
            del left[r][:k]
        rounds += 1
    assert rounds <= 6
