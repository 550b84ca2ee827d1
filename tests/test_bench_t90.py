"""Host logic of bench.py's budget search: the budget reported for "queries/s
at recall@10 = 0.9" is the smallest one reaching 0.9 within 1/64 of the
budget, and always one whose measured recall is >= 0.9."""
import types

import pytest

import bench


class _FakeAnn:
    """Search stand-in: returns the budget itself as the 'ids'."""

    @staticmethod
    def ann_search_batch(index, Q, k, T, kmax, mode):
        return T, None, None


_fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))


def _sweep(monkeypatch, recall_of_T):
    monkeypatch.setattr(bench, "recall_at_10", lambda torch, ids, W, k=None: recall_of_T(ids))
    args = types.SimpleNamespace(T=None)
    return bench.sweep_t90(args, _fake_torch, _FakeAnn, {"index": None, "Q": None}, lambda m: None)


@pytest.mark.parametrize("t_star", [100, 700, 2250, 2896, 5000])
def test_bisection_finds_the_smallest_budget_within_a_64th(monkeypatch, t_star):
    T90, r, table = _sweep(monkeypatch, lambda T: 0.9 if T >= t_star else 0.9 * T / t_star)
    assert r >= 0.9 and T90 >= t_star
    assert T90 - t_star <= max(1, T90 // 64)
    assert [t for t, _ in table] == sorted(t for t, _ in table)
    assert (T90, r) in table


def test_first_grid_point_already_reaching_the_target_is_kept(monkeypatch):
    T90, r, table = _sweep(monkeypatch, lambda T: 0.95)
    assert (T90, r) == (bench.T_GRID[0], 0.95) and table == [(bench.T_GRID[0], 0.95)]


def test_non_monotone_recall_still_returns_a_budget_at_or_above_the_target(monkeypatch):
    # dips below 0.9 inside the bracket: the returned budget must still reach 0.9
    def rec(T):
        if T >= 2896:
            return 0.92
        return 0.91 if 2500 <= T < 2600 else 0.85
    T90, r, _ = _sweep(monkeypatch, rec)
    assert r >= 0.9 and rec(T90) >= 0.9


def test_no_budget_reaching_the_target_reports_the_largest(monkeypatch):
    T90, r, table = _sweep(monkeypatch, lambda T: 0.5)
    assert T90 == bench.T_GRID[-1] and r == 0.5 and len(table) == len(bench.T_GRID)
