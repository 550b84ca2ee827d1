"""Pins for the oracle's approximate neighbourhood graph (the random
divide-and-conquer plus neighbourhood-propagation construction that Sec. 5.3
uses for its graphs, read as stated in oracle.c).

Each test checks the oracle against something other than itself: the exact
graph (a one-leaf partition reduces to it), the defining property of a median
split, and numpy brute force over the candidate sets the reading names.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1312_3062_gb300 import datagen


def sqd(X, i, js):
    d = X[js].astype(np.int64) - X[i].astype(np.int64)
    return (d * d).sum(axis=1)


def top_r(X, i, cands, R):
    """The R smallest (squared distance, id) over a candidate id set, by sort."""
    c = np.array(sorted(set(int(j) for j in cands) - {int(i)}), np.int64)
    if len(c) == 0:
        return np.full(R, -1), np.full(R, np.inf)
    k = sqd(X, i, c)
    order = np.lexsort((c, k))[:R]
    ids = np.full(R, -1, np.int64)
    keys = np.full(R, np.inf)
    ids[:len(order)] = c[order]
    keys[:len(order)] = k[order]
    return ids, keys


def halving(N, l, s):
    lo, hi = 0, N
    for bit in range(l - 1, -1, -1):
        m = lo + (hi - lo) // 2
        lo, hi = (m, hi) if (s >> bit) & 1 else (lo, m)
    return lo, hi


@pytest.fixture(scope="module")
def data():
    return datagen.mixture(31, 1537, 64, 24, np.uint8)


@pytest.mark.parametrize("iters", [0, 1, 2])
def test_one_leaf_is_the_exact_graph(data, iters):
    # levels = 0: the whole set is one leaf, so the leaf step is the exact
    # R-NN graph, and an exact row can only be kept by propagation
    X = data
    dirs = datagen.rp_directions(3, 2, 0, X.shape[1])
    ids, keys = oracle.knn_graph_approx(X, 12, dirs, iters)
    gi, gk = oracle.knn_graph(X, 12)
    assert np.array_equal(ids, gi) and np.array_equal(keys, gk)


@pytest.mark.parametrize("levels", [1, 3, 5])
def test_partition_is_a_median_split_at_every_node(data, levels):
    X = data
    N = len(X)
    dirs = datagen.rp_directions(7, 1, levels, X.shape[1])[0]
    perm = oracle.rp_partition(X, dirs)
    assert np.array_equal(np.sort(perm), np.arange(N))
    for l in range(levels):
        for s in range(1 << l):
            lo, hi = halving(N, l, s)
            m = lo + (hi - lo) // 2
            u = dirs[(1 << l) - 1 + s].astype(np.int64)
            proj = X[perm[lo:hi]].astype(np.int64) @ u
            key = [(int(p), int(i)) for p, i in zip(proj, perm[lo:hi])]
            assert max(key[:m - lo]) < min(key[m - lo:]), (l, s)


def test_leaf_step_is_brute_force_over_leaf_mates(data):
    X = data
    N, R, levels, rounds = len(X), 10, 4, 3
    dirs = datagen.rp_directions(11, rounds, levels, X.shape[1])
    ids, keys = oracle.knn_graph_approx(X, R, dirs, 0)
    mates = [set() for _ in range(N)]
    for r in range(rounds):
        perm = oracle.rp_partition(X, dirs[r])
        for s in range(1 << levels):
            lo, hi = halving(N, levels, s)
            members = perm[lo:hi]
            assert len(members) >= R + 1
            for i in members:
                mates[i].update(members.tolist())
    for i in range(N):
        ti, tk = top_r(X, i, mates[i], R)
        assert np.array_equal(ids[i], ti) and np.array_equal(keys[i], tk), i


def test_propagation_step_is_brute_force_over_neighbours_of_neighbours(data):
    X = data
    N, R = len(X), 8
    dirs = datagen.rp_directions(13, 1, 5, X.shape[1])
    g0, _ = oracle.knn_graph_approx(X, R, dirs, 0)
    g1, k1 = oracle.knn_graph_approx(X, R, dirs, 1)
    g2, k2 = oracle.knn_graph_approx(X, R, dirs, 2)
    for prev, cur, ck in ((g0, g1, k1), (g1, g2, k2)):
        for i in range(N):
            cands = set(prev[i].tolist())
            for j in prev[i]:
                if j >= 0:
                    cands.update(prev[j].tolist())
            cands.discard(-1)
            ti, tk = top_r(X, i, cands, R)
            assert np.array_equal(cur[i], ti) and np.array_equal(ck[i], tk), i


def test_rows_on_demand_match_the_whole_graph(data):
    X = data
    dirs = datagen.rp_directions(17, 2, 4, X.shape[1])
    ids, keys = oracle.knn_graph_approx(X, 10, dirs, 2)
    rows = np.array([0, 5, 1536, 700, 5], np.int64)
    si, sk = oracle.knn_graph_approx(X, 10, dirs, 2, rows=rows)
    assert np.array_equal(si, ids[rows]) and np.array_equal(sk, keys[rows])


def test_more_rounds_and_steps_only_lower_the_keys_and_reach_high_recall(data):
    X = data
    R = 10
    gi, gk = oracle.knn_graph(X, R)
    d = X.shape[1]
    prev = None
    for rounds, iters in ((1, 0), (2, 0), (4, 0), (4, 1), (4, 2)):
        dirs = datagen.rp_directions(19, 4, 4, d)[:rounds]
        ids, keys = oracle.knn_graph_approx(X, R, dirs, iters)
        assert np.all(keys >= gk)  # never better than exact
        if prev is not None:
            assert np.all(keys <= prev)  # a superset of candidates
        prev = keys
    recall = np.mean([len(set(ids[i]) & set(gi[i])) / R for i in range(len(X))])
    assert recall >= 0.9, recall


def test_input_helpers():
    # rp_levels: the fewest halvings after which no leaf exceeds leaf_max
    for N, leaf in ((1, 1), (97, 13), (1000, 1000), (1001, 1000), (10_000_000, 10_000), (1_000_000, 977)):
        L = datagen.rp_levels(N, leaf)
        assert -(-N // (1 << L)) <= leaf
        assert L == 0 or -(-N // (1 << (L - 1))) > leaf
    # rp_directions: one +-1 direction per segment of every level of every round, seeded
    dirs = datagen.rp_directions(4, 3, 5, 32)
    assert dirs.shape == (3, 31, 32) and dirs.dtype == np.int8
    assert set(np.unique(dirs).tolist()) == {-1, 1}
    assert np.array_equal(dirs, datagen.rp_directions(4, 3, 5, 32))
    assert not np.array_equal(dirs, datagen.rp_directions(5, 3, 5, 32))
    assert datagen.rp_directions(4, 2, 0, 16).shape == (2, 0, 16)


def test_duplicate_rows_break_ties_by_id():
    # 300 distinct rows, each five times: many equal keys (0 among copies),
    # so the id tie-break and the distinct-id rule decide the rows
    base = datagen.mixture(41, 300, 32, 6, np.uint8)
    X = np.repeat(base, 5, axis=0)
    N, R = len(X), 8
    dirs0 = datagen.rp_directions(43, 1, 0, 32)
    ids, keys = oracle.knn_graph_approx(X, R, dirs0, 1)
    gi, gk = oracle.knn_graph(X, R)
    assert np.array_equal(ids, gi) and np.array_equal(keys, gk)
    dirs = datagen.rp_directions(43, 2, 4, 32)
    ids, keys = oracle.knn_graph_approx(X, R, dirs, 0)
    mates = [set() for _ in range(N)]
    for r in range(2):
        perm = oracle.rp_partition(X, dirs[r])
        for s in range(16):
            lo, hi = halving(N, 4, s)
            for i in perm[lo:hi]:
                mates[i].update(perm[lo:hi].tolist())
    for i in range(N):
        ti, tk = top_r(X, i, mates[i], R)
        assert np.array_equal(ids[i], ti) and np.array_equal(keys[i], tk), i
        assert len(set(ids[i].tolist())) == R
