"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
brute force on tiny inputs, a textbook special case, or invariants of
Algorithm 1 (Sec. 4.2).  A plausible mistake anywhere in the oracle (a dropped
term, a wrong index, a flipped tie rule, an off-by-one in the budget) fails at
least one of them.
"""
from __future__ import annotations

import heapq
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle


# --------------------------------------------------------------------------
# helpers written independently of the oracle
# --------------------------------------------------------------------------

def nearest_f32(fr: Fraction) -> float:
    """The float32 nearest to an exact rational, ties to even mantissa."""
    f = np.float32(float(fr))
    best = None
    for c in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        if not np.isfinite(c):
            continue
        err = abs(Fraction(float(c)) - fr)
        even = (int(np.array(c, np.float32).view(np.uint32)) & 1) == 0
        cand = (err, 0 if even else 1)
        if best is None or cand < best[0]:
            best = (cand, float(c))
    return best[1]


def exact_key(a, b) -> float:
    """Squared L2 as the search compares it: exact integer for bytes, nearest
    float32 to the exact value for float32 inputs."""
    if a.dtype == np.uint8:
        diff = a.astype(np.int64) - b.astype(np.int64)
        return float(int((diff * diff).sum()))
    s = sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(a, b))
    return nearest_f32(s)


def part_tables(q, centers):
    P, n, dp = centers.shape
    return np.array([[exact_key(q[p * dp:(p + 1) * dp], centers[p, c]) for c in range(n)]
                     for p in range(P)])


def bridge_key_py(parts_keys, dtype):
    """Sec. 4.2's bridge key, sum_p of the part keys: the exact integer sum for
    bytes; for float32 the float32 nearest to the exact (rational) sum of the
    float32 part keys."""
    if np.dtype(dtype) == np.uint8:
        return float(sum(int(v) for v in parts_keys))
    return nearest_f32(sum(Fraction(float(np.float32(x))) for x in parts_keys))


def all_bridges_sorted(D, dtype):
    """Every bridge (center-id tuple) sorted by (bridge key, rank tuple)."""
    P, n = D.shape
    rank = np.empty((P, n), np.int64)
    for p in range(P):
        order = sorted(range(n), key=lambda c: (D[p, c], c))
        for r, c in enumerate(order):
            rank[p, c] = r
    out = []
    for cs in itertools.product(range(n), repeat=P):
        key = bridge_key_py([D[p, cs[p]] for p in range(P)], dtype)
        out.append((key, tuple(int(rank[p, cs[p]]) for p in range(P)), cs))
    out.sort(key=lambda e: (e[0], e[1]))
    return out


def bridge_id(cs, n):
    v = 0
    for c in cs:
        v = v * n + int(c)
    return v


def gmm(rng, N, d, ncomp, sigma, dtype):
    means = rng.uniform(0, 255 if dtype == np.uint8 else 1.0, size=(ncomp, d))
    comp = rng.integers(0, ncomp, size=N)
    x = means[comp] + rng.standard_normal((N, d)) * sigma
    if dtype == np.uint8:
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)
    x = np.abs(x)
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def tiny_index(rng, N, d, P, n, R, t, b, dtype, ncomp=6):
    sigma = 20.0 if dtype == np.uint8 else 0.15
    X = gmm(rng, N, d, ncomp, sigma, dtype)
    G, _ = oracle.knn_graph(X, R)
    init = rng.permutation(N)[:n]
    C = oracle.round_centers(oracle.kmeans(X, P, n, 4, init), dtype)
    bg = oracle.bridge_graph(X, C, t, b)
    return X, G, C, bg


# --------------------------------------------------------------------------
# distances and linear scan (Sec. 2, Sec. 5.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_exact_knn_keys_are_exact_squared_distances(oracle_lib, dtype):
    rng = np.random.default_rng(1)
    X = gmm(rng, 40, 12, 3, 20.0 if dtype == np.uint8 else 0.2, dtype)
    Qs = gmm(rng, 5, 12, 3, 20.0 if dtype == np.uint8 else 0.2, dtype)
    ids, keys = oracle.exact_knn(X, Qs, 40)
    for i in range(5):
        for r in range(40):
            assert keys[i, r] == exact_key(Qs[i], X[ids[i, r]])


def test_exact_knn_ties_break_by_id(oracle_lib):
    # duplicated rows give equal keys; the smaller id must come first
    rng = np.random.default_rng(2)
    base = rng.integers(0, 256, size=(10, 8)).astype(np.uint8)
    X = np.concatenate([base, base, base])          # ids i, i+10, i+20 identical
    q = base[3:4].copy()
    ids, keys = oracle.exact_knn(X, q, 6)
    assert list(ids[0, :3]) == [3, 13, 23] and list(keys[0, :3]) == [0, 0, 0]
    # brute force with numpy lexsort on (key, id)
    diff = X.astype(np.int64) - q.astype(np.int64)
    dk = (diff * diff).sum(1)
    order = np.lexsort((np.arange(len(X)), dk))[:6]
    assert list(ids[0]) == list(order)


def test_knn_graph_excludes_self_and_pads(oracle_lib):
    rng = np.random.default_rng(3)
    X = rng.integers(0, 256, size=(5, 4)).astype(np.uint8)
    G, K = oracle.knn_graph(X, 6)          # only 4 other rows exist
    for i in range(5):
        assert i not in G[i, :4]
        assert sorted(G[i, :4]) == sorted(set(range(5)) - {i})
        assert list(G[i, 4:]) == [-1, -1] and np.all(np.isinf(K[i, 4:]))
        assert np.all(np.diff(K[i, :4]) >= 0)


def test_f32_key_is_nearest_float32(oracle_lib):
    # a case where the plain float32 sum differs from the nearest float32 of
    # the exact value: keys must follow the exact value
    rng = np.random.default_rng(4)
    X = rng.random((64, 48)).astype(np.float32)
    q = rng.random((1, 48)).astype(np.float32)
    _, keys = oracle.exact_knn(X, q, 64)
    exact = sorted(exact_key(q[0], X[j]) for j in range(64))
    assert list(keys[0]) == exact


# --------------------------------------------------------------------------
# k-means per part (Sec. 3.2, Sec. 4.1)
# --------------------------------------------------------------------------

def test_kmeans_separated_clusters_give_cluster_means(oracle_lib):
    # closed form: well separated groups, init with one row per group ->
    # centres are the group means after the first update and stay there
    rng = np.random.default_rng(5)
    P, n, d = 2, 3, 4
    groups = [rng.integers(0, 10, size=(7, d)) + 80 * g for g in range(n)]
    X = np.concatenate(groups).astype(np.uint8)
    init = np.array([0, 7, 14])
    C = oracle.kmeans(X, P, n, 3, init)
    for g in range(n):
        mean = groups[g].astype(np.float64).mean(0)
        np.testing.assert_allclose(C[0, g], mean[:2], rtol=0, atol=1e-12)
        np.testing.assert_allclose(C[1, g], mean[2:], rtol=0, atol=1e-12)


def test_kmeans_matches_scipy_lloyd(oracle_lib):
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(6)
    X = gmm(rng, 300, 8, 5, 20.0, np.uint8)
    P, n = 2, 6
    init = rng.permutation(300)[:n]
    C = oracle.kmeans(X, P, n, 5, init)
    for p in range(P):
        part = X[:, p * 4:(p + 1) * 4].astype(np.float64)
        cent = part[init].copy()
        for _ in range(5):                 # textbook Lloyd via scipy's vq assignment
            lab, _ = vq.vq(part, cent)
            for j in range(n):
                if np.any(lab == j):
                    cent[j] = part[lab == j].mean(0)
        np.testing.assert_allclose(C[p], cent, rtol=1e-12, atol=1e-12)


def test_kmeans_objective_non_increasing(oracle_lib):
    rng = np.random.default_rng(7)
    X = gmm(rng, 400, 8, 8, 20.0, np.uint8)
    init = rng.permutation(400)[:10]
    prev = np.inf
    for it in range(1, 6):
        C = oracle.kmeans(X, 2, 10, it, init)
        obj = 0.0
        for p in range(2):
            part = X[:, p * 4:(p + 1) * 4].astype(np.float64)
            dd = ((part[:, None, :] - C[p][None]) ** 2).sum(-1)
            obj += dd.min(1).sum()
        assert obj <= prev + 1e-6
        prev = obj


def test_round_centers_half_even_and_clip(oracle_lib):
    C = np.array([[[0.5, 1.5, 2.5, -3.0, 255.6, 254.5]]])
    assert list(oracle.round_centers(C, np.uint8)[0, 0]) == [0, 2, 2, 0, 255, 254]


# --------------------------------------------------------------------------
# multi-sequence (Sec. 3.3) and the bridge-key identity (Sec. 4.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("P,n,dtype", [(2, 64, np.uint8), (3, 16, np.uint8), (4, 8, np.uint8),
                                       (2, 24, np.float32), (3, 10, np.float32),
                                       (4, 6, np.float32)])
def test_multiseq_equals_full_sort(oracle_lib, P, n, dtype):
    rng = np.random.default_rng(10 + P * n)
    if dtype == np.uint8:
        D = rng.integers(0, 12, size=(P, n)).astype(np.float64)   # many equal keys
    else:
        D = rng.random((P, n)).astype(np.float32).astype(np.float64)
        D[:, ::3] = D[:, :1]                                          # forced duplicates
    full = all_bridges_sorted(D, dtype)
    keys, ids, ranks, st = oracle.multiseq(D, dtype, n ** P + 5)
    assert len(keys) == n ** P
    assert [e[0] for e in full] == list(keys)
    assert [bridge_id(e[2], n) for e in full] == [int(v) for v in ids]
    assert [e[1] for e in full] == [tuple(r) for r in ranks]


def _f32(bits):
    return float(np.array([bits], np.uint32).view(np.float32)[0])


@pytest.mark.parametrize("P", [2, 3, 4])
def test_f32_bridge_key_is_nearest_float32_of_the_exact_sum(oracle_lib, P):
    # One center per part: the only bridge's key is the key of the part keys'
    # sum.  Cases where any grouped float32 sum (or a float64 sum rounded
    # again) would round differently: halfway cases broken by a tiny term,
    # exact halfway cases (ties to even), very wide exponent spreads,
    # subnormals, zeros, and random values.
    rng = np.random.default_rng(77 + P)
    eps = 2.0 ** -24
    cases = [
        [1.0, eps, 2.0 ** -60, 0.0],          # halfway + tiny: rounds up
        [1.0, eps, 0.0, 0.0],                 # exact halfway: ties to even (down)
        [1.0 + 2 * eps, eps, 0.0, 0.0],       # exact halfway, odd significand: up
        [1.0, 2.0 ** -25, 2.0 ** -25, 2.0 ** -80],  # two quarter-ulps make a half, plus tiny
        [3.0, 2.0 ** -120, 2.0 ** -149, 2.0 ** -140],
        [2.0 ** -149, 2.0 ** -149, 2.0 ** -148, 0.0],
        [0.0, 0.0, 0.0, 0.0],
        [2.0 ** 100, 1.0, 2.0 ** 76, 2.0 ** 75],
        [_f32(0x3f7fffff), _f32(0x33000000), _f32(0x2f000000), 0.0],
    ]
    for _ in range(300):
        e = rng.integers(-40, 10, size=4)
        cases.append([float(np.float32(rng.random() * 2.0 ** int(x))) for x in e])
    for c in cases:
        parts = np.array([[np.float32(v)] for v in c[:P]], np.float64)
        keys, ids, _, _ = oracle.multiseq(parts, np.float32, 1)
        assert keys[0] == bridge_key_py(parts[:, 0], np.float32), c[:P]


def test_multiseq_prefix_and_frontier_bound(oracle_lib):
    rng = np.random.default_rng(11)
    D = rng.integers(0, 1000, size=(4, 16)).astype(np.float64)
    full = all_bridges_sorted(D, np.uint8)
    keys, ids, _, st = oracle.multiseq(D, np.uint8, 100)
    assert [e[0] for e in full[:100]] == list(keys)
    # 'popped' push rule: every queued tuple has all predecessors popped, so the
    # queue never holds more than (P-1)*pops + 1 tuples
    assert st["max_frontier"] <= 3 * 100 + 1
    assert st["pushes"] <= 4 * 100 + 1


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_bridge_key_is_distance_to_concatenated_bridge(oracle_lib, dtype):
    # dist^2(q, y) = sum_p dist^2(q^p, y^p)  (Sec. 4.2)
    rng = np.random.default_rng(12)
    P, n, d = 3, 5, 12
    C = (rng.integers(0, 256, size=(P, n, d // P)).astype(np.uint8) if dtype == np.uint8
         else rng.random((P, n, d // P)).astype(np.float32))
    q = (rng.integers(0, 256, size=d).astype(np.uint8) if dtype == np.uint8
         else rng.random(d).astype(np.float32))
    D = part_tables(q, C)
    keys, ids, ranks, _ = oracle.multiseq(D, dtype, n ** P)
    for key, bid in zip(keys, ids):
        cs = []
        v = int(bid)
        for _ in range(P):
            cs.append(v % n)
            v //= n
        cs = cs[::-1]
        y = np.concatenate([C[p, cs[p]] for p in range(P)])
        if dtype == np.uint8:
            assert key == exact_key(q, y)
        else:
            assert abs(key - exact_key(q, y)) <= 4 * np.finfo(np.float32).eps * key + 1e-30


# --------------------------------------------------------------------------
# bridge graph (Sec. 4.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_bridge_graph_bruteforce(oracle_lib, dtype):
    rng = np.random.default_rng(13)
    N, d, P, n, t, b = 60, 8, 2, 8, 10, 3
    X = gmm(rng, N, d, 4, 20.0 if dtype == np.uint8 else 0.2, dtype)
    C = oracle.round_centers(oracle.kmeans(X, P, n, 3, rng.permutation(N)[:n]), dtype)
    bg = oracle.bridge_graph(X, C, t, b)
    named = {}
    for i in range(N):
        D = part_tables(X[i], C)
        for key, _, cs in all_bridges_sorted(D, dtype)[:t]:
            named.setdefault(bridge_id(cs, n), []).append((key, i))
    expect_ids = sorted(named)
    assert [int(v) for v in bg["bridges"]] == expect_ids
    for j, bid in enumerate(expect_ids):
        kept = sorted(named[bid])[:b]
        lo, hi = bg["offsets"][j], bg["offsets"][j + 1]
        assert list(bg["refs"][lo:hi]) == [r for _, r in kept]
        assert list(bg["keys"][lo:hi]) == [k for k, _ in kept]


# --------------------------------------------------------------------------
# Algorithm 1 (Sec. 4.2)
# --------------------------------------------------------------------------

def alg1_bruteforce(X, G, C, bg, q, k, T):
    """Algorithm 1 with bridges enumerated by a full sort instead of the
    multi-sequence, Python heapq / set, and the exact budget cap."""
    P, n, _ = C.shape
    D = part_tables(q, C)
    stream = iter(all_bridges_sorted(D, X.dtype))
    lists = {int(bg["bridges"][j]): list(bg["refs"][bg["offsets"][j]:bg["offsets"][j + 1]])
             for j in range(len(bg["bridges"]))}
    Q, seen, res, disc = [], set(), [], []
    cur = next(stream, None)
    if cur is not None:
        heapq.heappush(Q, (cur[0], 1, 0))
    t = 0
    while Q and t < T:
        key, kind, ident = heapq.heappop(Q)
        adj = G[ident] if kind == 0 else lists.get(bridge_id(cur[2], n), [])
        for x in adj:
            x = int(x)
            if x < 0 or x in seen:
                continue
            seen.add(x)
            dx = exact_key(q, X[x])
            heapq.heappush(Q, (dx, 0, x))
            res.append((dx, x))
            disc.append(x)
            t += 1
            if t == T:
                break
        if kind == 1 and t < T:
            cur = next(stream, None)
            if cur is not None:
                heapq.heappush(Q, (cur[0], 1, 0))
    res.sort()
    return res[:k], disc


@pytest.mark.parametrize("dtype,T", [(np.uint8, 7), (np.uint8, 40), (np.uint8, 500),
                                     (np.float32, 25), (np.float32, 500)])
def test_search_trace_matches_bruteforce_alg1(oracle_lib, dtype, T):
    rng = np.random.default_rng(20 + T)
    X, G, C, bg = tiny_index(rng, 120, 8, 2, 6, 4, 5, 2, dtype)
    Qs = gmm(rng, 6, 8, 6, 20.0 if dtype == np.uint8 else 0.15, dtype)
    k = 5
    ids, keys, st = oracle.search(X, G, C, bg, Qs, k, T, trace=True)
    for i in range(len(Qs)):
        res, disc = alg1_bruteforce(X, G, C, bg, Qs[i], k, T)
        assert list(st["trace"][i, :len(disc)]) == disc
        assert np.all(st["trace"][i, len(disc):] == -1)
        assert [r for _, r in res] == list(ids[i, :len(res)])
        assert [kk for kk, _ in res] == list(keys[i, :len(res)])
        assert np.all(ids[i, len(res):] == -1)


def reachable_from_bridges(G, bg, N):
    seen = set(int(r) for r in bg["refs"])
    stack = list(seen)
    while stack:
        v = stack.pop()
        for x in G[v]:
            x = int(x)
            if x >= 0 and x not in seen:
                seen.add(x)
                stack.append(x)
    return np.array(sorted(seen), np.int64)


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_large_budget_returns_exact_topk_of_reachable_set(oracle_lib, dtype):
    rng = np.random.default_rng(30)
    N = 300
    X, G, C, bg = tiny_index(rng, N, 16, 2, 8, 6, 10, 3, dtype)
    reach = reachable_from_bridges(G, bg, N)
    Qs = gmm(rng, 10, 16, 6, 20.0 if dtype == np.uint8 else 0.15, dtype)
    k = 10
    ids, keys, st = oracle.search(X, G, C, bg, Qs, k, N + 5)
    assert np.all(st["discovered"] == len(reach))
    for i in range(len(Qs)):
        kk = np.array([exact_key(Qs[i], X[j]) for j in reach])
        order = np.lexsort((reach, kk))[:k]
        assert list(ids[i]) == list(reach[order])
        assert list(keys[i]) == list(kk[order])


def test_budget_equal_to_n_returns_exact_nn(oracle_lib):
    # every reference reachable => T = N gives the exact k-NN (Sec. 2)
    rng = np.random.default_rng(31)
    N = 200
    X, G, C, bg = tiny_index(rng, N, 16, 2, 8, 12, 64, N, np.uint8, ncomp=2)
    assert len(reachable_from_bridges(G, bg, N)) == N
    Qs = gmm(rng, 8, 16, 2, 20.0, np.uint8)
    ids, keys, st = oracle.search(X, G, C, bg, Qs, 10, N)
    diff = Qs[:, None, :].astype(np.int64) - X[None].astype(np.int64)
    dk = (diff * diff).sum(-1)
    for i in range(len(Qs)):
        order = np.lexsort((np.arange(N), dk[i]))[:10]
        assert list(ids[i]) == list(order)
        assert list(keys[i]) == list(dk[i][order].astype(np.float64))


def test_search_invariants_and_monotone_discovery(oracle_lib):
    rng = np.random.default_rng(32)
    N = 400
    X, G, C, bg = tiny_index(rng, N, 16, 2, 8, 6, 10, 3, np.uint8)
    reach = len(reachable_from_bridges(G, bg, N))
    Qs = gmm(rng, 12, 16, 6, 20.0, np.uint8)
    prev = None
    for T in (1, 5, 17, 64, 150, 1000):
        _, _, st = oracle.search(X, G, C, bg, Qs, 10, T, trace=True)
        assert np.all(st["discovered"] == min(T, reach))          # exact budget
        assert np.all(st["max_q"] <= T + 1)                       # queue bound (Sec. 6)
        tr = st["trace"]
        for i in range(len(Qs)):
            got = tr[i][tr[i] >= 0]
            assert len(set(got.tolist())) == len(got)             # nothing discovered twice
            if prev is not None:                                  # deterministic prefix
                p = prev[i][prev[i] >= 0]
                assert list(got[:len(p)]) == list(p)
        prev = tr


def test_k_larger_than_budget_pads(oracle_lib):
    rng = np.random.default_rng(33)
    X, G, C, bg = tiny_index(rng, 100, 8, 2, 6, 4, 5, 2, np.uint8)
    Qs = gmm(rng, 3, 8, 6, 20.0, np.uint8)
    ids, keys, st = oracle.search(X, G, C, bg, Qs, 10, 4)
    assert np.all(ids[:, 4:] == -1) and np.all(np.isinf(keys[:, 4:]))
    assert np.all(ids[:, :4] >= 0)


def test_single_seed_reduces_to_best_first_graph_search(oracle_lib):
    # one non-empty bridge holding one reference = Arya-Mount best-first search
    # seeded at that reference (Sec. 3.1): textbook version written here
    rng = np.random.default_rng(34)
    N = 150
    X = gmm(rng, N, 8, 5, 20.0, np.uint8)
    G, _ = oracle.knn_graph(X, 5)
    C = oracle.round_centers(oracle.kmeans(X, 2, 4, 2, rng.permutation(N)[:4]), np.uint8)
    seed = 17
    bg = {"bridges": np.array([5], np.uint64), "offsets": np.array([0, 1], np.int64),
          "refs": np.array([seed], np.int32)}
    Qs = gmm(rng, 5, 8, 5, 20.0, np.uint8)
    T = 60
    _, _, st = oracle.search(X, G, C, bg, Qs, 5, T, trace=True)
    for i in range(len(Qs)):
        q = Qs[i]
        seen = {seed}
        order = [seed]
        heap = [(exact_key(q, X[seed]), seed)]
        while heap and len(order) < T:
            _, p = heapq.heappop(heap)
            for x in G[p]:
                x = int(x)
                if x not in seen:
                    seen.add(x)
                    order.append(x)
                    heapq.heappush(heap, (exact_key(q, X[x]), x))
                    if len(order) == T:
                        break
        assert list(st["trace"][i][:len(order)]) == order


def test_recall_counts_ties_at_kth(oracle_lib):
    X = np.array([[0], [1], [1], [5]], np.uint8)
    q = np.array([[0]], np.uint8)
    true_ids, true_keys = oracle.exact_knn(X, q, 2)        # keys 0, 1 (ids 0, 1)
    found = np.array([[0, 2]], np.int32)                   # id 2 ties with id 1
    assert oracle.recall_at_k(found, true_keys, X, q, 2)[0] == 1.0
    found = np.array([[0, 3]], np.int32)
    assert oracle.recall_at_k(found, true_keys, X, q, 2)[0] == 0.5


def test_on_demand_rows_equal_stored_graph(oracle_lib):
    # Adj[x] computed by linear scan when popped = the stored exact R-NN row
    rng = np.random.default_rng(35)
    X, G, C, bg = tiny_index(rng, 300, 16, 2, 6, 7, 10, 3, np.uint8)
    Qs = gmm(rng, 6, 16, 6, 20.0, np.uint8)
    a = oracle.search(X, G, C, bg, Qs, 5, 120, trace=True)
    b = oracle.search(X, 7, C, bg, Qs, 5, 120, trace=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2]["trace"], b[2]["trace"])
    # spare threads split each row's scan (6 queries, 16 threads: 2 per row)
    c = oracle.search(X, 7, C, bg, Qs, 5, 120, trace=True, nthreads=16)
    np.testing.assert_array_equal(a[0], c[0])
    np.testing.assert_array_equal(a[2]["trace"], c[2]["trace"])
    # ties across chunk boundaries: duplicated rows
    Xd = np.concatenate([X, X[:40]])
    Gd, _ = oracle.knn_graph(Xd, 7)
    bgd = oracle.bridge_graph(Xd, C, 10, 3)
    d1 = oracle.search(Xd, Gd, C, bgd, Qs, 5, 150, trace=True)
    d2 = oracle.search(Xd, 7, C, bgd, Qs[:2], 5, 150, trace=True, nthreads=16)
    np.testing.assert_array_equal(d1[0][:2], d2[0])
    np.testing.assert_array_equal(d1[2]["trace"][:2], d2[2]["trace"])


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_bridge_lists_of_selected_bridges_equal_the_bridge_graph(oracle_lib, dtype):
    # the restricted form (no global sort of all N*t triples) agrees with the
    # full bridge graph on present ids and gives empty lists for absent ids
    rng = np.random.default_rng(31)
    X = gmm(rng, 500, 16, 6, 20.0 if dtype == np.uint8 else 0.2, dtype)
    init = rng.permutation(len(X))[:8]
    C = oracle.round_centers(oracle.kmeans(X, 4, 8, 4, init), dtype)
    bg = oracle.bridge_graph(X, C, 30, 3)
    present = bg["bridges"][rng.choice(len(bg["bridges"]), 40, replace=False)]
    absent = np.setdiff1d(np.arange(8 ** 4, dtype=np.uint64), bg["bridges"])[:20]
    sel = np.sort(np.concatenate([present, absent]))
    counts, refs, keys = oracle.bridge_lists(X, C, 30, 3, sel, nthreads=4)
    where = {int(v): i for i, v in enumerate(bg["bridges"])}
    for i, y in enumerate(sel):
        if int(y) not in where:
            assert counts[i] == 0 and np.all(refs[i] == -1)
            continue
        j = where[int(y)]
        lo, hi = bg["offsets"][j], bg["offsets"][j + 1]
        assert counts[i] == hi - lo
        np.testing.assert_array_equal(refs[i, :counts[i]], bg["refs"][lo:hi])
        np.testing.assert_array_equal(keys[i, :counts[i]], bg["keys"][lo:hi])


# --------------------------------------------------------------------------
# bridge graph restricted to the bridges queries can reach (Sec. 4.1), and
# the search's bridge-key limit: the means of checking full-size searches
# whose whole bridge graph is too large to build
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_restricted_bridge_graph_holds_the_full_lists_of_reachable_bridges(oracle_lib, dtype):
    rng = np.random.default_rng(21)
    X, G, C, bg = tiny_index(rng, 400, 16, 2, 12, 8, 30, 3, dtype)
    Q = gmm(rng, 5, 16, 6, 20.0 if dtype == np.uint8 else 0.15, dtype)
    P, n, _ = C.shape
    full = {int(y): list(bg["refs"][bg["offsets"][i]:bg["offsets"][i + 1]]) for i, y in enumerate(bg["bridges"])}
    # each query's key to every bridge of the full graph (independent statement)
    qkeys = []
    for q in Q:
        D = part_tables(q, C)
        kq = {}
        for y in full:
            cs, v = [], y
            for _ in range(P):
                cs.append(v % n)
                v //= n
            cs = cs[::-1]
            kq[y] = bridge_key_py([D[p, cs[p]] for p in range(P)], dtype)
        qkeys.append(kq)
    for frac in (0.2, 0.5, 1.0):
        limits = np.array([np.quantile(list(kq.values()), frac) for kq in qkeys])
        near = oracle.bridge_graph_near(X, C, 30, 3, Q, limits)
        got = {int(y): list(near["refs"][near["offsets"][i]:near["offsets"][i + 1]])
               for i, y in enumerate(near["bridges"])}
        need = {y for y in full if any(qkeys[i][y] <= limits[i] for i in range(len(Q)))}
        assert need <= set(got)                                  # every reachable bridge is there
        for y, lst in got.items():
            assert lst == full[y]                                # with the full graph's list
            if y not in need:                                    # extras only within the float margin
                assert dtype == np.float32 and any(qkeys[i][y] <= limits[i] * (1 + 1e-5) for i in range(len(Q)))


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_search_with_restricted_bridges_equals_full_search_or_reports(oracle_lib, dtype):
    rng = np.random.default_rng(22)
    X, G, C, bg = tiny_index(rng, 800, 16, 2, 24, 6, 10, 3, dtype, ncomp=12)
    Q = gmm(rng, 12, 16, 12, 20.0 if dtype == np.uint8 else 0.15, dtype)
    want_i, want_k, want_s = oracle.search(X, G, C, bg, Q, 10, 60)
    assert not want_s["over_limit"].any()
    kth = oracle.exact_knn(X, Q, 20)[1][:, -1]
    partial = 0
    for scale in (0.5, 1.0, 1.2, 1.5, 2.0):
        limits = kth * scale
        near = oracle.bridge_graph_near(X, C, 10, 3, Q, limits)
        got_i, got_k, got_s = oracle.search(X, G, C, near, Q, 10, 60, bridge_key_limit=limits)
        ok = got_s["over_limit"] == 0
        np.testing.assert_array_equal(got_i[ok], want_i[ok])
        np.testing.assert_array_equal(got_k[ok], want_k[ok])
        if scale == 0.5:
            assert not ok.any()       # a tight limit is reported, not searched past
        partial += ok.any() and len(near["bridges"]) < len(bg["bridges"])
    assert partial >= 2               # complete searches on graphs missing some bridges
    # an unbounded limit over the full graph changes nothing
    i2, k2, s2 = oracle.search(X, G, C, bg, Q, 10, 60, bridge_key_limit=np.inf)
    np.testing.assert_array_equal(i2, want_i)
