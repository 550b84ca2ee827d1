"""Pins for the oracle's Graph-D-ADC statement (Sec. 5.4: the method as the
coarse quantizer of an inverted file whose residuals are product-quantized,
re-ranked by asymmetric distance).

Most cases use integer data, integer coarse centers and integer codewords,
so every key is an exact integer in the oracle's fp64 as in numpy's, and the
comparisons are exact; one case uses real-valued k-means centers and
codewords and bounds the fp64 rounding instead.
Each check uses something other than the oracle itself: explicit
reconstruction of the encoded vectors, a codebook that reproduces every
residual (asymmetric distance = true distance, so the result is the exact
k-NN), and brute force over the candidate lists."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1312_3062_gb300 import datagen


def setup(N=800, d=16, K=12, m=4, ks=16, vmax=255, seed=3):
    rng = np.random.default_rng(seed)
    X = np.minimum(datagen.mixture(seed, N, d, 10, np.uint8), vmax).astype(np.float32)
    C = X[rng.choice(N, K, replace=False)].copy()               # coarse centers: K data rows
    assign, _ = oracle.exact_knn(C, X, 1)                        # nearest coarse center
    assign = assign[:, 0]
    R = X.astype(np.float64) - C[assign].astype(np.float64)
    init = rng.choice(N, ks, replace=False)
    cb = np.rint(oracle.kmeans(R.astype(np.float32), m, ks, 4, init))   # integer codewords
    codes = oracle.pq_encode(X, C, assign, cb)
    offsets, members = oracle.ivf_lists(assign, K)
    return X, C, assign, R, cb, codes, offsets, members


def reconstruct(C, assign, cb, codes):
    m = cb.shape[0]
    parts = [cb[j][codes[:, j]] for j in range(m)]
    return C[assign].astype(np.float64) + np.concatenate(parts, axis=1)


def top_t(keys, ids, T):
    order = np.lexsort((ids, keys))[:T]
    return ids[order], keys[order]


def test_pq_encode_is_the_nearest_codeword_with_ties_to_the_lower_index():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 41, size=(300, 12)).astype(np.float32)
    C = rng.integers(0, 41, size=(5, 12)).astype(np.float32)
    assign = rng.integers(0, 5, size=300)
    R = X.astype(np.float64) - C[assign]
    cb = rng.integers(-20, 21, size=(3, 10, 4)).astype(np.float64)
    cb[1, 7] = cb[1, 3]          # a duplicated codeword: code 3 must win
    codes = oracle.pq_encode(X, C, assign, cb)
    for j in range(3):
        dist = ((R[:, None, 4 * j:4 * j + 4] - cb[j][None]) ** 2).sum(-1)
        assert np.array_equal(codes[:, j], dist.argmin(axis=1))   # argmin takes the first minimum
    assert not (codes[:, 1] == 7).any()


def test_inverted_lists_hold_each_reference_once_ascending():
    _, _, assign, _, _, _, offsets, members = setup()
    assert offsets[-1] == len(assign)
    for c in range(len(offsets) - 1):
        lst = members[offsets[c]:offsets[c + 1]]
        assert np.array_equal(lst, np.flatnonzero(assign == c))


def test_adc_key_is_the_distance_to_the_reconstructed_vector():
    X, C, assign, R, cb, codes, offsets, members = setup()
    Xr = reconstruct(C, assign, cb, codes)
    rng = np.random.default_rng(4)
    Q = np.rint(rng.uniform(0, 255, size=(6, X.shape[1])))
    lists = np.stack([rng.permutation(len(C))[:3] for _ in range(6)]).astype(np.int32)
    ids, keys, seen = oracle.adc_rerank(Q, lists, offsets, members, C, codes, cb, L=10 ** 9, T=25)
    for i in range(6):
        cand = np.concatenate([members[offsets[c]:offsets[c + 1]] for c in lists[i]])
        assert seen[i] == len(cand)
        k = ((Xr[cand] - Q[i]) ** 2).sum(1)
        ti, tk = top_t(k, cand, 25)
        n = min(25, len(cand))
        assert np.array_equal(ids[i, :n], ti) and np.array_equal(keys[i, :n], tk)
        assert (ids[i, n:] == -1).all() and np.isinf(keys[i, n:]).all()


def test_a_codebook_holding_every_residual_gives_the_exact_nearest_neighbours():
    # values <= 127 and integer centers: residuals lie in [-127, 127], so a
    # one-dimensional codebook of those 255 values (plus one spare) reproduces
    # every residual and the asymmetric distance is the true distance
    d, K = 8, 10
    X, C, assign, R, _, _, offsets, members = setup(N=700, d=d, K=K, vmax=127, seed=5)
    cb = np.tile(np.concatenate([np.arange(-127, 128), [128]]).astype(np.float64)[None, :, None], (d, 1, 1))
    codes = oracle.pq_encode(X, C, assign, cb)
    assert np.array_equal(reconstruct(C, assign, cb, codes), X.astype(np.float64))
    Q = datagen.mixture(6, 9, d, 4, np.uint8).astype(np.float32)
    lists = np.tile(np.arange(K, dtype=np.int32), (len(Q), 1))
    ids, keys, _ = oracle.adc_rerank(Q, lists, offsets, members, C, codes, cb, L=len(X), T=10)
    ei, ek = oracle.exact_knn(X, Q, 10)
    assert np.array_equal(ids, ei) and np.array_equal(keys, ek)


def test_candidates_are_the_first_L_members_in_list_order():
    X, C, assign, R, cb, codes, offsets, members = setup()
    Xr = reconstruct(C, assign, cb, codes)
    q = np.full((1, X.shape[1]), 100.0)
    order = np.array([[5, 2, 9, 0]], np.int32)
    full = np.concatenate([members[offsets[c]:offsets[c + 1]] for c in order[0]])
    L = len(members[offsets[5]:offsets[6]]) + 7      # the whole first list and 7 of the second
    ids, keys, seen = oracle.adc_rerank(q, order, offsets, members, C, codes, cb, L=L, T=12)
    assert seen[0] == L
    cand = full[:L]
    ti, tk = top_t(((Xr[cand] - q[0]) ** 2).sum(1), cand, 12)
    assert np.array_equal(ids[0], ti) and np.array_equal(keys[0], tk)


def test_graph_d_adc_search_over_all_lists_is_brute_force_over_all_codes():
    # coarse index: the K centers with their complete neighbourhood graph and
    # a bridge graph; w = Tc = K reaches every center, so with L = N every
    # reference is a candidate
    X, C, assign, R, cb, codes, offsets, members = setup(K=12)
    K = len(C)
    G, _ = oracle.knn_graph(C, K - 1)
    pc = oracle.kmeans(C, 2, 4, 5, np.arange(4)).astype(np.float32)
    bg = oracle.bridge_graph(C, pc, t=16, b=5)
    Q = datagen.mixture(8, 5, X.shape[1], 3, np.uint8).astype(np.float32)
    ids, keys, seen = oracle.graph_d_adc_search(C, G, pc, bg, offsets, members, codes, cb, Q,
                                                w=K, Tc=K, L=len(X), T=20)
    assert (seen == len(X)).all()
    Xr = reconstruct(C, assign, cb, codes)
    allids = np.arange(len(X))
    for i in range(len(Q)):
        ti, tk = top_t(((Xr - Q[i].astype(np.float64)) ** 2).sum(1), allids, 20)
        assert np.array_equal(ids[i], ti) and np.array_equal(keys[i], tk)


@pytest.mark.parametrize("w", [1, 3])
def test_graph_d_adc_search_visits_the_lists_algorithm_1_finds(w):
    # the lists visited are Algorithm 1's k = w result over the centers, in
    # its order: with T = the number of centers that is their exact order
    X, C, assign, R, cb, codes, offsets, members = setup(K=12)
    K = len(C)
    G, _ = oracle.knn_graph(C, K - 1)
    pc = oracle.kmeans(C, 2, 4, 5, np.arange(4)).astype(np.float32)
    bg = oracle.bridge_graph(C, pc, t=16, b=5)
    Q = datagen.mixture(9, 4, X.shape[1], 3, np.uint8).astype(np.float32)
    _, _, seen = oracle.graph_d_adc_search(C, G, pc, bg, offsets, members, codes, cb, Q, w=w, Tc=K,
                                           L=len(X), T=5)
    near, _ = oracle.exact_knn(C, Q, w)
    sizes = offsets[1:] - offsets[:-1]
    assert np.array_equal(seen, sizes[near].sum(1))


def test_real_valued_codes_and_keys_within_fp64_rounding():
    # real-valued centers and codewords: the oracle's codes are the nearest
    # codewords of numpy's explicit distances (up to fp64 near-ties) and its
    # keys the distances to numpy's explicit reconstruction c + r^, within
    # the rounding of fp64 sums of d terms
    rng = np.random.default_rng(11)
    X = datagen.mixture(12, 1500, 32, 8, np.float32)
    d, K, m, ks = 32, 9, 4, 12
    C = oracle.kmeans(X, 1, K, 3, rng.choice(len(X), K, replace=False))[0].astype(np.float32)
    assign, _ = oracle.exact_knn(C, X, 1)
    assign = assign[:, 0]
    R = X.astype(np.float64) - C[assign].astype(np.float64)
    cb = oracle.kmeans(R.astype(np.float32), m, ks, 3, rng.choice(len(X), ks, replace=False)).astype(np.float32)
    codes = oracle.pq_encode(X, C, assign, cb)
    dp = d // m
    for j in range(m):
        dist = ((R[:, None, j * dp:(j + 1) * dp] - cb[j].astype(np.float64)[None]) ** 2).sum(-1)
        best = dist.min(1)
        got = dist[np.arange(len(X)), codes[:, j]]
        assert np.all(got <= best + 1e-12 * (1 + best))
    Xr = reconstruct(C, assign, cb.astype(np.float64), codes)
    offsets, members = oracle.ivf_lists(assign, K)
    Q = datagen.mixture(13, 5, d, 8, np.float32)
    lists = np.tile(np.arange(K, dtype=np.int32), (len(Q), 1))
    ids, keys, _ = oracle.adc_rerank(Q, lists, offsets, members, C, codes, cb, L=len(X), T=40)
    for i in range(len(Q)):
        k = ((Xr - Q[i].astype(np.float64)) ** 2).sum(1)
        order = np.argsort(k, kind="stable")[:40]
        np.testing.assert_allclose(keys[i], k[order], rtol=1e-12, atol=0)
        np.testing.assert_allclose(k[ids[i]], keys[i], rtol=1e-12, atol=0)
        kc = oracle.adc_keys(Q[i], ids[i], assign, C, codes, cb)
        np.testing.assert_array_equal(kc, keys[i])
