"""Parity of the GPU Graph-D-ADC kernels (Sec. 5.4: product-quantized
residuals under coarse centers, asymmetric-distance re-ranking) with the
oracle, through the C ABI.

The oracle takes both distances of Sec. 5.4 in fp64; the kernels decide in
float32.  A float32 squared distance over a vector split into m parts of dp
dims is off the real one by at most (dp + m + 8) * 2^-24 * A, with
A = sum_t (|q_t - c_t| + |w_t|)^2 (one rounding per subtraction, product and
addition; the standard bound for sums of dp and m terms, rounded up).  The
tests allow twice that: a GPU code may differ from the oracle's only where
the two codewords' real distances lie within the sum of their bounds, a key
only by its bound, and a returned id only where its real key is within the
bounds of the T-th key (a near-tie at the cut).  Centers and codebooks are
real-valued k-means results, so rounding is exercised."""
from __future__ import annotations

import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1312_3062_gb300 import datagen  # noqa: E402


@pytest.fixture(scope="module")
def ann():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    _build.build()
    from paper_1312_3062_gb300 import ann as mod
    return mod


def quantizer(X, K, m, ks, seed):
    """Coarse centers (k-means), exact assignment, residual codebooks (k-means)."""
    rng = np.random.default_rng(seed)
    Xf = X.astype(np.float32)
    C = oracle.kmeans(Xf, 1, K, 3, rng.choice(len(X), K, replace=False))[0].astype(np.float32)
    assign, _ = oracle.exact_knn(C, Xf, 1)
    assign = assign[:, 0].astype(np.int32)
    R = (Xf - C[assign]).astype(np.float32)
    cb = oracle.kmeans(R, m, ks, 3, rng.choice(len(X), ks, replace=False)).astype(np.float32)
    return C, assign, cb


@functools.lru_cache(maxsize=None)
def rerank_case(K, m=8, ks=256, w=8):
    X = datagen.mixture(22, 20000, 128, 40, np.uint8)
    C, assign, cb = quantizer(X, K, m, ks, 6)
    codes = oracle.pq_encode(X, C, assign, cb)
    offsets, members = oracle.ivf_lists(assign, K)
    Q = datagen.mixture(23, 40, 128, 40, np.uint8).astype(np.float32)
    lists, _ = oracle.exact_knn(C, Q, w)          # nearest lists, ascending
    lists = lists.astype(np.int32)
    lists[::7, 2] = -1                             # absent entries are skipped
    return Q, lists, offsets, members, C, codes, cb, assign


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


U = 2.0 ** -24


def part_bound(a, w, dp, m):
    """Twice the float32 error bound of squared distances: a = q - c (or
    x - c) and w the codeword(s), fp64 arrays over the last axis."""
    A = ((np.abs(a) + np.abs(w)) ** 2).sum(-1)
    return 2.0 * (dp + m + 8) * U * A


@pytest.mark.parametrize("dtype,N,d,K,m,ks", [(np.uint8, 6000, 128, 64, 8, 256), (np.float32, 3001, 64, 40, 16, 64),
                                              (np.uint8, 2500, 32, 16, 1, 200)])
def test_pq_encode_matches_oracle(ann, dtype, N, d, K, m, ks):
    X = datagen.mixture(21, N, d, 30, dtype)
    C, assign, cb = quantizer(X, K, m, ks, 5)
    want = oracle.pq_encode(X, C, assign, cb)
    got = ann.ann_pq_encode(cuda(X), cuda(C), cuda(assign), cuda(cb)).cpu().numpy()
    diff = np.argwhere(got != want)
    dp = d // m
    R = X.astype(np.float64) - C[assign].astype(np.float64)
    for i, j in diff:
        r = R[i, j * dp:(j + 1) * dp]
        wg, wo = cb[j, got[i, j]].astype(np.float64), cb[j, want[i, j]].astype(np.float64)
        dg, do = ((r - wg) ** 2).sum(), ((r - wo) ** 2).sum()
        assert dg <= do + part_bound(r, wg, dp, 1) + part_bound(r, wo, dp, 1), (i, j, dg, do)
    assert len(diff) <= max(3, got.size // 2000)   # near-ties are rare


# K = 10: lists of ~2,000 members, so the merge buffer is flushed many times
@pytest.mark.parametrize("L,T,K", [(300, 10, 100), (10 ** 9, 100, 100), (2500, 1, 100), (20000, 128, 100),
                                   (10 ** 9, 128, 10), (9000, 37, 10)])
def test_adc_rerank_matches_oracle(ann, L, T, K):
    Q, lists, offsets, members, C, codes, cb, assign = rerank_case(K)
    oi, ok, oseen = oracle.adc_rerank(Q, lists, offsets, members, C, codes, cb, L, T)
    gi, gk, gseen = ann.ann_adc_rerank(cuda(Q), cuda(lists), cuda(offsets), cuda(members), cuda(C), cuda(codes),
                                       cuda(cb), L, T)
    assert np.array_equal(gseen.cpu().numpy(), oseen)
    check_rerank(gi.cpu().numpy(), gk.cpu().numpy().astype(np.float64), oi, ok, Q, assign, C, codes, cb)


def check_rerank(gi, gk, oi, ok, Q, assign, C, codes, cb):
    m, ks, dp = cb.shape
    Cd, cbd = C.astype(np.float64), cb.astype(np.float64)

    def bound(q, ids):
        a = q.astype(np.float64)[None, :] - Cd[assign[ids]]
        w = np.concatenate([cbd[j][codes[ids, j]] for j in range(m)], axis=1)
        return part_bound(a, w, dp, m)

    near = 0
    for i in range(len(Q)):
        g, o = gi[i][gi[i] >= 0], oi[i][oi[i] >= 0]
        assert len(g) == len(o)
        assert np.all(gi[i][len(g):] == -1) and np.all(np.isinf(gk[i][len(g):]))
        if len(g) == 0:
            continue
        kg = oracle.adc_keys(Q[i], g, assign, C, codes, cb)   # real keys of the GPU's ids
        tg = bound(Q[i], g)
        assert np.all(np.abs(gk[i][:len(g)] - kg) <= tg)
        assert np.all(np.diff(gk[i][:len(g)]) >= 0)
        if set(g.tolist()) != set(o.tolist()):
            kth, tk = ok[i][len(o) - 1], bound(Q[i], o[-1:])[0]
            for x in set(g.tolist()) ^ set(o.tolist()):
                kx = oracle.adc_keys(Q[i], np.array([x]), assign, C, codes, cb)[0]
                assert abs(kx - kth) <= bound(Q[i], np.array([x]))[0] + tk, (i, x, kx, kth)
            near += 1
    assert near <= max(1, len(Q) // 10)


@pytest.mark.parametrize("m,ks,L,T", [(8, 64, 1500, 100), (16, 32, 10 ** 9, 10)])
def test_graph_d_adc_end_to_end_matches_oracle(ann, m, ks, L, T):
    # the whole Graph-D-ADC query on the GPU: Algorithm 1 over a GPU-built
    # index of the coarse centers (seeded data rows), then re-ranking of the
    # first L members of the w lists it returns, against the oracle's
    # graph_d_adc_search on the same seeded inputs (codes from the oracle)
    X = datagen.mixture(31, 30000, 128, 60, np.uint8)
    rng = np.random.default_rng(32)
    K, w, Tc = 200, 12, 150   # lists of ~150 members: L = 1500 cuts inside the w-th list
    Cc = np.ascontiguousarray(X[np.sort(rng.choice(len(X), K, replace=False))])
    assign = oracle.exact_knn(Cc, X, 1)[0][:, 0].astype(np.int32)
    R = (X.astype(np.float64) - Cc[assign].astype(np.float64)).astype(np.float32)
    cb = oracle.kmeans(R, m, ks, 3, rng.choice(len(X), ks, replace=False)).astype(np.float32)
    codes = oracle.pq_encode(X, Cc, assign, cb)
    offsets, members = oracle.ivf_lists(assign, K)
    pc = oracle.round_centers(oracle.kmeans(Cc, 2, 16, 5, rng.permutation(K)[:16]), np.uint8)
    Gc = oracle.knn_graph(Cc, 10)[0]
    bgc = oracle.bridge_graph(Cc, pc, 100, 5)
    Q = datagen.mixture(33, 64, 128, 60, np.uint8)
    want_lists, _, _ = oracle.search(Cc, Gc, pc, bgc, Q, w, Tc)
    wi, wk, wseen = oracle.graph_d_adc_search(Cc, Gc, pc, bgc, offsets, members, codes, cb, Q, w, Tc, L, T)
    # the coarse index built on the GPU from the same centers
    Gd, _ = ann.ann_build_knn_graph(cuda(Cc), 10)
    ixc = ann.Index.create(cuda(Cc), Gd, cuda(pc), t=100, b=5)
    gi, gk, gseen, glists = ann.graph_d_adc_search(ixc, cuda(Q), w, Tc, cuda(offsets), cuda(members),
                                                   cuda(Cc.astype(np.float32)), cuda(codes), cuda(cb), L, T)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(glists.cpu().numpy(), want_lists)       # the coarse step is bit-exact
    np.testing.assert_array_equal(gseen.cpu().numpy(), wseen)
    check_rerank(gi.cpu().numpy(), gk.cpu().numpy().astype(np.float64), wi, wk, Q.astype(np.float32), assign,
                 Cc.astype(np.float32), codes, cb)
    ixc.free()


def test_adc_argument_checks(ann):
    Q = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    lists = torch.zeros((2, 1), dtype=torch.int32, device="cuda")
    offsets = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    members = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    codes = torch.zeros((1, 4), dtype=torch.uint8, device="cuda")
    cb = torch.zeros((4, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ann.AnnError):  # T above 128
        ann.ann_adc_rerank(Q, lists, offsets, members, C, codes, cb, 10, 129)
    ids, keys, seen = ann.ann_adc_rerank(Q, lists, offsets, members, C, codes, cb, 10, 3)
    assert ids.cpu().tolist() == [[0, -1, -1]] * 2 and seen.cpu().tolist() == [1, 1]
    assert np.isinf(keys.cpu().numpy()[:, 1:]).all()
