"""GPU parity: every CUDA step against the CPU oracle, element by element.

uint8 data: ids and integer keys bit-exact.  float32 data: ids identical and
keys within 1e-5 relative (the float32 key is the float32 nearest to the exact
squared distance on both sides).  All inputs are seeded synthetic data from
paper_1312_3062_gb300.datagen; every expected value comes from oracle/.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1312_3062_gb300 import datagen  # noqa: E402

F32_RTOL = 1e-5


@pytest.fixture(scope="module")
def ann():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    _build.build()
    from paper_1312_3062_gb300 import ann as mod
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


gmm = datagen.mixture


def gpu_keys(t, dtype):
    a = t.cpu().numpy()
    if dtype == np.uint8:
        a = a.view(np.uint32).astype(np.float64)
        a[a == 0xFFFFFFFF] = np.inf
        return a
    return a.astype(np.float64)


def assert_keys(got, want, dtype):
    if dtype == np.uint8:
        np.testing.assert_array_equal(got, want)
    else:
        fin = np.isfinite(want)
        assert np.array_equal(np.isfinite(got), fin)
        np.testing.assert_allclose(got[fin], want[fin], rtol=F32_RTOL, atol=0)


# --------------------------------------------------------------------------
# exact kNN / neighbourhood graph (Sec. 3.1, Sec. 5.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,N,d,R", [(np.uint8, 2500, 128, 20), (np.uint8, 777, 64, 32),
                                         (np.float32, 1500, 96, 16), (np.float32, 333, 384, 10)])
def test_knn_graph_matches_oracle(ann, dtype, N, d, R):
    X = gmm(N + d, N, d, 8, dtype)
    X[5] = X[3]          # exact duplicates: ties broken by id
    X[N - 1] = X[3]
    want_ids, want_keys = oracle.knn_graph(X, R)
    ids, keys = ann.ann_build_knn_graph(dev(X), R)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ids.cpu().numpy(), want_ids)
    assert_keys(gpu_keys(keys, dtype), want_keys, dtype)


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_exact_knn_queries_match_oracle(ann, dtype):
    X = gmm(7, 3001, 128, 16, dtype)
    Q = gmm(8, 130, 128, 16, dtype)
    want_ids, want_keys = oracle.exact_knn(X, Q, 10)
    ids, keys = ann.ann_exact_knn(dev(X), dev(Q), 10)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ids.cpu().numpy(), want_ids)
    assert_keys(gpu_keys(keys, dtype), want_keys, dtype)


def test_knn_pads_when_fewer_rows_than_k(ann):
    X = gmm(9, 5, 16, 2, np.uint8)
    want_ids, _ = oracle.knn_graph(X, 8)
    ids, keys = ann.ann_build_knn_graph(dev(X), 8)
    np.testing.assert_array_equal(ids.cpu().numpy(), want_ids)
    assert np.all(ids.cpu().numpy()[:, 4:] == -1)


# --------------------------------------------------------------------------
# part dictionaries (Sec. 4.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,P,n", [(np.uint8, 2, 16), (np.uint8, 4, 32), (np.float32, 3, 8)])
def test_kmeans_matches_oracle(ann, dtype, P, n):
    X = gmm(11 + P, 3000, 96, 20, dtype)
    init = np.random.default_rng(3).permutation(3000)[:n]
    want = oracle.kmeans(X, P, n, 6, init)
    got, got64 = ann.ann_train_centers(dev(X), P, n, 6, init, want_f64=True)
    torch.cuda.synchronize()
    g64 = got64.cpu().numpy()
    if dtype == np.uint8:
        np.testing.assert_array_equal(g64, want)                          # same fp64 operations
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.round_centers(want, np.uint8))
    else:
        np.testing.assert_allclose(g64, want, rtol=1e-9, atol=1e-12)     # sum order differs


# --------------------------------------------------------------------------
# bridge graph (Sec. 4.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,N,d,P,n,t,b", [(np.uint8, 2000, 128, 2, 16, 100, 5),
                                               (np.uint8, 1500, 128, 4, 8, 100, 5),
                                               (np.uint8, 1200, 96, 3, 16, 30, 3),
                                               (np.float32, 900, 64, 4, 6, 50, 4),
                                               (np.float32, 1000, 96, 3, 10, 100, 5)])
def test_bridge_graph_matches_oracle(ann, dtype, N, d, P, n, t, b):
    X = gmm(100 + N, N, d, 12, dtype)
    init = np.random.default_rng(4).permutation(N)[:n]
    C = oracle.round_centers(oracle.kmeans(X, P, n, 3, init), dtype)
    want = oracle.bridge_graph(X, C, t, b)
    G, _ = oracle.knn_graph(X, 4)
    ix = ann.Index.create(dev(X), dev(G), dev(C), t=t, b=b)
    ids, refs = ix.bridges()
    np.testing.assert_array_equal(ids, want["bridges"])
    for j in range(len(ids)):
        lo, hi = want["offsets"][j], want["offsets"][j + 1]
        row = refs[j]
        np.testing.assert_array_equal(row[:hi - lo], want["refs"][lo:hi])
        assert np.all(row[hi - lo:] == -1)
    info = ix.info()
    assert info["bridged_refs"] == len(np.unique(want["refs"]))
    assert info["alpha"] == pytest.approx(info["bridged_refs"] / n ** P)


# --------------------------------------------------------------------------
# Algorithm 1 (Sec. 4.2)
# --------------------------------------------------------------------------

def build_oracle_index(X, P, n, R, t, b, iters, seed):
    G, _ = oracle.knn_graph(X, R)
    init = np.random.default_rng(seed).permutation(len(X))[:n]
    C = oracle.round_centers(oracle.kmeans(X, P, n, iters, init), X.dtype)
    bg = oracle.bridge_graph(X, C, t, b)
    return G, C, bg


def run_both(ann, X, G, C, bg, Q, k, T, kmax, mode, b=5):
    want_ids, want_keys, want_st = oracle.search(X, G, C, bg, Q, k, T, kmax=kmax, nthreads=8)
    ix = ann.Index.create(dev(X), dev(G), dev(C), b=b, bridges=bg)
    karg = dev(np.asarray(k, np.int32)) if np.ndim(k) else int(k)
    Targ = dev(np.asarray(T, np.int32)) if np.ndim(T) else int(T)
    stats = torch.zeros((len(Q), ann.ANN_NSTATS), dtype=torch.int64, device="cuda")
    ids, keys, status = ann.ann_search_batch(ix, dev(Q), karg, Targ, kmax=kmax, mode=mode, out_stats=stats)
    torch.cuda.synchronize()
    return (want_ids, want_keys, want_st), (ids.cpu().numpy(), gpu_keys(keys, X.dtype), status.cpu().numpy(),
                                           stats.cpu().numpy()), ix


@pytest.fixture(scope="module")
def tiny_sift():
    """Workload 1 at full size: N=10,000 x 128 uint8, R=10, P=2 x 64, 200 queries."""
    X = datagen.references(1)
    Q = datagen.queries(1)
    G, _ = oracle.knn_graph(X, 10)
    init = datagen.kmeans_init_rows(1, len(X), 64)
    C = oracle.round_centers(oracle.kmeans(X, 2, 64, 10, init), np.uint8)
    bg = oracle.bridge_graph(X, C, 100, 5)
    return X, Q, G, C, bg


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_sift_bit_exact(ann, tiny_sift, mode):
    X, Q, G, C, bg = tiny_sift
    (wi, wk, wst), (gi, gk, gs, gst), _ = run_both(ann, X, G, C, bg, Q, 10, 256, 10, mode)
    assert np.all(gs == 0)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gk, wk)
    np.testing.assert_array_equal(gst[:, 0], wst["discovered"])
    np.testing.assert_array_equal(gst[:, 1], wst["ref_pops"])
    np.testing.assert_array_equal(gst[:, 2], wst["nonempty_bridge_pops"])


@pytest.mark.parametrize("dtype,P,n,R,d", [(np.uint8, 4, 16, 12, 128), (np.uint8, 3, 24, 16, 96),
                                           (np.float32, 3, 16, 12, 96), (np.float32, 4, 8, 10, 64),
                                           (np.float32, 2, 32, 8, 128)])
def test_search_mixed_budgets_matches_oracle(ann, dtype, P, n, R, d):
    N = 3000
    X = gmm(200 + P * n, N, d, 24, dtype)
    G, C, bg = build_oracle_index(X, P, n, R, 100, 5, 4, 5)
    Q = gmm(300 + P, 97, d, 24, dtype)
    rng = np.random.default_rng(6)
    k = rng.choice([1, 5, 10, 37], size=len(Q)).astype(np.int32)
    T = rng.choice([0, 1, 3, 20, 64, 200, 777, 2500], size=len(Q)).astype(np.int32)
    for mode in (0, 1):
        (wi, wk, wst), (gi, gk, gs, gst), _ = run_both(ann, X, G, C, bg, Q, k, T, 40, mode)
        assert np.all(gs == 0)
        np.testing.assert_array_equal(gi, wi)
        assert_keys(gk, wk, dtype)
        np.testing.assert_array_equal(gst[:, 0], wst["discovered"])
    if P == 4:
        # the c2 group level exists exactly when the bridges average >= 32 per
        # prefix node (c0, c1); the n = 8 case has it, so its walks ran over it
        ix = ann.Index.create(dev(X), dev(G), dev(C), t=100, b=5, bridges=bg)
        info = ix.info()
        assert (info["groups"] > 0) == (info["M"] >= 32 * n * n)
        if n == 8:
            assert info["groups"] > 0
        ix.free()


def test_search_edge_cases(ann, tiny_sift):
    X, Q, G, C, bg = tiny_sift
    Qs = Q[:40]
    # k = 0, T = 0, T < k, T >= N (whole reachable set), kmax padding
    k = np.array([0, 10, 10, 1, 10, 128] * 6 + [3, 3, 3, 3], np.int32)
    T = np.array([50, 0, 4, 1, 8192, 300] * 6 + [2, 7, 9, 11], np.int32)
    (wi, wk, wst), (gi, gk, gs, gst), _ = run_both(ann, X, G, C, bg, Qs, k, T, 128, 0)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gk, wk)
    assert np.all(gst[:, 0] <= T)
    assert np.all(gst[:, 6] <= T + 1)                                     # queue bound
    # empty batch
    ix = ann.Index.create(dev(X), dev(G), dev(C), bridges=bg)
    ids, keys, st = ann.ann_search_batch(ix, dev(Q[:0]), 10, 64, kmax=10)
    assert ids.shape == (0, 10)


def test_search_without_bridges_discovers_nothing(ann):
    X = gmm(400, 500, 64, 4, np.uint8)
    G, _ = oracle.knn_graph(X, 8)
    C = oracle.round_centers(oracle.kmeans(X, 2, 8, 2, np.arange(8)), np.uint8)
    bg = {"bridges": np.zeros(0, np.uint64), "offsets": np.zeros(1, np.int64), "refs": np.zeros(0, np.int32)}
    Q = gmm(401, 9, 64, 4, np.uint8)
    (wi, wk, _), (gi, gk, gs, gst), _ = run_both(ann, X, G, C, bg, Q, 5, 100, 5, 0)
    np.testing.assert_array_equal(gi, wi)
    assert np.all(gi == -1) and np.all(gst[:, 0] == 0)


def test_many_equal_bridge_keys_split_batches(ann):
    # constant data: every bridge key ties, so batches must split by ranks
    N = 600
    X = np.full((N, 32), 7, np.uint8)
    X[:, :4] = np.random.default_rng(1).integers(0, 3, size=(N, 4))
    G, C, bg = build_oracle_index(X, 4, 4, 6, 256, 8, 2, 7)
    Q = X[:20].copy()
    (wi, wk, _), (gi, gk, gs, _), _ = run_both(ann, X, G, C, bg, Q, 10, 400, 10, 0, b=8)
    assert np.all(gs == 0)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_array_equal(gk, wk)


def test_gpu_built_index_end_to_end(ann, tiny_sift):
    # every index step on the GPU, then the search; each step equals the oracle's
    X, Q, G, C, bg = tiny_sift
    Xd = dev(X)
    Gd, _ = ann.ann_build_knn_graph(Xd, 10)
    init = datagen.kmeans_init_rows(1, len(X), 64)
    Cd = ann.ann_train_centers(Xd, 2, 64, 10, init)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Gd.cpu().numpy(), G)
    np.testing.assert_array_equal(Cd.cpu().numpy(), C)
    ix = ann.Index.create(Xd, Gd, Cd, t=100, b=5)
    ids, _ = ix.bridges()
    np.testing.assert_array_equal(ids, bg["bridges"])
    gi, gk, gs = ann.ann_search_batch(ix, dev(Q), 10, 256)
    wi, wk, _ = oracle.search(X, G, C, bg, Q, 10, 256, nthreads=8)
    np.testing.assert_array_equal(gi.cpu().numpy(), wi)


def test_index_save_load_roundtrip(ann, tiny_sift, tmp_path):
    X, Q, G, C, bg = tiny_sift
    ix = ann.Index.create(dev(X), dev(G), dev(C), bridges=bg)
    p = str(tmp_path / "tiny.idx")
    ix.save(p)
    ix2 = ann.Index.load(p)
    a = ann.ann_search_batch(ix, dev(Q), 10, 256)[0].cpu().numpy()
    b = ann.ann_search_batch(ix2, dev(Q), 10, 256)[0].cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert ix2.info()["M"] == len(bg["bridges"])


def test_persistent_autotuned_plans_equal_oracle(ann, tiny_sift):
    # three budget buckets in one batch: the first persistent call measures
    # launch shapes per bucket on the batch itself; a second plan (new output
    # buffers) reuses the measured shapes; plain and both persistent plans
    # equal the oracle
    X, Q, G, C, bg = tiny_sift
    rng = np.random.default_rng(17)
    T = rng.choice(np.array([100, 200, 400], np.int32), size=len(Q)).astype(np.int32)
    wi, wk, _ = oracle.search(X, G, C, bg, Q, 10, T, kmax=10, nthreads=8)
    ix = ann.Index.create(dev(X), dev(G), dev(C), t=100, b=5, bridges=bg)
    Qd, Td = dev(Q), dev(T)
    for mode in (0, 1, 1):
        ids, keys, st = ann.ann_search_batch(ix, Qd, 10, Td, kmax=10, mode=mode)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        np.testing.assert_array_equal(ids.cpu().numpy(), wi)
        assert_keys(gpu_keys(keys, np.uint8), wk, np.uint8)
    ix.free()


@pytest.mark.parametrize("N,d,R", [(12000, 384, 20), (9000, 512, 16)])
def test_f32_tensor_knn_graph_sampled_rows(ann, N, d, R):
    # large enough for the tensor-core candidate path (N >= 8192); exact keys
    X = gmm(500 + d, N, d, 16, np.float32)
    G, K = ann.ann_build_knn_graph(dev(X), R)
    G, K = G.cpu().numpy(), K.cpu().numpy()
    rows = np.random.default_rng(d).choice(N, 64, replace=False)
    ids, keys = oracle.exact_knn(X, X[rows], R + 1)
    for i, r in enumerate(rows):
        keep = ids[i] != r
        np.testing.assert_array_equal(G[r], ids[i][keep][:R])
        np.testing.assert_allclose(K[r].astype(np.float64), keys[i][keep][:R], rtol=F32_RTOL, atol=0)


def test_f32_tensor_knn_rows_with_many_ties_fall_back_exactly(ann):
    # 700 copies of one row: its copies' candidate lists overflow and those
    # rows are recomputed exactly; every row still equals the oracle
    X = gmm(900, 10000, 64, 8, np.float32)
    X[1000:1700] = X[1000]
    Q = np.ascontiguousarray(X[::20])
    ids, keys = ann.ann_exact_knn(dev(X), dev(Q), 20)
    want_ids, want_keys = oracle.exact_knn(X, Q, 20)
    np.testing.assert_array_equal(ids.cpu().numpy(), want_ids)
    np.testing.assert_allclose(keys.cpu().numpy().astype(np.float64), want_keys, rtol=F32_RTOL, atol=0)


def test_persistent_plans_beyond_the_cache_limit_stay_correct(ann, tiny_sift):
    # every call with fresh output buffers is a new plan; past the cache limit
    # the least recently used plans are evicted and results do not change
    X, Q, G, C, bg = tiny_sift
    ix = ann.Index.create(dev(X), dev(G), dev(C), t=100, b=5, bridges=bg)
    Qd = dev(Q)
    want, _, _ = ann.ann_search_batch(ix, Qd, 10, 256, kmax=10, mode=0)
    want = want.cpu().numpy()
    for _ in range(40):
        ids, _, st = ann.ann_search_batch(ix, Qd, 10, 256, kmax=10, mode=1)
        np.testing.assert_array_equal(ids.cpu().numpy(), want)
        assert np.all(st.cpu().numpy() == 0)
    ix.free()


@pytest.mark.parametrize("dtype,P,n,R,d", [(np.uint8, 4, 16, 16, 128), (np.float32, 3, 16, 12, 96)])
def test_large_budgets_spill_queue_and_visited_set(ann, dtype, P, n, R, d):
    # budgets from 1024 on keep only 512 queue entries in shared memory, the
    # rest of the queue and the visited set in global scratch; budgets up to
    # the whole reachable set make the heap move entries out and take them
    # back many times per query
    N = 20000
    X = gmm(500 + P, N, d, 12, dtype)
    G, C, bg = build_oracle_index(X, P, n, R, 100, 5, 4, 5)
    Q = gmm(501 + P, 48, d, 12, dtype)
    rng = np.random.default_rng(7)
    k = rng.choice([1, 10, 100], size=len(Q)).astype(np.int32)
    T = rng.choice([1024, 1500, 3000, 6000, 8192], size=len(Q)).astype(np.int32)
    for mode in (0, 1):
        (wi, wk, wst), (gi, gk, gs, gst), _ = run_both(ann, X, G, C, bg, Q, k, T, 100, mode)
        assert np.all(gs == 0)
        np.testing.assert_array_equal(gi, wi)
        assert_keys(gk, wk, dtype)
        np.testing.assert_array_equal(gst[:, 0], wst["discovered"])
        np.testing.assert_array_equal(gst[:, 1], wst["ref_pops"])
        assert gst[:, 6].max() > 600          # queues longer than the shared-memory heap


@pytest.mark.parametrize("mode", [0, 1])
def test_invalid_per_query_parameters_fail_alone(ann, tiny_sift, mode):
    # a per-query k above kmax or below 0, or a budget below 0 or above the
    # largest one, fails that query alone (ANN_ERR_ARG, all padding); every
    # other query of the batch equals the oracle bit for bit
    X, Q, G, C, bg = tiny_sift
    Qs = Q[:48]
    k = np.full(len(Qs), 10, np.int32)
    T = np.full(len(Qs), 300, np.int32)
    k[3], T[17], T[30], k[41] = 11, -1, 9000, -2
    bad = np.zeros(len(Qs), bool)
    bad[[3, 17, 30, 41]] = True
    ix = ann.Index.create(dev(X), dev(G), dev(C), b=5, bridges=bg)
    ids, keys, st = ann.ann_search_batch(ix, dev(Qs), dev(k), dev(T), kmax=10, mode=mode)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    ids, keys = ids.cpu().numpy(), gpu_keys(keys, X.dtype)
    np.testing.assert_array_equal(st, np.where(bad, ann.ANN_ERR_ARG, ann.ANN_OK))
    assert np.all(ids[bad] == -1) and np.all(np.isinf(keys[bad]))
    wi, wk, _ = oracle.search(X, G, C, bg, Qs[~bad], 10, 300, kmax=10, nthreads=8)
    np.testing.assert_array_equal(ids[~bad], wi)
    np.testing.assert_array_equal(keys[~bad], wk)
    ix.free()
