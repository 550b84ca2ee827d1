"""Parity at the full size of the SIFT-shaped 1M workload (N = 1,000,000 x 128
uint8, R = 20, P = 4 x n = 256, t = 100, b <= 5), on sampled outputs the
oracle can compute: the whole bridge graph, sampled kNN rows, and the search
of sampled queries (the oracle computes each popped reference's row by
linear scan, so it needs no stored graph).  Every oracle input is the seeded
data; the part dictionaries are the oracle's own k-means on a seeded sample."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1312_3062_gb300 import datagen  # noqa: E402


@pytest.fixture(scope="module")
def sift1m():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    _build.build()
    from paper_1312_3062_gb300 import ann
    spec = datagen.WORKLOADS[2]
    X = datagen.references(2)
    Qall = datagen.queries(2)
    rng = np.random.default_rng(2024)
    train = np.sort(rng.choice(len(X), 20000, replace=False))
    C = oracle.round_centers(oracle.kmeans(X[train], 4, 256, 5, datagen.kmeans_init_rows(2, 20000, 256)), np.uint8)
    Xd = torch.from_numpy(X).cuda()
    G, _ = ann.ann_build_knn_graph(Xd, spec["R"])
    ix = ann.Index.create(Xd, G, torch.from_numpy(C).cuda(), t=100, b=5)
    return ann, X, Qall, C, G.cpu().numpy(), ix


def test_sampled_knn_rows(sift1m):
    ann, X, Qall, C, G, ix = sift1m
    rows = np.random.default_rng(1).choice(len(X), 48, replace=False)
    ids, keys = oracle.exact_knn(X, X[rows], 21)
    for i, r in enumerate(rows):
        want = [v for v in ids[i] if v != r][:20]
        np.testing.assert_array_equal(G[r], want)


def test_full_bridge_graph(sift1m):
    ann, X, Qall, C, G, ix = sift1m
    bg = oracle.bridge_graph(X, C, 100, 5)
    ids, refs = ix.bridges()
    np.testing.assert_array_equal(ids, bg["bridges"])
    lens = (refs >= 0).sum(1)
    np.testing.assert_array_equal(lens, np.diff(bg["offsets"]))
    np.testing.assert_array_equal(refs[refs >= 0], bg["refs"])
    sift1m_bg[0] = bg


sift1m_bg = [None]


@pytest.mark.parametrize("T,sel", [(64, [0, 1234, 5678, 9999, 42, 777, 3141, 2718]),
                                   (512, [11, 2222, 4444, 8888, 6060, 123, 9876, 5000]),
                                   (2048, [31, 7070])])
def test_sampled_search(sift1m, T, sel):
    ann, X, Qall, C, G, ix = sift1m
    bg = sift1m_bg[0] if sift1m_bg[0] is not None else oracle.bridge_graph(X, C, 100, 5)
    sift1m_bg[0] = bg
    Q = np.ascontiguousarray(Qall[sel])
    wi, wk, wst = oracle.search(X, 20, C, bg, Q, 10, T, kmax=10, nthreads=0)
    gi, gk, gs = ann.ann_search_batch(ix, torch.from_numpy(Q).cuda(), 10, T, kmax=10)
    torch.cuda.synchronize()
    assert np.all(gs.cpu().numpy() == 0)
    np.testing.assert_array_equal(gi.cpu().numpy(), wi)
    np.testing.assert_array_equal(gk.cpu().numpy().view(np.uint32).astype(np.float64), wk)


# ---------------------------------------------------------------------------
# GIST-shaped 1M workload: N = 1,000,000 x 384 float32, R = 20, P = 3 x n = 128,
# per-query k in {1, 10, 100} and T log-uniform in [64, 8192], persistent form
# ---------------------------------------------------------------------------

F32_RTOL = 1e-5


@pytest.fixture(scope="module")
def gist1m():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    _build.build()
    from paper_1312_3062_gb300 import ann
    spec = datagen.WORKLOADS[3]
    X = datagen.references(3)
    Q = datagen.queries(3)
    rng = np.random.default_rng(3033)
    train = np.sort(rng.choice(len(X), 20000, replace=False))
    C = oracle.round_centers(oracle.kmeans(X[train], 3, 128, 5, datagen.kmeans_init_rows(3, 20000, 128)),
                             np.float32)
    Xd = torch.from_numpy(X).cuda()
    G, _ = ann.ann_build_knn_graph(Xd, spec["R"])
    ix = ann.Index.create(Xd, G, torch.from_numpy(C).cuda(), t=100, b=5)
    k, T = datagen.per_query_params(3, len(Q))
    ids, keys, st = ann.ann_search_batch(ix, torch.from_numpy(Q).cuda(), torch.from_numpy(k).cuda(),
                                         torch.from_numpy(T).cuda(), kmax=100, mode=1)
    torch.cuda.synchronize()
    return ann, X, Q, C, G.cpu().numpy(), ix, k, T, ids.cpu().numpy(), keys.cpu().numpy(), st.cpu().numpy()


def test_gist1m_sampled_knn_rows(gist1m):
    ann, X, Q, C, G, ix, *_ = gist1m
    rows = np.random.default_rng(3).choice(len(X), 32, replace=False)
    ids, keys = oracle.exact_knn(X, X[rows], 21)
    for i, r in enumerate(rows):
        keep = ids[i] != r
        np.testing.assert_array_equal(G[r], ids[i][keep][:20])


gist1m_bg = [None]


def test_gist1m_full_bridge_graph(gist1m):
    ann, X, Q, C, G, ix, *_ = gist1m
    bg = oracle.bridge_graph(X, C, 100, 5)
    ids, refs = ix.bridges()
    np.testing.assert_array_equal(ids, bg["bridges"])
    np.testing.assert_array_equal(refs[refs >= 0], bg["refs"])
    gist1m_bg[0] = bg


def test_gist1m_sampled_uneven_search(gist1m):
    # the whole 10,000-query uneven batch ran in the persistent form; sampled
    # queries with budgets the oracle finishes quickly are checked one by one
    ann, X, Q, C, G, ix, k, T, ids, keys, st = gist1m
    assert np.all(st == 0)
    bg = gist1m_bg[0] if gist1m_bg[0] is not None else oracle.bridge_graph(X, C, 100, 5)
    small = np.where(T <= 256)[0]
    sel = np.random.default_rng(33).choice(small, 8, replace=False)
    wi, wk, _ = oracle.search(X, 20, C, bg, Q[sel], k[sel], T[sel], kmax=100, nthreads=0)
    np.testing.assert_array_equal(ids[sel], wi)
    fin = np.isfinite(wk)
    got = keys[sel].view(np.float32).astype(np.float64)
    np.testing.assert_allclose(got[fin], wk[fin], rtol=F32_RTOL, atol=0)
    assert np.all(np.isinf(got[~fin]))


def test_gist1m_sampled_large_budget_search(gist1m):
    # queries of the same batch with budgets in the storm regime (T >= 4096,
    # where the component is exhausted and hundreds of bridges are popped)
    # and in between (1024 <= T < 4096)
    ann, X, Q, C, G, ix, k, T, ids, keys, st = gist1m
    bg = gist1m_bg[0] if gist1m_bg[0] is not None else oracle.bridge_graph(X, C, 100, 5)
    rng = np.random.default_rng(34)
    sel = np.sort(np.concatenate([rng.choice(np.flatnonzero(T >= 4096), 6, replace=False),
                                  rng.choice(np.flatnonzero((T >= 1024) & (T < 4096)), 2, replace=False)]))
    wi, wk, wst = oracle.search(X, 20, C, bg, Q[sel], k[sel], T[sel], kmax=100, nthreads=0)
    assert (wst["bridge_pops"] > 100).sum() >= 4     # the storm regime is exercised
    np.testing.assert_array_equal(ids[sel], wi)
    fin = np.isfinite(wk)
    got = keys[sel].view(np.float32).astype(np.float64)
    np.testing.assert_allclose(got[fin], wk[fin], rtol=F32_RTOL, atol=0)


# ---------------------------------------------------------------------------
# The largest indexes: SIFT-shaped 10M uint8 (R = 16) and HOG-shaped 4M
# float32 (R = 16, 330M non-empty bridges).  Their full bridge graphs are too
# large for the oracle's global sort, so the oracle computes the lists of
# selected bridge ids (every reference's top-t scan, no sort) and the index
# is read back for the same ids.
# ---------------------------------------------------------------------------

def _big_index(workload, R, seed):
    from paper_1312_3062_gb300 import _build
    _build.build()
    from paper_1312_3062_gb300 import ann
    spec = datagen.WORKLOADS[workload]
    X = datagen.references(workload)
    rng = np.random.default_rng(seed)
    train = np.sort(rng.choice(len(X), 20000, replace=False))
    dt = np.uint8 if X.dtype == np.uint8 else np.float32
    C = oracle.round_centers(oracle.kmeans(X[train], spec["P"], spec["n"], 5,
                                           datagen.kmeans_init_rows(workload, 20000, spec["n"])), dt)
    Xd = torch.from_numpy(X).cuda()
    G, _ = ann.ann_build_knn_graph(Xd, R)
    ix = ann.Index.create(Xd, G, torch.from_numpy(C).cuda(), t=100, b=5)
    torch.cuda.synchronize()
    return ann, X, C, G, ix


def _selected_bridges(X, C, rng, n_random=400, n_refs=40):
    """Random bridge ids plus the first bridges of random references (these
    are chosen by a reference, hence non-empty)."""
    P, n, dp = C.shape
    ids = set(int(v) for v in rng.integers(0, n ** P, n_random, dtype=np.uint64))
    for r in rng.choice(len(X), n_refs, replace=False):
        x = X[r].astype(np.float64).reshape(P, dp)
        part = ((C.astype(np.float64) - x[:, None, :]) ** 2).sum(-1)
        _, bid, _, _ = oracle.multiseq(part, X.dtype, 3)
        ids.update(int(v) for v in bid)
    return np.array(sorted(ids), np.uint64)


def _check_big(ann, X, C, G, ix, R, seed):
    rng = np.random.default_rng(seed)
    rows = rng.choice(len(X), 16, replace=False)
    ids, _ = oracle.exact_knn(X, X[rows], R + 1)
    Gs = G[torch.from_numpy(rows).cuda()].cpu().numpy()
    for i, r in enumerate(rows):
        np.testing.assert_array_equal(Gs[i], ids[i][ids[i] != r][:R])
    sel = _selected_bridges(X, C, rng)
    counts, refs, _ = oracle.bridge_lists(X, C, 100, 5, sel)
    got = ix.lookup_bridges(sel)
    np.testing.assert_array_equal(got, refs)
    assert counts.max() > 0 and counts.min() == 0   # both present and absent ids were checked


def oracle_search_big(X, R, C, Q, k, T, kmax, limits):
    """Algorithm 1 for sampled queries of an index whose whole bridge graph is
    too large for the oracle: bridge lists restricted to the bridges each
    query can reach below a key limit (complete lists, computed from every
    reference), kNN rows computed on demand by linear scan.  A query that
    would pop a bridge above its limit is reported by the oracle and run
    again with the limit doubled."""
    nq = len(Q)
    k = np.broadcast_to(np.asarray(k, np.int32), (nq,))
    T = np.broadcast_to(np.asarray(T, np.int32), (nq,))
    limits = np.asarray(limits, np.float64).copy()
    ids = np.full((nq, kmax), -1, np.int32)
    keys = np.full((nq, kmax), np.inf)
    done = np.zeros(nq, bool)
    for _ in range(10):
        todo = np.flatnonzero(~done)
        bg = oracle.bridge_graph_near(X, C, 100, 5, Q[todo], limits[todo])
        wi, wk, st = oracle.search(X, R, C, bg, Q[todo], k[todo], T[todo], kmax=kmax, nthreads=0,
                                   bridge_key_limit=limits[todo])
        ok = st["over_limit"] == 0
        ids[todo[ok]], keys[todo[ok]] = wi[ok], wk[ok]
        done[todo[ok]] = True
        if done.all():
            return ids, keys
        limits[todo[~ok]] *= 2
    raise AssertionError("bridge key limits did not converge")


def first_limits(X, Q, T):
    """Starting key limits: the key of each query's min(T, 256)-th nearest
    reference (the doubling in oracle_search_big takes care of the rest)."""
    kk = int(min(256, np.max(T)))
    _, kd = oracle.exact_knn(X, Q, kk)
    col = np.minimum(np.broadcast_to(np.asarray(T), (len(Q),)), kk) - 1
    return kd[np.arange(len(Q)), col]


@pytest.fixture(scope="module")
def sift10m():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ann, X, C, G, ix = _big_index(5, 16, 5055)
    yield ann, X, C, G, ix
    ix.free()


@pytest.fixture(scope="module")
def hog4m():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ann, X, C, G, ix = _big_index(4, 16, 4044)
    yield ann, X, C, G, ix
    ix.free()


def test_sift10m_sampled_knn_rows_and_bridge_lists(sift10m):
    ann, X, C, G, ix = sift10m
    _check_big(ann, X, C, G, ix, 16, 55)


def test_sift10m_served_mix_search(sift10m):
    # the served workload's request mix (per query k in {1, 10, 100}, T in
    # {128, 512, 2048}) over all 10,000 queries in the persistent form, and
    # the same queries through the server; 16 sampled queries against the
    # oracle, bit-exact
    ann, X, C, G, ix = sift10m
    Q = datagen.queries(5)
    k, T = datagen.per_query_params(5, len(Q))
    ids, keys, st = ann.ann_search_batch(ix, torch.from_numpy(Q).cuda(), torch.from_numpy(k).cuda(),
                                         torch.from_numpy(T).cuda(), kmax=100, mode=1)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    ids, keys = ids.cpu().numpy(), ann.keys_as_uint32(keys)
    rng = np.random.default_rng(505)
    sel = np.sort(np.concatenate([rng.choice(np.flatnonzero(T == t), c, replace=False)
                                  for t, c in ((128, 5), (512, 5), (2048, 6))]))
    wi, wk = oracle_search_big(X, 16, C, Q[sel], k[sel], T[sel], 100, first_limits(X, Q[sel], T[sel]))
    np.testing.assert_array_equal(ids[sel], wi)
    got = keys[sel].astype(np.float64)
    got[got == 0xFFFFFFFF] = np.inf        # padding: UINT32_MAX on the GPU, +inf in the oracle
    np.testing.assert_array_equal(got, wk)
    # the same sampled queries submitted to the server, one request each
    import ctypes
    import time
    srv = ctypes.c_void_p()
    ann.check(ann.lib.ann_server_create(ix.handle, 64 << 20, 3, ctypes.byref(srv)))
    try:
        tickets = []
        for i in sel:
            q, kk, TT = (np.ascontiguousarray(a[i:i + 1]) for a in (Q, k, T))
            tk = ctypes.c_uint64()
            ann.check(ann.lib.ann_serve_submit(srv, q.ctypes.data, 1, kk.ctypes.data, TT.ctypes.data,
                                               ctypes.byref(tk)))
            tickets.append(tk.value)
        deadline = time.time() + 120
        for j, tk in enumerate(tickets):
            kj = int(k[sel[j]])
            si, sk, ss = np.empty((1, kj), np.int32), np.empty((1, kj), np.int32), np.empty(1, np.int32)
            while ann.lib.ann_serve_poll(srv, tk, si.ctypes.data, sk.ctypes.data, ss.ctypes.data) != ann.ANN_OK:
                assert time.time() < deadline, "server did not finish"
                time.sleep(0.001)
            assert ss[0] == 0
            np.testing.assert_array_equal(si[0], wi[j, :kj])
            sv = sk[0].view(np.uint32).astype(np.float64)
            sv[sv == 0xFFFFFFFF] = np.inf
            np.testing.assert_array_equal(sv, wk[j, :kj])
    finally:
        ann.lib.ann_server_destroy(srv)


def test_hog4m_sampled_knn_rows_and_bridge_lists(hog4m):
    ann, X, C, G, ix = hog4m
    assert ix.info()["groups"] > 0   # dense bridge graph: the c2 group level is built
    _check_big(ann, X, C, G, ix, 16, 44)


def test_hog4m_sampled_search(hog4m):
    # 20,000 queries at T in {256, 1024, 4096}, k = 10; 16 sampled queries
    # (8 / 6 / 2) against the oracle in one pass with per-query budgets:
    # identical ids, keys within 1e-5 relative
    ann, X, C, G, ix = hog4m
    Q = datagen.queries(4)
    rng = np.random.default_rng(404)
    sel_all, T_all, ids_all, keys_all = [], [], [], []
    for T, c in ((256, 8), (1024, 6), (4096, 2)):
        ids, keys, st = ann.ann_search_batch(ix, torch.from_numpy(Q).cuda(), 10, T, kmax=10, mode=1)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        sel = np.sort(rng.choice(len(Q), c, replace=False))
        sel_all.append(sel)
        T_all.append(np.full(c, T, np.int32))
        ids_all.append(ids.cpu().numpy()[sel])
        keys_all.append(keys.cpu().numpy()[sel])
    sel, T, ids, keys = (np.concatenate(v) for v in (sel_all, T_all, ids_all, keys_all))
    wi, wk = oracle_search_big(X, 16, C, Q[sel], 10, T, 10, first_limits(X, Q[sel], T))
    np.testing.assert_array_equal(ids, wi)
    got = keys.astype(np.float64)
    fin = np.isfinite(wk)
    np.testing.assert_allclose(got[fin], wk[fin], rtol=F32_RTOL, atol=0)
