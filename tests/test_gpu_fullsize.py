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
    wi, wk, wst = oracle.search(X, 20, C, bg, Q, 10, T, kmax=10, nthreads=len(sel))
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
    wi, wk, _ = oracle.search(X, 20, C, bg, Q[sel], k[sel], T[sel], kmax=100, nthreads=len(sel))
    np.testing.assert_array_equal(ids[sel], wi)
    fin = np.isfinite(wk)
    got = keys[sel].view(np.float32).astype(np.float64)
    np.testing.assert_allclose(got[fin], wk[fin], rtol=F32_RTOL, atol=0)
    assert np.all(np.isinf(got[~fin]))
