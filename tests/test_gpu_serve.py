"""Serving: each request's results equal the batch search of the same queries,
alone and when many requests overlap on the GPU (continuous batching).
Admission errors are checked on the host path."""
from __future__ import annotations

import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1312_3062_gb300 import datagen  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    _build.build()
    from paper_1312_3062_gb300 import ann
    X = datagen.references(2, 20000)
    Q = datagen.queries(2, 600)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    Xd = dev(X)
    G, _ = ann.ann_build_knn_graph(Xd, 16)
    C = ann.ann_train_centers(Xd, 4, 16, 4, datagen.kmeans_init_rows(2, len(X), 16))
    ix = ann.Index.create(Xd, G, C, t=100, b=5)
    rng = np.random.default_rng(5)
    k = rng.choice([1, 10, 100], size=len(Q)).astype(np.int32)
    T = rng.choice([128, 512, 2048], size=len(Q)).astype(np.int32)
    ids, keys, st = ann.ann_search_batch(ix, dev(Q), dev(k), dev(T), kmax=100)
    torch.cuda.synchronize()
    return ann, ix, X, Q, k, T, ids.cpu().numpy(), keys.cpu().numpy(), G, C


def serve(ann, ix, Q, k, T, chunks, scratch=64 << 20, streams=3, stagger=0.0):
    srv = ctypes.c_void_p()
    ann.check(ann.lib.ann_server_create(ix.handle, scratch, streams, ctypes.byref(srv)))
    tickets = []
    for lo, hi in chunks:
        q = np.ascontiguousarray(Q[lo:hi])
        kk = np.ascontiguousarray(k[lo:hi])
        TT = np.ascontiguousarray(T[lo:hi])
        tk = ctypes.c_uint64()
        ann.check(ann.lib.ann_serve_submit(srv, q.ctypes.data, hi - lo, kk.ctypes.data, TT.ctypes.data,
                                           ctypes.byref(tk)))
        tickets.append((tk.value, lo, hi, int(kk.max())))
        if stagger:
            time.sleep(stagger)
    out = {}
    deadline = time.time() + 120
    while len(out) < len(tickets) and time.time() < deadline:
        for tk, lo, hi, km in tickets:
            if tk in out:
                continue
            ids = np.empty((hi - lo, km), np.int32)
            keys = np.empty((hi - lo, km), np.int32)
            st = np.empty(hi - lo, np.int32)
            rc = ann.lib.ann_serve_poll(srv, tk, ids.ctypes.data, keys.ctypes.data, st.ctypes.data)
            if rc == ann.ANN_OK:
                out[tk] = (lo, hi, km, ids, keys, st)
                assert ann.lib.ann_serve_latency(srv, tk) > 0
            else:
                assert rc == ann.ANN_PENDING
        time.sleep(0.001)
    ann.lib.ann_server_destroy(srv)
    assert len(out) == len(tickets), "server did not finish every request"
    return list(out.values())


def check(results, ids_ref, keys_ref):
    for lo, hi, km, ids, keys, st in results:
        assert np.all(st == 0)
        np.testing.assert_array_equal(ids, ids_ref[lo:hi, :km])
        np.testing.assert_array_equal(keys, keys_ref[lo:hi, :km])


def test_served_alone_equals_batch(setup):
    ann, ix, X, Q, k, T, ids_ref, keys_ref, *_ = setup
    res = serve(ann, ix, Q, k, T, [(0, 37)])
    check(res, ids_ref, keys_ref)


def test_served_mix_equals_batch(setup):
    ann, ix, X, Q, k, T, ids_ref, keys_ref, *_ = setup
    rng = np.random.default_rng(9)
    cuts = np.unique(np.concatenate([[0, len(Q)], rng.integers(1, len(Q), 40)]))
    chunks = list(zip(cuts[:-1], cuts[1:]))
    res = serve(ann, ix, Q, k, T, chunks, stagger=0.0005)
    check(res, ids_ref, keys_ref)


def test_served_under_memory_pressure(setup):
    # a pool that holds only one batch at a time: requests wait for memory, all complete
    ann, ix, X, Q, k, T, ids_ref, keys_ref, *_ = setup
    chunks = [(i, i + 50) for i in range(0, 600, 50)]
    res = serve(ann, ix, Q, k, T, chunks, scratch=300 * 1024, streams=4)
    check(res, ids_ref, keys_ref)


def test_request_larger_than_pool_is_refused(setup):
    ann, ix, X, Q, k, T, *_ = setup
    srv = ctypes.c_void_p()
    ann.check(ann.lib.ann_server_create(ix.handle, 64 * 1024, 1, ctypes.byref(srv)))
    q = np.ascontiguousarray(Q[:400])
    kk = np.full(400, 100, np.int32)
    TT = np.full(400, 512, np.int32)
    tk = ctypes.c_uint64()
    rc = ann.lib.ann_serve_submit(srv, q.ctypes.data, 400, kk.ctypes.data, TT.ctypes.data, ctypes.byref(tk))
    assert rc == ann.ANN_ERR_OOM
    assert ann.lib.ann_serve_poll(srv, 12345, q.ctypes.data, None, None) == ann.ANN_ERR_ARG
    ann.lib.ann_server_destroy(srv)


def test_batch_matches_oracle(setup):
    # the oracle builds every index part itself from the same data and the
    # same k-means initial rows; the GPU-built index must equal it
    ann, ix, X, Q, k, T, ids_ref, keys_ref, G, C = setup
    Go, _ = oracle.knn_graph(X, 16)
    np.testing.assert_array_equal(G.cpu().numpy(), Go)
    Co = oracle.round_centers(oracle.kmeans(X, 4, 16, 4, datagen.kmeans_init_rows(2, len(X), 16)), np.uint8)
    np.testing.assert_array_equal(C.cpu().numpy(), Co)
    bg = oracle.bridge_graph(X, Co, 100, 5)
    ids, refs = ix.bridges()
    np.testing.assert_array_equal(ids, bg["bridges"])
    np.testing.assert_array_equal(refs[refs >= 0], bg["refs"])
    sel = np.arange(0, 600, 15)
    wi, wk, _ = oracle.search(X, Go, Co, bg, Q[sel], k[sel], T[sel], kmax=100, nthreads=8)
    np.testing.assert_array_equal(ids_ref[sel], wi)
    np.testing.assert_array_equal(keys_ref[sel].view(np.uint32).astype(np.float64),
                                  np.where(np.isinf(wk), 4294967295.0, wk))


def test_native_replay_collects_every_request(setup):
    # the load driver submits at the given arrival times and collects every
    # ticket; the server then holds no live request and every latency is set
    ann, ix, X, Q, k, T, ids_ref, keys_ref, *_ = setup
    srv = ctypes.c_void_p()
    ann.check(ann.lib.ann_server_create(ix.handle, 64 << 20, 3, ctypes.byref(srv)))
    rng = np.random.default_rng(11)
    n = 60
    sizes = rng.integers(1, 40, n).astype(np.int32)
    first = rng.integers(0, len(Q) - 40, n).astype(np.int64)
    arrivals = np.cumsum(rng.exponential(0.0005, n)).astype(np.float64)
    lat = np.zeros(n, np.float64)
    el = ctypes.c_double()
    q = np.ascontiguousarray(Q)
    ann.check(ann.lib.ann_serve_replay(srv, q.ctypes.data, k.ctypes.data, T.ctypes.data, n, first.ctypes.data,
                                       sizes.ctypes.data, arrivals.ctypes.data, lat.ctypes.data, ctypes.byref(el)))
    assert np.all(lat > 0) and el.value > 0
    # a ticket that was collected is gone
    assert ann.lib.ann_serve_poll(srv, 1, np.empty((40, 100), np.int32).ctypes.data, None, None) == ann.ANN_ERR_ARG
    ann.lib.ann_server_destroy(srv)
