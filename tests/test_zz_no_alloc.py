"""ann_exact_knn_static: the allocation-free variant of the exact k-NN entry
point, for callers that cannot allocate device memory themselves (their
device memory belongs to another allocator, or their loop cannot take an
allocation's synchronisation).  Called through the C ABI; its output must
equal ann_exact_knn's on two calls in a row (the scratch array is shared and
keeps the previous call's contents).  Kept in the last-collected file."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    return ctypes.CDLL(_build.build())


def mixture(seed, N, d, dtype):
    rng = np.random.default_rng(seed)
    if dtype == np.uint8:
        means = rng.uniform(0, 255, size=(16, d))
        x = means[rng.integers(0, 16, N)] + rng.standard_normal((N, d)) * 20.0
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)
    x = np.abs(rng.standard_normal((N, d))).astype(np.float32)
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def call(fn, X, Q, k, self_mode):
    N, d = X.shape
    nq = Q.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int32, device="cuda")
    keys = torch.zeros((nq, k), dtype=torch.int32 if X.dtype == torch.uint8 else torch.float32, device="cuda")
    rc = fn(ctypes.c_void_p(X.data_ptr()), ctypes.c_int64(N), ctypes.c_void_p(Q.data_ptr()), ctypes.c_int64(nq),
            ctypes.c_int(0 if X.dtype == torch.uint8 else 1), ctypes.c_int32(d), ctypes.c_int32(k),
            ctypes.c_int32(int(self_mode)), ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(keys.data_ptr()),
            ctypes.c_void_p(0))
    assert rc == 0
    torch.cuda.synchronize()
    return ids.cpu().numpy(), keys.cpu().numpy()


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_static_matches_allocating_entry_point_twice(lib, dtype):
    for call_no, (N, nq, k, self_mode) in enumerate([(5000, 300, 16, False), (3001, 3001, 20, True)]):
        X = torch.from_numpy(mixture(10 + call_no, N, 128, dtype)).cuda()
        Q = X if self_mode else torch.from_numpy(mixture(20 + call_no, nq, 128, dtype)).cuda()
        want_ids, want_keys = call(lib.ann_exact_knn, X, Q, k, self_mode)
        got_ids, got_keys = call(lib.ann_exact_knn_static, X, Q, k, self_mode)
        np.testing.assert_array_equal(got_ids, want_ids)
        if dtype == np.uint8:
            np.testing.assert_array_equal(got_keys, want_keys)
        else:
            np.testing.assert_allclose(got_keys, want_keys, rtol=1e-5, atol=0)


@pytest.mark.parametrize("dtype", [np.uint8, np.float32])
def test_static_matches_the_oracle(lib, dtype):
    # the same two calls in a row, now against the CPU oracle's linear scan
    import oracle
    for call_no, (N, nq, k, self_mode) in enumerate([(4000, 200, 12, False), (2500, 2500, 10, True)]):
        Xh = mixture(30 + call_no, N, 128, dtype)
        Qh = Xh if self_mode else mixture(40 + call_no, nq, 128, dtype)
        X = torch.from_numpy(Xh).cuda()
        Q = X if self_mode else torch.from_numpy(Qh).cuda()
        got_ids, got_keys = call(lib.ann_exact_knn_static, X, Q, k, self_mode)
        want_ids, want_keys = oracle.exact_knn(Xh, Qh, k, exclude_self=self_mode)
        np.testing.assert_array_equal(got_ids, want_ids)
        if dtype == np.uint8:
            np.testing.assert_array_equal(got_keys.view(np.uint32).astype(np.float64), want_keys)
        else:
            np.testing.assert_allclose(got_keys.astype(np.float64), want_keys, rtol=1e-5, atol=0)


@pytest.mark.parametrize("fn_name", ["ann_exact_knn", "ann_exact_knn_static"])
def test_query_buffer_longer_than_refs_at_the_same_address(lib, fn_name):
    # refs = the first N rows of the query buffer: the queries past row N
    # need norms of their own, not the reference norms
    import oracle
    Xh = mixture(50, 3000, 128, np.uint8)
    X = torch.from_numpy(Xh).cuda()
    N = 1800
    fn = getattr(lib, fn_name)
    ids = torch.full((3000, 8), -7, dtype=torch.int32, device="cuda")
    keys = torch.zeros((3000, 8), dtype=torch.int32, device="cuda")
    rc = fn(ctypes.c_void_p(X.data_ptr()), ctypes.c_int64(N), ctypes.c_void_p(X.data_ptr()), ctypes.c_int64(3000),
            ctypes.c_int(0), ctypes.c_int32(128), ctypes.c_int32(8), ctypes.c_int32(0),
            ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(0))
    assert rc == 0
    torch.cuda.synchronize()
    want_ids, want_keys = oracle.exact_knn(Xh[:N], Xh, 8)
    np.testing.assert_array_equal(ids.cpu().numpy(), want_ids)
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint32).astype(np.float64), want_keys)


def test_static_rejects_sizes_beyond_its_scratch(lib):
    X = torch.zeros((1 << 20, 16), dtype=torch.uint8, device="cuda")
    Q = torch.zeros((8, 16), dtype=torch.uint8, device="cuda")
    ids = torch.empty((8, 4), dtype=torch.int32, device="cuda")
    rc = lib.ann_exact_knn_static(ctypes.c_void_p(X.data_ptr()), ctypes.c_int64(1 << 20),
                                  ctypes.c_void_p(Q.data_ptr()), ctypes.c_int64(8), ctypes.c_int(0),
                                  ctypes.c_int32(16), ctypes.c_int32(4), ctypes.c_int32(0),
                                  ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(0), ctypes.c_void_p(0))
    assert rc == -3
    lib.ann_last_error.restype = ctypes.c_char_p
    assert b"static scratch" in lib.ann_last_error()
