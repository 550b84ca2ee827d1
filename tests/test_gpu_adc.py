"""Parity of the GPU Graph-D-ADC kernels (Sec. 5.4: product-quantized
residuals under coarse centers, asymmetric-distance re-ranking) with the
oracle, through the C ABI.

Codes and keys are decided in float32 in one fixed operation order on both
sides, so codes, ids and keys must match bit for bit.  Centers and codebooks
are real-valued k-means results, so float32 rounding is exercised."""
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
    return Q, lists, offsets, members, C, codes, cb


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dtype,N,d,K,m,ks", [(np.uint8, 6000, 128, 64, 8, 256), (np.float32, 3001, 64, 40, 16, 64),
                                              (np.uint8, 2500, 32, 16, 1, 200)])
def test_pq_encode_matches_oracle(ann, dtype, N, d, K, m, ks):
    X = datagen.mixture(21, N, d, 30, dtype)
    C, assign, cb = quantizer(X, K, m, ks, 5)
    want = oracle.pq_encode(X, C, assign, cb)
    got = ann.ann_pq_encode(cuda(X), cuda(C), cuda(assign), cuda(cb)).cpu().numpy()
    assert np.array_equal(got, want)


# K = 10: lists of ~2,000 members, so the merge buffer is flushed many times
@pytest.mark.parametrize("L,T,K", [(300, 10, 100), (10 ** 9, 100, 100), (2500, 1, 100), (20000, 128, 100),
                                   (10 ** 9, 128, 10), (9000, 37, 10)])
def test_adc_rerank_matches_oracle(ann, L, T, K):
    Q, lists, offsets, members, C, codes, cb = rerank_case(K)
    oi, ok, oseen = oracle.adc_rerank(Q, lists, offsets, members, C, codes, cb, L, T)
    gi, gk, gseen = ann.ann_adc_rerank(cuda(Q), cuda(lists), cuda(offsets), cuda(members), cuda(C), cuda(codes),
                                       cuda(cb), L, T)
    assert np.array_equal(gseen.cpu().numpy(), oseen)
    assert np.array_equal(gi.cpu().numpy(), oi)
    assert np.array_equal(gk.cpu().numpy().astype(np.float64), ok)


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
