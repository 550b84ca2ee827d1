"""Parity of the GPU approximate neighbourhood graph (random median-split
partitions, leaf brute force, neighbourhood propagation; the construction
Sec. 5.3 uses for its graphs) with the oracle, through the C ABI.

uint8 keys are exact integers, so ids and keys must match bit for bit:
whole graphs at sizes the oracle finishes in seconds (several leaves, ragged
leaf sizes, R up to 32, d from 16 to 512, 0 to 2 propagation steps, leaves
staged whole and leaves streamed through shared memory), and
sampled rows at the full 1M size of the SIFT-shaped workload, which the
oracle evaluates on demand."""
from __future__ import annotations

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


def gpu_graph(ann, X, R, dirs, iters):
    ids, keys = ann.ann_build_knn_graph_approx(torch.from_numpy(X).cuda(), R,
                                               torch.from_numpy(dirs).cuda(), iters)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), keys.cpu().numpy().view(np.uint32)


CASES = [
    # (seed, N, d, ncomp, R, rounds, leaf_max, iters)
    (1, 20000, 128, 60, 20, 2, 400, 1),
    (2, 12345, 64, 40, 16, 3, 300, 2),
    (3, 5003, 128, 30, 10, 1, 1500, 0),
    (4, 97, 16, 4, 5, 2, 13, 2),
    (5, 3001, 512, 20, 12, 2, 380, 1),
    (6, 4096, 32, 16, 32, 2, 512, 1),
    # leaves beyond one CTA's shared memory: streamed through it (d <= 128)
    (7, 9001, 128, 8, 16, 1, 5000, 1),
    (8, 6000, 64, 6, 10, 2, 3000, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[1]}_d{c[2]}_R{c[4]}_it{c[7]}" for c in CASES])
def test_graph_matches_oracle(ann, case):
    seed, N, d, ncomp, R, rounds, leaf_max, iters = case
    X = datagen.mixture(100 + seed, N, d, ncomp, np.uint8)
    levels = datagen.rp_levels(N, leaf_max)
    dirs = datagen.rp_directions(seed, rounds, levels, d)
    gi, gk = gpu_graph(ann, X, R, dirs, iters)
    oi, ok = oracle.knn_graph_approx(X, R, dirs, iters)
    assert np.array_equal(gi, oi)
    assert np.array_equal(gk.astype(np.float64), ok)


@pytest.mark.parametrize("N", [1200, 6007])
def test_one_leaf_is_the_exact_graph(ann, N):
    # 1,200 rows fit in shared memory; 6,007 rows are streamed through it
    X = datagen.mixture(7, N, 128, 10, np.uint8)
    dirs = datagen.rp_directions(7, 1, 0, 128)
    gi, gk = gpu_graph(ann, X, 20, dirs, 1)
    ei, ek = ann.ann_build_knn_graph(torch.from_numpy(X).cuda(), 20)
    assert np.array_equal(gi, ei.cpu().numpy())
    assert np.array_equal(gk, ek.cpu().numpy().view(np.uint32))


def test_deterministic_and_argument_checks(ann):
    X = datagen.mixture(8, 8000, 128, 20, np.uint8)
    dirs = datagen.rp_directions(8, 2, 4, 128)
    a = gpu_graph(ann, X, 16, dirs, 1)
    b = gpu_graph(ann, X, 16, dirs, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    Xd = torch.from_numpy(X).cuda()
    Xw = torch.from_numpy(datagen.mixture(9, 3000, 256, 4, np.uint8)).cuda()
    with pytest.raises(ann.AnnError):  # d > 128 and a leaf of 3,000 rows beyond shared memory
        ann.ann_build_knn_graph_approx(Xw, 16, torch.from_numpy(datagen.rp_directions(8, 1, 0, 256)).cuda(), 0)
    with pytest.raises(ann.AnnError):  # leaves of 7-8 points cannot fill R = 16
        ann.ann_build_knn_graph_approx(Xd, 16, torch.from_numpy(datagen.rp_directions(8, 1, 10, 128)).cuda(), 0)
    with pytest.raises(ann.AnnError):  # float32 data
        ann.ann_build_knn_graph_approx(Xd.float(), 16, torch.from_numpy(dirs).cuda(), 0)


def test_full_size_sampled_rows(ann):
    """SIFT-shaped 1M x 128 uint8, R = 20, 4 partitions into leaves of <= 977
    points, one propagation step: sampled rows bit-exact against the oracle,
    every row valid, and a good part of the exact neighbours found."""
    X = datagen.references(2)
    N, d, R = X.shape[0], X.shape[1], 20
    levels = datagen.rp_levels(N, 1024)
    dirs = datagen.rp_directions(2, 4, levels, d)
    gi, gk = gpu_graph(ann, X, R, dirs, 1)
    rows = np.random.default_rng(5).choice(N, 12, replace=False).astype(np.int64)
    oi, ok = oracle.knn_graph_approx(X, R, dirs, 1, rows=rows)
    assert np.array_equal(gi[rows], oi)
    assert np.array_equal(gk[rows].astype(np.float64), ok)
    # every row: R distinct ids, no self, ascending (key, id)
    assert (gi >= 0).all() and (gi != np.arange(N)[:, None]).all()
    packed = (gk.astype(np.uint64) << np.uint64(32)) | gi.astype(np.uint64)
    assert (packed[:, 1:] > packed[:, :-1]).all()
    ei, _ = ann.ann_build_knn_graph(torch.from_numpy(X).cuda(), R)
    ei = ei.cpu().numpy()
    sample = np.random.default_rng(6).choice(N, 20000, replace=False)
    recall = np.mean([len(np.intersect1d(gi[i], ei[i])) / R for i in sample])
    print(f"graph recall of the approximate rows: {recall:.4f}")
    assert recall >= 0.5, recall
