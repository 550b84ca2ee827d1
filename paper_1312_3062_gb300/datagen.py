"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5.1: SIFT,
GIST and HOG features).  The real datasets are not available; these mixtures
stand in for them.

This module holds input generation only (random numbers, shapes, per-query
parameters).  It contains none of the search method's arithmetic and is the
one module that both the CUDA path's tests/benchmark and the CPU oracle's
tests consume.

Workloads (seed = SeedSequence(13123062 + workload number)):
  1 tiny_sift   N=10,000 x 128 uint8, 64-component isotropic Gaussian mixture,
                means U[0,255], sigma 20, rint + clip; 200 queries; R=10;
                P=2 x n=64; T=256, k=10
  2 sift1m      N=1,000,000 x 128 uint8, 1,000 components (as 1); 10,000
                queries; R=20; P=4 x n=256; T in {64,256,1024,4096}, k in {1,10,100}
  3 gist1m      N=1,000,000 x 384 float32, 500-component mixture, means U[0,1],
                sigma 0.15, folded at 0 (abs), L2-normalised; 10,000 queries with
                per-query k in {1,10,100}, T log-uniform in [64, 8192]; R=20; P=3 x 128
  4 hog4m       N=4,000,000 x 512 float32, 2,000 clusters; per cluster and dim a
                scale s ~ LogUniform[0.01, 1]; x ~ Exp(mean s); L2-normalised;
                20,000 queries; R=16; P=4 x 256; T in {256,1024,4096}, k=10
  5 sift10m     N=10,000,000 x 128 uint8 (mixture of 2); R=16; P=4 x 256; requests
                of 1-512 queries, per-query k in {1,10,100}, T in {128,512,2048}
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 13123062
CHUNK = 1_000_000

WORKLOADS = {
    1: dict(name="tiny_sift", N=10_000, d=128, dtype="u8", ncomp=64, sigma=20.0, nq=200,
            R=10, P=2, n=64, t=100, b=5, T=(256,), k=(10,)),
    2: dict(name="sift1m", N=1_000_000, d=128, dtype="u8", ncomp=1000, sigma=20.0, nq=10_000,
            R=20, P=4, n=256, t=100, b=5, T=(64, 256, 1024, 4096), k=(1, 10, 100)),
    3: dict(name="gist1m", N=1_000_000, d=384, dtype="f32", ncomp=500, sigma=0.15, nq=10_000,
            R=20, P=3, n=128, t=100, b=5, T=(64, 8192), k=(1, 10, 100)),
    4: dict(name="hog4m", N=4_000_000, d=512, dtype="f32", ncomp=2000, nq=20_000,
            R=16, P=4, n=256, t=100, b=5, T=(256, 1024, 4096), k=(10,)),
    5: dict(name="sift10m", N=10_000_000, d=128, dtype="u8", ncomp=1000, sigma=20.0, nq=10_000,
            R=16, P=4, n=256, t=100, b=5, T=(128, 512, 2048), k=(1, 10, 100)),
}


def _seq(workload: int, salt: int = 0) -> np.random.SeedSequence:
    return np.random.SeedSequence([SEED_BASE + workload, salt])


def _mixture_params(workload: int, d: int, ncomp: int, kind: str):
    rng = np.random.Generator(np.random.PCG64(_seq(workload, 1)))
    if kind == "u8":
        return rng.uniform(0.0, 255.0, size=(ncomp, d))
    if kind == "gist":
        return rng.uniform(0.0, 1.0, size=(ncomp, d))
    if kind == "hog":
        return np.exp(rng.uniform(np.log(0.01), np.log(1.0), size=(ncomp, d)))
    raise ValueError(kind)


def _draw_rows(workload: int, spec: dict, rows: int, stream: int, start_chunk: int = 0):
    """rows vectors from the workload's mixture; stream 0 = references, 1 = queries."""
    d, ncomp = spec["d"], spec["ncomp"]
    kind = "u8" if spec["dtype"] == "u8" else ("gist" if workload == 3 else "hog")
    params = _mixture_params(workload, d, ncomp, kind)
    out = np.empty((rows, d), np.uint8 if kind == "u8" else np.float32)
    root = _seq(workload, 2 + stream)
    nchunks = (rows + CHUNK - 1) // CHUNK
    children = root.spawn(start_chunk + nchunks)[start_chunk:]
    for c in range(nchunks):
        lo, hi = c * CHUNK, min(rows, (c + 1) * CHUNK)
        rng = np.random.Generator(np.random.PCG64(children[c]))
        comp = rng.integers(0, ncomp, size=hi - lo)
        if kind == "u8":
            x = params[comp] + rng.standard_normal((hi - lo, d)) * spec["sigma"]
            out[lo:hi] = np.clip(np.rint(x), 0, 255).astype(np.uint8)
        elif kind == "gist":
            x = np.abs(params[comp] + rng.standard_normal((hi - lo, d)) * spec["sigma"])
            x /= np.maximum(np.linalg.norm(x, axis=1, keepdims=True), 1e-30)
            out[lo:hi] = x.astype(np.float32)
        else:
            x = rng.standard_exponential((hi - lo, d)) * params[comp]
            x /= np.maximum(np.linalg.norm(x, axis=1, keepdims=True), 1e-30)
            out[lo:hi] = x.astype(np.float32)
    return out


def references(workload: int, N: int | None = None) -> np.ndarray:
    """Reference set X (N rows; default the workload's full size)."""
    spec = WORKLOADS[workload]
    return _draw_rows(workload, spec, spec["N"] if N is None else N, stream=0)


def queries(workload: int, nq: int | None = None) -> np.ndarray:
    """Query set drawn from the same mixture as the references."""
    spec = WORKLOADS[workload]
    return _draw_rows(workload, spec, spec["nq"] if nq is None else nq, stream=1)


def kmeans_init_rows(workload: int, N: int, n: int) -> np.ndarray:
    """n distinct training-row indices (a seeded permutation prefix) for k-means init."""
    rng = np.random.Generator(np.random.PCG64(_seq(workload, 10)))
    return rng.permutation(N)[:n].astype(np.int64)


def training_rows(workload: int, N: int, cap: int = 1_000_000) -> np.ndarray | None:
    """Rows used to train the part dictionaries: all rows when N <= cap, else a
    seeded sample of cap rows (sorted).  None means all rows."""
    if N <= cap:
        return None
    rng = np.random.Generator(np.random.PCG64(_seq(workload, 11)))
    return np.sort(rng.choice(N, size=cap, replace=False)).astype(np.int64)


def coarse_rows(workload: int, N: int, K: int) -> np.ndarray:
    """K distinct data rows (sorted) serving as the coarse centers of the
    Graph-D-ADC stand-in (seeded)."""
    rng = np.random.Generator(np.random.PCG64(_seq(workload, 60)))
    return np.sort(rng.choice(N, size=K, replace=False)).astype(np.int64)


def per_query_params(workload: int, nq: int, seed_salt: int = 20):
    """Per-query (k, T) for the uneven-batch workloads (3: log-uniform T in
    [64, 8192]; 5: k in {1,10,100}, T in {128,512,2048})."""
    spec = WORKLOADS[workload]
    rng = np.random.Generator(np.random.PCG64(_seq(workload, seed_salt)))
    k = rng.choice(np.asarray(spec["k"], np.int32), size=nq).astype(np.int32)
    if workload == 3:
        lo, hi = spec["T"]
        T = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nq))).astype(np.int32)
    else:
        T = rng.choice(np.asarray(spec["T"], np.int32), size=nq).astype(np.int32)
    return k, T


def uneven_budgets(workload: int, nq: int, choices, seed_salt: int = 40) -> np.ndarray:
    """Per-query budgets drawn uniformly from `choices` (an uneven batch)."""
    rng = np.random.Generator(np.random.PCG64(_seq(workload, seed_salt)))
    return rng.choice(np.asarray(choices, np.int32), size=nq).astype(np.int32)


def mixture(seed: int, N: int, d: int, ncomp: int, dtype) -> np.ndarray:
    """Small seeded mixtures for parity cases: uint8 rows as in workload 1
    (means U[0,255], sigma 20, rint + clip), float32 rows as in workload 3
    (means U[0,1], sigma 0.15, folded at 0, L2-normalised)."""
    rng = np.random.default_rng(seed)
    if dtype == np.uint8:
        means = rng.uniform(0, 255, size=(ncomp, d))
        x = means[rng.integers(0, ncomp, N)] + rng.standard_normal((N, d)) * 20.0
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)
    means = rng.uniform(0, 1, size=(ncomp, d))
    x = np.abs(means[rng.integers(0, ncomp, N)] + rng.standard_normal((N, d)) * 0.15)
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def rp_directions(seed: int, rounds: int, levels: int, d: int) -> np.ndarray:
    """Random split directions for the approximate kNN-graph construction:
    int8 entries +-1 (Rademacher), shape (rounds, 2^levels - 1, d), one per
    segment of every level of every round."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, 50, seed])))
    signs = rng.integers(0, 2, size=(rounds, (1 << levels) - 1, d), dtype=np.int8)
    return (2 * signs - 1).astype(np.int8)


def rp_levels(N: int, leaf_max: int) -> int:
    """Smallest number of halvings after which no leaf exceeds leaf_max points."""
    levels = 0
    while -(-N // (1 << levels)) > leaf_max:
        levels += 1
    return levels


def poisson_requests(workload: int, nreq: int, rate_qps: float, seed_salt: int = 30):
    """Poisson arrivals of request batches: (arrival_s, batch_size) arrays;
    batch sizes log-uniform integers in [1, 512]."""
    rng = np.random.Generator(np.random.PCG64(_seq(workload, seed_salt)))
    sizes = np.floor(np.exp(rng.uniform(0.0, np.log(513.0), size=nreq))).astype(np.int32)
    sizes = np.clip(sizes, 1, 512)
    mean_size = float(sizes.mean())
    gaps = rng.exponential(mean_size / rate_qps, size=nreq)
    return np.cumsum(gaps), sizes
