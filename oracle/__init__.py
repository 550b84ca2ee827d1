"""CPU oracle for augmented-neighbourhood-graph ANN search (arXiv:1312.3062).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference legs may import this package.
It wraps ``oracle.c`` (plain C, fp64 / exact integers) through ctypes and
shares no code with the CUDA library.

Functions and the passages they follow:
  exact_knn      Sec. 2 (NN definition), Sec. 5.1 (ground truth by linear scan)
  knn_graph      Sec. 3.1 / Sec. 5.3 (R-NN neighbourhood graph), exact
  kmeans         Sec. 3.2 / Sec. 4.1 (PQ dictionaries per part, Lloyd, fp64)
  round_centers  reading of Sec. 4.1 for byte data (centres rounded to bytes)
  multiseq       Sec. 3.3 (multi-sequence algorithm)
  bridge_graph   Sec. 4.1 (top-t bridges per ref, top-b refs per bridge)
  search         Sec. 4.2, Algorithm 1 (ANN search over the augmented graph)
  recall_at_k    Sec. 5.1 (accuracy r/k)
  rp_partition   Sec. 5.3 / 5.5 reading: one random partition of the approximate
                 neighbourhood-graph construction (recursive median splits)
  knn_graph_approx  the same reading: leaf brute force over random partitions,
                 then neighbourhood propagation (rows on demand)
  ivf_lists, pq_encode, adc_rerank, graph_d_adc_search
                 Sec. 5.4 (Graph-D-ADC): inverted lists under coarse centers,
                 product-quantized residuals, lists found by Algorithm 1 over
                 the centers, asymmetric-distance re-ranking
Every function is pinned by the ``-m "not gpu"`` tests in ``tests/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

U8, F32 = 0, 1
STAT_NAMES = ("discovered", "ref_pops", "bridge_pops", "nonempty_bridge_pops", "max_q",
              "max_frontier", "ms_pushes", "over_limit")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=c11", "-shared", "-fPIC", "-ffp-contract=off",
                           "-o", tmp, _SRC, "-lpthread", "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.oracle_exact_knn.argtypes = [P, i64, P, i64, i32, i32, i32, i32, P, P, i32]
            lib.oracle_exact_knn.restype = None
            lib.oracle_kmeans.argtypes = [P, i64, i32, i32, i32, i32, i32, P, P]
            lib.oracle_kmeans.restype = None
            lib.oracle_multiseq.argtypes = [P, i32, i32, i32, i64, P, P, P, P]
            lib.oracle_multiseq.restype = i64
            lib.oracle_bridge_graph.argtypes = [P, i64, i32, i32, i32, i32, P, i32, i32, P, P, P, P, i32]
            lib.oracle_bridge_graph.restype = i64
            lib.oracle_bridge_lists.argtypes = [P, i64, i32, i32, i32, i32, P, i32, i32, P, i64, P, P, P, i32]
            lib.oracle_bridge_lists.restype = None
            lib.oracle_search.argtypes = [P, i64, i32, i32, P, i32, i32, i32, P, i64, P, P, P, P,
                                          i64, P, P, i32, P, P, P, P, i32, P, i32]
            PP = ctypes.POINTER(ctypes.c_void_p)
            lib.oracle_bridge_graph_near.argtypes = [P, i64, i32, i32, i32, i32, P, i32, i32, P, i32, P,
                                                     PP, PP, PP, PP, i32]
            lib.oracle_bridge_graph_near.restype = i64
            lib.oracle_free.argtypes = [P]
            lib.oracle_free.restype = None
            lib.oracle_search.restype = i32
            lib.oracle_num_stats.restype = i32
            lib.oracle_pq_encode.argtypes = [P, i64, i32, P, P, i32, i32, P, P]
            lib.oracle_pq_encode.restype = None
            lib.oracle_adc_rerank.argtypes = [P, i32, P, i32, P, P, P, P, i32, i32, P, i64, i32, P, P]
            lib.oracle_adc_rerank.restype = i64
            lib.oracle_adc_keys.argtypes = [P, i32, P, i64, P, P, P, i32, i32, P, P]
            lib.oracle_adc_keys.restype = None
            lib.oracle_rp_partition.argtypes = [P, i64, i32, P, i32, P]
            lib.oracle_rp_partition.restype = None
            lib.oracle_knn_graph_approx.argtypes = [P, i64, i32, i32, P, i32, i32, i32, P, i64, P, P]
            lib.oracle_knn_graph_approx.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _dtype_code(X: np.ndarray) -> int:
    if X.dtype == np.uint8:
        return U8
    if X.dtype == np.float32:
        return F32
    raise TypeError(f"unsupported dtype {X.dtype}")


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def exact_knn(X: np.ndarray, Qs: np.ndarray, k: int, exclude_self: bool = False, nthreads: int = 0):
    """Linear-scan k-NN by (squared distance, id); pads with -1 / +inf.
    Query rows are independent; nthreads (0 = all cores) only splits them."""
    lib = _load()
    X = np.ascontiguousarray(X)
    Qs = np.ascontiguousarray(Qs)
    assert X.dtype == Qs.dtype and X.shape[1] == Qs.shape[1]
    nq = Qs.shape[0]
    ids = np.empty((nq, k), np.int32)
    keys = np.empty((nq, k), np.float64)
    lib.oracle_exact_knn(_ptr(X), X.shape[0], _ptr(Qs), nq, X.shape[1], _dtype_code(X), k,
                         int(exclude_self), _ptr(ids), _ptr(keys), _threads(nthreads))
    return ids, keys


def knn_graph(X: np.ndarray, R: int, nthreads: int = 0):
    """Exact R-NN graph: each row ascending by (key, id), self excluded."""
    return exact_knn(X, X, R, exclude_self=True, nthreads=nthreads)


def kmeans(X: np.ndarray, P: int, n: int, iters: int, init_rows: np.ndarray) -> np.ndarray:
    """Per-part Lloyd k-means in fp64; returns centres of shape (P, n, d/P) float64."""
    lib = _load()
    X = np.ascontiguousarray(X)
    N, d = X.shape
    assert d % P == 0
    init_rows = np.ascontiguousarray(init_rows, dtype=np.int64)
    assert init_rows.shape == (n,) and len(np.unique(init_rows)) == n
    C = np.empty((P, n, d // P), np.float64)
    lib.oracle_kmeans(_ptr(X), N, d, _dtype_code(X), P, n, iters, _ptr(init_rows), _ptr(C))
    return C


def round_centers(C: np.ndarray, dtype) -> np.ndarray:
    """Store the fp64 centres in the data type: bytes by round-half-even and clip."""
    if np.dtype(dtype) == np.uint8:
        return np.clip(np.rint(C), 0, 255).astype(np.uint8)
    return C.astype(np.float32)


def multiseq(part_keys: np.ndarray, dtype, m: int):
    """First m bridges in multi-sequence order for part keys of shape (P, n).

    Returns (keys, bridge_ids, ranks (m, P), stats {max_frontier, pushes})."""
    lib = _load()
    part_keys = np.ascontiguousarray(part_keys, dtype=np.float64)
    P, n = part_keys.shape
    keys = np.empty(m, np.float64)
    ids = np.empty(m, np.uint64)
    ranks = np.empty((m, P), np.int32)
    st = np.zeros(2, np.int64)
    got = lib.oracle_multiseq(_ptr(part_keys), P, n, U8 if np.dtype(dtype) == np.uint8 else F32,
                              m, _ptr(keys), _ptr(ids), _ptr(ranks), _ptr(st))
    return keys[:got], ids[:got], ranks[:got], {"max_frontier": int(st[0]), "pushes": int(st[1])}


def bridge_graph(X: np.ndarray, centers: np.ndarray, t: int, b: int, nthreads: int = 0):
    """Bridge graph: dict with ascending 'bridges' (uint64), CSR 'offsets', 'refs', 'keys'.
    References are independent in the top-t step; nthreads (0 = all cores) splits them."""
    lib = _load()
    X = np.ascontiguousarray(X)
    centers = np.ascontiguousarray(centers)
    assert centers.dtype == X.dtype
    P, n, dp = centers.shape
    N, d = X.shape
    assert dp * P == d
    cap = N * t
    bridges = np.empty(cap, np.uint64)
    offsets = np.empty(cap + 1, np.int64)
    refs = np.empty(cap, np.int32)
    keys = np.empty(cap, np.float64)
    M = lib.oracle_bridge_graph(_ptr(X), N, d, _dtype_code(X), P, n, _ptr(centers), t, b,
                                _ptr(bridges), _ptr(offsets), _ptr(refs), _ptr(keys), _threads(nthreads))
    nnz = int(offsets[M])
    return {"bridges": bridges[:M].copy(), "offsets": offsets[:M + 1].copy(),
            "refs": refs[:nnz].copy(), "keys": keys[:nnz].copy(), "P": P, "n": n}


def bridge_lists(X: np.ndarray, centers: np.ndarray, t: int, b: int, sel: np.ndarray, nthreads: int = 0):
    """The bridge graph's reference lists of the selected bridge ids only (same
    definition as bridge_graph, without sorting all N*t triples).  sel: strictly
    ascending bridge ids.  Returns (counts (nsel,), refs (nsel, b) -1 padded,
    keys (nsel, b) +inf padded)."""
    lib = _load()
    X = np.ascontiguousarray(X)
    centers = np.ascontiguousarray(centers)
    assert centers.dtype == X.dtype
    sel = np.ascontiguousarray(sel, dtype=np.uint64)
    assert np.all(np.diff(sel.astype(np.float64)) > 0)
    P, n, dp = centers.shape
    N, d = X.shape
    counts = np.empty(len(sel), np.int32)
    refs = np.full((len(sel), b), -1, np.int32)
    keys = np.full((len(sel), b), np.inf, np.float64)
    lib.oracle_bridge_lists(_ptr(X), N, d, _dtype_code(X), P, n, _ptr(centers), t, b, _ptr(sel), len(sel),
                            _ptr(counts), _ptr(refs), _ptr(keys), _threads(nthreads))
    for i, c in enumerate(counts):
        refs[i, c:] = -1
        keys[i, c:] = np.inf
    return counts, refs, keys


def bridge_graph_near(X: np.ndarray, centers: np.ndarray, t: int, b: int, queries: np.ndarray, limits,
                      nthreads: int = 0):
    """The bridge graph restricted to the bridges whose key to at least one of
    the queries is <= that query's limit (a bridge a little above may be kept
    too).  Each kept bridge has its complete list (the b nearest of ALL the
    references that chose it), as in bridge_graph.  Same dict as
    bridge_graph; pass `limits` to search(..., bridge_key_limit=) so that a
    query reaching past its limit is reported instead of searched wrongly."""
    lib = _load()
    X = np.ascontiguousarray(X)
    centers = np.ascontiguousarray(centers)
    queries = np.ascontiguousarray(queries)
    assert centers.dtype == X.dtype == queries.dtype
    P, n, dp = centers.shape
    N, d = X.shape
    lim = np.ascontiguousarray(np.broadcast_to(np.asarray(limits, np.float64), (len(queries),)))
    pb, po, pr, pk = (ctypes.c_void_p() for _ in range(4))
    M = lib.oracle_bridge_graph_near(_ptr(X), N, d, _dtype_code(X), P, n, _ptr(centers), t, b, _ptr(queries),
                                     len(queries), _ptr(lim), ctypes.byref(pb), ctypes.byref(po), ctypes.byref(pr),
                                     ctypes.byref(pk), _threads(nthreads))
    if M < 0:
        raise ValueError("oracle_bridge_graph_near: bad arguments")
    try:
        offsets = np.ctypeslib.as_array(ctypes.cast(po, ctypes.POINTER(ctypes.c_int64)), (M + 1,)).copy()
        nnz = int(offsets[M])
        bridges = (np.ctypeslib.as_array(ctypes.cast(pb, ctypes.POINTER(ctypes.c_uint64)), (M,)).copy()
                   if M else np.zeros(0, np.uint64))
        refs = (np.ctypeslib.as_array(ctypes.cast(pr, ctypes.POINTER(ctypes.c_int32)), (nnz,)).copy()
                if nnz else np.zeros(0, np.int32))
        keys = (np.ctypeslib.as_array(ctypes.cast(pk, ctypes.POINTER(ctypes.c_double)), (nnz,)).copy()
                if nnz else np.zeros(0, np.float64))
    finally:
        for p_ in (pb, po, pr, pk):
            lib.oracle_free(p_)
    return {"bridges": bridges, "offsets": offsets, "refs": refs, "keys": keys, "P": P, "n": n}


def search(X: np.ndarray, graph: np.ndarray, centers: np.ndarray, bg: dict, queries: np.ndarray,
           k, T, kmax: int | None = None, nthreads: int = 1, trace: bool = False, bridge_key_limit=None):
    """Algorithm 1 for each query.  k, T: scalars or per-query arrays.
    nthreads: threads (0 = all cores); one query per thread, and threads left
    over share each query's on-demand kNN row scans.
    graph: (N, R) int32 rows, or an int R to compute each popped row on demand
    (its R nearest other references by linear scan).

    Returns (ids (nq, kmax) int32, keys (nq, kmax) float64, stats dict of arrays);
    with trace=True the stats dict also holds 'trace' (nq, max T): the
    discovered ids in discovery order, -1 after the last.
    bridge_key_limit (scalar or per query): bg's lists are complete only for
    bridges with key <= the limit; a query that would pop a bridge above it
    stops there and gets stats['over_limit'] = 1."""
    lib = _load()
    X = np.ascontiguousarray(X)
    queries = np.ascontiguousarray(queries)
    if isinstance(graph, (int, np.integer)):
        R_on_demand = int(graph)      # rows computed on demand by linear scan
        graph = None
    else:
        graph = np.ascontiguousarray(graph, dtype=np.int32)
    centers = np.ascontiguousarray(centers)
    assert X.dtype == queries.dtype == centers.dtype
    N, d = X.shape
    nq = queries.shape[0]
    P, n, _ = centers.shape
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (nq,)))
    T = np.ascontiguousarray(np.broadcast_to(np.asarray(T, np.int32), (nq,)))
    if kmax is None:
        kmax = int(k.max()) if nq else 1
    ids = np.empty((nq, kmax), np.int32)
    keys = np.empty((nq, kmax), np.float64)
    ns = lib.oracle_num_stats()
    st = np.zeros((nq, ns), np.int64)
    bridges = np.ascontiguousarray(bg["bridges"], dtype=np.uint64)
    offs = np.ascontiguousarray(bg["offsets"], dtype=np.int64)
    refs = np.ascontiguousarray(bg["refs"], dtype=np.int32)
    cap = int(T.max()) if (trace and nq) else 0
    disc = np.empty((nq, max(cap, 1)), np.int32)
    lim = None if bridge_key_limit is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(bridge_key_limit, np.float64), (nq,)))
    rc = lib.oracle_search(_ptr(X), N, d, _dtype_code(X), None if graph is None else _ptr(graph),
                           R_on_demand if graph is None else graph.shape[1], P, n,
                           _ptr(centers), len(bridges), _ptr(bridges), _ptr(offs), _ptr(refs),
                           _ptr(queries), nq, _ptr(k), _ptr(T), kmax, _ptr(ids), _ptr(keys),
                           _ptr(st), _ptr(disc) if trace else None, cap, None if lim is None else _ptr(lim),
                           _threads(nthreads))
    if rc != 0:
        raise ValueError("oracle_search: bad arguments")
    out = {name: st[:, i] for i, name in enumerate(STAT_NAMES)}
    if trace:
        out["trace"] = disc[:, :cap]
    return ids, keys, out


def recall_at_k(found_ids: np.ndarray, true_keys: np.ndarray, X: np.ndarray, queries: np.ndarray,
                k: int) -> np.ndarray:
    """Accuracy r/k per query (Sec. 5.1), tie-tolerant: a returned id counts when
    its true key is <= the true k-th key.  found_ids: (nq, >=k)."""
    nq = found_ids.shape[0]
    out = np.zeros(nq)
    for i in range(nq):
        ids = found_ids[i, :k]
        ids = ids[ids >= 0]
        if len(ids) == 0:
            continue
        kth = true_keys[i, k - 1]
        if X.dtype == np.uint8:
            diff = X[ids].astype(np.int64) - queries[i].astype(np.int64)
            dk = (diff * diff).sum(1).astype(np.float64)
        else:
            diff = X[ids].astype(np.float64) - queries[i].astype(np.float64)
            dk = (diff * diff).sum(1).astype(np.float32).astype(np.float64)
        out[i] = np.count_nonzero(dk <= kth) / k
    return out


def _levels_of(dirs: np.ndarray) -> int:
    nseg = dirs.shape[1]
    levels = (nseg + 1).bit_length() - 1
    assert (1 << levels) - 1 == nseg, "dirs must hold 2^levels - 1 directions per round"
    return levels


def rp_partition(X: np.ndarray, dirs_round: np.ndarray) -> np.ndarray:
    """One random partition of the approximate graph construction: the point
    at every position after the recursive median splits along dirs_round
    (shape (2^levels - 1, d), int8).  Leaves are the 2^levels segments of
    the recursive halving of [0, N)."""
    lib = _load()
    X = np.ascontiguousarray(X)
    assert X.dtype == np.uint8
    dirs_round = np.ascontiguousarray(dirs_round, dtype=np.int8)
    levels = _levels_of(dirs_round[None])
    perm = np.empty(X.shape[0], np.int32)
    lib.oracle_rp_partition(_ptr(X), X.shape[0], X.shape[1], _ptr(dirs_round), levels, _ptr(perm))
    return perm


def knn_graph_approx(X: np.ndarray, R: int, dirs: np.ndarray, iters: int, rows=None):
    """Approximate R-NN graph of uint8 rows: leaf brute force over
    dirs.shape[0] random partitions, then `iters` propagation steps.
    dirs: (rounds, 2^levels - 1, d) int8.  rows: the points whose rows are
    wanted (None = all).  Returns (ids int32, keys float64), each (nrows, R),
    ascending (key, id)."""
    lib = _load()
    X = np.ascontiguousarray(X)
    assert X.dtype == np.uint8 and R <= 64
    dirs = np.ascontiguousarray(dirs, dtype=np.int8)
    rounds, levels = dirs.shape[0], _levels_of(dirs)
    assert dirs.shape[2] == X.shape[1]
    sel = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nrows = X.shape[0] if sel is None else len(sel)
    ids = np.empty((nrows, R), np.int32)
    keys = np.empty((nrows, R), np.float64)
    lib.oracle_knn_graph_approx(_ptr(X), X.shape[0], X.shape[1], R, _ptr(dirs), rounds, levels, iters,
                                None if sel is None else _ptr(sel), nrows, _ptr(ids), _ptr(keys))
    return ids, keys


def ivf_lists(assign: np.ndarray, K: int):
    """Inverted lists of the coarse quantizer: offsets (K + 1) and members,
    each list ascending by reference id."""
    assign = np.asarray(assign, np.int64)
    assert assign.min() >= 0 and assign.max() < K
    members = np.argsort(assign, kind="stable").astype(np.int32)
    offsets = np.zeros(K + 1, np.int64)
    offsets[1:] = np.cumsum(np.bincount(assign, minlength=K))
    return offsets, members


def pq_encode(X: np.ndarray, centers: np.ndarray, assign: np.ndarray, codebooks: np.ndarray) -> np.ndarray:
    """Product-quantization codes of the residuals X[i] - centers[assign[i]]:
    for each of the m parts the nearest of its ks codewords (distances in
    fp64), ties to the lower index.
    codebooks: (m, ks, d / m).  Returns (N, m) uint8."""
    lib = _load()
    Xf = np.ascontiguousarray(X, dtype=np.float32)
    Cf = np.ascontiguousarray(centers, dtype=np.float32)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    cb = np.ascontiguousarray(codebooks, dtype=np.float32)
    m, ks, dp = cb.shape
    N, d = Xf.shape
    assert m * dp == d and ks <= 256 and assign.shape == (N,)
    codes = np.empty((N, m), np.uint8)
    lib.oracle_pq_encode(_ptr(Xf), N, d, _ptr(Cf), _ptr(assign), m, ks, _ptr(cb), _ptr(codes))
    return codes


def adc_rerank(queries: np.ndarray, lists: np.ndarray, offsets: np.ndarray, members: np.ndarray,
               centers: np.ndarray, codes: np.ndarray, codebooks: np.ndarray, L: int, T: int):
    """Asymmetric-distance re-ranking: for query i, the first L members of
    the lists lists[i] (visited in that order; -1 entries skipped) ranked by
    (||q - c - r^||^2 in fp64, id).  Returns (ids (nq, T), keys (nq, T)
    float64, examined (nq,))."""
    lib = _load()
    Qd = np.ascontiguousarray(queries, dtype=np.float32)
    lists = np.ascontiguousarray(lists, dtype=np.int32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    members = np.ascontiguousarray(members, dtype=np.int32)
    Cd = np.ascontiguousarray(centers, dtype=np.float32)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    cb = np.ascontiguousarray(codebooks, dtype=np.float32)
    m, ks, _ = cb.shape
    nq, d = Qd.shape
    ids = np.empty((nq, T), np.int32)
    keys = np.empty((nq, T), np.float64)
    seen = np.empty(nq, np.int64)
    for i in range(nq):
        li = np.ascontiguousarray(lists[i])
        seen[i] = lib.oracle_adc_rerank(_ptr(Qd[i]), d, _ptr(li), len(li), _ptr(offsets), _ptr(members),
                                        _ptr(Cd), _ptr(codes), m, ks, _ptr(cb), L, T,
                                        ids[i:].ctypes.data_as(ctypes.c_void_p),
                                        keys[i:].ctypes.data_as(ctypes.c_void_p))
    return ids, keys, seen


def adc_keys(q: np.ndarray, cand: np.ndarray, assign: np.ndarray, centers: np.ndarray, codes: np.ndarray,
             codebooks: np.ndarray) -> np.ndarray:
    """fp64 asymmetric distances ||q - c(x) - r^(x)||^2 of the candidates cand
    (ids; x is listed under assign[x]) to the one query q."""
    lib = _load()
    qd = np.ascontiguousarray(q, dtype=np.float32)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    Cd = np.ascontiguousarray(centers, dtype=np.float32)
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    cb = np.ascontiguousarray(codebooks, dtype=np.float32)
    m, ks, _ = cb.shape
    out = np.empty(len(cand), np.float64)
    lib.oracle_adc_keys(_ptr(qd), qd.shape[0], _ptr(cand), len(cand), _ptr(assign), _ptr(Cd), _ptr(codes), m, ks,
                        _ptr(cb), _ptr(out))
    return out


def graph_d_adc_search(coarse: np.ndarray, coarse_graph, part_centers: np.ndarray, bg: dict,
                       offsets: np.ndarray, members: np.ndarray, codes: np.ndarray, codebooks: np.ndarray,
                       queries: np.ndarray, w: int, Tc: int, L: int, T: int):
    """Graph-D-ADC search (Sec. 5.4): Algorithm 1 over the index of the coarse
    centers (k = w lists, budget Tc), then asymmetric-distance re-ranking of
    the first L members of those lists.  Returns (ids, keys, examined)."""
    lists, _, _ = search(coarse, coarse_graph, part_centers, bg, queries, w, Tc)
    return adc_rerank(queries, lists, offsets, members, coarse, codes, codebooks, L, T)
