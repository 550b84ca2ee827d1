"""Thin Python binding of the C ABI in include/ann.h (argument marshalling only).

Every function has the name of its C entry point and forwards device
pointers taken from torch CUDA tensors (or plain integers).  All computation
happens in libann.so; if the library is missing this module raises at import
time -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

ANN_U8, ANN_F32 = 0, 1
ANN_OK, ANN_PENDING = 0, 1
ANN_ERR_ARG, ANN_ERR_OOM, ANN_ERR_CAPACITY, ANN_ERR_TIMEOUT, ANN_ERR_CUDA, ANN_ERR_FORMAT = -1, -2, -3, -4, -5, -6
ANN_MODE_PLAIN, ANN_MODE_PERSISTENT = 0, 1
STAT_NAMES = ("discovered", "ref_pops", "bridge_pops", "walks", "walk_nodes", "walk_leaves", "max_q",
              "preloaded")
ANN_NSTATS = len(STAT_NAMES)

if not os.path.exists(_build.LIB):
    raise ImportError(f"{_build.LIB} is missing: run paper_1312_3062_gb300._build.build() "
                      "(or __graft_entry__.build()) first")

lib = ctypes.CDLL(_build.LIB)

P_ = ctypes.c_void_p
i32, i64, u64, f64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t


class ann_index_desc(ctypes.Structure):
    _fields_ = [("dtype", i32), ("N", i64), ("d", i32), ("R", i32), ("P", i32), ("n", i32), ("t", i32),
                ("b", i32), ("data", P_), ("graph", P_), ("centers", P_), ("M", i64), ("bridge_ids", P_),
                ("bridge_offsets", P_), ("bridge_refs", P_)]


class ann_index_info(ctypes.Structure):
    _fields_ = [("N", i64), ("M", i64), ("d", i32), ("R", i32), ("P", i32), ("n", i32), ("b", i32),
                ("dtype", i32), ("bridged_refs", i64), ("alpha", f64), ("bytes_vectors", i64),
                ("bytes_graph", i64), ("bytes_bridges", i64), ("groups", i64)]


def _sig(name, argtypes, restype=ctypes.c_int):
    fn = getattr(lib, name)
    fn.argtypes = argtypes
    fn.restype = restype
    return fn


_sig("ann_last_error", [], ctypes.c_char_p)
_sig("ann_exact_knn", [P_, i64, P_, i64, ctypes.c_int, i32, i32, i32, P_, P_, P_])
_sig("ann_exact_knn_static", [P_, i64, P_, i64, ctypes.c_int, i32, i32, i32, P_, P_, P_])
_sig("ann_build_knn_graph", [P_, ctypes.c_int, i64, i32, i32, P_, P_, P_])
_sig("ann_build_knn_graph_approx", [P_, ctypes.c_int, i64, i32, i32, P_, i32, i32, i32, P_, P_, P_])
_sig("ann_pq_encode", [P_, ctypes.c_int, i64, i32, P_, i64, P_, i32, i32, P_, P_, P_])
_sig("ann_adc_rerank", [P_, i64, i32, P_, i32, P_, i64, P_, P_, P_, i32, i32, P_, i64, i32, P_, P_, P_, P_])
_sig("ann_train_centers", [P_, ctypes.c_int, i64, i32, i32, i32, i32, P_, P_, P_, P_])
_sig("ann_index_create", [ctypes.POINTER(ann_index_desc), ctypes.POINTER(P_)])
_sig("ann_index_load", [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(P_)])
_sig("ann_index_save", [P_, ctypes.c_char_p])
_sig("ann_index_free", [P_])
_sig("ann_index_get_info", [P_, ctypes.POINTER(ann_index_info)])
_sig("ann_index_get_bridges", [P_, P_, P_])
_sig("ann_index_lookup_bridges", [P_, P_, i64, P_])
_sig("ann_search_batch", [P_, P_, i64, P_, P_, i32, i32, i32, i32, P_, P_, P_, P_, P_])
_sig("ann_server_create", [P_, sz, i32, ctypes.POINTER(P_)])
_sig("ann_server_destroy", [P_])
_sig("ann_serve_submit", [P_, P_, i32, P_, P_, ctypes.POINTER(u64)])
_sig("ann_serve_poll", [P_, u64, P_, P_, P_])
_sig("ann_serve_latency", [P_, u64], f64)
_sig("ann_serve_replay", [P_, P_, P_, P_, i32, P_, P_, P_, P_, P_])

EXPORTED = ("ann_last_error", "ann_exact_knn", "ann_exact_knn_static", "ann_build_knn_graph", "ann_build_knn_graph_approx",
            "ann_pq_encode", "ann_adc_rerank", "ann_train_centers", "ann_index_create",
            "ann_index_load", "ann_index_save", "ann_index_free", "ann_index_get_info", "ann_index_get_bridges", "ann_index_lookup_bridges",
            "ann_search_batch", "ann_server_create", "ann_server_destroy", "ann_serve_submit", "ann_serve_poll",
            "ann_serve_latency", "ann_serve_replay")


class AnnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ann error {code}: {msg}")
        self.code = code


def check(rc: int) -> int:
    if rc < 0:
        raise AnnError(rc, lib.ann_last_error().decode(errors="replace"))
    return rc


def ptr(x) -> int | None:
    """Device/host address of a torch tensor or numpy array (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous(), "tensor must be contiguous"
    return x.data_ptr()


def stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(t) -> int:
    import torch
    if t.dtype == torch.uint8:
        return ANN_U8
    if t.dtype == torch.float32:
        return ANN_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


# ---- entry points (same names as the C ABI) ----

def ann_exact_knn(refs, queries, k, exclude_self=False, out_ids=None, out_keys=None, stream=None):
    import torch
    N, d = refs.shape
    nq = queries.shape[0]
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=refs.device)
    if out_keys is None:
        out_keys = torch.empty((nq, k), dtype=torch.int32 if refs.dtype == torch.uint8 else torch.float32,
                               device=refs.device)
    check(lib.ann_exact_knn(ptr(refs), N, ptr(queries), nq, dtype_code(refs), d, k, int(exclude_self),
                            ptr(out_ids), ptr(out_keys), stream_ptr(stream)))
    return out_ids, out_keys


def ann_build_knn_graph(data, R, out_ids=None, out_keys=None, stream=None):
    import torch
    N, d = data.shape
    if out_ids is None:
        out_ids = torch.empty((N, R), dtype=torch.int32, device=data.device)
    if out_keys is None:
        out_keys = torch.empty((N, R), dtype=torch.int32 if data.dtype == torch.uint8 else torch.float32,
                               device=data.device)
    check(lib.ann_build_knn_graph(ptr(data), dtype_code(data), N, d, R, ptr(out_ids), ptr(out_keys),
                                  stream_ptr(stream)))
    return out_ids, out_keys


def ann_build_knn_graph_approx(data, R, dirs, iters, out_ids=None, out_keys=None, stream=None):
    """dirs: device int8 tensor (rounds, 2^levels - 1, d) of split directions."""
    import torch
    N, d = data.shape
    rounds, nseg = dirs.shape[0], dirs.shape[1]
    levels = (nseg + 1).bit_length() - 1
    if (1 << levels) - 1 != nseg or dirs.shape[2] != d:
        raise ValueError("dirs must have shape (rounds, 2^levels - 1, d)")
    if out_ids is None:
        out_ids = torch.empty((N, R), dtype=torch.int32, device=data.device)
    if out_keys is None:
        out_keys = torch.empty((N, R), dtype=torch.int32, device=data.device)
    check(lib.ann_build_knn_graph_approx(ptr(data), dtype_code(data), N, d, R, ptr(dirs) if nseg else None,
                                         rounds, levels, iters, ptr(out_ids), ptr(out_keys), stream_ptr(stream)))
    return out_ids, out_keys


def ann_pq_encode(data, centers, assign, codebooks, out=None, stream=None):
    """codebooks: device float32 (m, ks, d / m); returns device uint8 (N, m)."""
    import torch
    N, d = data.shape
    m, ks, _ = codebooks.shape
    if out is None:
        out = torch.empty((N, m), dtype=torch.uint8, device=data.device)
    check(lib.ann_pq_encode(ptr(data), dtype_code(data), N, d, ptr(centers), centers.shape[0], ptr(assign), m, ks,
                            ptr(codebooks), ptr(out), stream_ptr(stream)))
    return out


def ann_adc_rerank(queries, lists, offsets, members, centers, codes, codebooks, L, T, stream=None):
    """lists: device int32 (nq, w); returns (ids int32 (nq, T), keys float32 (nq, T), seen int64 (nq,))."""
    import torch
    nq, d = queries.shape
    w = lists.shape[1]
    m, ks, _ = codebooks.shape
    ids = torch.empty((nq, T), dtype=torch.int32, device=queries.device)
    keys = torch.empty((nq, T), dtype=torch.float32, device=queries.device)
    seen = torch.empty((nq,), dtype=torch.int64, device=queries.device)
    check(lib.ann_adc_rerank(ptr(queries), nq, d, ptr(lists), w, ptr(offsets), offsets.shape[0] - 1, ptr(members),
                             ptr(centers), ptr(codes), m, ks, ptr(codebooks), L, T, ptr(ids), ptr(keys), ptr(seen),
                             stream_ptr(stream)))
    return ids, keys, seen


def graph_d_adc_search(coarse_index, queries, w, Tc, offsets, members, centers_f32, codes, codebooks, L, T,
                       stream=None):
    """Graph-D-ADC (Sec. 5.4) end to end: Algorithm 1 over the index of the
    coarse centers (k = w lists, budget Tc) gives each query's lists, then
    ann_adc_rerank ranks the first L members of those lists.  queries: device
    tensor of the coarse index's dtype (uint8 queries are widened to float32
    for the re-ranking).  Returns (ids, keys, examined, lists)."""
    import torch
    lists, _, _ = ann_search_batch(coarse_index, queries, w, Tc, kmax=w, stream=stream)
    qf = queries if queries.dtype == torch.float32 else queries.to(torch.float32)
    ids, keys, seen = ann_adc_rerank(qf, lists, offsets, members, centers_f32, codes, codebooks, L, T, stream)
    return ids, keys, seen, lists


def ann_train_centers(train, P, n, iters, init_rows: np.ndarray, want_f64=False, stream=None):
    import torch
    ntrain, d = train.shape
    init_rows = np.ascontiguousarray(init_rows, dtype=np.int64)
    out = torch.empty((P, n, d // P), dtype=train.dtype, device=train.device)
    out64 = torch.empty((P, n, d // P), dtype=torch.float64, device=train.device) if want_f64 else None
    check(lib.ann_train_centers(ptr(train), dtype_code(train), ntrain, d, P, n, iters, ptr(init_rows), ptr(out),
                                ptr(out64), stream_ptr(stream)))
    return (out, out64) if want_f64 else out


class Index:
    """Owner of an ann_index handle."""

    def __init__(self, handle: int):
        self.handle = handle

    @classmethod
    def create(cls, data, graph, centers, t=100, b=5, bridges: dict | None = None):
        N, d = data.shape
        P, n, _ = centers.shape
        desc = ann_index_desc(dtype=dtype_code(data), N=N, d=d, R=graph.shape[1], P=P, n=n, t=t, b=b,
                              data=ptr(data), graph=ptr(graph), centers=ptr(centers))
        keep = []
        if bridges is not None:
            ids = np.ascontiguousarray(bridges["bridges"], dtype=np.uint64)
            offs = np.ascontiguousarray(bridges["offsets"], dtype=np.int64)
            refs = np.ascontiguousarray(bridges["refs"], dtype=np.int32)
            keep = [ids, offs, refs]
            desc.M = len(ids)
            desc.bridge_ids, desc.bridge_offsets, desc.bridge_refs = ptr(ids), ptr(offs), ptr(refs)
        h = P_()
        check(lib.ann_index_create(ctypes.byref(desc), ctypes.byref(h)))
        del keep
        return cls(h.value)

    @classmethod
    def load(cls, path: str, device: int = -1):
        h = P_()
        check(lib.ann_index_load(path.encode(), device, ctypes.byref(h)))
        return cls(h.value)

    def save(self, path: str):
        check(lib.ann_index_save(self.handle, path.encode()))

    def info(self) -> dict:
        inf = ann_index_info()
        check(lib.ann_index_get_info(self.handle, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in ann_index_info._fields_}

    def bridges(self):
        inf = self.info()
        M, b = inf["M"], inf["b"]
        ids = np.empty(max(M, 1), np.uint64)
        refs = np.empty(max(M * b, 1), np.int32)
        check(lib.ann_index_get_bridges(self.handle, ptr(ids), ptr(refs)))
        return ids[:M], refs[:M * b].reshape(M, b)

    def lookup_bridges(self, ids):
        """Reference lists (-1 padded) of the selected bridge ids."""
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        refs = np.empty((max(len(ids), 1), self.info()["b"]), np.int32)
        check(lib.ann_index_lookup_bridges(self.handle, ptr(ids), len(ids), ptr(refs)))
        return refs[:len(ids)]

    def free(self):
        if self.handle:
            lib.ann_index_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ann_search_batch(index: Index, queries, k, T, kmax=None, mode=ANN_MODE_PLAIN, out_ids=None, out_keys=None,
                     out_status=None, out_stats=None, stream=None):
    """k, T: ints (uniform) or device int32 tensors (per query)."""
    import torch
    nq = queries.shape[0]
    k_arr = k if torch.is_tensor(k) else None
    T_arr = T if torch.is_tensor(T) else None
    k_all = 0 if k_arr is not None else int(k)
    T_all = 0 if T_arr is not None else int(T)
    if kmax is None:
        kmax = int(k_arr.max().item()) if k_arr is not None else k_all
        kmax = max(kmax, 1)
    dev = queries.device
    if out_ids is None:
        out_ids = torch.empty((nq, kmax), dtype=torch.int32, device=dev)
    if out_keys is None:
        out_keys = torch.empty((nq, kmax), dtype=torch.int32 if queries.dtype == torch.uint8 else torch.float32,
                               device=dev)
    if out_status is None:
        out_status = torch.empty((nq,), dtype=torch.int32, device=dev)
    check(lib.ann_search_batch(index.handle, ptr(queries), nq, ptr(k_arr), ptr(T_arr), k_all, T_all, kmax, mode,
                               ptr(out_ids), ptr(out_keys), ptr(out_status), ptr(out_stats), stream_ptr(stream)))
    return out_ids, out_keys, out_status


def keys_as_uint32(keys):
    """View int32 key storage of uint8 indexes as exact uint32 numpy values."""
    a = keys.cpu().numpy() if hasattr(keys, "cpu") else np.asarray(keys)
    return a.view(np.uint32) if a.dtype == np.int32 else a
