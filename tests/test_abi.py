"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ann.h declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1312_3062_gb300 import _build
    return _build.build()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ann.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ann_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ann_index_load", "ann_build_knn_graph", "ann_search_batch", "ann_serve_submit",
                 "ann_serve_poll"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header(libpath):
    from paper_1312_3062_gb300 import ann
    assert sorted(ann.EXPORTED) == declared_symbols()


def test_argument_errors_need_no_gpu(libpath):
    # argument validation happens before any CUDA call
    from paper_1312_3062_gb300 import ann
    rc = ann.lib.ann_exact_knn(None, 0, None, 0, 0, 128, 10, 0, None, None, None)
    assert rc == ann.ANN_ERR_ARG
    assert b"N or nq" in ann.lib.ann_last_error()
    rc = ann.lib.ann_search_batch(None, None, 1, None, None, 1, 1, 1, 0, None, None, None, None, None)
    assert rc == ann.ANN_ERR_ARG and b"index is NULL" in ann.lib.ann_last_error()
    # approximate graph: dtype, leaf size, d and alignment are checked on the
    # host; the (never dereferenced) addresses only have to look aligned
    cases = [((16, ann.ANN_F32, 1000, 128, 10, 32, 1, 2, 0, 48), b"ANN_U8"),
             ((16, ann.ANN_U8, 1000, 128, 10, 32, 1, 7, 0, 48), b"R + 1"),
             ((16, ann.ANN_U8, 1000, 120, 10, 32, 1, 2, 0, 48), b"multiple of 16"),
             ((8, ann.ANN_U8, 1000, 128, 10, 32, 1, 2, 0, 48), b"16-byte aligned"),
             ((16, ann.ANN_U8, 1000, 128, 33, 32, 1, 2, 0, 48), b"R must be"),
             ((16, ann.ANN_U8, 1000, 128, 10, None, 1, 2, 0, 48), b"dirs are required")]
    for a, msg in cases:
        rc = ann.lib.ann_build_knn_graph_approx(*a, None, None)
        assert rc == ann.ANN_ERR_ARG and msg in ann.lib.ann_last_error(), (a, ann.lib.ann_last_error())
    # Graph-D-ADC entry points: shapes and limits are checked on the host
    enc = [((16, ann.ANN_U8, 100, 128, 16, 10, 16, 2, 256, 16, 16, None), b"32 dims per part"),
           ((16, ann.ANN_U8, 100, 128, 16, 10, 16, 7, 256, 16, 16, None), b"multiple of m"),
           ((16, ann.ANN_U8, 100, 128, 16, 10, 16, 8, 257, 16, 16, None), b"ks must be"),
           ((16, 7, 100, 128, 16, 10, 16, 8, 256, 16, 16, None), b"dtype")]
    for a, msg in enc:
        rc = ann.lib.ann_pq_encode(*a)
        assert rc == ann.ANN_ERR_ARG and msg in ann.lib.ann_last_error(), (a, ann.lib.ann_last_error())
    rr = [((16, 4, 128, 16, 8, 16, 10, 16, 16, 16, 8, 256, 16, 1000, 129, 16, None, None, None), b"T must be"),
          ((16, 4, 128, 16, 8, 16, 10, 16, 16, 16, 65, 256, 16, 1000, 10, 16, None, None, None), b"m <= 64"),
          ((16, 4, 128, 16, 0, 16, 10, 16, 16, 16, 8, 256, 16, 1000, 10, 16, None, None, None), b"w >= 1"),
          ((16, 4, 128, None, 8, 16, 10, 16, 16, 16, 8, 256, 16, 1000, 10, 16, None, None, None), b"null")]
    for a, msg in rr:
        rc = ann.lib.ann_adc_rerank(*a)
        assert rc == ann.ANN_ERR_ARG and msg in ann.lib.ann_last_error(), (a, ann.lib.ann_last_error())
