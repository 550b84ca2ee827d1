"""The error bound behind the exact float32 k-NN (candidates from bf16 split
dot products, float32 accumulation): for each pair the approximate key
|q|^2 + |x|^2 - 2 (qh.xh + ql.xh + qh.xl) must lie within
eps = (gamma_{3d+16} + 3 * 2^-18) * (|q|^2 + max |x|^2) of the exact one (the
kernel uses four times this).  Emulated here in numpy: bf16 round to nearest
even, products and a sequential float32 sum; checked on vectors shaped like
the float32 workloads, including the worst case of equal positive vectors."""
from __future__ import annotations

import numpy as np

from paper_1312_3062_gb300 import datagen


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest, ties to even), returned as float32."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def approx_key(q: np.ndarray, x: np.ndarray) -> float:
    qh, xh = bf16(q), bf16(x)
    ql, xl = bf16(q - qh), bf16(x - xh)
    acc = np.float32(0)
    for a, b in ((qh, xh), (ql, xh), (qh, xl)):
        for t in (a * b).astype(np.float32):     # exact products of bf16 values
            acc = np.float32(acc + t)
    qn = np.float32(np.dot(q.astype(np.float64), q.astype(np.float64)))
    xn = np.float32(np.dot(x.astype(np.float64), x.astype(np.float64)))
    a = np.float32(np.float32(qn + xn) - np.float32(2) * acc)
    return float(max(a, np.float32(0)))


def eps(d: int, qn: float, xn: float) -> float:
    u = 2.0 ** -24
    n = 3 * d + 16
    return (n * u / (1 - n * u) + 3 * 2.0 ** -18) * (qn + xn)


def test_margin_covers_the_split_product_error():
    worst = 0.0
    for w, d in ((3, 384), (4, 512)):
        X = datagen.references(w, 64)
        Q = datagen.queries(w, 8)
        xmax = float(max(np.dot(r.astype(np.float64), r.astype(np.float64)) for r in X))
        for q in Q:
            qn = float(np.dot(q.astype(np.float64), q.astype(np.float64)))
            for x in X[:24]:
                exact = float(np.sum((q.astype(np.float64) - x.astype(np.float64)) ** 2))
                err = abs(approx_key(q, x) - exact)
                bound = eps(d, qn, xmax)
                assert err <= bound
                worst = max(worst, err / bound)
    # the worst case for cancellation: identical positive vectors
    x = np.abs(datagen.queries(4, 1)[0])
    xn = float(np.dot(x.astype(np.float64), x.astype(np.float64)))
    assert abs(approx_key(x, x) - 0.0) <= eps(512, xn, xn)
    assert worst < 1.0
