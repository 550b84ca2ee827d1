"""The float32 bridge key of the GPU path (Sec. 4.2: the sum over parts of
the part keys, taken as the float32 nearest to the exact sum) checked on its
own: a small kernel compiled from the library's device header applies the
same device functions the search and the bridge-graph build use to
adversarial and random inputs, and every result must equal the float32
nearest to the exact rational sum (ties to even), computed here with
fractions.  Also checks the directed-rounding bounds the walk skips work on:
lower bound <= key <= upper bound."""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include "ann_device.cuh"
using namespace ann;
__global__ void k(const uint32_t *in, uint32_t *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t a = in[4 * i], b = in[4 * i + 1], c = in[4 * i + 2], d = in[4 * i + 3];
    out[3 * i] = KeyOps<ANN_F32>::sum4(a, b, c, d);
    out[3 * i + 1] = KeyOps<ANN_F32>::add_lo(KeyOps<ANN_F32>::add_lo(a, b), KeyOps<ANN_F32>::add_lo(c, d));
    out[3 * i + 2] = KeyOps<ANN_F32>::add_hi(KeyOps<ANN_F32>::up(KeyOps<ANN_F32>::add_lo(a, b)),
                                              KeyOps<ANN_F32>::up(KeyOps<ANN_F32>::add_lo(c, d)));
}
extern "C" int run(const uint32_t *in, uint32_t *out, int n) {
    uint32_t *di, *dout;
    if (cudaMalloc(&di, 16 * (size_t)n) || cudaMalloc(&dout, 12 * (size_t)n)) return 1;
    cudaMemcpy(di, in, 16 * (size_t)n, cudaMemcpyHostToDevice);
    k<<<(n + 127) / 128, 128>>>(di, dout, n);
    cudaMemcpy(out, dout, 12 * (size_t)n, cudaMemcpyDeviceToHost);
    int e = (int)cudaGetLastError();
    cudaFree(di);
    cudaFree(dout);
    return e;
}
'''


@pytest.fixture(scope="module")
def keysum():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1312_3062_gb300 import _build
    d = tempfile.mkdtemp()
    src, lib = os.path.join(d, "keysum.cu"), os.path.join(d, "libkeysum.so")
    open(src, "w").write(SRC)
    subprocess.check_call([_build.nvcc(), *_build.ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           f"-I{os.path.join(ROOT, 'paper_1312_3062_gb300', 'csrc')}",
                           f"-I{os.path.join(ROOT, 'include')}", "-o", lib, src])
    return ctypes.CDLL(lib)


def nearest_f32_bits(fr: Fraction) -> int:
    """Bit pattern of the float32 nearest to a non-negative rational, ties to even."""
    if fr == 0:
        return 0
    # find e with 2^e <= fr < 2^(e+1)
    e = fr.numerator.bit_length() - fr.denominator.bit_length()
    if Fraction(2) ** e > fr:
        e -= 1
    q_exp = max(e - 23, -149)                 # spacing of float32 values near fr
    scaled = fr / Fraction(2) ** q_exp
    q = scaled.numerator // scaled.denominator
    rem = scaled - q
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q % 2 == 1):
        q += 1
    v = Fraction(q) * Fraction(2) ** q_exp
    if v >= Fraction(2) ** 128:
        return 0x7F800000
    return int(np.array([float(v)], np.float32).view(np.uint32)[0])


def f32(bits):
    return Fraction(float(np.array([bits], np.uint32).view(np.float32)[0]))


def cases(rng):
    b = lambda x: int(np.array([x], np.float32).view(np.uint32)[0])  # noqa: E731
    eps = 2.0 ** -24
    fixed = [
        [1.0, eps, 2.0 ** -60, 0.0], [1.0, eps, 0.0, 0.0], [1.0 + 2 * eps, eps, 0.0, 0.0],
        [1.0, 2.0 ** -25, 2.0 ** -25, 2.0 ** -80], [3.0, 2.0 ** -120, 2.0 ** -149, 2.0 ** -140],
        [2.0 ** -149, 2.0 ** -149, 2.0 ** -148, 0.0], [0.0] * 4, [2.0 ** 100, 1.0, 2.0 ** 76, 2.0 ** 75],
        [2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 0.0], [2.0 ** 127, 2.0 ** 127, 0.0, 0.0],
        [1.0, 2.0 ** -37, 2.0 ** -37, 0.0], [1.0, 2.0 ** -36, 2.0 ** -61, 2.0 ** -61],
    ]
    out = [[b(x) for x in c] for c in fixed]
    for _ in range(20000):
        spread = int(rng.integers(0, 60))
        e = rng.integers(-20, 20) - rng.integers(0, spread + 1, size=4)
        v = [float(np.float32(rng.random() * 2.0 ** int(x))) for x in e]
        if rng.random() < 0.2:
            v[int(rng.integers(0, 4))] = 0.0
        out.append([b(x) for x in v])
    # halfway cases: a + b exactly at a midpoint, then nudged by c
    for _ in range(2000):
        a = float(np.float32(1.0 + rng.integers(0, 2 ** 23) * eps * 2))
        out.append([b(a), b(eps * a), b(float(np.float32(2.0 ** -int(rng.integers(30, 140))))), 0])
        out.append([b(a), b(eps * a), 0, 0])
    return np.array(out, np.uint32)


def test_exact_key_sum_and_bounds(keysum):
    inp = cases(np.random.default_rng(5))
    out = np.zeros((len(inp), 3), np.uint32)
    assert keysum.run(inp.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                      ctypes.c_int(len(inp))) == 0
    INF = 0x7F800000
    for row, (key, lo, hi) in zip(inp, out):
        exact = sum(f32(x) for x in row)
        assert int(key) == nearest_f32_bits(exact), [hex(int(x)) for x in row]
        # bounds (an infinite upper bound is a valid one)
        assert f32(lo) <= exact
        if int(hi) != INF:
            assert f32(hi) >= exact
        if int(key) != INF:
            assert f32(lo) <= f32(key) and (int(hi) == INF or f32(key) <= f32(hi))
