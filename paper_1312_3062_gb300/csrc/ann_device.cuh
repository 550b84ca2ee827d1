// ann_device.cuh -- device helpers shared by the search and index-build kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ann.h"

namespace ann {

__host__ __device__ inline uint32_t align_up16(uint32_t x) { return (x + 15u) & ~15u; }

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

// float32 exact-ish squared distance pieces: error-free transforms
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// accumulate (x - y)^2 into the double-float (hi, lo)
__device__ __forceinline__ void df_acc_sqdiff(float x, float y, float &hi, float &lo) {
    float dh, dl;
    two_sum(x, -y, dh, dl);                 // dh + dl = x - y exactly
    float p = __fmul_rn(dh, dh);
    float pe = __fmaf_rn(dh, dh, -p);       // p + pe = dh^2 exactly
    pe = __fmaf_rn(__fmul_rn(2.0f, dh), dl, pe);  // + 2 dh dl (dl^2 is below 2^-48 of dh^2)
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ void df_add(float &hi, float &lo, float h2, float l2) {
    float s, e;
    two_sum(hi, h2, s, e);
    float l = __fadd_rn(__fadd_rn(lo, l2), e);
    float s2 = __fadd_rn(s, l);                  // fast renormalisation
    lo = __fsub_rn(l, __fsub_rn(s2, s));
    hi = s2;
}

// bitonic sort of keys (and optional values) in shared memory by one warp; L power of two
__device__ inline void warp_sort_pairs(uint64_t *keys, uint32_t *vals, int L) {
    const int lane = lane_id();
    for (int k = 2; k <= L; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < L; i += 32) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool up = (i & k) == 0;
                    uint64_t a = keys[i], b = keys[ixj];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[ixj] = a;
                        if (vals) {
                            uint32_t t = vals[i];
                            vals[i] = vals[ixj];
                            vals[ixj] = t;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Bitonic sort of 32*EPL keys held in registers, ascending in the blocked
// order (element i = lane*EPL + slot).  Pairs in different lanes exchange
// through shuffles; pairs in the same lane swap registers.
template <int EPL, typename K>
__device__ __forceinline__ void reg_bitonic_sort_t(K (&v)[EPL]) {
    const int lane = lane_id();
    constexpr int L = 32 * EPL;
#pragma unroll
    for (int k = 2; k <= L; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= EPL) {
#pragma unroll
                for (int s = 0; s < EPL; s++) {
                    const int i = lane * EPL + s;
                    const K o = __shfl_xor_sync(0xffffffffu, v[s], j / EPL);
                    const bool up = (i & k) == 0, lower = (i & j) == 0;
                    const K mn = v[s] < o ? v[s] : o, mx = v[s] < o ? o : v[s];
                    v[s] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int s = 0; s < EPL; s++) {
                    const int p = s ^ j;
                    if (p > s) {
                        const bool up = ((lane * EPL + s) & k) == 0;
                        const K a = v[s], b = v[p];
                        if ((a > b) == up) {
                            v[s] = b;
                            v[p] = a;
                        }
                    }
                }
            }
        }
    }
}

template <int EPL>
__device__ __forceinline__ void reg_bitonic_sort(uint64_t (&v)[EPL]) {
    reg_bitonic_sort_t<EPL, uint64_t>(v);
}

// ---------------------------------------------------------------------------
// per-part key of one part of the query against one center, computed by one lane
// ---------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ uint32_t part_key_lane(const uint8_t *qbytes, const void *C, int p, int c,
                                                  int n, int dp);

template <>
__device__ __forceinline__ uint32_t part_key_lane<ANN_U8>(const uint8_t *qbytes, const void *C, int p,
                                                          int c, int n, int dp) {
    const uint8_t *cent = (const uint8_t *)C + ((int64_t)p * n + c) * dp;
    const uint8_t *qp = qbytes + p * dp;
    uint32_t acc = 0;
    int e = 0;
    if ((dp & 3) == 0) {
        for (; e < dp; e += 4) {
            uint32_t a = *(const uint32_t *)(qp + e);
            uint32_t b = __ldg((const unsigned int *)(cent + e));
            uint32_t df = __vabsdiffu4(a, b);
            acc = __dp4a(df, df, acc);
        }
    }
    for (; e < dp; e++) {
        int t = (int)qp[e] - (int)cent[e];
        acc += (uint32_t)(t * t);
    }
    return acc;
}

template <>
__device__ __forceinline__ uint32_t part_key_lane<ANN_F32>(const uint8_t *qbytes, const void *C, int p,
                                                           int c, int n, int dp) {
    const float *cent = (const float *)C + ((int64_t)p * n + c) * dp;
    const float *qp = (const float *)qbytes + p * dp;
    float hi = 0.f, lo = 0.f;
    for (int e = 0; e < dp; e++) df_acc_sqdiff(qp[e], __ldg(cent + e), hi, lo);
    return __float_as_uint(__fadd_rn(hi, lo));
}

// ---------------------------------------------------------------------------
// bridge-key arithmetic (grouping (D0 + D1) + (D2 + D3 + ...))
// ---------------------------------------------------------------------------
template <int DT> struct KeyOps;
template <> struct KeyOps<ANN_U8> {
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) { return a + b; }
};
template <> struct KeyOps<ANN_F32> {
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) {
        return __float_as_uint(__fadd_rn(__uint_as_float(a), __uint_as_float(b)));
    }
};

}  // namespace ann
