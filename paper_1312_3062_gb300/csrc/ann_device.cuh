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
// bridge-key arithmetic (Sec. 4.2: the bridge key is the sum over parts of the
// part keys).  uint8: exact integer sums.  float32: the key is the float32
// nearest to the EXACT sum of the float32 part keys (ties to even), one
// rounding of the real sum; bounds used to skip work are taken with directed
// rounding, so they never exclude a key they should admit.
// ---------------------------------------------------------------------------

// Exact sum of four finite non-negative floats (bit patterns), rounded once to
// float32, for any exponent spread: each value is an integer count of 2^-149
// below 2^277, so ten 32-bit limbs hold the sum exactly.  Rarely taken (the
// caller's fast path covers spreads up to 36 bits).
static __device__ __noinline__ uint32_t f32_exact_sum_wide(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    uint32_t acc[10];
#pragma unroll
    for (int j = 0; j < 10; j++) acc[j] = 0;
    const uint32_t v[4] = {a, b, c, d};
    for (int i = 0; i < 4; i++) {
        const uint32_t ex = (v[i] >> 23) & 0xffu;
        uint32_t man = v[i] & 0x7fffffu;
        int sh = 0;
        if (ex) {
            man |= 0x800000u;
            sh = (int)ex - 1;  // normal: (2^23 + m) * 2^(ex - 1) units of 2^-149
        }
        const uint64_t part = (uint64_t)man << (sh & 31);
        uint64_t carry = 0;
        for (int j = sh >> 5; j < 10; j++) {
            const uint64_t add = j == (sh >> 5) ? (part & 0xffffffffu) : (j == (sh >> 5) + 1 ? part >> 32 : 0);
            const uint64_t t = (uint64_t)acc[j] + add + carry;
            acc[j] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    int top = -1;
    for (int j = 9; j >= 0 && top < 0; j--)
        if (acc[j]) top = 32 * j + 31 - __clz(acc[j]);
    if (top < 24) return acc[0];  // below 2^24 units: the count is the float's own bit pattern
    auto bit = [&](int pos) -> uint32_t { return (acc[pos >> 5] >> (pos & 31)) & 1u; };
    int low = top - 23;
    uint32_t q = 0;
    for (int p2 = top; p2 >= low; p2--) q = (q << 1) | bit(p2);
    const uint32_t rnd = bit(low - 1);
    uint32_t sticky = 0;
    for (int p2 = low - 2; p2 >= 0 && !sticky; p2--) sticky = bit(p2);
    if (rnd && (sticky || (q & 1u))) q++;
    if (q == (1u << 24)) {
        q >>= 1;
        low++;
    }
    // q * 2^(low - 149) = (2^23 + m) * 2^(E - 150) with E = low + 1
    const int E = low + 1;
    if (E >= 255) return 0x7f800000u;
    return ((uint32_t)E << 23) | (q & 0x7fffffu);
}

// The float32 nearest to a + b + c + d (finite, non-negative; bit patterns).
// Fast path: align the four significands to the largest exponent in one
// 64-bit integer (exact while the exponents differ by at most 36), round once.
__device__ __forceinline__ uint32_t f32_exact_sum(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    const uint32_t v[4] = {a, b, c, d};
    uint32_t emax = 1;
#pragma unroll
    for (int i = 0; i < 4; i++) emax = max(emax, (v[i] >> 23) & 0xffu);
    uint64_t acc = 0;
    bool wide = false;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t ex = (v[i] >> 23) & 0xffu;
        const uint32_t man = (v[i] & 0x7fffffu) | (ex ? 0x800000u : 0u);
        const uint32_t e = ex ? ex : 1u;  // subnormals scale like exponent field 1
        const uint32_t sh = emax - e;
        if (man != 0 && sh > 36) wide = true;
        acc += sh > 36 ? 0ull : ((uint64_t)man << (36 - sh));
    }
    // acc counts units of 2^(emax - 186); a result below the normal range
    // (all inputs tiny) also goes the wide way
    if (wide || acc == 0 || emax < 2) return acc == 0 && !wide ? 0u : f32_exact_sum_wide(a, b, c, d);
    const int top = 63 - __clzll((long long)acc);
    int shift = top - 23;  // >= 13: a normal input sets a bit at 59 or above
    uint64_t q = acc >> shift;
    const uint64_t rem = acc & ((1ull << shift) - 1), half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (q & 1ull))) q++;
    if (q == (1ull << 24)) {
        q >>= 1;
        shift++;
    }
    // value = q * 2^(shift + emax - 186), biased exponent E = shift + emax - 186 + 150
    const int E = shift + (int)emax - 36;
    if (E < 1) return f32_exact_sum_wide(a, b, c, d);
    if (E >= 255) return 0x7f800000u;
    return ((uint32_t)E << 23) | ((uint32_t)q & 0x7fffffu);
}

// out of line: the walks call it only for leaves that may lie in the window,
// and keeping its registers out of the search loop avoids spills there
static __device__ __noinline__ uint32_t f32_exact_sum_call(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    return f32_exact_sum(a, b, c, d);
}

__device__ __forceinline__ uint32_t f32_next_up(uint32_t x) { return x == 0x7f800000u ? x : x + 1; }

template <int DT> struct KeyOps;
template <> struct KeyOps<ANN_U8> {
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) { return a + b; }
    // lower / upper bounds of a sum (exact for integers)
    static __device__ __forceinline__ uint32_t add_lo(uint32_t a, uint32_t b) { return a + b; }
    static __device__ __forceinline__ uint32_t up(uint32_t a) { return a; }
    static __device__ __forceinline__ uint32_t add_hi(uint32_t a, uint32_t b) { return a + b; }
    static __device__ __forceinline__ uint32_t sum4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        return a + b + c + d;
    }
};
template <> struct KeyOps<ANN_F32> {
    // rounded sum (used only where any monotone estimate will do)
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) {
        return __float_as_uint(__fadd_rn(__uint_as_float(a), __uint_as_float(b)));
    }
    // a float32 never above the exact sum
    static __device__ __forceinline__ uint32_t add_lo(uint32_t a, uint32_t b) {
        return __float_as_uint(__fadd_rd(__uint_as_float(a), __uint_as_float(b)));
    }
    // a float32 never below the exact value whose round-down is a
    static __device__ __forceinline__ uint32_t up(uint32_t a) { return f32_next_up(a); }
    // a float32 never below the exact sum
    static __device__ __forceinline__ uint32_t add_hi(uint32_t a, uint32_t b) {
        return __float_as_uint(__fadd_ru(__uint_as_float(a), __uint_as_float(b)));
    }
    static __device__ __forceinline__ uint32_t sum4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        return f32_exact_sum_call(a, b, c, d);
    }
};

}  // namespace ann
