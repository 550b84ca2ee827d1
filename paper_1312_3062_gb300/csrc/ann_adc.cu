// ann_adc.cu -- Graph-D-ADC (Sec. 5.4) on sm_103a: the method as the coarse
// quantizer of an inverted file whose residuals are product-quantized.
//
//  - pq_encode_kernel: the code of every reference, one thread per
//    (reference, part); the part's codebook sits in shared memory and every
//    lane of a warp reads the same codeword (broadcast).
//  - adc_rerank_kernel: one CTA per query.  For each visited list (the
//    coarse search's result, in order) the CTA builds the asymmetric-distance
//    table of (q - c) against every codeword in shared memory, then keys the
//    list's members by m table lookups.  A candidate enters a pending buffer
//    only when it beats the current T-th best; the buffer and the best T are
//    merged by a bitonic sort when the buffer fills.  The result, the T
//    smallest (key, id) of all candidates, does not depend on the order in
//    which candidates arrive.
// Codes and keys are decided in float32 (the precision of the lookup tables
// of asymmetric distance computation) with every operation rounded: each
// distance is within (dp + m + 8) * 2^-24 * sum_t (|a_t| + |w_t|)^2 of the
// real one (a = x - c or q - c, w the codeword), so a code or a rank differs
// from the real-valued one of Sec. 5.4 only at near-ties of that size.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {
namespace {

constexpr int ENC_THREADS = 128;
constexpr int ENC_MAX_DP = 32;       // dims per part held in registers
constexpr int RR_THREADS = 256;
constexpr int RR_PER_THREAD = 4;
constexpr int RR_CHUNK = RR_THREADS * RR_PER_THREAD;  // candidates keyed per pass
constexpr int RR_SORT = 2048;        // merge buffer: best T + pending candidates
constexpr int RR_MAX_T = 128;

template <int DT>
__device__ __forceinline__ float elem(const void *X, int64_t i) {
    if (DT == ANN_U8) return (float)((const uint8_t *)X)[i];
    return ((const float *)X)[i];
}

template <int DT>
__global__ void __launch_bounds__(ENC_THREADS) pq_encode_kernel(const void *__restrict__ X, int64_t N, int d,
                                                                const float *__restrict__ centers, int64_t K,
                                                                const int32_t *__restrict__ assign, int m, int ks,
                                                                const float *__restrict__ codebooks,
                                                                uint8_t *__restrict__ codes) {
    extern __shared__ float cbs[];  // part j's codebook, ks * dp
    const int j = blockIdx.y;
    const int dp = d / m;
    for (int e = threadIdx.x; e < ks * dp; e += blockDim.x) cbs[e] = codebooks[(int64_t)j * ks * dp + e];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t a = assign[i];
    if (a < 0 || a >= K) {  // no such list: code 0 (rejected on the host for valid inputs)
        codes[i * m + j] = 0;
        return;
    }
    float r[ENC_MAX_DP];
#pragma unroll
    for (int t = 0; t < ENC_MAX_DP; t++)
        if (t < dp) r[t] = __fsub_rn(elem<DT>(X, i * d + j * dp + t), centers[a * d + j * dp + t]);
    float best = INFINITY;
    int arg = 0;
    for (int k = 0; k < ks; k++) {
        const float *w = cbs + k * dp;
        float s = 0.0f;
#pragma unroll
        for (int t = 0; t < ENC_MAX_DP; t++)
            if (t < dp) {
                const float e = __fsub_rn(r[t], w[t]);
                s = __fadd_rn(s, __fmul_rn(e, e));
            }
        if (s < best) {
            best = s;
            arg = k;
        }
    }
    codes[i * m + j] = (uint8_t)arg;
}

// ascending bitonic sort of buf[0 .. RR_SORT) by the whole CTA
__device__ void cta_bitonic_sort(uint64_t *buf) {
    for (int k = 2; k <= RR_SORT; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < RR_SORT; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = buf[i], b = buf[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(RR_THREADS) adc_rerank_kernel(
    const float *__restrict__ Q, int d, const int32_t *__restrict__ lists, int w, const int64_t *__restrict__ offsets,
    int64_t K, const int32_t *__restrict__ members, const float *__restrict__ centers,
    const uint8_t *__restrict__ codes, int m, int ks, const float *__restrict__ codebooks, int64_t L, int T,
    int32_t *__restrict__ out_ids, float *__restrict__ out_keys, int64_t *__restrict__ out_seen) {
    extern __shared__ __align__(16) uint8_t sm[];
    uint64_t *buf = (uint64_t *)sm;                             // RR_SORT: [0, T) best, then pending
    float *table = (float *)(sm + sizeof(uint64_t) * RR_SORT);  // m * ks
    float *rq = table + m * ks;                                 // d: q - c of the current list
    __shared__ unsigned pending;
    __shared__ uint64_t thr;
    const int64_t b = blockIdx.x;
    const float *q = Q + b * d;
    const int dp = d / m;
    const int cap = RR_SORT - T;  // pending slots
    for (int i = threadIdx.x; i < RR_SORT; i += blockDim.x) buf[i] = ~0ull;
    if (threadIdx.x == 0) {
        pending = 0;
        thr = ~0ull;
    }
    __syncthreads();
    int64_t seen = 0;
    for (int li = 0; li < w && seen < L; li++) {
        const int64_t c = lists[b * w + li];
        if (c < 0 || c >= K) continue;  // uniform
        const float *cv = centers + c * d;
        for (int t = threadIdx.x; t < d; t += blockDim.x) rq[t] = __fsub_rn(q[t], cv[t]);
        __syncthreads();
        for (int e = threadIdx.x; e < m * ks; e += blockDim.x) {
            const int j = e / ks, k = e - j * ks;
            const float *cw = codebooks + ((int64_t)j * ks + k) * dp;
            const float *r = rq + j * dp;
            float s = 0.0f;
            if ((dp & 3) == 0) {
                // the codeword as 16-byte loads; the same operations in the same order
                for (int t = 0; t < dp; t += 4) {
                    const float4 w4 = __ldg((const float4 *)(cw + t));
                    const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const float ee = __fsub_rn(r[t + u], ww[u]);
                        s = __fadd_rn(s, __fmul_rn(ee, ee));
                    }
                }
            } else {
                for (int t = 0; t < dp; t++) {
                    const float ee = __fsub_rn(r[t], __ldg(cw + t));
                    s = __fadd_rn(s, __fmul_rn(ee, ee));
                }
            }
            table[e] = s;
        }
        __syncthreads();
        const int64_t lo = offsets[c];
        const int64_t size = offsets[c + 1] - lo;
        const int64_t take = size < L - seen ? size : L - seen;
        for (int64_t base = 0; base < take; base += RR_CHUNK) {
            const uint64_t th = thr;
#pragma unroll
            for (int u = 0; u < RR_PER_THREAD; u++) {
                const int64_t p = base + u * RR_THREADS + threadIdx.x;
                if (p < take) {
                    const int32_t x = members[lo + p];
                    const uint8_t *cx = codes + (int64_t)x * m;
                    float key = 0.0f;
                    for (int j = 0; j < m; j++) key = __fadd_rn(key, table[j * ks + cx[j]]);
                    const uint64_t v = ((uint64_t)__float_as_uint(key) << 32) | (uint32_t)x;
                    if (v < th) buf[T + atomicAdd(&pending, 1u)] = v;
                }
            }
            __syncthreads();
            // every thread takes the count of this chunk into a register, and
            // no thread may add to it for the next chunk before all have read
            // it, so the merge decision is the same in every thread
            const unsigned pend = pending;
            __syncthreads();
            if (pend > (unsigned)(cap - RR_CHUNK)) {
                for (int i = T + (int)pend + threadIdx.x; i < RR_SORT; i += blockDim.x) buf[i] = ~0ull;
                __syncthreads();
                cta_bitonic_sort(buf);
                if (threadIdx.x == 0) {
                    thr = buf[T - 1];
                    pending = 0;
                }
                __syncthreads();
            }
        }
        seen += take;
        __syncthreads();  // the table is rebuilt for the next list
    }
    if (pending > 0) {
        for (int i = T + (int)pending + threadIdx.x; i < RR_SORT; i += blockDim.x) buf[i] = ~0ull;
        __syncthreads();
        cta_bitonic_sort(buf);
    }
    for (int r = threadIdx.x; r < T; r += blockDim.x) {
        const uint64_t v = buf[r];
        out_ids[b * T + r] = v == ~0ull ? -1 : (int32_t)(uint32_t)v;
        if (out_keys) out_keys[b * T + r] = v == ~0ull ? INFINITY : __uint_as_float((uint32_t)(v >> 32));
    }
    if (out_seen && threadIdx.x == 0) out_seen[b] = seen;
}

}  // namespace
}  // namespace ann

extern "C" int ann_pq_encode(const void *data, int dtype, int64_t N, int32_t d, const float *centers, int64_t K,
                             const int32_t *assign, int32_t m, int32_t ks, const float *codebooks, uint8_t *codes,
                             void *stream) {
    using namespace ann;
    ANN_ARG(dtype == ANN_U8 || dtype == ANN_F32, "dtype must be ANN_U8 or ANN_F32");
    ANN_ARG(N >= 0 && N < (1ll << 31), "N out of range");
    ANN_ARG(m >= 1 && m <= 65535 && d >= m && d % m == 0, "d must be a positive multiple of m");
    ANN_ARG(d / m <= ENC_MAX_DP, "at most 32 dims per part");
    ANN_ARG(ks >= 1 && ks <= 256, "ks must be in [1, 256]");
    ANN_ARG(K >= 1, "K must be >= 1");
    ANN_ARG(N == 0 || (data && centers && assign && codebooks && codes), "null pointer");
    if (N == 0) return ANN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(float) * (size_t)ks * (size_t)(d / m);
    dim3 grid((unsigned)((N + ENC_THREADS - 1) / ENC_THREADS), (unsigned)m);
    if (dtype == ANN_U8)
        pq_encode_kernel<ANN_U8><<<grid, ENC_THREADS, smem, s>>>(data, N, d, centers, K, assign, m, ks,
                                                                 codebooks, codes);
    else
        pq_encode_kernel<ANN_F32><<<grid, ENC_THREADS, smem, s>>>(data, N, d, centers, K, assign, m, ks,
                                                                  codebooks, codes);
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

extern "C" int ann_adc_rerank(const float *queries, int64_t nq, int32_t d, const int32_t *lists, int32_t w,
                              const int64_t *offsets, int64_t K, const int32_t *members, const float *centers,
                              const uint8_t *codes, int32_t m, int32_t ks, const float *codebooks, int64_t L,
                              int32_t T, int32_t *out_ids, float *out_keys, int64_t *out_seen, void *stream) {
    using namespace ann;
    ANN_ARG(nq >= 0 && nq < (1ll << 31), "nq out of range");
    ANN_ARG(m >= 1 && m <= 64 && d >= m && d % m == 0, "d must be a multiple of m, m <= 64");
    ANN_ARG(ks >= 1 && ks <= 256, "ks must be in [1, 256]");
    ANN_ARG(T >= 1 && T <= RR_MAX_T, "T must be in [1, 128]");
    ANN_ARG(w >= 1 && K >= 1 && L >= 0, "w >= 1, K >= 1, L >= 0");
    ANN_ARG(nq == 0 || (queries && lists && offsets && members && centers && codes && codebooks && out_ids),
            "null pointer");
    if (nq == 0) return ANN_OK;
    int dev = 0, optin = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    ANN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t smem = sizeof(uint64_t) * RR_SORT + sizeof(float) * ((size_t)m * (size_t)ks + (size_t)d);
    ANN_ARG(smem + 64 <= (size_t)optin, "m * ks tables too large for shared memory");
    cudaStream_t s = (cudaStream_t)stream;
    ANN_CUDA(cudaFuncSetAttribute(adc_rerank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    adc_rerank_kernel<<<(unsigned)nq, RR_THREADS, smem, s>>>(queries, d, lists, w, offsets, K, members, centers, codes,
                                                             m, ks, codebooks, L, T, out_ids, out_keys, out_seen);
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}
