// ann_knn_f32.cu -- exact k-NN of float32 rows (ground truth of Sec. 5.1 and
// the exact R-NN graph of Sec. 3.1 / Sec. 4.1) with the dot products on the
// tensor cores.
//
// Keys are the float32 nearest to the exact squared distance, exactly as in
// the SIMT kernel of ann_knn.cu.  The tensor cores only choose candidates:
//   1. Every row is split into bf16 parts, x = xh + xl + (dropped rest);
//      one bf16 tensor-core GEMM (cuBLAS, float32 accumulation) over the
//      concatenations [xh | xh | xl] and [qh | ql | qh] (inner length 3 d)
//      gives <q, x> ~ qh.xh + ql.xh + qh.xl for a tile of query rows against
//      every reference row; the approximate key a(x) = |q|^2 + |x|^2 - 2<q, x> is off
//      the exact one by at most eps(q) (a bound from the dropped terms and the
//      accumulation length, times a safety factor; see eps_row).
//   2. Pass 1: a warp per query row finds a_k, the k-th smallest a(x).  The k
//      references with a(x) <= a_k have exact keys <= a_k + eps, so the true
//      k-th key is <= a_k + eps, and every true neighbour y has
//      a(y) <= exact(y) + eps <= a_k + 2 eps.
//   3. Pass 2: every x with a(x) <= a_k + 2 eps is a candidate (at most
//      kCap per row); the candidates' exact keys (double-float, one
//      rounding) decide the k smallest by (key, id).
// Rows whose candidate list overflows are recomputed by the exact SIMT kernel.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {

constexpr int kCap = 512;  // candidates per row kept for exact rescoring

static std::mutex g_blas_mu;
static cublasHandle_t g_blas[64];
static std::mutex g_blas_use[64];  // a handle's stream is set per call: one caller at a time

static int blas_handle(cublasHandle_t *out) {
    int dev = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(ANN_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_blas_mu);
    if (!g_blas[dev]) {
        if (cublasCreate(&g_blas[dev]) != CUBLAS_STATUS_SUCCESS) return fail(ANN_ERR_CUDA, "cublasCreate failed");
    }
    *out = g_blas[dev];
    return ANN_OK;
}

// |x|^2 of every row in fp64 (products of floats are exact in fp64)
__global__ void norms_f32_kernel(const float *X, int64_t N, int d, double *n64, float *n32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float *row = X + i * d;
    double s = 0.0;
    for (int j = 0; j < d; j++) {
        const double v = (double)__ldg(row + j);
        s += v * v;
    }
    n64[i] = s;
    n32[i] = (float)s;
}

__global__ void max_norm_kernel(const double *n64, int64_t N, unsigned long long *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) atomicMax(out, (unsigned long long)__double_as_longlong(n64[i]));  // non-negative doubles order as bits
}

// split x into bf16 xh = rn(x) and xl = rn(x - xh), |x - xh - xl| <= 2^-18 |x|,
// and store each row as three blocks of d: (h, h, l) for references,
// (h, l, h) for queries, so that one inner product of length 3 d pairs
// xh.qh + xh.ql + xl.qh
__global__ void split_bf16_kernel(const float *X, int64_t rows, int d, int query_order, __nv_bfloat16 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * d) return;
    const int64_t r = i / d;
    const int j = (int)(i - r * d);
    const float v = X[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    __nv_bfloat16 *o = out + r * 3 * d;
    o[j] = h;
    o[d + j] = query_order ? l : h;
    o[2 * d + j] = query_order ? h : l;
}

// Error bound of a(x) for query norm qn and the largest reference norm xn.
// Per coordinate the three products miss at most 3 * 2^-18 |q_i x_i| (the
// dropped ql.xl term and the rounding of ql, xl); the float32 sum of the
// n = 3 d + 16 rounded terms adds at most gamma_n times their magnitudes.
// All magnitudes sum to at most (qn + xn) / 2 (Cauchy-Schwarz), and the key
// doubles the dot product; the bound is then taken four times over.
__device__ __forceinline__ double eps_row(int d, double qn, double xn) {
    const double u = 1.0 / 16777216.0;
    const double n = 3.0 * d + 16.0;
    return 4.0 * (n * u / (1.0 - n * u) + 3.0 / 262144.0) * (qn + xn) + 1e-30;
}

__device__ __forceinline__ float approx_key(float dot, float qn, float xn) {
    const float a = qn + xn - 2.0f * dot;
    return a > 0.f ? a : 0.f;
}

// Both passes give each row one CTA of kSegWarps warps; warp w scans columns
// [w * seg, (w + 1) * seg) of the row, kUnroll loads in flight per lane.
constexpr int kSegWarps = 4;
constexpr int kUnroll = 8;

__device__ __forceinline__ void list_insert_k(uint64_t &mine, uint64_t &thr, uint64_t cv, int k) {
    const int lane = threadIdx.x & 31;
    const int pos = __popc(__ballot_sync(0xffffffffu, mine < cv));
    const uint64_t up = __shfl_up_sync(0xffffffffu, mine, 1);
    if (lane == pos) mine = cv;
    else if (lane > pos) mine = up;
    thr = __shfl_sync(0xffffffffu, mine, k - 1);
}

// Pass 1: the k-th smallest approximate key of each row (ties by id).  D holds
// the tile's rows (row r at D + r * N).  Each warp keeps the k best of its
// segment in a sorted warp list (entry `lane`); warp 0 merges the lists.
__global__ void __launch_bounds__(32 * kSegWarps) f32_kth_kernel(const float *D, int64_t rows, int64_t q0, int64_t N,
                                                                 const float *qn32, const float *rn32,
                                                                 int exclude_self, int k, float *akth) {
    __shared__ uint64_t lists[kSegWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = blockIdx.x;
    if (r >= rows) return;
    const int64_t q = q0 + r;
    const float qn = qn32[q];
    const float *row = D + r * N;
    const int64_t seg = ((N + kSegWarps - 1) / kSegWarps + 31) / 32 * 32;
    const int64_t cbeg = warp * seg, cend = cbeg + seg < N ? cbeg + seg : N;
    uint64_t mine = ~0ull, thr = ~0ull;
    for (int64_t c0 = cbeg; c0 < cend; c0 += 32 * kUnroll) {  // warp-uniform bounds
        float dv[kUnroll], xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int64_t c = c0 + 32 * u + lane;
            dv[u] = c < cend ? __ldg(row + c) : 0.f;
            xv[u] = c < cend ? __ldg(rn32 + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int64_t c = c0 + 32 * u + lane;
            uint64_t v = ~0ull;
            if (c < cend && !(exclude_self && c == q))
                v = ((uint64_t)__float_as_uint(approx_key(dv[u], qn, xv[u])) << 32) | (uint32_t)c;
            unsigned m = __ballot_sync(0xffffffffu, v < thr);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const uint64_t cv = __shfl_sync(0xffffffffu, v, src);
                if (cv < thr) list_insert_k(mine, thr, cv, k);
            }
        }
    }
    lists[warp][lane] = mine;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < kSegWarps; w++) {
            const uint64_t v = lists[w][lane];
            unsigned m = __ballot_sync(0xffffffffu, v < thr);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const uint64_t cv = __shfl_sync(0xffffffffu, v, src);
                if (cv < thr) list_insert_k(mine, thr, cv, k);
            }
        }
        if (lane == 0) akth[r] = thr == ~0ull ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(thr >> 32));
    }
}

// Pass 2: candidates a(x) <= a_k + 2 eps (any order, at most kCap stored).
__global__ void __launch_bounds__(32 * kSegWarps) f32_cand_kernel(const float *D, int64_t rows, int64_t q0, int64_t N,
                                                                  int d, const float *qn32, const float *rn32,
                                                                  const double *qn64, const unsigned long long *xmax,
                                                                  int exclude_self, const float *akth, uint32_t *cand,
                                                                  int32_t *ncand) {
    __shared__ int cnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = blockIdx.x;
    if (r >= rows) return;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int64_t q = q0 + r;
    const float qn = qn32[q];
    const double e = eps_row(d, qn64[q], __longlong_as_double((long long)*xmax));
    const double lim = (double)akth[r] + 2.0 * e;
    // compare in float32 against the limit rounded up: never fewer candidates
    // than the fp64 comparison (fp64 throughput is low on this part)
    float limf = (float)lim;
    if ((double)limf < lim) limf = nextafterf(limf, __int_as_float(0x7f800000));
    const float *row = D + r * N;
    uint32_t *out = cand + r * kCap;
    const int64_t seg = ((N + kSegWarps - 1) / kSegWarps + 31) / 32 * 32;
    const int64_t cbeg = warp * seg, cend = cbeg + seg < N ? cbeg + seg : N;
    for (int64_t c0 = cbeg; c0 < cend; c0 += 32 * kUnroll) {  // warp-uniform bounds
        float dv[kUnroll], xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int64_t c = c0 + 32 * u + lane;
            dv[u] = c < cend ? __ldg(row + c) : 0.f;
            xv[u] = c < cend ? __ldg(rn32 + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const int64_t c = c0 + 32 * u + lane;
            const bool take = c < cend && !(exclude_self && c == q) && approx_key(dv[u], qn, xv[u]) <= limf;
            const unsigned m = __ballot_sync(0xffffffffu, take);
            if (m) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&cnt, __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                const int pos = base + __popc(m & ((1u << lane) - 1));
                if (take && pos < kCap) out[pos] = (uint32_t)c;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) ncand[r] = cnt;
}

// Exact keys of the candidates and the k smallest by (key, id).  Rows whose
// candidates overflowed go to the fallback list.
__global__ void f32_rescore_kernel(const float *X, const float *Qm, int d, int64_t rows, int64_t q0,
                                   const uint32_t *cand, const int32_t *ncand, int k, int32_t *out_ids,
                                   uint32_t *out_keys, int32_t *fb_rows, int32_t *fb_count) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= rows) return;
    const int64_t q = q0 + r;
    const int nc = ncand[r];
    if (nc > kCap) {
        if (lane == 0) fb_rows[atomicAdd(fb_count, 1)] = (int32_t)q;
        return;
    }
    const float *qv = Qm + q * d;
    uint64_t mine = ~0ull;
    for (int b0 = 0; b0 < nc; b0 += 32) {
        const int i = b0 + lane;
        uint64_t v = ~0ull;
        if (i < nc) {
            const uint32_t x = cand[r * kCap + i];
            const float *xv = X + (int64_t)x * d;
            float hi = 0.f, lo = 0.f;
            for (int j = 0; j < d; j++) df_acc_sqdiff(__ldg(xv + j), __ldg(qv + j), hi, lo);
            v = ((uint64_t)__float_as_uint(__fadd_rn(hi, lo)) << 32) | x;
        }
        unsigned m = __ballot_sync(0xffffffffu, v < __shfl_sync(0xffffffffu, mine, k - 1));
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t cv = __shfl_sync(0xffffffffu, v, src);
            if (cv < __shfl_sync(0xffffffffu, mine, k - 1)) {
                const int pos = __popc(__ballot_sync(0xffffffffu, mine < cv));
                const uint64_t up = __shfl_up_sync(0xffffffffu, mine, 1);
                if (lane == pos) mine = cv;
                else if (lane > pos) mine = up;
            }
        }
    }
    if (lane < k) {
        const bool have = mine != ~0ull;
        out_ids[q * k + lane] = have ? (int32_t)(uint32_t)mine : -1;
        if (out_keys) out_keys[q * k + lane] = have ? (uint32_t)(mine >> 32) : 0x7f800000u;
    }
}

// implemented in ann_knn.cu: exact SIMT k-NN of the selected query rows
int knn_f32_rows(const float *refs, int64_t N, const float *queries, const int32_t *rows, int64_t nrows, int d,
                 int k, int exclude_self, int32_t *out_ids, uint32_t *out_keys, cudaStream_t s);

int knn_f32_tensor(const float *refs, int64_t N, const float *queries, int64_t nq, int d, int k, int exclude_self,
                   int32_t *out_ids, uint32_t *out_keys, cudaStream_t s) {
    cublasHandle_t h;
    int rc = blas_handle(&h);
    if (rc != ANN_OK) return rc;
    int dev = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> use(g_blas_use[dev]);
    // tile of query rows: the tile's dot products take at most 2^31 floats
    int64_t tm = std::max<int64_t>(32, std::min<int64_t>(nq, ((int64_t)1 << 31) / N) / 32 * 32);
    if (tm > nq) tm = nq;
    const bool shared = queries == refs && nq <= N;  // queries are the first nq reference rows
    __nv_bfloat16 *x3 = nullptr, *q3 = nullptr;
    double *rn64 = nullptr, *qn64 = nullptr;
    float *rn32 = nullptr, *qn32 = nullptr, *D = nullptr, *akth = nullptr;
    unsigned long long *xmax = nullptr;
    uint32_t *cand = nullptr;
    int32_t *ncand = nullptr, *fb_rows = nullptr, *fb_count = nullptr;
    auto release = [&]() {
        void *ps[] = {rn64, rn32, shared ? nullptr : qn64, shared ? nullptr : qn32, D, akth, xmax, cand, ncand,
                      fb_rows, fb_count, x3, q3};
        for (void *p : ps)
            if (p) cudaFreeAsync(p, s);
    };
#define F32_ALLOC(p, bytes)                                                     \
    do {                                                                        \
        cudaError_t _e = cudaMallocAsync((void **)&(p), (bytes), s);            \
        if (_e != cudaSuccess) {                                                \
            release();                                                          \
            return cuda_fail(_e, "cudaMallocAsync(float32 k-NN workspace)");    \
        }                                                                       \
    } while (0)
    F32_ALLOC(rn64, 8 * N);
    F32_ALLOC(rn32, 4 * N);
    if (shared) {
        qn64 = rn64;
        qn32 = rn32;
    } else {
        F32_ALLOC(qn64, 8 * nq);
        F32_ALLOC(qn32, 4 * nq);
    }
    F32_ALLOC(D, 4 * (size_t)tm * N);
    F32_ALLOC(akth, 4 * tm);
    F32_ALLOC(xmax, 8);
    F32_ALLOC(cand, 4 * (size_t)tm * kCap);
    F32_ALLOC(ncand, 4 * tm);
    F32_ALLOC(fb_rows, 4 * nq);
    F32_ALLOC(fb_count, 4);
    F32_ALLOC(x3, 6 * (size_t)N * d);
    F32_ALLOC(q3, 6 * (size_t)nq * d);
#undef F32_ALLOC
    split_bf16_kernel<<<(unsigned)((N * d + 255) / 256), 256, 0, s>>>(refs, N, d, 0, x3);
    split_bf16_kernel<<<(unsigned)((nq * d + 255) / 256), 256, 0, s>>>(queries, nq, d, 1, q3);
    norms_f32_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(refs, N, d, rn64, rn32);
    if (!shared) norms_f32_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(queries, nq, d, qn64, qn32);
    cudaMemsetAsync(xmax, 0, 8, s);
    cudaMemsetAsync(fb_count, 0, 4, s);
    max_norm_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(rn64, N, xmax);
    if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) {
        release();
        return fail(ANN_ERR_CUDA, "cublasSetStream failed");
    }
    const float one = 1.f, zero = 0.f;
    for (int64_t q0 = 0; q0 < nq; q0 += tm) {
        const int64_t rows = std::min<int64_t>(tm, nq - q0);
        // D (column-major N x rows) = X3^T Q3: row r of the tile is D + r * N
        const cublasStatus_t st = cublasGemmEx(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)N, (int)rows, 3 * d, &one, x3,
                                               CUDA_R_16BF, 3 * d, q3 + q0 * 3 * d, CUDA_R_16BF, 3 * d, &zero, D,
                                               CUDA_R_32F, (int)N, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
        if (st != CUBLAS_STATUS_SUCCESS) {
            release();
            return fail(ANN_ERR_CUDA, "cublasGemmEx (float32 k-NN) failed: status " + std::to_string((int)st));
        }
        const unsigned grid = (unsigned)((rows * 32 + 255) / 256);
        f32_kth_kernel<<<(unsigned)rows, 32 * kSegWarps, 0, s>>>(D, rows, q0, N, qn32, rn32, exclude_self, k, akth);
        f32_cand_kernel<<<(unsigned)rows, 32 * kSegWarps, 0, s>>>(D, rows, q0, N, d, qn32, rn32, qn64, xmax,
                                                                 exclude_self, akth, cand, ncand);
        f32_rescore_kernel<<<grid, 256, 0, s>>>(refs, queries, d, rows, q0, cand, ncand, k, out_ids, out_keys,
                                                fb_rows, fb_count);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            release();
            return cuda_fail(e, "float32 k-NN kernels");
        }
    }
    int32_t nfb = 0;
    cudaError_t e = cudaMemcpyAsync(&nfb, fb_count, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "float32 k-NN fallback count");
    }
    if (nfb > 0) rc = knn_f32_rows(refs, N, queries, fb_rows, nfb, d, k, exclude_self, out_ids, out_keys, s);
    release();
    return rc;
}

}  // namespace ann
