// ann_knn.cu -- exact k nearest neighbours by linear scan on sm_103a: the
// ground truth of Sec. 5.1 and, with self excluded, the exact R-NN
// neighbourhood graph of Sec. 3.1 / Sec. 4.1.
//
// A CTA owns 64 query rows and streams every reference row through shared
// memory in tiles of 64.  Keys are exact: uint8 rows use
// ||a||^2 + ||b||^2 - 2 a.b with __dp4a (integers, no rounding); float32 rows
// accumulate (a - b)^2 in double-float and round once to float32.  Each warp
// keeps the running k best (key, id) of its 8 rows in registers, one entry per
// lane, and merges every tile's candidates with ballots.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {

constexpr int KB_M = 64;   // query rows per CTA
constexpr int KB_N = 64;   // reference rows per tile
constexpr int KB_THREADS = 256;

__global__ void norms_u8_kernel(const uint8_t *X, int64_t N, int d, uint32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t *row = (const uint32_t *)(X + i * d);
    uint32_t s = 0;
    for (int w = 0; w < d / 4; w++) {
        uint32_t v = __ldg(row + w);
        s = __dp4a(v, v, s);
    }
    out[i] = s;
}

// insert candidate v into the warp-held ascending list (entry `lane` in `mine`)
__device__ __forceinline__ void list_insert(uint64_t &mine, uint64_t v) {
    const int lane = lane_id();
    unsigned lt = __ballot_sync(0xffffffffu, mine < v);
    int pos = __popc(lt);
    uint64_t up = __shfl_up_sync(0xffffffffu, mine, 1);
    if (lane == pos) mine = v;
    else if (lane > pos) mine = up;
}

__device__ __forceinline__ void merge_row(uint64_t &mine, const uint32_t *drow, int64_t ref0, int nvalid,
                                          int64_t self_id, int k) {
    const int lane = lane_id();
    for (int half = 0; half < KB_N / 32; half++) {
        int c = half * 32 + lane;
        uint64_t v = ~0ull;
        if (c < nvalid && ref0 + c != self_id) v = ((uint64_t)drow[c] << 32) | (uint32_t)(ref0 + c);
        uint64_t thr = __shfl_sync(0xffffffffu, mine, k - 1);
        unsigned m = __ballot_sync(0xffffffffu, v < thr);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1;
            uint64_t cv = __shfl_sync(0xffffffffu, v, src);
            uint64_t t2 = __shfl_sync(0xffffffffu, mine, k - 1);
            if (cv < t2) list_insert(mine, cv);
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(KB_THREADS) knn_kernel(const void *refs, int64_t N, const void *queries, int64_t nq,
                                                       int d, int k, int exclude_self, const uint32_t *rnorm,
                                                       const uint32_t *qnorm, int32_t *out_ids, uint32_t *out_keys,
                                                       const int32_t *qsel = nullptr) {
    // qsel (optional): the tile's row i is query row qsel[i] (its id for
    // exclude_self and its output row); otherwise row i itself
#define QROW(i) (qsel ? (int64_t)qsel[(i)] : (int64_t)(i))
    extern __shared__ __align__(16) uint8_t sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * KB_M;
    const int qrows = (int)(nq - q0 < KB_M ? nq - q0 : KB_M);
    // tile layout: words per row, padded by 4 words to spread banks
    const int KW = DT == ANN_U8 ? d / 4 : 64;  // f32 streams K in chunks of 64 floats
    const int SW = KW + 4;
    uint32_t *As = (uint32_t *)sm;
    uint32_t *Bs = As + KB_M * SW;
    uint32_t *Ds = Bs + KB_N * SW;   // KB_M x (KB_N + 1)
    uint32_t *qn = Ds + KB_M * (KB_N + 1);
    uint32_t *rn = qn + KB_M;
    const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 4x4 outputs each

    uint64_t mine[KB_M / 8];
#pragma unroll
    for (int r = 0; r < KB_M / 8; r++) mine[r] = ~0ull;

    if (DT == ANN_U8) {
        // queries stay resident
        const int words = d / 4;
        for (int i = tid; i < KB_M * words; i += KB_THREADS) {
            int r = i / words, w = i % words;
            As[r * SW + w] = r < qrows ? __ldg((const uint32_t *)((const uint8_t *)queries + QROW(q0 + r) * d) + w) : 0u;
        }
        for (int r = tid; r < KB_M; r += KB_THREADS) qn[r] = r < qrows ? qnorm[QROW(q0 + r)] : 0u;
    }
    for (int64_t r0 = 0; r0 < N; r0 += KB_N) {
        const int nvalid = (int)(N - r0 < KB_N ? N - r0 : KB_N);
        uint32_t acc[4][4];
        float hi[4][4], lo[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                acc[i][j] = 0;
                hi[i][j] = 0.f;
                lo[i][j] = 0.f;
            }
        if (DT == ANN_U8) {
            const int words = d / 4;
            __syncthreads();
            for (int i = tid; i < KB_N * words; i += KB_THREADS) {
                int r = i / words, w = i % words;
                Bs[r * SW + w] = r < nvalid ? __ldg((const uint32_t *)((const uint8_t *)refs + (r0 + r) * d) + w) : 0u;
            }
            for (int r = tid; r < KB_N; r += KB_THREADS) rn[r] = r < nvalid ? rnorm[r0 + r] : 0u;
            __syncthreads();
            for (int w = 0; w < words; w += 4) {
                uint4 a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = *(const uint4 *)&As[(ty * 4 + i) * SW + w];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = *(const uint4 *)&Bs[(tx * 4 + j) * SW + w];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        acc[i][j] = __dp4a(a[i].x, b[j].x, acc[i][j]);
                        acc[i][j] = __dp4a(a[i].y, b[j].y, acc[i][j]);
                        acc[i][j] = __dp4a(a[i].z, b[j].z, acc[i][j]);
                        acc[i][j] = __dp4a(a[i].w, b[j].w, acc[i][j]);
                    }
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    int r = ty * 4 + i, c = tx * 4 + j;
                    Ds[r * (KB_N + 1) + c] = qn[r] + rn[c] - 2u * acc[i][j];
                }
        } else {
            const float *Q = (const float *)queries;
            const float *X = (const float *)refs;
            for (int k0 = 0; k0 < d; k0 += 64) {
                const int kc = d - k0 < 64 ? d - k0 : 64;
                __syncthreads();
                for (int i = tid; i < KB_M * 64; i += KB_THREADS) {
                    int r = i / 64, w = i % 64;
                    As[r * SW + w] = (r < qrows && w < kc) ? __float_as_uint(__ldg(Q + QROW(q0 + r) * d + k0 + w)) : 0u;
                }
                for (int i = tid; i < KB_N * 64; i += KB_THREADS) {
                    int r = i / 64, w = i % 64;
                    Bs[r * SW + w] = (r < nvalid && w < kc) ? __float_as_uint(__ldg(X + (r0 + r) * d + k0 + w)) : 0u;
                }
                __syncthreads();
                for (int w = 0; w < kc; w++) {
                    float a[4], b[4];
#pragma unroll
                    for (int i = 0; i < 4; i++) a[i] = __uint_as_float(As[(ty * 4 + i) * SW + w]);
#pragma unroll
                    for (int j = 0; j < 4; j++) b[j] = __uint_as_float(Bs[(tx * 4 + j) * SW + w]);
#pragma unroll
                    for (int i = 0; i < 4; i++)
#pragma unroll
                        for (int j = 0; j < 4; j++) df_acc_sqdiff(a[i], b[j], hi[i][j], lo[i][j]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    int r = ty * 4 + i, c = tx * 4 + j;
                    Ds[r * (KB_N + 1) + c] = __float_as_uint(__fadd_rn(hi[i][j], lo[i][j]));
                }
        }
        __syncthreads();
        // merge: warp w owns rows w*8 .. w*8+7
#pragma unroll
        for (int rr = 0; rr < KB_M / 8; rr++) {
            int r = warp * (KB_M / 8) + rr;
            if (r < qrows)
                merge_row(mine[rr], &Ds[r * (KB_N + 1)], r0, nvalid, exclude_self ? QROW(q0 + r) : -1, k);
        }
    }
#pragma unroll
    for (int rr = 0; rr < KB_M / 8; rr++) {
        int r = warp * (KB_M / 8) + rr;
        if (r < qrows && lane < k) {
            uint64_t v = mine[rr];
            bool have = v != ~0ull;
            out_ids[QROW(q0 + r) * k + lane] = have ? (int32_t)(uint32_t)v : -1;
            if (out_keys)
                out_keys[QROW(q0 + r) * k + lane] =
                    have ? (uint32_t)(v >> 32) : (DT == ANN_U8 ? 0xffffffffu : 0x7f800000u);
        }
    }
#undef QROW
}

// exact SIMT k-NN of the selected float32 query rows (fallback of the
// tensor-core path for rows it cannot certify)
int knn_f32_rows(const float *refs, int64_t N, const float *queries, const int32_t *rows, int64_t nrows, int d,
                 int k, int exclude_self, int32_t *out_ids, uint32_t *out_keys, cudaStream_t s) {
    const int SW = 64 + 4;
    size_t smem = 4 * ((size_t)(KB_M + KB_N) * SW + (size_t)KB_M * (KB_N + 1) + KB_M + KB_N);
    ANN_CUDA(cudaFuncSetAttribute(knn_kernel<ANN_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    knn_kernel<ANN_F32><<<(unsigned)((nrows + KB_M - 1) / KB_M), KB_THREADS, smem, s>>>(
        refs, N, queries, nrows, d, k, exclude_self, nullptr, nullptr, out_ids, out_keys, rows);
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

// implemented in ann_knn_f32.cu
int knn_f32_tensor(const float *refs, int64_t N, const float *queries, int64_t nq, int d, int k, int exclude_self,
                   int32_t *out_ids, uint32_t *out_keys, cudaStream_t s);

}  // namespace ann

using namespace ann;

extern "C" int ann_exact_knn(const void *refs, int64_t N, const void *queries, int64_t nq, int dtype, int32_t d,
                             int32_t k, int32_t exclude_self, int32_t *out_ids, void *out_keys, void *stream) {
    ANN_ARG(dtype == ANN_U8 || dtype == ANN_F32, "dtype must be ANN_U8 or ANN_F32");
    ANN_ARG(N >= 1 && N < (1ll << 31) && nq >= 0 && nq < (1ll << 31), "N or nq out of range");
    ANN_ARG(k >= 1 && k <= 32, "k must be in [1, 32]");
    ANN_ARG(dtype == ANN_U8 ? (d >= 16 && d % 16 == 0) : (d >= 4 && d % 4 == 0),
            "d must be a multiple of 16 (u8) or 4 (f32)");
    ANN_ARG(refs && (nq == 0 || (queries && out_ids)), "refs, queries and out_ids are required");
    ANN_ARG(!exclude_self || (queries == refs && nq == N), "exclude_self needs queries == refs");
    if (nq == 0) return ANN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == ANN_U8 && (d == 64 || d == 128) && knn_u8_tensor_fits(d, k))
        return knn_u8_tensor((const uint8_t *)refs, N, (const uint8_t *)queries, nq, d, k, exclude_self, out_ids,
                             (uint32_t *)out_keys, s);
    // float32 at scale: candidates from tensor-core dot products, exact keys
    if (dtype == ANN_F32 && N >= 8192 && nq >= 256)
        return knn_f32_tensor((const float *)refs, N, (const float *)queries, nq, d, k, exclude_self, out_ids,
                              (uint32_t *)out_keys, s);
    uint32_t *rn = nullptr, *qn = nullptr;
    AsyncBufs bufs(s);  // released on return
    if (dtype == ANN_U8) {
        ANN_CUDA(bufs.alloc(&rn, 4 * N));
        norms_u8_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>((const uint8_t *)refs, N, d, rn);
        if (queries == refs && nq <= N) {  // the query rows are the first nq reference rows
            qn = rn;
        } else {
            ANN_CUDA(bufs.alloc(&qn, 4 * nq));
            norms_u8_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>((const uint8_t *)queries, nq, d, qn);
        }
    }
    const int KW = dtype == ANN_U8 ? d / 4 : 64;
    const int SW = KW + 4;
    size_t smem = 4 * ((size_t)(KB_M + KB_N) * SW + (size_t)KB_M * (KB_N + 1) + KB_M + KB_N);
    unsigned grid = (unsigned)((nq + KB_M - 1) / KB_M);
    if (dtype == ANN_U8) {
        ANN_CUDA(cudaFuncSetAttribute(knn_kernel<ANN_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        knn_kernel<ANN_U8><<<grid, KB_THREADS, smem, s>>>(refs, N, queries, nq, d, k, exclude_self, rn, qn, out_ids,
                                                          (uint32_t *)out_keys);
    } else {
        ANN_CUDA(cudaFuncSetAttribute(knn_kernel<ANN_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        knn_kernel<ANN_F32><<<grid, KB_THREADS, smem, s>>>(refs, N, queries, nq, d, k, exclude_self, rn, qn, out_ids,
                                                           (uint32_t *)out_keys);
    }
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

extern "C" int ann_build_knn_graph(const void *data, int dtype, int64_t N, int32_t d, int32_t R, int32_t *out_ids,
                                   void *out_keys, void *stream) {
    return ann_exact_knn(data, N, data, N, dtype, d, R, 1, out_ids, out_keys, stream);
}

// ---------------------------------------------------------------------------
// Exact k-NN without any allocation: the row norms live in a file-scope
// device array instead of memory obtained from cudaMallocAsync.  Meant for
// callers that may not allocate device memory themselves, such as a host
// program whose device memory is owned entirely by another allocator (a
// framework's caching allocator or a fixed pool that must remain the only
// owner), or a latency-critical loop that cannot afford an allocation's
// device-wide synchronisation and unbounded latency.
// ---------------------------------------------------------------------------
namespace ann {

static const int64_t kStaticNormRows = 1 << 20;  // 4 MiB of uint32 norms
static __device__ __align__(256) uint32_t g_static_norms[kStaticNormRows];

static std::mutex g_static_mu;
static uint32_t *g_static_ptr[64];  // device address of g_static_norms, per device ordinal

// Device address of the array on the current device; looked up once per device.
static int static_norms_ptr(uint32_t **out) {
    int dev = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(ANN_ERR_ARG, "device ordinal out of range for the static scratch table");
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_norms);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static norms)");
        g_static_ptr[dev] = (uint32_t *)p;
    }
    *out = g_static_ptr[dev];
    return ANN_OK;
}

}  // namespace ann

extern "C" int ann_exact_knn_static(const void *refs, int64_t N, const void *queries, int64_t nq, int dtype,
                                    int32_t d, int32_t k, int32_t exclude_self, int32_t *out_ids, void *out_keys,
                                    void *stream) {
    ANN_ARG(dtype == ANN_U8 || dtype == ANN_F32, "dtype must be ANN_U8 or ANN_F32");
    ANN_ARG(N >= 1 && N < (1ll << 31) && nq >= 0 && nq < (1ll << 31), "N or nq out of range");
    ANN_ARG(k >= 1 && k <= 32, "k must be in [1, 32]");
    ANN_ARG(dtype == ANN_U8 ? (d >= 16 && d % 16 == 0) : (d >= 4 && d % 4 == 0),
            "d must be a multiple of 16 (u8) or 4 (f32)");
    ANN_ARG(refs && (nq == 0 || (queries && out_ids)), "refs, queries and out_ids are required");
    ANN_ARG(!exclude_self || (queries == refs && nq == N), "exclude_self needs queries == refs");
    // the queries reuse the reference norms only when they are the first nq
    // reference rows; a longer query buffer at the same address gets its own
    const bool shared = queries == refs && nq <= N;
    const int64_t rows = dtype == ANN_U8 ? N + (shared ? 0 : nq) : 0;
    if (rows > kStaticNormRows)
        return fail(ANN_ERR_CAPACITY, "ann_exact_knn_static: N (+ nq when queries differ from refs) exceeds the "
                                      "static scratch of 1048576 rows; use ann_exact_knn");
    if (nq == 0) return ANN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *rn = nullptr, *qn = nullptr;
    if (dtype == ANN_U8) {
        uint32_t *base = nullptr;
        int r = static_norms_ptr(&base);
        if (r != ANN_OK) return r;
        // every norm used below is written here first: nothing must start at zero
        rn = base;
        qn = shared ? rn : base + N;
        norms_u8_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>((const uint8_t *)refs, N, d, rn);
        if (!shared)
            norms_u8_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>((const uint8_t *)queries, nq, d, qn);
    }
    const int KW = dtype == ANN_U8 ? d / 4 : 64;
    const int SW = KW + 4;
    size_t smem = 4 * ((size_t)(KB_M + KB_N) * SW + (size_t)KB_M * (KB_N + 1) + KB_M + KB_N);
    unsigned grid = (unsigned)((nq + KB_M - 1) / KB_M);
    if (dtype == ANN_U8) {
        ANN_CUDA(cudaFuncSetAttribute(knn_kernel<ANN_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        knn_kernel<ANN_U8><<<grid, KB_THREADS, smem, s>>>(refs, N, queries, nq, d, k, exclude_self, rn, qn, out_ids,
                                                          (uint32_t *)out_keys);
    } else {
        ANN_CUDA(cudaFuncSetAttribute(knn_kernel<ANN_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        knn_kernel<ANN_F32><<<grid, KB_THREADS, smem, s>>>(refs, N, queries, nq, d, k, exclude_self, rn, qn, out_ids,
                                                           (uint32_t *)out_keys);
    }
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}
