// ann_knn_approx.cu -- approximate R-NN neighbourhood graph of uint8 rows on
// sm_103a.  Sec. 5.3 builds its neighbourhood graphs with an approximate
// construction (random divide-and-conquer, then neighbourhood propagation;
// Sec. 5.5 puts its cost at O(N log N)); the steps are fixed as follows.
//
//  1. `rounds` random partitions.  Positions [0, N) are halved recursively
//     `levels` times (segment [lo, hi) -> [lo, m), [m, hi), m = lo + (hi-lo)/2).
//     At level l every segment s reorders its members ascending by
//     (<u, x>, id), u = dirs[round][2^l - 1 + s].  One level is one radix sort
//     of the 64-bit keys (segment, <u, x> + bias, id) over all N positions:
//     a segment's members occupy the same positions before and after, so a
//     global sort is the per-segment sort.
//  2. Leaf step: every point is offered every other leaf member.  A leaf that
//     fits in shared memory is staged whole by one CTA (one warp per point);
//     a larger one (d <= 128) is streamed through shared memory by CTAs of
//     32 members each, two per warp.
//  3. `iters` propagation steps (one warp per point): row i is offered the
//     rows of its neighbours, read from the previous step's graph.
// A row is a warp-held ascending list of packed (key << 32 | id) values, one
// per lane; offering keeps the R smallest with distinct ids, so every row is
// the R best of all candidates offered, whatever the order -- the result is
// deterministic and bit-exact against a plain CPU statement.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cub/device/device_radix_sort.cuh>
#include <utility>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {
namespace {

constexpr int LEAF_THREADS = 512;
constexpr int PROP_THREADS = 256;
constexpr int TILE_THREADS = 512;
constexpr int TILE_I = 2 * TILE_THREADS / 32;  // members per CTA of the streamed leaf kernel
constexpr int TILE_J = 256;                    // leaf rows per shared-memory pass
constexpr unsigned FULL = 0xffffffffu;

// sum of x_b * u_b over 4 byte pairs: x unsigned, u signed (PTX dp4a with
// mixed operand types)
__device__ __forceinline__ int dp4a_us(uint32_t x, uint32_t u, int c) {
    int r;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(u), "r"(c));
    return r;
}

// squared distance of 16 byte pairs, accumulated
__device__ __forceinline__ uint32_t sqd16(uint4 a, uint4 b, uint32_t acc) {
    uint32_t t;
    t = __vabsdiffu4(a.x, b.x);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.y, b.y);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.z, b.z);
    acc = __dp4a(t, t, acc);
    t = __vabsdiffu4(a.w, b.w);
    acc = __dp4a(t, t, acc);
    return acc;
}

// offer one candidate per lane (~0 = none) to the warp-held ascending list;
// the list keeps its R smallest values with distinct ids (a repeated id comes
// with the same key, so equal packed values are the same candidate)
__device__ __forceinline__ void offer_lanes(uint64_t &mine, uint64_t v, int R) {
    const int lane = lane_id();
    unsigned m = __ballot_sync(FULL, v < __shfl_sync(FULL, mine, R - 1));
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const uint64_t cv = __shfl_sync(FULL, v, src);
        const uint64_t thr = __shfl_sync(FULL, mine, R - 1);
        if (cv < thr && !__any_sync(FULL, mine == cv)) {
            const int pos = __popc(__ballot_sync(FULL, mine < cv));
            const uint64_t up = __shfl_up_sync(FULL, mine, 1);
            if (lane == pos) mine = cv;
            else if (lane > pos) mine = up;
        }
    }
}

// key of position p at level l: (segment, <u, x> + bias, id)
__global__ void rp_key_kernel(const uint8_t *__restrict__ X, int64_t N, int d, const int8_t *__restrict__ u_level,
                              int l, const uint64_t *__restrict__ prev, uint64_t idmask, int id_bits, int seg_shift,
                              int bias, uint64_t *__restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const uint32_t id = prev ? (uint32_t)(prev[p] & idmask) : (uint32_t)p;
    int64_t lo = 0, hi = N;
    uint64_t s = 0;
    for (int k = 0; k < l; k++) {
        const int64_t m = lo + (hi - lo) / 2;
        if (p >= m) {
            lo = m;
            s = 2 * s + 1;
        } else {
            hi = m;
            s = 2 * s;
        }
    }
    const uint4 *x = (const uint4 *)(X + (int64_t)id * d);
    const uint4 *u = (const uint4 *)(u_level + (int64_t)s * d);
    int acc = 0;
    for (int w = 0; w < d / 16; w++) {
        const uint4 xv = __ldg(x + w), uv = __ldg(u + w);
        acc = dp4a_us(xv.x, uv.x, acc);
        acc = dp4a_us(xv.y, uv.y, acc);
        acc = dp4a_us(xv.z, uv.z, acc);
        acc = dp4a_us(xv.w, uv.w, acc);
    }
    out[p] = (s << seg_shift) | ((uint64_t)(uint32_t)(acc + bias) << id_bits) | id;
}

// one CTA per leaf: stage the leaf's rows, offer every leaf-mate to each
// member's row (rows: N*R packed values, updated in place; a point lies in
// exactly one leaf per round)
__global__ void __launch_bounds__(LEAF_THREADS) rp_leaf_kernel(const uint8_t *__restrict__ X, int64_t N, int d,
                                                               int R, int levels, const uint64_t *__restrict__ sorted,
                                                               uint64_t idmask, uint64_t *__restrict__ rows) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int64_t leaf = blockIdx.x;
    int64_t lo = 0, hi = N;
    for (int k = levels - 1; k >= 0; k--) {
        const int64_t m = lo + (hi - lo) / 2;
        if ((leaf >> k) & 1) lo = m;
        else hi = m;
    }
    const int S = (int)(hi - lo);
    const int W = d / 16;
    const int stride = d + 16;  // 16-byte units per row: odd, so a quarter-warp's rows hit distinct banks
    uint32_t *ids = (uint32_t *)(sm + (size_t)S * stride);
    for (int m = threadIdx.x; m < S; m += blockDim.x)
        ids[m] = sorted ? (uint32_t)(sorted[lo + m] & idmask) : (uint32_t)(lo + m);
    __syncthreads();
    for (int e = threadIdx.x; e < S * W; e += blockDim.x) {
        const int m = e / W, w = e - m * W;
        *(uint4 *)(sm + (size_t)m * stride + 16 * w) = __ldg((const uint4 *)(X + (int64_t)ids[m] * d) + w);
    }
    __syncthreads();
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int i = warp; i < S; i += nwarps) {
        const uint32_t gi = ids[i];
        uint64_t mine = lane < R ? rows[(int64_t)gi * R + lane] : ~0ull;
        const uint4 *ri = (const uint4 *)(sm + (size_t)i * stride);
        uint4 a[8];
#pragma unroll
        for (int w = 0; w < 8; w++)
            if (w < W) a[w] = ri[w];
        for (int j0 = 0; j0 < S; j0 += 32) {
            const int j = j0 + lane;
            uint64_t v = ~0ull;
            if (j < S && j != i) {
                const uint4 *rj = (const uint4 *)(sm + (size_t)j * stride);
                uint32_t acc = 0;
#pragma unroll
                for (int w = 0; w < 8; w++)
                    if (w < W) acc = sqd16(a[w], rj[w], acc);
                for (int w = 8; w < W; w++) acc = sqd16(ri[w], rj[w], acc);
                v = ((uint64_t)acc << 32) | ids[j];
            }
            offer_lanes(mine, v, R);
        }
        if (lane < R) rows[(int64_t)gi * R + lane] = mine;
    }
}

__device__ __forceinline__ uint32_t dot16(uint4 a, uint4 b, uint32_t acc) {
    acc = __dp4a(a.x, b.x, acc);
    acc = __dp4a(a.y, b.y, acc);
    acc = __dp4a(a.z, b.z, acc);
    acc = __dp4a(a.w, b.w, acc);
    return acc;
}

// leaves larger than shared memory (d <= 128): CTA (leaf, chunk) owns TILE_I
// members, two per warp with their rows in registers, and streams the whole
// leaf through shared memory TILE_J rows at a time.  Keys are
// ||x||^2 + ||y||^2 - 2 x.y in exact integers (the squared distance itself).
__global__ void __launch_bounds__(TILE_THREADS) rp_leaf_tiled_kernel(const uint8_t *__restrict__ X, int64_t N,
                                                                     int d, int R, int levels, int chunks,
                                                                     const uint64_t *__restrict__ sorted,
                                                                     uint64_t idmask, uint64_t *__restrict__ rows) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int64_t leaf = blockIdx.x / chunks;
    const int chunk = (int)(blockIdx.x % chunks);
    int64_t lo = 0, hi = N;
    for (int k = levels - 1; k >= 0; k--) {
        const int64_t m = lo + (hi - lo) / 2;
        if ((leaf >> k) & 1) lo = m;
        else hi = m;
    }
    const int S = (int)(hi - lo);
    const int W = d / 16;
    const int stride = d + 16;
    uint32_t *tids = (uint32_t *)(sm + (size_t)TILE_J * stride);
    uint32_t *tnorm = tids + TILE_J;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int i1 = chunk * TILE_I + 2 * warp, i2 = i1 + 1;
    const bool v1 = i1 < S, v2 = i2 < S;  // warp-uniform
    const uint32_t g1 = v1 ? (sorted ? (uint32_t)(sorted[lo + i1] & idmask) : (uint32_t)(lo + i1)) : 0u;
    const uint32_t g2 = v2 ? (sorted ? (uint32_t)(sorted[lo + i2] & idmask) : (uint32_t)(lo + i2)) : 0u;
    uint4 a1[8], a2[8];
    uint32_t n1 = 0, n2 = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        a1[w] = make_uint4(0, 0, 0, 0);
        a2[w] = make_uint4(0, 0, 0, 0);
        if (w < W) {
            if (v1) a1[w] = __ldg((const uint4 *)(X + (int64_t)g1 * d) + w);
            if (v2) a2[w] = __ldg((const uint4 *)(X + (int64_t)g2 * d) + w);
            n1 = dot16(a1[w], a1[w], n1);
            n2 = dot16(a2[w], a2[w], n2);
        }
    }
    uint64_t m1 = (v1 && lane < R) ? rows[(int64_t)g1 * R + lane] : ~0ull;
    uint64_t m2 = (v2 && lane < R) ? rows[(int64_t)g2 * R + lane] : ~0ull;
    for (int t0 = 0; t0 < S; t0 += TILE_J) {
        const int TJ = min(TILE_J, S - t0);
        __syncthreads();  // the previous tile is consumed
        for (int m = threadIdx.x; m < TJ; m += blockDim.x)
            tids[m] = sorted ? (uint32_t)(sorted[lo + t0 + m] & idmask) : (uint32_t)(lo + t0 + m);
        __syncthreads();
        for (int e = threadIdx.x; e < TJ * W; e += blockDim.x) {
            const int m = e / W, w = e - m * W;
            *(uint4 *)(sm + (size_t)m * stride + 16 * w) = __ldg((const uint4 *)(X + (int64_t)tids[m] * d) + w);
        }
        __syncthreads();
        for (int m = threadIdx.x; m < TJ; m += blockDim.x) {
            const uint4 *r = (const uint4 *)(sm + (size_t)m * stride);
            uint32_t n = 0;
            for (int w = 0; w < W; w++) {
                const uint4 b = r[w];
                n = dot16(b, b, n);
            }
            tnorm[m] = n;
        }
        __syncthreads();
        if (!v1) continue;  // warp-uniform; the barriers above are reached by every warp
        for (int jb = 0; jb < TJ; jb += 32) {
            const int jl = jb + lane, j = t0 + jl;
            uint64_t c1 = ~0ull, c2 = ~0ull;
            if (jl < TJ) {
                const uint4 *rj = (const uint4 *)(sm + (size_t)jl * stride);
                uint32_t d1 = 0, d2 = 0;
#pragma unroll
                for (int w = 0; w < 8; w++)
                    if (w < W) {
                        const uint4 b = rj[w];
                        d1 = dot16(a1[w], b, d1);
                        d2 = dot16(a2[w], b, d2);
                    }
                const uint32_t nj = tnorm[jl], idj = tids[jl];
                if (j != i1) c1 = ((uint64_t)(n1 + nj - 2u * d1) << 32) | idj;
                if (v2 && j != i2) c2 = ((uint64_t)(n2 + nj - 2u * d2) << 32) | idj;
            }
            offer_lanes(m1, c1, R);
            offer_lanes(m2, c2, R);
        }
    }
    if (v1 && lane < R) rows[(int64_t)g1 * R + lane] = m1;
    if (v2 && lane < R) rows[(int64_t)g2 * R + lane] = m2;
}

// one warp per point: offer the rows of its neighbours (from rin) to its row
__global__ void __launch_bounds__(PROP_THREADS) rp_prop_kernel(const uint8_t *__restrict__ X, int64_t N, int d, int R,
                                                               const uint64_t *__restrict__ rin,
                                                               uint64_t *__restrict__ rout) {
    const int lane = lane_id();
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;  // whole warps
    const uint64_t orig = lane < R ? rin[i * R + lane] : ~0ull;
    uint64_t mine = orig;
    const int W = d / 16;
    const uint4 *xi = (const uint4 *)(X + i * d);
    uint4 a[8];
#pragma unroll
    for (int w = 0; w < 8; w++)
        if (w < W) a[w] = __ldg(xi + w);
    const int RR = R * R;
    for (int e0 = 0; e0 < RR; e0 += 32) {
        const int e = e0 + lane;
        const int jj = e < RR ? e / R : 0;
        const uint32_t j = (uint32_t)__shfl_sync(FULL, orig, jj);
        uint32_t c = 0xffffffffu;
        if (e < RR && j != 0xffffffffu) c = (uint32_t)__ldg(rin + (int64_t)j * R + (e - jj * R));
        bool fresh = c != 0xffffffffu && c != (uint32_t)i;
        for (int q = 0; q < R; q++)  // already in the row: nothing to compute
            if ((uint32_t)__shfl_sync(FULL, mine, q) == c) fresh = false;
        uint64_t v = ~0ull;
        if (fresh) {
            const uint4 *xc = (const uint4 *)(X + (int64_t)c * d);
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < 8; w++)
                if (w < W) acc = sqd16(a[w], __ldg(xc + w), acc);
            for (int w = 8; w < W; w++) acc = sqd16(__ldg(xi + w), __ldg(xc + w), acc);
            v = ((uint64_t)acc << 32) | c;
        }
        offer_lanes(mine, v, R);
    }
    if (lane < R) rout[i * R + lane] = mine;
}

__global__ void rp_export_kernel(const uint64_t *__restrict__ rows, int64_t n, int32_t *__restrict__ ids,
                                 uint32_t *__restrict__ keys) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint64_t v = rows[e];
    ids[e] = (int32_t)(uint32_t)v;  // an empty slot (~0) becomes id -1, key UINT32_MAX
    if (keys) keys[e] = (uint32_t)(v >> 32);
}

int bit_length(uint64_t v) {
    int b = 0;
    while (v) {
        b++;
        v >>= 1;
    }
    return b;
}

}  // namespace

size_t knn_approx_leaf_smem(int64_t leaf_rows, int d) { return (size_t)leaf_rows * (size_t)(d + 16 + 4); }
size_t knn_approx_tile_smem(int d) { return (size_t)TILE_J * (size_t)(d + 16 + 8); }

}  // namespace ann

extern "C" int ann_build_knn_graph_approx(const void *data, int dtype, int64_t N, int32_t d, int32_t R,
                                          const int8_t *dirs, int32_t rounds, int32_t levels, int32_t iters,
                                          int32_t *out_ids, void *out_keys, void *stream) {
    using namespace ann;
    ANN_ARG(dtype == ANN_U8, "the approximate graph is built for ANN_U8 data only");
    ANN_ARG(N >= 2 && N < (1ll << 31), "N out of range");
    ANN_ARG(d >= 16 && d <= 4096 && d % 16 == 0, "d must be a multiple of 16 in [16, 4096]");
    ANN_ARG(R >= 1 && R <= 32, "R must be in [1, 32]");
    ANN_ARG(rounds >= 1 && levels >= 0 && levels <= 30 && iters >= 0, "rounds >= 1, 0 <= levels <= 30, iters >= 0");
    ANN_ARG(data && out_ids && (levels == 0 || dirs), "data, out_ids and (levels > 0) dirs are required");
    ANN_ARG(((uintptr_t)data & 15) == 0 && ((uintptr_t)dirs & 15) == 0, "data and dirs must be 16-byte aligned");
    const int64_t nleaves = 1ll << levels;
    const int64_t smallest = N / nleaves, largest = (N + nleaves - 1) / nleaves;
    ANN_ARG(smallest >= R + 1, "every leaf must hold at least R + 1 points: use fewer levels");
    const int id_bits = std::max(1, bit_length((uint64_t)(N - 1)));
    const int bias = 128 * 255 * d;
    const int proj_bits = bit_length((uint64_t)255 * 255 * (uint64_t)d);
    ANN_ARG(levels + proj_bits + id_bits <= 64, "levels, d and N too large for one 64-bit sort key");
    int dev = 0, optin = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    ANN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // leaves that fit in one CTA's shared memory are staged whole; larger
    // ones (d <= 128) are streamed through it
    const bool tiled = knn_approx_leaf_smem(largest, d) > (size_t)optin;
    ANN_ARG(!tiled || d <= 128, "with d > 128 the largest leaf must fit in shared memory: use more levels");
    const size_t smem = tiled ? knn_approx_tile_smem(d) : knn_approx_leaf_smem(largest, d);
    const int chunks = (int)((largest + TILE_I - 1) / TILE_I);
    ANN_ARG(!tiled || nleaves * chunks < (1ll << 31), "too many leaf chunks for one launch");
    cudaStream_t s = (cudaStream_t)stream;

    const uint64_t idmask = (1ull << id_bits) - 1;
    uint64_t *k0 = nullptr, *k1 = nullptr, *ra = nullptr, *rb = nullptr;
    void *temp = nullptr;
    size_t temp_bytes = 0;
    auto release = [&]() {
        if (k0) cudaFreeAsync(k0, s);
        if (k1) cudaFreeAsync(k1, s);
        if (ra) cudaFreeAsync(ra, s);
        if (rb) cudaFreeAsync(rb, s);
        if (temp) cudaFreeAsync(temp, s);
    };
#define AP_CUDA(call)                                          \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) {                               \
            release();                                         \
            return cuda_fail(_e, #call);                       \
        }                                                      \
    } while (0)
    AP_CUDA(cudaMallocAsync((void **)&ra, sizeof(uint64_t) * (size_t)N * R, s));
    if (iters > 0) AP_CUDA(cudaMallocAsync((void **)&rb, sizeof(uint64_t) * (size_t)N * R, s));
    if (levels > 0) {
        AP_CUDA(cudaMallocAsync((void **)&k0, sizeof(uint64_t) * (size_t)N, s));
        AP_CUDA(cudaMallocAsync((void **)&k1, sizeof(uint64_t) * (size_t)N, s));
        cub::DoubleBuffer<uint64_t> probe(k0, k1);
        AP_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, temp_bytes, probe, (int)N, 0, 64, s));
        AP_CUDA(cudaMallocAsync(&temp, temp_bytes, s));
    }
    AP_CUDA(cudaMemsetAsync(ra, 0xff, sizeof(uint64_t) * (size_t)N * R, s));
    if (tiled) AP_CUDA(cudaFuncSetAttribute(rp_leaf_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    else AP_CUDA(cudaFuncSetAttribute(rp_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t nseg = nleaves - 1;
    const unsigned gridN = (unsigned)((N + 255) / 256);
    for (int r = 0; r < rounds; r++) {
        cub::DoubleBuffer<uint64_t> keys(k0, k1);
        for (int l = 0; l < levels; l++) {
            const int8_t *u = dirs + ((int64_t)r * nseg + ((1ll << l) - 1)) * d;
            const uint64_t *prev = l == 0 ? nullptr : keys.Current();
            uint64_t *out = l == 0 ? keys.Current() : keys.Alternate();
            rp_key_kernel<<<gridN, 256, 0, s>>>((const uint8_t *)data, N, d, u, l, prev, idmask, id_bits,
                                                proj_bits + id_bits, bias, out);
            AP_CUDA(cudaGetLastError());
            if (l > 0) keys.selector ^= 1;
            size_t tb = temp_bytes;
            AP_CUDA(cub::DeviceRadixSort::SortKeys(temp, tb, keys, (int)N, 0, l + proj_bits + id_bits, s));
        }
        const uint64_t *sorted = levels > 0 ? keys.Current() : nullptr;
        if (tiled)
            rp_leaf_tiled_kernel<<<(unsigned)(nleaves * chunks), TILE_THREADS, smem, s>>>(
                (const uint8_t *)data, N, d, R, levels, chunks, sorted, idmask, ra);
        else
            rp_leaf_kernel<<<(unsigned)nleaves, LEAF_THREADS, smem, s>>>((const uint8_t *)data, N, d, R, levels,
                                                                         sorted, idmask, ra);
        AP_CUDA(cudaGetLastError());
    }
    const unsigned gridW = (unsigned)((N * 32 + PROP_THREADS - 1) / PROP_THREADS);
    for (int it = 0; it < iters; it++) {
        rp_prop_kernel<<<gridW, PROP_THREADS, 0, s>>>((const uint8_t *)data, N, d, R, ra, rb);
        AP_CUDA(cudaGetLastError());
        std::swap(ra, rb);
    }
    const int64_t n = N * R;
    rp_export_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ra, n, out_ids, (uint32_t *)out_keys);
    AP_CUDA(cudaGetLastError());
#undef AP_CUDA
    release();
    return ANN_OK;
}
