// ann_index.cu -- index construction on sm_103a: per-part dictionaries
// (Sec. 4.1 "Computing bridge vectors"), the bridge graph (Sec. 4.1
// "Augmented neighborhood graph") and the index handle, file format and
// statistics (Table 1).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cub/cub.cuh>
#include <functional>
#include <string>
#include <vector>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA;
}

// RAII device buffer used inside this file
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        n = count;
        return cudaMalloc((void **)&p, sizeof(T) * (count ? count : 1));
    }
    ~DBuf() {
        if (p) cudaFree(p);
    }
    T *release() {
        T *q = p;
        p = nullptr;
        return q;
    }
};

#define ANN_CUDA_ALLOC(buf, count) ANN_CUDA((buf).alloc(count))

// ---------------------------------------------------------------------------
// k-means per part, fp64 (Sec. 4.1)
// ---------------------------------------------------------------------------
// One thread per training row.  The row's part is staged in shared memory as
// float (exact for bytes and float32); the distance to each center is summed
// in dimension order with separate multiply and add (no FMA), the same
// arithmetic as a plain sequential fp64 loop.
template <int DT>
__global__ void km_assign_kernel(const void *X, int64_t N, int d, int dp, int p, int n, const double *C,
                                 int32_t *assign) {
    extern __shared__ float srow[];  // dp * blockDim.x
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int tid = threadIdx.x, B = blockDim.x;
    if (i < N) {
        for (int e = 0; e < dp; e++) {
            int64_t at = i * d + (int64_t)p * dp + e;
            srow[e * B + tid] = DT == ANN_U8 ? (float)((const uint8_t *)X)[at] : ((const float *)X)[at];
        }
    }
    if (i >= N) return;
    double best = 0.0;
    int arg = -1;
    for (int j = 0; j < n; j++) {
        const double *cj = C + (int64_t)j * dp;
        double s = 0.0;
        for (int e = 0; e < dp; e++) {
            double t = __dsub_rn((double)srow[e * B + tid], cj[e]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        if (arg < 0 || s < best) {
            best = s;
            arg = j;
        }
    }
    assign[i] = arg;
}

template <int DT>
__global__ void km_accumulate_kernel(const void *X, int64_t N, int d, int dp, int p, const int32_t *assign,
                                     unsigned long long *isums, double *fsums, unsigned long long *counts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int j = assign[i];
    atomicAdd(&counts[j], 1ull);
    for (int e = 0; e < dp; e++) {
        int64_t at = i * d + (int64_t)p * dp + e;
        if (DT == ANN_U8) atomicAdd(&isums[(int64_t)j * dp + e], (unsigned long long)((const uint8_t *)X)[at]);
        else atomicAdd(&fsums[(int64_t)j * dp + e], (double)((const float *)X)[at]);
    }
}

template <int DT>
__global__ void km_update_kernel(int n, int dp, const unsigned long long *isums, const double *fsums,
                                 const unsigned long long *counts, double *C) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * dp) return;
    int j = idx / dp;
    unsigned long long c = counts[j];
    if (c == 0) return;  // empty cluster keeps its center
    double s = DT == ANN_U8 ? (double)isums[idx] : fsums[idx];
    C[idx] = __ddiv_rn(s, (double)c);
}

template <int DT>
__global__ void km_init_kernel(const void *X, int d, int dp, int P, int n, const int64_t *rows, double *C) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over P*n*dp
    if (idx >= P * n * dp) return;
    int p = idx / (n * dp), j = (idx / dp) % n, e = idx % dp;
    int64_t at = rows[j] * d + (int64_t)p * dp + e;
    C[idx] = DT == ANN_U8 ? (double)((const uint8_t *)X)[at] : (double)((const float *)X)[at];
}

__global__ void km_store_kernel(int total, int dtype, const double *C, void *out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    if (dtype == ANN_U8) {
        double r = rint(C[idx]);  // round half to even
        r = r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);
        ((uint8_t *)out)[idx] = (uint8_t)r;
    } else {
        ((float *)out)[idx] = __double2float_rn(C[idx]);
    }
}

// ---------------------------------------------------------------------------
// bridge graph (Sec. 4.1): top-t bridge vectors of every reference vector,
// then the b nearest references of every bridge vector.
// ---------------------------------------------------------------------------
// A tuple of ranks r can be among the t smallest only if prod_p (r_p + 1) <= t
// (every tuple below it in every coordinate precedes it).  Each warp scores
// all such candidate tuples for its reference and sorts them by
// (key, ranks): exactly the first t tuples of the multi-sequence order.
template <int DT>
__global__ void bg_topt_kernel(const void *X, int64_t N, int d, int P, int n, const void *C,
                               const uint32_t *cands, int ncand, int Lc, int t_eff, uint32_t slice,
                               uint64_t *out_keys, uint32_t *out_vals) {
    extern __shared__ __align__(16) uint8_t smem_all[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    uint8_t *sm = smem_all + (size_t)warp * slice;
    const int vb = d * (DT == ANN_U8 ? 1 : 4);
    uint8_t *qb = sm;
    uint32_t *D = (uint32_t *)(sm + align_up16(vb));
    uint32_t *skey = D + P * n;
    uint8_t *scid = (uint8_t *)(skey + P * n);
    uint64_t *tmp = (uint64_t *)(sm + align_up16(align_up16(vb) + 8 * P * n + P * n));
    const int dp = d / P;
    int Lp = 1;
    while (Lp < n) Lp <<= 1;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = gw; i < N; i += nw) {
        const uint4 *src = (const uint4 *)((const uint8_t *)X + i * (int64_t)vb);
        for (int c = lane; c < (vb >> 4); c += 32) ((uint4 *)qb)[c] = __ldg(src + c);
        __syncwarp();
        for (int idx = lane; idx < P * n; idx += 32) D[idx] = part_key_lane<DT>(qb, C, idx / n, idx % n, n, dp);
        __syncwarp();
        for (int p = 0; p < P; p++) {
            for (int r = lane; r < Lp; r += 32)
                tmp[r] = r < n ? (((uint64_t)D[p * n + r]) << 32) | (uint32_t)r : ~0ull;
            __syncwarp();
            warp_sort_pairs(tmp, nullptr, Lp);
            for (int r = lane; r < n; r += 32) {
                skey[p * n + r] = (uint32_t)(tmp[r] >> 32);
                scid[p * n + r] = (uint8_t)(uint32_t)tmp[r];
            }
            __syncwarp();
        }
        for (int c = lane; c < Lc; c += 32) {
            uint64_t v = ~0ull;
            if (c < ncand) {
                uint32_t rr = cands[c];
                uint32_t r[kMaxP];
                for (int p = 0; p < P; p++) r[p] = (rr >> (8 * (P - 1 - p))) & 255u;
                // Sec. 4.2: the sum of the part keys (float32: nearest to the exact sum)
                const uint32_t key = KeyOps<DT>::sum4(skey[r[0]], skey[n + r[1]], P > 2 ? skey[2 * n + r[2]] : 0u,
                                                      P > 3 ? skey[3 * n + r[3]] : 0u);
                v = ((uint64_t)key << 32) | rr;
            }
            tmp[c] = v;
        }
        __syncwarp();
        warp_sort_pairs(tmp, nullptr, Lc);
        for (int j = lane; j < t_eff; j += 32) {
            uint64_t v = tmp[j];
            uint32_t rr = (uint32_t)v;
            uint64_t bid = 0;
            for (int p = 0; p < P; p++) {
                uint32_t r = (rr >> (8 * (P - 1 - p))) & 255u;
                bid = bid * (uint64_t)n + scid[p * n + r];
            }
            out_keys[i * t_eff + j] = (bid << 32) | (v >> 32);
            out_vals[i * t_eff + j] = (uint32_t)i;
        }
        __syncwarp();
    }
}

__global__ void bg_keep_kernel(const uint64_t *keys, int64_t m, int b, uint8_t *flags) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    flags[j] = (j < b) || ((keys[j - b] >> 32) != (keys[j] >> 32));
}

__global__ void bg_first_kernel(const uint64_t *keys, int64_t m, uint32_t *first) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    first[j] = (j == 0 || (keys[j - 1] >> 32) != (keys[j] >> 32)) ? 1u : 0u;
}

// seg = inclusive scan of first, minus one
__global__ void bg_scatter_kernel(const uint64_t *keys, const uint32_t *vals, const uint32_t *seg_incl,
                                  const uint32_t *first, int64_t m, uint32_t *ustart, uint32_t *ubid) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (first[j]) {
        uint32_t s = seg_incl[j] - 1;
        ustart[s] = (uint32_t)j;
        ubid[s] = (uint32_t)(keys[j] >> 32);
    }
}

__global__ void bg_refs_kernel(const uint32_t *vals, const uint32_t *seg_incl, const uint32_t *ustart, int64_t m,
                               int b, int32_t *brefs) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    uint32_t s = seg_incl[j] - 1;
    brefs[(int64_t)s * b + (j - ustart[s])] = (int32_t)vals[j];
}

__global__ void bg_leaf_kernel(const uint32_t *ubid, int64_t M, uint32_t suf, uint32_t *leaf) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    leaf[j] = ubid[j] % suf;
}

// offA[a] = first bridge index whose prefix is >= a  (a in [0, nA])
__global__ void bg_offa_kernel(const uint32_t *ubid, int64_t M, uint32_t suf, int64_t nA, uint32_t *offA) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a > nA) return;
    int64_t lo = 0, hi = M;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(ubid[mid] / suf) < a) lo = mid + 1;
        else hi = mid;
    }
    offA[a] = (uint32_t)lo;
}

__global__ void bg_bits_kernel(const uint32_t *offA, int64_t nA, uint32_t *bmA) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t words = (nA + 31) / 32;
    if (w >= words) return;
    uint32_t v = 0;
    for (int i = 0; i < 32; i++) {
        int64_t a = w * 32 + i;
        if (a < nA && offA[a + 1] > offA[a]) v |= 1u << i;
    }
    bmA[w] = v;
}

// groups of bridges sharing (prefix node, c2): flag the first of each
__global__ void bg_gflag_kernel(const uint32_t *ubid, int64_t M, uint32_t n, uint32_t *flag) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    flag[j] = (j == 0 || ubid[j] / n != ubid[j - 1] / n) ? 1u : 0u;
}

__global__ void bg_gscatter_kernel(const uint32_t *ubid, const uint32_t *flag, const uint32_t *gincl, int64_t M,
                                   uint32_t n, uint32_t *gstart, uint8_t *gc2) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > M) return;
    if (j == M) {
        gstart[M > 0 ? gincl[M - 1] : 0] = (uint32_t)M;
        return;
    }
    if (flag[j]) {
        const uint32_t g = gincl[j] - 1;
        gstart[g] = (uint32_t)j;
        gc2[g] = (uint8_t)((ubid[j] / n) % n);
    }
}

// goff[a] = first group whose prefix node is >= a  (a in [0, nA])
__global__ void bg_goff_kernel(const uint32_t *ubid, const uint32_t *gstart, int64_t G, uint32_t suf, int64_t nA,
                               uint32_t *goff) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a > nA) return;
    int64_t lo = 0, hi = G;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(ubid[gstart[mid]] / suf) < a) lo = mid + 1;
        else hi = mid;
    }
    goff[a] = (uint32_t)lo;
}

// suffix-major order: key s * nA + a of every bridge (a = prefix, s = suffix)
__global__ void bg_skey_kernel(const uint32_t *ubid, int64_t M, uint32_t suf, uint32_t nA, uint32_t *key,
                               uint32_t *pos) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    key[j] = (ubid[j] % suf) * nA + ubid[j] / suf;
    pos[j] = (uint32_t)j;
}

__global__ void bg_sleaf_kernel(const uint32_t *skey, int64_t M, uint32_t nA, uint32_t *sleaf) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    sleaf[j] = skey[j] % nA;
}

// offS[s] = first suffix-major entry whose suffix is >= s  (s in [0, nS])
__global__ void bg_offs_kernel(const uint32_t *skey, int64_t M, uint32_t nA, int64_t nS, uint32_t *offS) {
    int64_t sfx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sfx > nS) return;
    int64_t lo = 0, hi = M;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(skey[mid] / nA) < sfx) lo = mid + 1;
        else hi = mid;
    }
    offS[sfx] = (uint32_t)lo;
}

__global__ void mark_refs_kernel(const int32_t *brefs, int64_t total, uint8_t *mark) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= total) return;
    int32_t r = brefs[j];
    if (r >= 0) mark[r] = 1;
}

static inline unsigned nblk(int64_t m, int t = 256) { return (unsigned)((m + t - 1) / t); }

static int64_t ipow(int64_t a, int e) {
    int64_t r = 1;
    for (int i = 0; i < e; i++) r *= a;
    return r;
}

static int count_bridged(ann_index *ix, cudaStream_t s) {
    DBuf<uint8_t> mark;
    ANN_CUDA_ALLOC(mark, ix->dev.N);
    ANN_CUDA(cudaMemsetAsync(mark.p, 0, ix->dev.N, s));
    int64_t tot = ix->dev.M * ix->dev.b;
    if (tot > 0) mark_refs_kernel<<<nblk(tot), 256, 0, s>>>(ix->brefs, tot, mark.p);
    std::vector<uint8_t> h(ix->dev.N);
    ANN_CUDA(cudaMemcpyAsync(h.data(), mark.p, ix->dev.N, cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaStreamSynchronize(s));
    int64_t c = 0;
    for (uint8_t v : h) c += v;
    ix->bridged_refs = c;
    return ANN_OK;
}

// Build the device bridge index from sorted unique bridge ids (device,
// uint32) and the padded reference lists (device, M*b) -- both already owned.
static int finish_bridge_index(ann_index *ix, DBuf<uint32_t> &ubid, int64_t M, cudaStream_t s) {
    DevIndex &dv = ix->dev;
    uint32_t suf = (uint32_t)ipow(dv.n, dv.P - dv.PA);
    DBuf<uint32_t> leaf, offA, bmA;
    ANN_CUDA_ALLOC(leaf, M);
    ANN_CUDA_ALLOC(offA, dv.nA + 1);
    ANN_CUDA_ALLOC(bmA, (dv.nA + 31) / 32);
    if (M > 0) bg_leaf_kernel<<<nblk(M), 256, 0, s>>>(ubid.p, M, suf, leaf.p);
    bg_offa_kernel<<<nblk(dv.nA + 1), 256, 0, s>>>(ubid.p, M, suf, dv.nA, offA.p);
    bg_bits_kernel<<<nblk((dv.nA + 31) / 32), 256, 0, s>>>(offA.p, dv.nA, bmA.p);
    ANN_CUDA(cudaGetLastError());
    // c2 groups inside each prefix node: two suffix parts, and on average at
    // least 32 bridges per prefix node (otherwise reading the leaves is cheaper)
    int64_t G = 0;
    DBuf<uint32_t> goff, gstart;
    DBuf<uint8_t> gc2;
    if (dv.P - dv.PA == 2 && M >= 32 * dv.nA) {
        DBuf<uint32_t> flag, gincl;
        ANN_CUDA_ALLOC(flag, M);
        ANN_CUDA_ALLOC(gincl, M);
        bg_gflag_kernel<<<nblk(M), 256, 0, s>>>(ubid.p, M, (uint32_t)dv.n, flag.p);
        size_t tb = 0;
        ANN_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb, flag.p, gincl.p, M, s));
        DBuf<uint8_t> temp;
        ANN_CUDA_ALLOC(temp, tb);
        ANN_CUDA(cub::DeviceScan::InclusiveSum(temp.p, tb, flag.p, gincl.p, M, s));
        uint32_t g32 = 0;
        ANN_CUDA(cudaMemcpyAsync(&g32, gincl.p + (M - 1), 4, cudaMemcpyDeviceToHost, s));
        ANN_CUDA(cudaStreamSynchronize(s));
        G = g32;
        ANN_CUDA_ALLOC(gstart, G + 1);
        ANN_CUDA_ALLOC(gc2, G);
        ANN_CUDA_ALLOC(goff, dv.nA + 1);
        bg_gscatter_kernel<<<nblk(M + 1), 256, 0, s>>>(ubid.p, flag.p, gincl.p, M, (uint32_t)dv.n, gstart.p, gc2.p);
        bg_goff_kernel<<<nblk(dv.nA + 1), 256, 0, s>>>(ubid.p, gstart.p, G, suf, dv.nA, goff.p);
        ANN_CUDA(cudaGetLastError());
    }
    // suffix-major copy for the split walks (indexes without the group level)
    DBuf<uint32_t> bmS, offS, sleaf, sidx;
    const int64_t nS = suf;
    if (G == 0 && M > 0) {
        DBuf<uint32_t> k0, k1, v0;
        ANN_CUDA_ALLOC(k0, M);
        ANN_CUDA_ALLOC(k1, M);
        ANN_CUDA_ALLOC(v0, M);
        ANN_CUDA_ALLOC(sidx, M);
        ANN_CUDA_ALLOC(sleaf, M);
        ANN_CUDA_ALLOC(offS, nS + 1);
        ANN_CUDA_ALLOC(bmS, (nS + 31) / 32);
        bg_skey_kernel<<<nblk(M), 256, 0, s>>>(ubid.p, M, suf, (uint32_t)dv.nA, k0.p, v0.p);
        size_t tb = 0;
        ANN_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, k0.p, k1.p, v0.p, sidx.p, M, 0, 32, s));
        DBuf<uint8_t> temp;
        ANN_CUDA_ALLOC(temp, tb);
        ANN_CUDA(cub::DeviceRadixSort::SortPairs(temp.p, tb, k0.p, k1.p, v0.p, sidx.p, M, 0, 32, s));
        bg_sleaf_kernel<<<nblk(M), 256, 0, s>>>(k1.p, M, (uint32_t)dv.nA, sleaf.p);
        bg_offs_kernel<<<nblk(nS + 1), 256, 0, s>>>(k1.p, M, (uint32_t)dv.nA, nS, offS.p);
        bg_bits_kernel<<<nblk((nS + 31) / 32), 256, 0, s>>>(offS.p, nS, bmS.p);
        ANN_CUDA(cudaGetLastError());
        ANN_CUDA(cudaStreamSynchronize(s));
    }
    ANN_CUDA(cudaStreamSynchronize(s));
    ix->bmS = bmS.release();
    ix->offS = offS.release();
    ix->sleaf = sleaf.release();
    ix->sidx = sidx.release();
    dv.nS = nS;
    dv.bmS = ix->bmS;
    dv.offS = ix->offS;
    dv.sleaf = ix->sleaf;
    dv.sidx = ix->sidx;
    ix->leaf = leaf.release();
    ix->offA = offA.release();
    ix->bmA = bmA.release();
    ix->goff = goff.release();
    ix->gstart = gstart.release();
    ix->gc2 = gc2.release();
    dv.leaf = ix->leaf;
    dv.offA = ix->offA;
    dv.bmA = ix->bmA;
    dv.ngroups = G;
    dv.goff = ix->goff;
    dv.gstart = ix->gstart;
    dv.gc2 = ix->gc2;
    dv.M = M;
    return count_bridged(ix, s);
}

template <int DT>
static int build_bridges_gpu(ann_index *ix, cudaStream_t s) {
    DevIndex &dv = ix->dev;
    const int P = dv.P, n = dv.n, b = dv.b;
    const int64_t N = dv.N;
    const int64_t nb = ipow(n, P);
    const int t_eff = (int)std::min<int64_t>(dv.t, nb);
    // candidate rank tuples with prod(r_p + 1) <= t_eff
    std::vector<uint32_t> cands;
    {
        std::vector<int> r(P, 0);
        std::function<void(int, int64_t)> rec = [&](int p, int64_t prod) {
            if (p == P) {
                uint32_t v = 0;
                for (int q = 0; q < P; q++) v = (v << 8) | (uint32_t)r[q];
                cands.push_back(v);
                return;
            }
            for (int x = 0; x < n && prod * (x + 1) <= t_eff; x++) {
                r[p] = x;
                rec(p + 1, prod * (x + 1));
            }
        };
        rec(0, 1);
    }
    const int ncand = (int)cands.size();
    int Lc = 1;
    while (Lc < ncand) Lc <<= 1;
    int Lp = 1;
    while (Lp < n) Lp <<= 1;
    DBuf<uint32_t> dcand;
    ANN_CUDA_ALLOC(dcand, ncand);
    ANN_CUDA(cudaMemcpyAsync(dcand.p, cands.data(), 4 * ncand, cudaMemcpyHostToDevice, s));
    const int vb = dv.d * (DT == ANN_U8 ? 1 : 4);
    uint32_t slice = align_up16(align_up16(vb) + 8 * P * n + P * n) + 8 * std::max(Lc, Lp);
    slice = align_up16(slice);
    int dev;
    ANN_CUDA(cudaGetDevice(&dev));
    int optin = 0, nsm = 0;
    ANN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    ANN_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int warps = (int)std::min<int64_t>(8, optin / slice);
    if (warps < 1) return fail(ANN_ERR_CAPACITY, "bridge builder: per-reference state exceeds shared memory");
    size_t smem = (size_t)warps * slice;
    ANN_CUDA(cudaFuncSetAttribute(bg_topt_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t m = N * t_eff;
    DBuf<uint64_t> k0, k1;
    DBuf<uint32_t> v0, v1;
    ANN_CUDA_ALLOC(k0, m);
    ANN_CUDA_ALLOC(k1, m);
    ANN_CUDA_ALLOC(v0, m);
    ANN_CUDA_ALLOC(v1, m);
    int64_t blocks = std::min<int64_t>((N + warps - 1) / warps, (int64_t)nsm * 16);
    if (N > 0)
        bg_topt_kernel<DT><<<(unsigned)blocks, warps * 32, smem, s>>>(dv.X, N, dv.d, P, n, dv.C, dcand.p, ncand,
                                                                       Lc, t_eff, slice, k0.p, v0.p);
    ANN_CUDA(cudaGetLastError());
    // sort by (bridge id, key); stable, so references stay in id order within ties
    size_t tb = 0;
    ANN_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, k0.p, k1.p, v0.p, v1.p, m, 0, 64, s));
    DBuf<uint8_t> temp;
    ANN_CUDA_ALLOC(temp, tb);
    ANN_CUDA(cub::DeviceRadixSort::SortPairs(temp.p, tb, k0.p, k1.p, v0.p, v1.p, m, 0, 64, s));
    // keep the first b of every bridge
    DBuf<uint8_t> flags;
    ANN_CUDA_ALLOC(flags, m);
    if (m > 0) bg_keep_kernel<<<nblk(m), 256, 0, s>>>(k1.p, m, b, flags.p);
    DBuf<int64_t> nsel;
    ANN_CUDA_ALLOC(nsel, 1);
    size_t tb2 = 0;
    ANN_CUDA(cub::DeviceSelect::Flagged(nullptr, tb2, k1.p, flags.p, k0.p, nsel.p, m, s));
    DBuf<uint8_t> temp2;
    ANN_CUDA_ALLOC(temp2, tb2);
    ANN_CUDA(cub::DeviceSelect::Flagged(temp2.p, tb2, k1.p, flags.p, k0.p, nsel.p, m, s));
    ANN_CUDA(cub::DeviceSelect::Flagged(temp2.p, tb2, v1.p, flags.p, v0.p, nsel.p, m, s));
    int64_t mk = 0;
    ANN_CUDA(cudaMemcpyAsync(&mk, nsel.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaStreamSynchronize(s));
    // segments = distinct bridges
    DBuf<uint32_t> first, seg;
    ANN_CUDA_ALLOC(first, mk);
    ANN_CUDA_ALLOC(seg, mk);
    if (mk > 0) bg_first_kernel<<<nblk(mk), 256, 0, s>>>(k0.p, mk, first.p);
    size_t tb3 = 0;
    ANN_CUDA(cub::DeviceScan::InclusiveSum(nullptr, tb3, first.p, seg.p, mk, s));
    DBuf<uint8_t> temp3;
    ANN_CUDA_ALLOC(temp3, tb3);
    ANN_CUDA(cub::DeviceScan::InclusiveSum(temp3.p, tb3, first.p, seg.p, mk, s));
    uint32_t M32 = 0;
    if (mk > 0) ANN_CUDA(cudaMemcpyAsync(&M32, seg.p + mk - 1, 4, cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaStreamSynchronize(s));
    const int64_t M = M32;
    DBuf<uint32_t> ustart, ubid;
    DBuf<int32_t> brefs;
    ANN_CUDA_ALLOC(ustart, M);
    ANN_CUDA_ALLOC(ubid, M);
    ANN_CUDA_ALLOC(brefs, M * b);
    ANN_CUDA(cudaMemsetAsync(brefs.p, 0xff, sizeof(int32_t) * std::max<int64_t>(M * b, 1), s));
    if (mk > 0) {
        bg_scatter_kernel<<<nblk(mk), 256, 0, s>>>(k0.p, v0.p, seg.p, first.p, mk, ustart.p, ubid.p);
        bg_refs_kernel<<<nblk(mk), 256, 0, s>>>(v0.p, seg.p, ustart.p, mk, b, brefs.p);
    }
    ANN_CUDA(cudaGetLastError());
    ix->brefs = brefs.release();
    dv.brefs = ix->brefs;
    return finish_bridge_index(ix, ubid, M, s);
}

int build_bridge_index_from_host(ann_index *ix, int64_t M, const uint64_t *ids, const int64_t *offsets,
                                 const int32_t *refs) {
    DevIndex &dv = ix->dev;
    const int b = dv.b;
    std::vector<uint32_t> hb(M > 0 ? M : 1);
    std::vector<int32_t> hr((size_t)std::max<int64_t>(M * b, 1), -1);
    for (int64_t j = 0; j < M; j++) {
        if (ids[j] >= (uint64_t)ipow(dv.n, dv.P)) return fail(ANN_ERR_ARG, "bridge id out of range");
        if (j > 0 && ids[j] <= ids[j - 1]) return fail(ANN_ERR_ARG, "bridge ids must be strictly ascending");
        int64_t len = offsets[j + 1] - offsets[j];
        if (len < 1 || len > b) return fail(ANN_ERR_ARG, "each bridge list must hold 1..b references");
        hb[j] = (uint32_t)ids[j];
        for (int64_t i = 0; i < len; i++) {
            int32_t r = refs[offsets[j] + i];
            if (r < 0 || r >= dv.N) return fail(ANN_ERR_ARG, "bridge reference out of range");
            hr[j * b + i] = r;
        }
    }
    DBuf<uint32_t> ubid;
    DBuf<int32_t> brefs;
    ANN_CUDA_ALLOC(ubid, M);
    ANN_CUDA_ALLOC(brefs, M * b);
    ANN_CUDA(cudaMemcpy(ubid.p, hb.data(), 4 * std::max<int64_t>(M, 0), cudaMemcpyHostToDevice));
    ANN_CUDA(cudaMemcpy(brefs.p, hr.data(), 4 * std::max<int64_t>(M * b, 0), cudaMemcpyHostToDevice));
    ix->brefs = brefs.release();
    dv.brefs = ix->brefs;
    return finish_bridge_index(ix, ubid, M, 0);
}

static void destroy(ann_index *ix) {
    if (!ix) return;
    free_plans(ix);
    cudaFree(ix->X);
    cudaFree(ix->G);
    cudaFree(ix->C);
    cudaFree(ix->bmA);
    cudaFree(ix->offA);
    cudaFree(ix->leaf);
    cudaFree(ix->brefs);
    cudaFree(ix->goff);
    cudaFree(ix->gstart);
    cudaFree(ix->gc2);
    cudaFree(ix->bmS);
    cudaFree(ix->offS);
    cudaFree(ix->sleaf);
    cudaFree(ix->sidx);
    delete ix;
}

static int check_desc(const ann_index_desc *d) {
    ANN_ARG(d != nullptr, "desc is NULL");
    ANN_ARG(d->dtype == ANN_U8 || d->dtype == ANN_F32, "dtype must be ANN_U8 or ANN_F32");
    ANN_ARG(d->N >= 1 && d->N < (1ll << 31), "N must be in [1, 2^31)");
    ANN_ARG(d->P >= 2 && d->P <= kMaxP, "P must be in [2, 4]");
    ANN_ARG(d->n >= 1 && d->n <= kMaxN, "n must be in [1, 256]");
    ANN_ARG(d->d >= d->P && d->d % d->P == 0, "d must be a multiple of P");
    ANN_ARG(d->dtype == ANN_F32 ? d->d % 4 == 0 : d->d % 16 == 0, "d must be a multiple of 16 (u8) or 4 (f32)");
    ANN_ARG(d->R >= 1 && d->R <= kMaxR, "R must be in [1, 32]");
    ANN_ARG(d->b >= 1 && d->b <= kMaxB, "b must be in [1, 8]");
    ANN_ARG(d->t >= 1, "t must be >= 1");
    ANN_ARG(ipow(d->n, d->P) <= (1ll << 32), "n^P must be <= 2^32");
    ANN_ARG(d->data && d->graph && d->centers, "data, graph and centers are required");
    return ANN_OK;
}

}  // namespace ann

using namespace ann;

extern "C" const char *ann_last_error(void) { return g_err.c_str(); }

extern "C" int ann_train_centers(const void *train, int dtype, int64_t ntrain, int32_t d, int32_t P, int32_t n,
                                 int32_t iters, const int64_t *init_rows, void *out_centers,
                                 double *out_centers_f64, void *stream) {
    ANN_ARG(dtype == ANN_U8 || dtype == ANN_F32, "dtype must be ANN_U8 or ANN_F32");
    ANN_ARG(P >= 1 && P <= kMaxP && d % P == 0, "P must divide d and be <= 4");
    ANN_ARG(n >= 1 && n <= kMaxN && ntrain >= n, "need 1 <= n <= 256 and ntrain >= n");
    ANN_ARG(iters >= 0, "iters must be >= 0");
    ANN_ARG(train && init_rows && out_centers, "train, init_rows and out_centers are required");
    for (int j = 0; j < n; j++) ANN_ARG(init_rows[j] >= 0 && init_rows[j] < ntrain, "init row out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const int dp = d / P;
    DBuf<double> C;
    DBuf<int64_t> rows;
    DBuf<int32_t> assign;
    DBuf<unsigned long long> isums, counts;
    DBuf<double> fsums;
    ANN_CUDA_ALLOC(C, (size_t)P * n * dp);
    ANN_CUDA_ALLOC(rows, n);
    ANN_CUDA_ALLOC(assign, ntrain);
    ANN_CUDA_ALLOC(isums, (size_t)n * dp);
    ANN_CUDA_ALLOC(fsums, (size_t)n * dp);
    ANN_CUDA_ALLOC(counts, n);
    ANN_CUDA(cudaMemcpyAsync(rows.p, init_rows, 8 * n, cudaMemcpyHostToDevice, s));
    const int total = P * n * dp;
    if (dtype == ANN_U8) km_init_kernel<ANN_U8><<<nblk(total), 256, 0, s>>>(train, d, dp, P, n, rows.p, C.p);
    else km_init_kernel<ANN_F32><<<nblk(total), 256, 0, s>>>(train, d, dp, P, n, rows.p, C.p);
    const int TB = 128;
    size_t sm = sizeof(float) * dp * TB;
    if (dtype == ANN_U8)
        ANN_CUDA(cudaFuncSetAttribute(km_assign_kernel<ANN_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    else
        ANN_CUDA(cudaFuncSetAttribute(km_assign_kernel<ANN_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    for (int p = 0; p < P; p++) {
        double *Cp = C.p + (size_t)p * n * dp;
        for (int it = 0; it < iters; it++) {
            ANN_CUDA(cudaMemsetAsync(isums.p, 0, 8 * (size_t)n * dp, s));
            ANN_CUDA(cudaMemsetAsync(fsums.p, 0, 8 * (size_t)n * dp, s));
            ANN_CUDA(cudaMemsetAsync(counts.p, 0, 8 * (size_t)n, s));
            if (dtype == ANN_U8) {
                km_assign_kernel<ANN_U8><<<nblk(ntrain, TB), TB, sm, s>>>(train, ntrain, d, dp, p, n, Cp, assign.p);
                km_accumulate_kernel<ANN_U8><<<nblk(ntrain), 256, 0, s>>>(train, ntrain, d, dp, p, assign.p, isums.p,
                                                                          fsums.p, counts.p);
                km_update_kernel<ANN_U8><<<nblk(n * dp), 256, 0, s>>>(n, dp, isums.p, fsums.p, counts.p, Cp);
            } else {
                km_assign_kernel<ANN_F32><<<nblk(ntrain, TB), TB, sm, s>>>(train, ntrain, d, dp, p, n, Cp, assign.p);
                km_accumulate_kernel<ANN_F32><<<nblk(ntrain), 256, 0, s>>>(train, ntrain, d, dp, p, assign.p, isums.p,
                                                                           fsums.p, counts.p);
                km_update_kernel<ANN_F32><<<nblk(n * dp), 256, 0, s>>>(n, dp, isums.p, fsums.p, counts.p, Cp);
            }
            ANN_CUDA(cudaGetLastError());
        }
    }
    km_store_kernel<<<nblk(total), 256, 0, s>>>(total, dtype, C.p, out_centers);
    if (out_centers_f64)
        ANN_CUDA(cudaMemcpyAsync(out_centers_f64, C.p, 8 * (size_t)total, cudaMemcpyDeviceToDevice, s));
    ANN_CUDA(cudaGetLastError());
    ANN_CUDA(cudaStreamSynchronize(s));
    return ANN_OK;
}

extern "C" int ann_index_create(const ann_index_desc *desc, ann_index **out) {
    int r = check_desc(desc);
    if (r != ANN_OK) return r;
    ANN_ARG(out != nullptr, "out is NULL");
    ann_index *ix = new ann_index();
    memset(ix, 0, sizeof(*ix));
    ANN_CUDA(cudaGetDevice(&ix->device));
    DevIndex &dv = ix->dev;
    dv.dtype = desc->dtype;
    dv.N = desc->N;
    dv.d = desc->d;
    dv.R = desc->R;
    dv.P = desc->P;
    dv.n = desc->n;
    dv.b = desc->b;
    dv.t = desc->t;
    dv.PA = desc->P >= 3 ? 2 : 1;
    dv.nA = ipow(desc->n, dv.PA);
    const size_t es = desc->dtype == ANN_U8 ? 1 : 4;
    const size_t xb = (size_t)desc->N * desc->d * es;
    const size_t gb = (size_t)desc->N * desc->R * 4;
    const size_t cb = (size_t)desc->P * desc->n * (desc->d / desc->P) * es;
    cudaError_t e;
    if ((e = cudaMalloc(&ix->X, xb)) != cudaSuccess || (e = cudaMalloc((void **)&ix->G, gb)) != cudaSuccess ||
        (e = cudaMalloc(&ix->C, cb)) != cudaSuccess) {
        destroy(ix);
        return cuda_fail(e, "cudaMalloc(index arrays)");
    }
    if ((e = cudaMemcpy(ix->X, desc->data, xb, cudaMemcpyDefault)) != cudaSuccess ||
        (e = cudaMemcpy(ix->G, desc->graph, gb, cudaMemcpyDefault)) != cudaSuccess ||
        (e = cudaMemcpy(ix->C, desc->centers, cb, cudaMemcpyDefault)) != cudaSuccess) {
        destroy(ix);
        return cuda_fail(e, "cudaMemcpy(index arrays)");
    }
    dv.X = ix->X;
    dv.G = ix->G;
    dv.C = ix->C;
    if (desc->bridge_ids) {
        ANN_ARG(desc->bridge_offsets && desc->bridge_refs && desc->M >= 0, "incomplete host bridge graph");
        r = build_bridge_index_from_host(ix, desc->M, desc->bridge_ids, desc->bridge_offsets, desc->bridge_refs);
    } else {
        r = desc->dtype == ANN_U8 ? build_bridges_gpu<ANN_U8>(ix, 0) : build_bridges_gpu<ANN_F32>(ix, 0);
    }
    if (r != ANN_OK) {
        std::string keep = g_err;
        destroy(ix);
        g_err = keep;
        return r;
    }
    *out = ix;
    return ANN_OK;
}

extern "C" int ann_index_free(ann_index *index) {
    destroy(index);
    return ANN_OK;
}

extern "C" int ann_index_get_info(const ann_index *index, ann_index_info *out) {
    ANN_ARG(index && out, "index and out are required");
    const DevIndex &dv = index->dev;
    out->N = dv.N;
    out->M = dv.M;
    out->d = dv.d;
    out->R = dv.R;
    out->P = dv.P;
    out->n = dv.n;
    out->b = dv.b;
    out->dtype = dv.dtype;
    out->bridged_refs = index->bridged_refs;
    out->alpha = (double)index->bridged_refs / (double)ipow(dv.n, dv.P);
    const size_t es = dv.dtype == ANN_U8 ? 1 : 4;
    out->bytes_vectors = (int64_t)(dv.N * dv.d * es);
    out->bytes_graph = dv.N * dv.R * 4;
    out->bytes_bridges = dv.M * (4 + 4 * dv.b) + (dv.nA + 1) * 4 + (dv.nA + 31) / 32 * 4 +
                         (dv.ngroups ? (dv.ngroups + 1) * 4 + dv.ngroups + (dv.nA + 1) * 4 : 0) +
                         (dv.sidx ? dv.M * 8 + (dv.nS + 1) * 4 + (dv.nS + 31) / 32 * 4 : 0);
    out->groups = dv.ngroups;
    return ANN_OK;
}

extern "C" int ann_index_get_bridges(const ann_index *index, uint64_t *ids, int32_t *refs) {
    ANN_ARG(index && ids && refs, "index, ids and refs are required");
    const DevIndex &dv = index->dev;
    std::vector<uint32_t> offA(dv.nA + 1), leaf(dv.M > 0 ? dv.M : 1);
    ANN_CUDA(cudaMemcpy(offA.data(), dv.offA, 4 * (dv.nA + 1), cudaMemcpyDeviceToHost));
    if (dv.M > 0) {
        ANN_CUDA(cudaMemcpy(leaf.data(), dv.leaf, 4 * dv.M, cudaMemcpyDeviceToHost));
        ANN_CUDA(cudaMemcpy(refs, dv.brefs, 4 * dv.M * dv.b, cudaMemcpyDeviceToHost));
    }
    const uint64_t suf = (uint64_t)ipow(dv.n, dv.P - dv.PA);
    for (int64_t a = 0; a < dv.nA; a++)
        for (uint32_t j = offA[a]; j < offA[a + 1]; j++) ids[j] = (uint64_t)a * suf + leaf[j];
    return ANN_OK;
}

extern "C" int ann_index_lookup_bridges(const ann_index *index, const uint64_t *ids, int64_t nids, int32_t *refs) {
    ANN_ARG(index && (nids == 0 || (ids && refs)), "index, ids and refs are required");
    ANN_ARG(nids >= 0, "nids must be >= 0");
    const DevIndex &dv = index->dev;
    const uint64_t suf = (uint64_t)ipow(dv.n, dv.P - dv.PA);
    const uint64_t nb = (uint64_t)ipow(dv.n, dv.P);
    std::vector<uint32_t> offA(dv.nA + 1);
    ANN_CUDA(cudaMemcpy(offA.data(), dv.offA, 4 * (dv.nA + 1), cudaMemcpyDeviceToHost));
    std::vector<uint32_t> leaves;
    for (int64_t q = 0; q < nids; q++) {
        int32_t *out = refs + q * dv.b;
        for (int i = 0; i < dv.b; i++) out[i] = -1;
        ANN_ARG(ids[q] < nb, "bridge id out of range");
        const uint64_t a = ids[q] / suf, lf = ids[q] % suf;
        const uint32_t j0 = offA[a], j1 = offA[a + 1];
        if (j1 == j0) continue;
        leaves.resize(j1 - j0);
        ANN_CUDA(cudaMemcpy(leaves.data(), dv.leaf + j0, 4 * (size_t)(j1 - j0), cudaMemcpyDeviceToHost));
        const auto it = std::lower_bound(leaves.begin(), leaves.end(), (uint32_t)lf);
        if (it == leaves.end() || *it != (uint32_t)lf) continue;
        const int64_t j = j0 + (it - leaves.begin());
        ANN_CUDA(cudaMemcpy(out, dv.brefs + j * dv.b, 4 * (size_t)dv.b, cudaMemcpyDeviceToHost));
    }
    return ANN_OK;
}

// ---- file format: header, X, graph, centers, bridge ids (uint64), refs (M*b) ----
struct FileHeader {
    char magic[8];
    int32_t version, dtype;
    int64_t N;
    int32_t d, R, P, n, t, b;
    int64_t M;
};

extern "C" int ann_index_save(const ann_index *index, const char *path) {
    ANN_ARG(index && path, "index and path are required");
    const DevIndex &dv = index->dev;
    FileHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "ANNIDX1", 8);
    h.version = 1;
    h.dtype = dv.dtype;
    h.N = dv.N;
    h.d = dv.d;
    h.R = dv.R;
    h.P = dv.P;
    h.n = dv.n;
    h.t = dv.t;
    h.b = dv.b;
    h.M = dv.M;
    const size_t es = dv.dtype == ANN_U8 ? 1 : 4;
    std::vector<uint8_t> X((size_t)dv.N * dv.d * es), C((size_t)dv.P * dv.n * (dv.d / dv.P) * es);
    std::vector<int32_t> G((size_t)dv.N * dv.R), refs((size_t)std::max<int64_t>(dv.M * dv.b, 1));
    std::vector<uint64_t> ids((size_t)std::max<int64_t>(dv.M, 1));
    ANN_CUDA(cudaMemcpy(X.data(), dv.X, X.size(), cudaMemcpyDeviceToHost));
    ANN_CUDA(cudaMemcpy(G.data(), dv.G, 4 * G.size(), cudaMemcpyDeviceToHost));
    ANN_CUDA(cudaMemcpy(C.data(), dv.C, C.size(), cudaMemcpyDeviceToHost));
    int r = ann_index_get_bridges(index, ids.data(), refs.data());
    if (r != ANN_OK) return r;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ANN_ERR_ARG, std::string("cannot open for writing: ") + path);
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(X.data(), 1, X.size(), f) == X.size() &&
              fwrite(G.data(), 4, G.size(), f) == G.size() && fwrite(C.data(), 1, C.size(), f) == C.size() &&
              fwrite(ids.data(), 8, (size_t)dv.M, f) == (size_t)dv.M &&
              fwrite(refs.data(), 4, (size_t)(dv.M * dv.b), f) == (size_t)(dv.M * dv.b);
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(ANN_ERR_ARG, std::string("write failed: ") + path);
    return ANN_OK;
}

extern "C" int ann_index_load(const char *path, int device, ann_index **out) {
    ANN_ARG(path && out, "path and out are required");
    if (device >= 0) ANN_CUDA(cudaSetDevice(device));
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ANN_ERR_ARG, std::string("cannot open: ") + path);
    FileHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, "ANNIDX1", 8) != 0 || h.version != 1) {
        fclose(f);
        return fail(ANN_ERR_FORMAT, "not an index file (bad magic or version)");
    }
    if ((h.dtype != ANN_U8 && h.dtype != ANN_F32) || h.N < 1 || h.P < 2 || h.P > kMaxP || h.n < 1 ||
        h.n > kMaxN || h.d < 1 || h.d % h.P || h.R < 1 || h.R > kMaxR || h.b < 1 || h.b > kMaxB || h.M < 0 ||
        h.M > h.N * (int64_t)h.t) {
        fclose(f);
        return fail(ANN_ERR_FORMAT, "index header out of range");
    }
    const size_t es = h.dtype == ANN_U8 ? 1 : 4;
    std::vector<uint8_t> X((size_t)h.N * h.d * es), C((size_t)h.P * h.n * (h.d / h.P) * es);
    std::vector<int32_t> G((size_t)h.N * h.R), refs((size_t)std::max<int64_t>(h.M * h.b, 1));
    std::vector<uint64_t> ids((size_t)std::max<int64_t>(h.M, 1));
    bool ok = fread(X.data(), 1, X.size(), f) == X.size() && fread(G.data(), 4, G.size(), f) == G.size() &&
              fread(C.data(), 1, C.size(), f) == C.size() && fread(ids.data(), 8, (size_t)h.M, f) == (size_t)h.M &&
              fread(refs.data(), 4, (size_t)(h.M * h.b), f) == (size_t)(h.M * h.b);
    fclose(f);
    if (!ok) return fail(ANN_ERR_FORMAT, "index file truncated");
    // CSR offsets from the padded lists
    std::vector<int64_t> offs((size_t)h.M + 1);
    std::vector<int32_t> flat;
    flat.reserve((size_t)h.M * h.b);
    offs[0] = 0;
    for (int64_t j = 0; j < h.M; j++) {
        for (int i = 0; i < h.b; i++)
            if (refs[j * h.b + i] >= 0) flat.push_back(refs[j * h.b + i]);
        offs[j + 1] = (int64_t)flat.size();
    }
    void *dX = nullptr, *dC = nullptr;
    int32_t *dG = nullptr;
    // staging copies on the device, freed on every return (the index copies them)
    struct Staged {
        void *p[3] = {};
        ~Staged() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } staged;
    ANN_CUDA(cudaMalloc(&staged.p[0], X.size()));
    ANN_CUDA(cudaMalloc(&staged.p[1], 4 * G.size()));
    ANN_CUDA(cudaMalloc(&staged.p[2], C.size()));
    dX = staged.p[0];
    dG = (int32_t *)staged.p[1];
    dC = staged.p[2];
    ANN_CUDA(cudaMemcpy(dX, X.data(), X.size(), cudaMemcpyHostToDevice));
    ANN_CUDA(cudaMemcpy(dG, G.data(), 4 * G.size(), cudaMemcpyHostToDevice));
    ANN_CUDA(cudaMemcpy(dC, C.data(), C.size(), cudaMemcpyHostToDevice));
    ann_index_desc d;
    memset(&d, 0, sizeof(d));
    d.dtype = h.dtype;
    d.N = h.N;
    d.d = h.d;
    d.R = h.R;
    d.P = h.P;
    d.n = h.n;
    d.t = h.t;
    d.b = h.b;
    d.data = dX;
    d.graph = dG;
    d.centers = dC;
    d.M = h.M;
    d.bridge_ids = ids.data();
    d.bridge_offsets = offs.data();
    d.bridge_refs = flat.data();
    return ann_index_create(&d, out);
}
