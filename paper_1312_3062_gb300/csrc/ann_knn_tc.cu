// ann_knn_tc.cu -- exact k nearest neighbours of uint8 vectors on the 5th
// generation tensor cores (tcgen05) of sm_103a: the R-NN neighbourhood graph
// of Sec. 3.1 / Sec. 4.1 and the linear-scan ground truth of Sec. 5.1.
//
// Keys are ||a||^2 + ||b||^2 - 2 a.b.  Bytes 0..255 are exact in bf16, every
// product is an integer below 2^16 and every partial sum of a row of d <= 128
// products is an integer below 2^24, so the bf16 MMA with fp32 accumulation
// returns the exact integer dot product; the key is then formed exactly in
// fp32 (all terms below 2^24) and compared as an integer.
//
// One CTA per SM, persistent over blocks of 128 query rows:
//   warp 0      TMA producer: the query block (A, 128 x d bf16) once per
//               block, reference tiles (B, 256 x d bf16) through a 2-stage ring
//   warp 1      allocates 512 TMEM columns; one lane issues tcgen05.mma
//               (M=128, N=256, K=16) into one of two 256-column accumulators
//   warps 2..9  epilogue: tcgen05.ld of the accumulator, key, threshold test
//               against the row's current k-th best, rare sorted insertion.
//               Two warps share each TMEM lane quadrant (one per column half)
//               and keep separate lists that are merged at the end of a block.
// Every mbarrier wait is bounded; on timeout the CTA records an error and
// every role leaves its loop, so the kernel always returns and frees TMEM.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ann_device.cuh"
#include "ann_internal.cuh"

namespace ann {
namespace tc {

constexpr int BM = 128;           // query rows per block (TMEM lanes)
constexpr int BN = 256;           // reference rows per tile (accumulator columns)
constexpr int BK = 64;            // bf16 elements per TMA box row (128 B, one swizzle row)
constexpr int STAGES = 2;
constexpr int NUM_THREADS = 320;  // 10 warps

struct Params {
    int64_t nq, N;
    int d, k, exclude_self;
    const uint32_t *qnorm, *rnorm;
    int32_t *out_ids;
    uint32_t *out_keys;
    int *error;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait (2 s) for the phase with the given parity; false on timeout or
// when another role has already recorded an error
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *err) {
    const uint32_t a = smem_u32(bar);
    if (*err) return false;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0;; it++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 255) {
            if (*err) return false;
            if (globaltimer_ns() - t0 > 2000000000ull) break;
        }
    }
    *err = 1;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;            // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                  // descriptor version for sm_100-class tensor cores
    d |= (uint64_t)2 << 61;                  // layout: 128-byte swizzle
    return d;
}

// instruction descriptor: kind::f16, A and B bf16, D f32, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4)                   // D format f32
           | (1u << 7)                 // A format bf16
           | (1u << 10)                // B format bf16
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// shared memory plan (bytes, 1024-aligned tiles)
struct Smem {
    __host__ __device__ static constexpr int a_bytes(int d) { return BM * d * 2; }
    __host__ __device__ static constexpr int b_bytes(int d) { return BN * d * 2; }
};

__global__ void __launch_bounds__(NUM_THREADS, 1)
    knn_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Params prm,
                  uint64_t *half_lists) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // align the dynamic shared memory base to 1024 bytes (swizzle atoms)
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int d = prm.d, k = prm.k;
    const int kch = d / BK;                       // TMA boxes per row block
    uint8_t *sA = smem;                           // kch x [BM rows x 128 B]
    uint8_t *sB = sA + Smem::a_bytes(d);          // STAGES x kch x [BN rows x 128 B]
    uint64_t *lists = (uint64_t *)(sB + STAGES * Smem::b_bytes(d));  // [8 epilogue warps][32 rows][k]
    uint32_t *rn_s = (uint32_t *)(lists + 8 * 32 * k);                // [8 epilogue warps][BN/2]
    uint64_t *bars = (uint64_t *)(rn_s + 8 * (BN / 2));
    uint64_t *full = bars;                        // STAGES
    uint64_t *empty = bars + STAGES;              // STAGES
    uint64_t *tfull = bars + 2 * STAGES;          // 2
    uint64_t *tempty = bars + 2 * STAGES + 2;     // 2
    uint64_t *afull = bars + 2 * STAGES + 4;      // 1
    uint64_t *aempty = bars + 2 * STAGES + 5;     // 1
    uint64_t *mdone = bars + 2 * STAGES + 6;      // 1: every MMA issued so far has completed
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 7);
    __shared__ int s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nblocks = (prm.nq + BM - 1) / BM;
    const int64_t ntiles = (prm.N + BN - 1) / BN;

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 8);  // one arrival per epilogue warp
        }
        mbar_init(afull, 1);
        mbar_init(aempty, 1);
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_base = *tmem_slot;
    volatile int *err = &s_err;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int64_t g = 0;  // global tile counter (ring position)
            int64_t nb = 0;
            int64_t last_use[STAGES];
            for (int s = 0; s < STAGES; s++) last_use[s] = -1;
            int64_t a_loads = 0;
            for (int64_t blk = blockIdx.x; blk < nblocks && !*err; blk += gridDim.x, nb++) {
                if (nb > 0 && !mbar_wait(aempty, (uint32_t)((nb - 1) & 1), err)) break;
                mbar_expect_tx(afull, (uint32_t)Smem::a_bytes(d));
                for (int c = 0; c < kch; c++)
                    tma_load_2d(sA + c * BM * 128, &mapA, afull, c * BK, (int)(blk * BM));
                a_loads++;
                bool ok = true;
                for (int64_t t = 0; t < ntiles; t++, g++) {
                    const int s = (int)(g % STAGES);
                    const int64_t use = g / STAGES;
                    if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), err)) {
                        ok = false;
                        break;
                    }
                    uint8_t *dst = sB + s * Smem::b_bytes(d);
                    mbar_expect_tx(&full[s], (uint32_t)Smem::b_bytes(d));
                    for (int c = 0; c < kch; c++)
                        tma_load_2d(dst + c * BN * 128, &mapB, &full[s], c * BK, (int)(t * BN));
                    last_use[s] = use;
                }
                if (!ok) break;
            }
            // do not leave copies in flight: wait (bounded) for the last load of every buffer
            volatile int drain_err = 0;
            for (int s = 0; s < STAGES; s++)
                if (last_use[s] >= 0) mbar_wait(&full[s], (uint32_t)(last_use[s] & 1), &drain_err);
            if (a_loads > 0) mbar_wait(afull, (uint32_t)((a_loads - 1) & 1), &drain_err);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc(BM, BN);
            int64_t g = 0, u = 0;  // ring position, accumulator use counter
            int64_t nb = 0;
            for (int64_t blk = blockIdx.x; blk < nblocks && !*err; blk += gridDim.x, nb++) {
                if (!mbar_wait(afull, (uint32_t)(nb & 1), err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool ok = true;
                for (int64_t t = 0; t < ntiles; t++, g++, u++) {
                    const int s = (int)(g % STAGES);
                    const int acc = (int)(u & 1);
                    const int64_t ause = u >> 1;
                    if ((ause > 0 && !mbar_wait(&tempty[acc], (uint32_t)((ause - 1) & 1), err)) ||
                        !mbar_wait(&full[s], (uint32_t)((g / STAGES) & 1), err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dcol = tmem_base + (uint32_t)(acc * BN);
                    const uint8_t *b0 = sB + s * Smem::b_bytes(d);
                    for (int c = 0; c < kch; c++)
                        for (int kk = 0; kk < BK / 16; kk++) {
                            uint64_t ad = smem_desc(sA + c * BM * 128 + kk * 32);
                            uint64_t bd = smem_desc(b0 + c * BN * 128 + kk * 32);
                            mma_bf16(dcol, ad, bd, idesc, (c | kk) != 0);
                        }
                    mma_commit(&empty[s]);     // B stage free once these MMAs are done
                    mma_commit(&tfull[acc]);   // accumulator ready for the epilogue
                }
                if (!ok) break;
                mma_commit(aempty);            // query block may be replaced
            }
            // every MMA issued has completed before TMEM is released (bounded wait)
            mma_commit(mdone);
            volatile int drain_err = 0;
            mbar_wait(mdone, 0, &drain_err);
        }
    } else {
        // ---------------- epilogue ----------------
        const int ew = warp - 2;              // 0..7
        const int quad = warp & 3;            // TMEM lane quadrant this warp may access
        const int half = ew >> 2;             // column half
        const int row = quad * 32 + lane;     // row of the block
        uint64_t *mylist = lists + ((size_t)ew * 32 + lane) * k;
        float *myrn = (float *)(rn_s + ew * (BN / 2));
        int64_t u = 0;
        for (int64_t blk = blockIdx.x; blk < nblocks && !*err; blk += gridDim.x) {
            const int64_t qrow = blk * BM + row;
            const bool valid_row = qrow < prm.nq;
            const float qn = valid_row ? (float)prm.qnorm[qrow] : 0.f;
            for (int i = 0; i < k; i++) mylist[i] = ~0ull;
            uint64_t thr = ~0ull;             // current k-th entry of this list
            float thr_f = 1.0e20f;            // above every key (keys are below 2^25)
            bool ok = true;
            for (int64_t t = 0; t < ntiles; t++, u++) {
                const int acc = (int)(u & 1);
                // reference norms of this tile's column half as floats (exact below 2^24);
                // padding rows get a key no list accepts
                const int64_t r0 = t * BN;
                for (int c = lane; c < BN / 2; c += 32) {
                    const int64_t rid = r0 + half * (BN / 2) + c;
                    myrn[c] = rid < prm.N ? (float)prm.rnorm[rid] : 1.0e30f;
                }
                __syncwarp();
                if (!mbar_wait(&tfull[acc], (uint32_t)((u >> 1) & 1), err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int cb = 0; cb < BN / 2; cb += 32) {
                    const int col0 = half * (BN / 2) + cb;
                    uint32_t v[32];
                    __syncwarp();
                    tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * BN + col0), v);
                    // 32 exact keys without branches; the list is touched only when one beats its k-th entry
                    float kk[32];
                    float mn = 1.0e30f;
#pragma unroll
                    for (int j4 = 0; j4 < 8; j4++) {
                        const float4 r4 = *(const float4 *)(myrn + cb + 4 * j4);
                        const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const int j = 4 * j4 + q;
                            kk[j] = __fmaf_rn(-2.0f, __uint_as_float(v[j]), qn + rr[q]);
                            mn = fminf(mn, kk[j]);
                        }
                    }
                    if (valid_row && mn <= thr_f) {
#pragma unroll
                        for (int j = 0; j < 32; j++) {
                            const float kf = kk[j];
                            if (kf <= thr_f) {
                                const int64_t rid = r0 + col0 + j;
                                if (rid < prm.N && !(prm.exclude_self && rid == qrow)) {
                                    const uint64_t e = ((uint64_t)(uint32_t)kf << 32) | (uint32_t)rid;
                                    if (e < thr) {
                                        int p = k - 1;
                                        while (p > 0 && mylist[p - 1] > e) {
                                            mylist[p] = mylist[p - 1];
                                            p--;
                                        }
                                        mylist[p] = e;
                                        thr = mylist[k - 1];
                                        thr_f = thr == ~0ull ? 1.0e20f : (float)(uint32_t)(thr >> 32);
                                    }
                                }
                            }
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[acc]);
            }
            if (!ok) break;
            // this warp's list for its rows and column half; merged by a second kernel
            if (valid_row) {
                uint64_t *dst = half_lists + ((size_t)qrow * 2 + half) * k;
                for (int i = 0; i < k; i++) dst[i] = mylist[i];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base));
    }
    if (threadIdx.x == 0 && s_err) atomicExch(prm.error, 1);
}

// merge the two column halves' sorted lists of every row
__global__ void merge_halves_kernel(const uint64_t *half_lists, int64_t nq, int k, int32_t *out_ids,
                                    uint32_t *out_keys) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const uint64_t *la = half_lists + (size_t)q * 2 * k;
    const uint64_t *lb = la + k;
    int ia = 0, ib = 0;
    for (int i = 0; i < k; i++) {
        uint64_t e;
        if (ia < k && (ib >= k || la[ia] <= lb[ib])) e = la[ia++];
        else e = lb[ib++];
        const bool have = e != ~0ull;
        out_ids[q * k + i] = have ? (int32_t)(uint32_t)e : -1;
        if (out_keys) out_keys[q * k + i] = have ? (uint32_t)(e >> 32) : 0xffffffffu;
    }
}

__global__ void to_bf16_kernel(const uint8_t *src, int64_t n, uint16_t *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // bytes are exact in bf16: the bf16 bits of an integer 0..255 via float
    const float f = (float)src[i];
    dst[i] = (uint16_t)(__float_as_uint(f) >> 16);
}

__global__ void norms_kernel(const uint8_t *X, int64_t N, int d, uint32_t *out) {
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

// ---- driver entry point for tensor-map encoding (no link against libcuda) ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

static int make_map(CUtensorMap *map, const uint16_t *base, int64_t rows, int d, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(ANN_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)d * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ANN_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return ANN_OK;
}

size_t smem_bytes(int d, int k) {
    return 1024 /* alignment slack */ + (size_t)Smem::a_bytes(d) + (size_t)STAGES * Smem::b_bytes(d) +
           (size_t)8 * 32 * k * 8 + (size_t)8 * (BN / 2) * 4 + (2 * STAGES + 7) * 8 + 16;
}

}  // namespace tc

// Whether the tensor-core kernel's shared memory for (d, k) fits a CTA.
bool knn_u8_tensor_fits(int d, int k) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return tc::smem_bytes(d, k) <= (size_t)optin;
}

// Exact k-NN of uint8 rows on the tensor cores.  Requires d in {64, 128}.
int knn_u8_tensor(const uint8_t *refs, int64_t N, const uint8_t *queries, int64_t nq, int d, int k,
                  int exclude_self, int32_t *out_ids, uint32_t *out_keys, cudaStream_t s) {
    using namespace tc;
    const size_t smem = smem_bytes(d, k);
    int dev = 0, nsm = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    ANN_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const bool shared = queries == refs && nq <= N;  // queries are the first nq reference rows
    uint16_t *rb = nullptr, *qb = nullptr;
    uint32_t *rn = nullptr, *qn = nullptr;
    int *derr = nullptr;
    uint64_t *hl = nullptr;
    AsyncBufs bufs(s);  // every buffer below is released on return
    ANN_CUDA(bufs.alloc(&hl, (size_t)nq * 2 * k * 8));
    ANN_CUDA(bufs.alloc(&rb, (size_t)N * d * 2));
    ANN_CUDA(bufs.alloc(&rn, (size_t)N * 4));
    ANN_CUDA(bufs.alloc(&derr, sizeof(int)));
    ANN_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s));
    to_bf16_kernel<<<(unsigned)((N * d + 255) / 256), 256, 0, s>>>(refs, N * d, rb);
    norms_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(refs, N, d, rn);
    if (shared) {
        qb = rb;
        qn = rn;
    } else {
        ANN_CUDA(bufs.alloc(&qb, (size_t)nq * d * 2));
        ANN_CUDA(bufs.alloc(&qn, (size_t)nq * 4));
        to_bf16_kernel<<<(unsigned)((nq * d + 255) / 256), 256, 0, s>>>(queries, nq * d, qb);
        norms_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(queries, nq, d, qn);
    }
    CUtensorMap mapA, mapB;
    int r = make_map(&mapA, qb, nq, d, BM);
    if (r == ANN_OK) r = make_map(&mapB, rb, N, d, BN);
    if (r == ANN_OK) {
        Params prm{nq, N, d, k, exclude_self, qn, rn, out_ids, out_keys, derr};
        cudaError_t e = cudaFuncSetAttribute(knn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            r = cuda_fail(e, "cudaFuncSetAttribute(knn_tc_kernel)");
        } else {
            const int64_t nblocks = (nq + BM - 1) / BM;
            const unsigned grid = (unsigned)(nblocks < nsm ? nblocks : nsm);
            knn_tc_kernel<<<grid, NUM_THREADS, smem, s>>>(mapA, mapB, prm, hl);
            merge_halves_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(hl, nq, k, out_ids, out_keys);
            e = cudaGetLastError();
            if (e != cudaSuccess) r = cuda_fail(e, "knn_tc_kernel launch");
        }
    }
    int herr = 0;
    if (r == ANN_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) r = cuda_fail(e, "knn_tc_kernel");
    }
    if (r == ANN_OK && herr) r = fail(ANN_ERR_TIMEOUT, "knn_tc_kernel: a pipeline wait timed out");
    return r;
}

}  // namespace ann
