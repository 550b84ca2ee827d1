// ann_search.cu -- host side of Algorithm 1 (Sec. 4.2): launch planning, the
// plain, persistent (CUDA graph, autotuned) forms and the C entry point.  The
// device code is in ann_search_dev.cuh.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ann_search_dev.cuh"

namespace ann {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int g_num_sms = 0;
static size_t g_smem_optin = 0;

static int device_props() {
    if (g_num_sms) return ANN_OK;
    int dev;
    ANN_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    ANN_CUDA(cudaGetDeviceProperties(&prop, dev));
    g_num_sms = prop.multiProcessorCount;
    g_smem_optin = prop.sharedMemPerBlockOptin;
    // stream-ordered scratch allocations reuse the pool instead of returning memory at every sync
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return ANN_OK;
}

// Budgets from this size on use per-warp global scratch: sorted bridge windows
// (one walk then serves many batches, which pays off when queries pop many
// bridges), and the queue's overflow and the visited set, so the shared-memory
// slice of a query no longer grows with its budget.
static const int kWindowedFromT = 1024;

// Launch configuration for a budget bucket: warps per CTA and batch capacity.
struct Tune {
    int warps;
    int bcap;
    bool stage;         // stage the next pop's neighbour vectors (cp.async)
    bool tickets = true;  // persistent form: pull queries from a ticket (else a fixed grid-stride share)
    int spill_heap = (int)kSpillHeap;  // large budgets: queue entries kept in shared memory
};

// Warps per CTA: the count that keeps the most warps resident per SM given
// the per-warp shared-memory slice (ties go to more warps per CTA).
static Tune choose_tune_heap(const DevIndex &ix, int capT, int kmax, int spill_heap) {
    Tune t;
    t.spill_heap = spill_heap;
    // bridge batch: budgets below the windowed kernels pop few bridges
    t.bcap = capT >= kWindowedFromT ? 128 : 64;
    t.stage = true;
    WarpLayout L = make_layout(ix.dtype, ix.d, ix.P, ix.n, ix.PA, capT, kmax, t.bcap, ix.b, ix.R, true,
                               ix.ngroups > 0, capT >= kWindowedFromT, (uint32_t)t.spill_heap);
    const size_t per_sm = 228 * 1024, per_cta_reserved = 1024;
    size_t budget = g_smem_optin ? g_smem_optin : 227 * 1024;
    // register-file limit of the kernel (both instantiations use the same budget)
    static int regs = 0;
    if (!regs) {
        cudaFuncAttributes fa;
        regs = cudaFuncGetAttributes(&fa, search_kernel<ANN_U8, false, false>) == cudaSuccess ? fa.numRegs : 168;
        if (regs < 32) regs = 32;
    }
    const int warps_by_regs = 65536 / (regs * 32);
    int best_w = 1, best_res = 0;
    for (int w = 1; w <= 6; w++) {
        size_t cta = (size_t)w * L.total;
        if (cta > budget) break;
        int ctas = (int)(per_sm / (cta + per_cta_reserved));
        if (ctas > 32 / w) ctas = 32 / w;
        if (ctas > warps_by_regs / w) ctas = warps_by_regs / w;
        int res = ctas * w;
        if (res >= best_res) {
            best_res = res;
            best_w = w;
        }
    }
    t.warps = best_w;
    return t;
}

static Tune choose_tune(const DevIndex &ix, int capT, int kmax) {
    return choose_tune_heap(ix, capT, kmax, (int)kSpillHeap);
}


// The dynamic shared-memory limit of a kernel is a property of the function,
// read again whenever a launch (or a graph node) is checked, so it is raised
// once to the device's opt-in maximum rather than set per launch: a captured
// graph may hold nodes of one kernel with different sizes.
template <int DT, bool WIN>
static cudaError_t config_kernel(size_t smem, int threads, int *blocks_per_sm) {
    static bool raised = false;
    if (!raised) {
        cudaError_t e = cudaFuncSetAttribute(search_kernel<DT, WIN, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_smem_optin);
        if (e != cudaSuccess) return e;
        raised = true;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<DT, WIN, false>, threads, smem);
}

// Launch configuration of one search launch: layout, grid and the size of the
// per-warp global scratch (windowed kernels only).
struct LaunchCfg {
    SearchArgs A;
    dim3 grid, block;
    size_t smem;
    bool win;
    size_t scratch_bytes;
};

static int plan_launch(const SearchArgs &base, int capT, bool persistent, const int32_t *list,
                       const int32_t *list_count, int64_t list_len, int32_t *ticket, LaunchCfg &cfg,
                       const Tune *tune = nullptr) {
    SearchArgs A = base;
    A.capT = capT;
    const Tune tn = tune ? *tune : choose_tune(A.ix, capT, A.kmax);
    A.bcap = tn.bcap;
    A.L = make_layout(A.ix.dtype, A.ix.d, A.ix.P, A.ix.n, A.ix.PA, capT, A.kmax, tn.bcap, A.ix.b, A.ix.R,
                      tn.stage, A.ix.ngroups > 0, capT >= kWindowedFromT, (uint32_t)tn.spill_heap);
    A.list = list;
    A.list_count = list_count;
    A.list_len = list_len;
    A.ticket = (persistent && tn.tickets) ? ticket : nullptr;
    const bool win = capT >= kWindowedFromT;
    uint32_t gcap = (uint32_t)(2 * capT);
    if (gcap > 8192) gcap = 8192;
    A.gcap = win ? gcap : 0;
    // per-warp scratch: windows, then the queue's overflow, then the visited set
    auto al = [](uint64_t x) { return (x + 255) & ~(uint64_t)255; };
    A.spill_off = win ? al((uint64_t)gcap * 24) : 0;
    A.hash_off = win ? A.spill_off + al(8ull * (uint64_t)capT) : 0;
    A.wstride = win ? A.hash_off + al(4ull << A.L.hash_log) : 0;
    size_t smem = (size_t)A.L.total * tn.warps;
    if (smem > g_smem_optin) return fail(ANN_ERR_CAPACITY, "per-query state exceeds shared memory");
    int blocks_per_sm = 0;
    const int threads = tn.warps * 32;
    cudaError_t e;
    if (A.ix.ngroups > 0)
        e = config_grouped(A.ix.dtype, win, smem, threads, &blocks_per_sm);
    else if (A.ix.dtype == ANN_U8)
        e = win ? config_kernel<ANN_U8, true>(smem, threads, &blocks_per_sm)
                : config_kernel<ANN_U8, false>(smem, threads, &blocks_per_sm);
    else
        e = win ? config_kernel<ANN_F32, true>(smem, threads, &blocks_per_sm)
                : config_kernel<ANN_F32, false>(smem, threads, &blocks_per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "search kernel configuration");
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const int64_t cap = (int64_t)g_num_sms * blocks_per_sm;
    // ticket queue: one wave; fixed shares: up to four waves, sized by the
    // query count when it is known on the host
    const bool by_ticket = persistent && ticket && tn.tickets;
    int64_t want = by_ticket ? cap : (list_count ? cap * 4 : (list_len + tn.warps - 1) / tn.warps);
    // plain launches grid-stride beyond four waves; windowed ones beyond one wave (bounded scratch)
    const int64_t lim = win ? cap : cap * 4;
    if (want > lim) want = lim;
    if (want < 1) want = 1;
    cfg.A = A;
    cfg.grid = dim3((unsigned)want);
    cfg.block = dim3(threads);
    cfg.smem = smem;
    cfg.win = win;
    cfg.scratch_bytes = win ? (size_t)want * tn.warps * A.wstride : 0;
    return ANN_OK;
}

static int do_launch(LaunchCfg &cfg, uint8_t *scratch, cudaStream_t stream) {
    cfg.A.gscratch = scratch;
    if (cfg.A.ix.ngroups > 0) {
        launch_grouped(cfg.A.ix.dtype, cfg.win, cfg.grid, cfg.block, cfg.smem, stream, cfg.A);
    } else if (cfg.A.ix.dtype == ANN_U8) {
        if (cfg.win) search_kernel<ANN_U8, true, false><<<cfg.grid, cfg.block, cfg.smem, stream>>>(cfg.A);
        else search_kernel<ANN_U8, false, false><<<cfg.grid, cfg.block, cfg.smem, stream>>>(cfg.A);
    } else {
        if (cfg.win) search_kernel<ANN_F32, true, false><<<cfg.grid, cfg.block, cfg.smem, stream>>>(cfg.A);
        else search_kernel<ANN_F32, false, false><<<cfg.grid, cfg.block, cfg.smem, stream>>>(cfg.A);
    }
    ANN_CUDA(cudaGetLastError());
    return ANN_OK;
}

// plan + stream-ordered scratch (windowed kernels) + launch
static int launch_search(const SearchArgs &base, int capT, cudaStream_t stream, bool persistent,
                         const int32_t *list, const int32_t *list_count, int64_t list_len,
                         int32_t *ticket) {
    LaunchCfg cfg;
    int r = plan_launch(base, capT, persistent, list, list_count, list_len, ticket, cfg);
    if (r != ANN_OK) return r;
    uint8_t *scratch = nullptr;
    if (cfg.scratch_bytes) ANN_CUDA(cudaMallocAsync((void **)&scratch, cfg.scratch_bytes, stream));
    r = do_launch(cfg, scratch, stream);
    if (scratch) cudaFreeAsync(scratch, stream);
    return r;
}

__global__ void max_kernel(const int32_t *v, int64_t n, int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(out, v[i]);
}

// ---- persistent mode: bucket queries by budget on the device ----
static const int kBuckets = 7;  // capT = 128 << i  (128 .. 8192)

__global__ void bucket_kernel(int64_t nq, const int32_t *T, int32_t T_all, int32_t *counts,
                              int32_t *lists, int32_t *tickets) {
    // counts[kBuckets], lists[kBuckets * nq]
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int t = T ? T[i] : T_all;
    int bkt = 0;
    while (bkt < kBuckets - 1 && t > (128 << bkt)) bkt++;
    int pos = atomicAdd(&counts[bkt], 1);
    lists[(int64_t)bkt * nq + pos] = (int32_t)i;
}

struct Plan {
    cudaGraphExec_t exec = nullptr;
    int32_t *scratch = nullptr;   // counts[kBuckets] + tickets[kBuckets] + lists[kBuckets*nq]
    uint8_t *wscratch = nullptr;  // per-warp sorted bridge windows (largest windowed bucket's need)
    uint64_t last_use = 0;        // for evicting the least recently used plan
};

// plans kept per index; the least recently used one goes beyond this
static const size_t kMaxPlans = 32;

struct PlanKey {
    const void *queries;
    int64_t nq;
    const int32_t *k, *T;
    int32_t k_all, T_all, kmax;
    int32_t *out_ids;
    void *out_keys;
    int32_t *out_status;
    int64_t *out_stats;
    cudaStream_t stream;
    bool operator<(const PlanKey &o) const {
        return std::tie(queries, nq, k, T, k_all, T_all, kmax, out_ids, out_keys, out_status, out_stats, stream) <
               std::tie(o.queries, o.nq, o.k, o.T, o.k_all, o.T_all, o.kmax, o.out_ids, o.out_keys, o.out_status,
                        o.out_stats, o.stream);
    }
};

struct PlanCache {
    std::mutex mu;
    uint64_t clock = 0;
    std::map<PlanKey, Plan> plans;
    std::map<std::pair<int, int>, Tune> tuned;  // (bucket capacity, kmax) -> measured best launch shape
};

void free_plans(ann_index *ix) {
    if (!ix->plans) return;
    PlanCache *pc = (PlanCache *)ix->plans;
    for (auto &kv : pc->plans) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.scratch) cudaFree(kv.second.scratch);
        if (kv.second.wscratch) cudaFree(kv.second.wscratch);
    }
    delete pc;
    ix->plans = nullptr;
}

// budgets of the buckets one persistent batch may use
static void bucket_range(const int32_t *T, int32_t T_all, int &b0, int &b1) {
    b1 = kBuckets - 1;
    if (!T) {
        b1 = 0;
        while (b1 < kBuckets - 1 && T_all > (128 << b1)) b1++;
    }
    b0 = T ? 0 : b1;
}

static const Tune *tuned_for(const PlanCache *pc, int capT, int kmax) {
    auto it = pc->tuned.find({capT, kmax});
    return it == pc->tuned.end() ? nullptr : &it->second;
}

static int bucket_cap(int bkt) { return (128 << bkt) > kMaxT ? kMaxT : (128 << bkt); }

// One replay of the persistent form.  A uniform budget is one bucket and the
// queries are taken in order; otherwise a device pass sorts them into
// buckets first.  Every bucket's kernel pulls its queries from a ticket.
// Buckets without global scratch run concurrently on forked streams (largest
// budget first), so the smaller ones fill the SMs the larger leave idle at
// their tail; windowed buckets share one scratch and run one after another.
// streams and events of the fork/join; they must outlive the capture
struct ForkSet {
    cudaStream_t side[kBuckets] = {};
    cudaEvent_t fork = nullptr, join[kBuckets] = {};
    int nside = 0;
    ~ForkSet() {
        for (int i = 0; i < nside; i++) {
            if (join[i]) cudaEventDestroy(join[i]);
            if (side[i]) cudaStreamDestroy(side[i]);
        }
        if (fork) cudaEventDestroy(fork);
    }
};

static int record_persistent(const PlanCache *pc, const SearchArgs &A, int64_t nq, const int32_t *T, int32_t T_all,
                             int32_t *scratch, uint8_t *wscratch, cudaStream_t s, ForkSet &fs) {
    int32_t *counts = scratch, *tickets = scratch + kBuckets, *lists = scratch + 2 * kBuckets;
    ANN_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int32_t) * 2 * kBuckets, s));
    if (T) {
        bucket_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(nq, T, T_all, counts, lists, tickets);
        ANN_CUDA(cudaGetLastError());
    }
    int b0, b1;
    bucket_range(T, T_all, b0, b1);
    int rc = ANN_OK;
    for (int bkt = b1; bkt >= b0 && rc == ANN_OK; bkt--) {
        const int capT = bucket_cap(bkt);
        LaunchCfg cfg;
        rc = T ? plan_launch(A, capT, true, lists + (int64_t)bkt * nq, counts + bkt, nq, tickets + bkt, cfg,
                             tuned_for(pc, capT, A.kmax))
               : plan_launch(A, capT, true, nullptr, nullptr, nq, tickets + bkt, cfg, tuned_for(pc, capT, A.kmax));
        if (rc != ANN_OK) break;
        if (cfg.win || b0 == b1) {
            rc = do_launch(cfg, wscratch, s);
            continue;
        }
        if (!fs.fork) {
            if (cudaEventCreateWithFlags(&fs.fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(fs.fork, s) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "fork event");
                break;
            }
        }
        const int i = fs.nside;
        if (cudaStreamCreateWithFlags(&fs.side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fs.join[i], cudaEventDisableTiming) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "side stream");
            break;
        }
        fs.nside++;
        if (cudaStreamWaitEvent(fs.side[i], fs.fork, 0) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "fork");
            break;
        }
        rc = do_launch(cfg, nullptr, fs.side[i]);
        if (rc != ANN_OK) break;
        if (cudaEventRecord(fs.join[i], fs.side[i]) != cudaSuccess || cudaStreamWaitEvent(s, fs.join[i], 0) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "join");
            break;
        }
    }
    return rc;
}

// Launch shapes worth measuring for a bucket: the analytic choice, fewer warps
// per CTA (finer CTA granularity, fewer registers per SM in use), the
// analytic choice without cp.async staging, with fixed shares instead of the
// ticket, and, for large budgets, other shared-memory heap capacities (a
// smaller heap leaves room for more resident queries, a larger one moves
// entries out less often).  All give identical results.
static std::vector<Tune> tune_candidates(const DevIndex &ix, int capT, int kmax) {
    const Tune d = choose_tune(ix, capT, kmax);
    std::vector<Tune> c{d};
    for (int w : {1, 2, 3, 4})
        if (w < d.warps) c.push_back(Tune{w, d.bcap, true, true});
    c.push_back(Tune{d.warps, d.bcap, false, true});
    c.push_back(Tune{d.warps, d.bcap, true, false});  // the plain form's fixed grid-stride shares
    if (capT >= kWindowedFromT)
        for (int hc : {256, 1024, 2048})
            if (hc < capT) {
                Tune t = d;
                t.spill_heap = hc;
                Tune a = choose_tune_heap(ix, capT, kmax, hc);
                t.warps = a.warps;
                c.push_back(t);
            }
    return c;
}

// Measure the candidates of every bucket this batch uses that has no measured
// choice yet, on (a prefix of) the batch itself, and keep the fastest.
static int autotune(PlanCache *pc, const SearchArgs &A, int64_t nq, const int32_t *T, int32_t T_all,
                    int32_t *scratch, cudaStream_t s) {
    int b0, b1;
    bucket_range(T, T_all, b0, b1);
    bool todo = false;
    for (int bkt = b0; bkt <= b1; bkt++) todo |= tuned_for(pc, bucket_cap(bkt), A.kmax) == nullptr;
    if (!todo) return ANN_OK;
    int32_t *counts = scratch, *tickets = scratch + kBuckets, *lists = scratch + 2 * kBuckets;
    int32_t *tcount = scratch + kBuckets * (2 + nq);  // one extra word: queries per tuning run
    ANN_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int32_t) * 2 * kBuckets, s));
    int32_t hc[kBuckets] = {0};
    if (T) {
        bucket_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(nq, T, T_all, counts, lists, tickets);
        ANN_CUDA(cudaGetLastError());
        ANN_CUDA(cudaMemcpyAsync(hc, counts, sizeof(hc), cudaMemcpyDeviceToHost, s));
        ANN_CUDA(cudaStreamSynchronize(s));
    } else {
        hc[b1] = (int32_t)nq;
    }
    cudaEvent_t e0, e1;
    ANN_CUDA(cudaEventCreate(&e0));
    ANN_CUDA(cudaEventCreate(&e1));
    int rc = ANN_OK;
    for (int bkt = b0; bkt <= b1 && rc == ANN_OK; bkt++) {
        const int capT = bucket_cap(bkt);
        if (tuned_for(pc, capT, A.kmax) || hc[bkt] == 0) continue;
        const std::vector<Tune> cands = tune_candidates(A.ix, capT, A.kmax);
        // tune on up to four rounds of the default shape's resident warps
        LaunchCfg c0;
        rc = plan_launch(A, capT, true, nullptr, nullptr, nq, tickets + bkt, c0, &cands[0]);
        if (rc != ANN_OK) break;
        const int64_t resident = (int64_t)c0.grid.x * (c0.block.x / 32);
        const int32_t ntune = (int32_t)std::min<int64_t>(hc[bkt], 4 * resident);
        ANN_CUDA(cudaMemcpyAsync(tcount, &ntune, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        const int32_t *list = T ? lists + (int64_t)bkt * nq : nullptr;
        float best_ms = 0.f;
        int best = -1;
        for (size_t ci = 0; ci < cands.size() && rc == ANN_OK; ci++) {
            float ms_min = 0.f;
            for (int rep = 0; rep < 2; rep++) {
                LaunchCfg cfg;
                if (plan_launch(A, capT, true, list, tcount, nq, tickets + bkt, cfg, &cands[ci]) != ANN_OK) break;
                uint8_t *ws = nullptr;
                if (cfg.scratch_bytes && cudaMallocAsync((void **)&ws, cfg.scratch_bytes, s) != cudaSuccess) break;
                cudaMemsetAsync(tickets + bkt, 0, sizeof(int32_t), s);
                cudaEventRecord(e0, s);
                rc = do_launch(cfg, ws, s);
                cudaEventRecord(e1, s);
                if (ws) cudaFreeAsync(ws, s);
                if (rc != ANN_OK) break;
                cudaError_t ce = cudaEventSynchronize(e1);
                if (ce != cudaSuccess) {
                    rc = cuda_fail(ce, "autotune run");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 0 || ms < ms_min) ms_min = ms;
                if (ms > 50.f) break;  // long runs: one measurement is enough
            }
            if (rc == ANN_OK && ms_min > 0.f && (best < 0 || ms_min < best_ms)) {
                best_ms = ms_min;
                best = (int)ci;
            }
        }
        cudaGetLastError();  // a candidate that failed to configure is simply not chosen
        if (rc == ANN_OK) pc->tuned[{capT, A.kmax}] = cands[best < 0 ? 0 : best];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int search_launch_plain(const ann_index *ix, const void *queries, int64_t nq, const int32_t *k, const int32_t *T,
                        int32_t kmax, int capT, int32_t *out_ids, void *out_keys, int32_t *out_status,
                        cudaStream_t stream) {
    int r = device_props();
    if (r != ANN_OK) return r;
    if (nq == 0) return ANN_OK;
    SearchArgs A{};
    A.ix = ix->dev;
    A.queries = queries;
    A.nq = nq;
    A.k = k;
    A.T = T;
    A.kmax = kmax;
    A.out_ids = out_ids;
    A.out_keys = out_keys;
    A.out_status = out_status;
    if (capT > kMaxT) capT = kMaxT;
    if (capT < 32) capT = 32;
    return launch_search(A, capT, stream, false, nullptr, nullptr, nq, nullptr);
}

int search_launch_list(const ann_index *ix, const void *queries, int64_t nq, const int32_t *k, const int32_t *T,
                       int32_t kmax, int capT, const int32_t *list, int64_t count, int32_t *out_ids, void *out_keys,
                       int32_t *out_status, cudaStream_t stream) {
    int r = device_props();
    if (r != ANN_OK) return r;
    if (nq == 0 || count == 0) return ANN_OK;
    SearchArgs A{};
    A.ix = ix->dev;
    A.queries = queries;
    A.nq = nq;
    A.k = k;
    A.T = T;
    A.kmax = kmax;
    A.out_ids = out_ids;
    A.out_keys = out_keys;
    A.out_status = out_status;
    if (capT > kMaxT) capT = kMaxT;
    if (capT < 32) capT = 32;
    return launch_search(A, capT, stream, false, list, nullptr, count, nullptr);
}

int search_bucket_of(int32_t T) {
    int b = 0;
    while (b < kBuckets - 1 && T > (128 << b)) b++;
    return b;
}

int search_bucket_cap(int bucket) { return bucket_cap(bucket); }

int search_num_buckets() { return kBuckets; }

}  // namespace ann

using namespace ann;

extern "C" int ann_search_batch(const ann_index *index, const void *queries, int64_t nq, const int32_t *k,
                                const int32_t *T, int32_t k_all, int32_t T_all, int32_t kmax, int32_t mode,
                                int32_t *out_ids, void *out_keys, int32_t *out_status, int64_t *out_stats,
                                void *stream) {
    ANN_ARG(index != nullptr, "index is NULL");
    ANN_ARG(nq >= 0 && nq < (1ll << 31), "nq out of range");
    ANN_ARG(kmax >= 1 && kmax <= kMaxK, "kmax must be in [1, 128]");
    ANN_ARG(mode == ANN_MODE_PLAIN || mode == ANN_MODE_PERSISTENT, "mode must be 0 (plain) or 1 (persistent)");
    ANN_ARG(nq == 0 || (queries && out_ids), "queries and out_ids are required");
    ANN_ARG(((uintptr_t)queries & 15) == 0, "queries must be 16-byte aligned");
    if (!k) ANN_ARG(k_all >= 0 && k_all <= kmax, "k_all must be in [0, kmax]");
    if (!T) ANN_ARG(T_all >= 0 && T_all <= kMaxT, "T_all must be in [0, 8192]");
    int r = device_props();
    if (r != ANN_OK) return r;
    if (nq == 0) return ANN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SearchArgs A{};
    A.ix = index->dev;
    A.queries = queries;
    A.nq = nq;
    A.k = k;
    A.T = T;
    A.k_all = k_all;
    A.T_all = T_all;
    A.kmax = kmax;
    A.out_ids = out_ids;
    A.out_keys = out_keys;
    A.out_status = out_status;
    A.out_stats = out_stats;
    if (mode == ANN_MODE_PLAIN) {
        // one launch sized for the largest budget in the batch
        int capT = T_all;
        if (T) {
            int32_t *dmax = nullptr, hmax = 0;
            AsyncBufs bufs(s);  // released at the end of this block
            ANN_CUDA(bufs.alloc(&dmax, sizeof(int32_t)));
            ANN_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int32_t), s));
            max_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(T, nq, dmax);
            ANN_CUDA(cudaMemcpyAsync(&hmax, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            ANN_CUDA(cudaStreamSynchronize(s));
            capT = hmax;
        }
        if (capT > kMaxT) capT = kMaxT;
        if (capT < 32) capT = 32;
        return launch_search(A, capT, s, false, nullptr, nullptr, nq, nullptr);
    }
    // persistent: bucket by budget, one persistent kernel per bucket, replayed as a CUDA graph
    ann_index *ixm = const_cast<ann_index *>(index);
    if (!ixm->plans) ixm->plans = new PlanCache();
    PlanCache *pc = (PlanCache *)ixm->plans;
    PlanKey key{queries, nq, k, T, k_all, T_all, kmax, out_ids, out_keys, out_status, out_stats, s};
    std::lock_guard<std::mutex> g(pc->mu);
    auto it = pc->plans.find(key);
    if (it == pc->plans.end() && pc->plans.size() >= kMaxPlans) {
        // evict the least recently used plan once its stream has finished with it
        auto old = pc->plans.begin();
        for (auto jt = pc->plans.begin(); jt != pc->plans.end(); ++jt)
            if (jt->second.last_use < old->second.last_use) old = jt;
        ANN_CUDA(cudaStreamSynchronize(old->first.stream));
        cudaGraphExecDestroy(old->second.exec);
        cudaFree(old->second.scratch);
        if (old->second.wscratch) cudaFree(old->second.wscratch);
        pc->plans.erase(old);
    }
    if (it == pc->plans.end()) {
        Plan p;
        ANN_CUDA(cudaMalloc(&p.scratch, sizeof(int32_t) * (2 * kBuckets + (size_t)kBuckets * nq + 1)));
        {
            int r = autotune(pc, A, nq, T, T_all, p.scratch, s);
            if (r != ANN_OK) {
                cudaFree(p.scratch);
                return r;
            }
            size_t need = 0;
            int b0, b1;
            bucket_range(T, T_all, b0, b1);
            for (int bkt = b0; bkt <= b1; bkt++) {
                LaunchCfg cfg;
                r = plan_launch(A, bucket_cap(bkt), true, nullptr, p.scratch, nq, p.scratch, cfg,
                                tuned_for(pc, bucket_cap(bkt), kmax));
                if (r != ANN_OK) {
                    cudaFree(p.scratch);
                    return r;
                }
                need = cfg.scratch_bytes > need ? cfg.scratch_bytes : need;
            }
            if (need) {
                cudaError_t ae = cudaMalloc(&p.wscratch, need);
                if (ae != cudaSuccess) {
                    cudaFree(p.scratch);
                    return cuda_fail(ae, "cudaMalloc(search scratch)");
                }
            }
        }
        auto drop = [&p]() {
            cudaFree(p.scratch);
            if (p.wscratch) cudaFree(p.wscratch);
        };
        cudaStream_t cap;
        cudaError_t ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            drop();
            return cuda_fail(ce, "cudaStreamCreateWithFlags");
        }
        cudaGraph_t graph;
        ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
            cudaStreamDestroy(cap);
            drop();
            return cuda_fail(ce, "cudaStreamBeginCapture");
        }
        int rr;
        {
            ForkSet fs;
            rr = record_persistent(pc, A, nq, T, T_all, p.scratch, p.wscratch, cap, fs);
            ce = cudaStreamEndCapture(cap, &graph);
        }
        cudaStreamDestroy(cap);
        if (rr != ANN_OK || ce != cudaSuccess) {
            if (ce == cudaSuccess) cudaGraphDestroy(graph);
            drop();
            return rr != ANN_OK ? rr : cuda_fail(ce, "cudaStreamEndCapture");
        }
        ce = cudaGraphInstantiate(&p.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            drop();
            return cuda_fail(ce, "cudaGraphInstantiate");
        }
        it = pc->plans.emplace(key, p).first;
    }
    it->second.last_use = ++pc->clock;
    ANN_CUDA(cudaGraphLaunch(it->second.exec, s));
    return ANN_OK;
}
