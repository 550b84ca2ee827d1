// ann_serve.cu -- serving loop: continuous batching with memory-based
// admission over a resident index.
//
// Submitted requests wait in a FIFO.  A host thread admits as many waiting
// requests as fit both a free stream slot and the device scratch pool
// (inputs + outputs of the merged batch), packs their queries into one pinned
// staging buffer, sorts them on the host into the persistent form's budget
// buckets, and launches copy-in, one Algorithm 1 launch per non-empty bucket
// (each sized for its own budget, largest first) and copy-out on the slot's
// stream.  Batches on different slots overlap on the
// GPU; requests that arrive while others run are admitted as soon as a slot
// and scratch free up.  Completion is signalled by a host function enqueued
// behind the copy-out (no device-side waiting).  Each query's result does not
// depend on which other queries share its batch.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ann_internal.cuh"

namespace ann {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    int32_t nq, kmax;
    std::vector<uint8_t> queries;
    std::vector<int32_t> k, T;
    std::vector<int32_t> ids;
    std::vector<uint32_t> keys;
    std::vector<int32_t> status;
    Clock::time_point t_submit, t_done;
    bool done = false;
};

// first-fit allocator over [0, size)
struct Pool {
    size_t size;
    std::map<size_t, size_t> free_;  // offset -> length
    explicit Pool(size_t s) : size(s) { free_[0] = s; }
    bool alloc(size_t len, size_t &off) {
        len = (len + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                off = it->first;
                size_t rest = it->second - len;
                size_t o2 = it->first + len;
                free_.erase(it);
                if (rest) free_[o2] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len) {
        len = (len + 255) & ~size_t(255);
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Slot {
    std::condition_variable *cv = nullptr;  // the server's wake-up
    cudaStream_t stream = nullptr;
    uint8_t *h_in = nullptr;   // pinned: queries, then k, then T
    uint8_t *h_out = nullptr;  // pinned: ids, keys, status
    bool busy = false;
    std::atomic<bool> finished{false};
    size_t pool_off = 0, pool_len = 0;
    std::vector<std::shared_ptr<Request>> reqs;
    int32_t nq = 0, kmax = 0;
};

static const int kServeMaxBatch = 8192;

}  // namespace ann

struct ann_server {
    const ann_index *index;
    size_t vbytes;  // bytes per query vector
    uint8_t *pool_base = nullptr;
    std::unique_ptr<ann::Pool> pool;
    std::vector<std::unique_ptr<ann::Slot>> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<ann::Request>> waiting;
    std::unordered_map<uint64_t, std::shared_ptr<ann::Request>> live;
    std::unordered_map<uint64_t, double> done_latency;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int device = 0;
    std::string thread_error;
};

namespace ann {

static size_t batch_bytes(const ann_server *s, int64_t nq, int32_t kmax) {
    size_t a = ((size_t)nq * s->vbytes + 255) & ~size_t(255);
    a += ((size_t)nq * 12 + 255) & ~size_t(255);             // k, T, query order by bucket
    a += ((size_t)nq * kmax * 8 + 255) & ~size_t(255);       // ids, keys
    a += ((size_t)nq * 4 + 255) & ~size_t(255);              // status
    return a;
}

static void CUDART_CB on_done(void *p) {
    Slot *sl = (Slot *)p;
    sl->finished.store(true, std::memory_order_release);
    sl->cv->notify_all();
}

// launch one merged batch on a free slot (called with the lock held)
static bool launch_batch(ann_server *S, Slot &sl, std::vector<std::shared_ptr<Request>> &batch, int32_t nq,
                         int32_t kmax, size_t off, size_t len) {
    const size_t vb = S->vbytes;
    uint8_t *h = sl.h_in;
    size_t qo = 0;
    int32_t *hk = (int32_t *)(h + (size_t)kServeMaxBatch * vb);
    int32_t *hT = hk + kServeMaxBatch;
    int32_t *hl = hT + kServeMaxBatch;  // batch positions grouped by budget bucket
    int32_t at = 0;
    for (auto &r : batch) {
        memcpy(h + qo, r->queries.data(), (size_t)r->nq * vb);
        qo += (size_t)r->nq * vb;
        memcpy(hk + at, r->k.data(), 4 * (size_t)r->nq);
        memcpy(hT + at, r->T.data(), 4 * (size_t)r->nq);
        at += r->nq;
    }
    const int nb = search_num_buckets();
    std::vector<int32_t> bstart(nb + 1, 0), bfill(nb, 0);
    for (int32_t i = 0; i < nq; i++) bstart[search_bucket_of(hT[i]) + 1]++;
    for (int b = 0; b < nb; b++) bstart[b + 1] += bstart[b];
    for (int32_t i = 0; i < nq; i++) {
        const int b = search_bucket_of(hT[i]);
        hl[bstart[b] + bfill[b]++] = i;
    }
    uint8_t *d = S->pool_base + off;
    uint8_t *dq = d;
    size_t o = ((size_t)nq * vb + 255) & ~size_t(255);
    int32_t *dk = (int32_t *)(d + o);
    int32_t *dT = dk + nq;
    int32_t *dl = dT + nq;
    o += ((size_t)nq * 12 + 255) & ~size_t(255);
    int32_t *dids = (int32_t *)(d + o);
    uint32_t *dkeys = (uint32_t *)(dids + (size_t)nq * kmax);
    o += ((size_t)nq * kmax * 8 + 255) & ~size_t(255);
    int32_t *dst = (int32_t *)(d + o);
    cudaStream_t s = sl.stream;
    bool ok = cudaMemcpyAsync(dq, h, (size_t)nq * vb, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(dk, hk, 4 * (size_t)nq, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(dT, hT, 4 * (size_t)nq, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(dl, hl, 4 * (size_t)nq, cudaMemcpyHostToDevice, s) == cudaSuccess;
    for (int b = nb - 1; ok && b >= 0; b--)
        if (bstart[b + 1] > bstart[b])
            ok = search_launch_list(S->index, dq, nq, dk, dT, kmax, search_bucket_cap(b), dl + bstart[b],
                                    bstart[b + 1] - bstart[b], dids, dkeys, dst, s) == ANN_OK;
    uint8_t *ho = sl.h_out;
    if (ok)
        ok = cudaMemcpyAsync(ho, dids, (size_t)nq * kmax * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
             cudaMemcpyAsync(ho + (size_t)nq * kmax * 8, dst, 4 * (size_t)nq, cudaMemcpyDeviceToHost, s) ==
                 cudaSuccess;
    sl.finished.store(false);
    if (ok) ok = cudaLaunchHostFunc(s, on_done, &sl) == cudaSuccess;
    if (!ok) {
        S->thread_error = cudaGetErrorString(cudaGetLastError());
        return false;
    }
    sl.busy = true;
    sl.pool_off = off;
    sl.pool_len = len;
    sl.reqs = batch;
    sl.nq = nq;
    sl.kmax = kmax;
    return true;
}

// collect results of a finished slot (called with the lock held)
static void finish_slot(ann_server *S, Slot &sl) {
    const int32_t nq = sl.nq, kmax = sl.kmax;
    const int32_t *ids = (const int32_t *)sl.h_out;
    const uint32_t *keys = (const uint32_t *)(ids + (size_t)nq * kmax);
    const int32_t *st = (const int32_t *)(sl.h_out + (size_t)nq * kmax * 8);
    int32_t at = 0;
    auto now = Clock::now();
    for (auto &r : sl.reqs) {
        r->ids.resize((size_t)r->nq * r->kmax);
        r->keys.resize((size_t)r->nq * r->kmax);
        r->status.resize(r->nq);
        for (int32_t i = 0; i < r->nq; i++) {
            memcpy(&r->ids[(size_t)i * r->kmax], ids + (size_t)(at + i) * kmax, 4 * (size_t)r->kmax);
            memcpy(&r->keys[(size_t)i * r->kmax], keys + (size_t)(at + i) * kmax, 4 * (size_t)r->kmax);
            r->status[i] = st[at + i];
        }
        at += r->nq;
        r->t_done = now;
        r->done = true;
    }
    S->pool->release(sl.pool_off, sl.pool_len);
    sl.reqs.clear();
    sl.busy = false;
}

static void serve_loop(ann_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // completions
        for (auto &sp : S->slots)
            if (sp->busy && sp->finished.load(std::memory_order_acquire)) finish_slot(S, *sp);
        if (S->stop) {
            bool any = false;
            for (auto &sp : S->slots) any |= sp->busy;
            if (!any) break;
        }
        // admission: fill free slots with as many waiting requests as fit
        for (auto &sp : S->slots) {
            if (sp->busy || S->waiting.empty()) continue;
            std::vector<std::shared_ptr<Request>> batch;
            int32_t nq = 0, kmax = 1;
            size_t off = 0, len = 0;
            // greedy prefix of the FIFO that fits in one launch and in the pool
            size_t take = 0;
            for (size_t i = 0; i < S->waiting.size(); i++) {
                auto &r = S->waiting[i];
                if (nq + r->nq > kServeMaxBatch) break;
                int32_t km = std::max(kmax, r->kmax);
                size_t need = batch_bytes(S, nq + r->nq, km);
                size_t o2;
                if (!S->pool->alloc(need, o2)) break;
                S->pool->release(o2, need);
                nq += r->nq;
                kmax = km;
                take = i + 1;
            }
            if (take == 0) break;  // head of the queue does not fit yet: wait for memory
            len = batch_bytes(S, nq, kmax);
            if (!S->pool->alloc(len, off)) break;
            for (size_t i = 0; i < take; i++) {
                batch.push_back(S->waiting.front());
                S->waiting.pop_front();
            }
            if (!launch_batch(S, *sp, batch, nq, kmax, off, len)) {
                S->pool->release(off, len);
                for (auto &r : batch) {
                    r->ids.assign((size_t)r->nq * r->kmax, -1);
                    r->keys.assign((size_t)r->nq * r->kmax, 0xffffffffu);
                    r->status.assign(r->nq, ANN_ERR_CUDA);
                    r->t_done = Clock::now();
                    r->done = true;
                }
            }
        }
        bool busy = false;
        for (auto &sp : S->slots) busy |= sp->busy;
        if (busy) S->cv.wait_for(lk, std::chrono::microseconds(200));
        else S->cv.wait(lk, [&] { return S->stop || !S->waiting.empty(); });
    }
}

}  // namespace ann

using namespace ann;

extern "C" int ann_server_create(const ann_index *index, size_t scratch_bytes, int32_t max_streams,
                                 ann_server **out) {
    ANN_ARG(index && out, "index and out are required");
    ANN_ARG(max_streams >= 1 && max_streams <= 64, "max_streams must be in [1, 64]");
    ANN_ARG(scratch_bytes >= 4096, "scratch_bytes too small");
    ann_server *S = new ann_server();
    S->index = index;
    S->vbytes = (size_t)index->dev.d * (index->dev.dtype == ANN_U8 ? 1 : 4);
    ANN_CUDA(cudaGetDevice(&S->device));
    cudaError_t e = cudaMalloc((void **)&S->pool_base, scratch_bytes);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "cudaMalloc(scratch pool)");
    }
    S->pool.reset(new Pool(scratch_bytes));
    for (int i = 0; i < max_streams; i++) {
        std::unique_ptr<Slot> sl(new Slot());
        sl->cv = &S->cv;
        size_t in_b = (size_t)kServeMaxBatch * (S->vbytes + 12);
        size_t out_b = (size_t)kServeMaxBatch * (kMaxK * 8 + 4);
        if ((e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaHostAlloc((void **)&sl->h_in, in_b, cudaHostAllocDefault)) != cudaSuccess ||
            (e = cudaHostAlloc((void **)&sl->h_out, out_b, cudaHostAllocDefault)) != cudaSuccess) {
            S->slots.push_back(std::move(sl));
            ann_server_destroy(S);
            return cuda_fail(e, "server slot setup");
        }
        S->slots.push_back(std::move(sl));
    }
    S->worker = std::thread(serve_loop, S);
    *out = S;
    return ANN_OK;
}

extern "C" int ann_server_destroy(ann_server *S) {
    if (!S) return ANN_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->waiting.clear();
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &sl : S->slots) {
        if (sl->stream) {
            cudaStreamSynchronize(sl->stream);
            cudaStreamDestroy(sl->stream);
        }
        if (sl->h_in) cudaFreeHost(sl->h_in);
        if (sl->h_out) cudaFreeHost(sl->h_out);
    }
    if (S->pool_base) cudaFree(S->pool_base);
    delete S;
    return ANN_OK;
}

extern "C" int ann_serve_submit(ann_server *S, const void *host_queries, int32_t nq, const int32_t *k,
                                const int32_t *T, uint64_t *ticket) {
    ANN_ARG(S && ticket, "server and ticket are required");
    ANN_ARG(nq >= 1 && nq <= kServeMaxBatch, "nq must be in [1, 8192]");
    ANN_ARG(host_queries && k && T, "queries, k and T are required");
    int32_t kmax = 1;
    for (int32_t i = 0; i < nq; i++) {
        ANN_ARG(k[i] >= 0 && k[i] <= kMaxK, "k out of range");
        ANN_ARG(T[i] >= 0 && T[i] <= kMaxT, "T out of range");
        kmax = std::max(kmax, k[i]);
    }
    if (batch_bytes(S, nq, kmax) > S->pool->size)
        return fail(ANN_ERR_OOM, "request can never fit in the server's scratch pool");
    auto r = std::make_shared<Request>();
    r->nq = nq;
    r->kmax = kmax;
    r->queries.assign((const uint8_t *)host_queries, (const uint8_t *)host_queries + (size_t)nq * S->vbytes);
    r->k.assign(k, k + nq);
    r->T.assign(T, T + nq);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        r->ticket = S->next_ticket++;
        S->waiting.push_back(r);
        S->live[r->ticket] = r;
        *ticket = r->ticket;
    }
    S->cv.notify_all();
    return ANN_OK;
}

extern "C" int ann_serve_poll(ann_server *S, uint64_t ticket, int32_t *host_ids, void *host_keys,
                              int32_t *host_status) {
    ANN_ARG(S && host_ids, "server and host_ids are required");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->live.find(ticket);
        if (it == S->live.end()) return fail(ANN_ERR_ARG, "unknown or already collected ticket");
        if (!it->second->done) return ANN_PENDING;
        r = it->second;
    }
    memcpy(host_ids, r->ids.data(), 4 * r->ids.size());
    if (host_keys) memcpy(host_keys, r->keys.data(), 4 * r->keys.size());
    if (host_status) memcpy(host_status, r->status.data(), 4 * r->status.size());
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->live.erase(ticket);
        S->done_latency[ticket] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    }
    return ANN_OK;
}

extern "C" double ann_serve_latency(ann_server *S, uint64_t ticket) {
    if (!S) return -1.0;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->done_latency.find(ticket);
    return it == S->done_latency.end() ? -1.0 : it->second;
}

// Load replay (a measurement tool; the paper has no counterpart): requests are
// submitted from the calling thread at their arrival times and collected by a
// second native thread, so the measured rate and latencies are the server's,
// not those of a scripting-language driver.
extern "C" int ann_serve_replay(ann_server *S, const void *host_queries, const int32_t *k, const int32_t *T,
                                int32_t nreq, const int64_t *first, const int32_t *size, const double *arrival_s,
                                double *out_latency_s, double *out_elapsed_s) {
    ANN_ARG(S && host_queries && k && T && first && size && arrival_s && out_latency_s && out_elapsed_s,
            "all arguments are required");
    ANN_ARG(nreq >= 1, "nreq must be >= 1");
    for (int32_t r = 0; r < nreq; r++) {
        ANN_ARG(size[r] >= 1 && size[r] <= kServeMaxBatch && first[r] >= 0, "request size or offset out of range");
        ANN_ARG(r == 0 || arrival_s[r] >= arrival_s[r - 1], "arrival times must not decrease");
    }
    const size_t vb = S->vbytes;
    std::vector<uint64_t> tickets((size_t)nreq, 0);
    std::atomic<int32_t> submitted{0};
    std::atomic<bool> failed{false}, submit_done{false};
    std::atomic<int> poll_error{ANN_OK};
    const auto t0 = Clock::now();
    Clock::time_point t_last = t0;
    std::thread collector([&] {
        std::vector<int32_t> ids((size_t)kServeMaxBatch * kMaxK);
        std::vector<int32_t> pending;
        int32_t seen = 0, done = 0;
        // until every submitted request is collected (or a poll fails)
        while (poll_error.load() == ANN_OK) {
            const bool last = submit_done.load(std::memory_order_acquire);
            const int32_t ns = submitted.load(std::memory_order_acquire);
            if (last && done == ns) break;
            while (seen < ns) pending.push_back(seen++);
            for (size_t i = 0; i < pending.size();) {
                const int32_t r = pending[i];
                const int rc = ann_serve_poll(S, tickets[(size_t)r], ids.data(), nullptr, nullptr);
                if (rc == ANN_OK) {
                    out_latency_s[r] = ann_serve_latency(S, tickets[(size_t)r]);
                    t_last = Clock::now();
                    done++;
                    pending[i] = pending.back();
                    pending.pop_back();
                } else if (rc == ANN_PENDING) {
                    i++;
                } else {
                    poll_error.store(rc);
                    failed.store(true);
                    break;
                }
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    });
    int rc = ANN_OK;
    for (int32_t r = 0; r < nreq && !failed.load(); r++) {
        const auto at = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[r]));
        for (auto now = Clock::now(); now < at; now = Clock::now()) {
            if (at - now > std::chrono::microseconds(300))
                std::this_thread::sleep_for(at - now - std::chrono::microseconds(200));
        }
        uint64_t tk = 0;
        rc = ann_serve_submit(S, (const uint8_t *)host_queries + (size_t)first[r] * vb, size[r], k + first[r],
                              T + first[r], &tk);
        if (rc != ANN_OK) {
            failed.store(true);
            break;
        }
        tickets[(size_t)r] = tk;
        submitted.store(r + 1, std::memory_order_release);
    }
    submit_done.store(true, std::memory_order_release);
    collector.join();
    if (rc == ANN_OK) rc = poll_error.load();
    *out_elapsed_s = std::chrono::duration<double>(t_last - t0).count() - arrival_s[0];
    return rc;
}
