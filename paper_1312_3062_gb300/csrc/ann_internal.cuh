// ann_internal.cuh -- shared internals of the sm_103a library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/ann.h"

namespace ann {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// Stream-ordered device buffers (cudaMallocAsync) released by cudaFreeAsync
// on the same stream when the owner goes out of scope, so that an early
// error return frees whatever was already taken.
class AsyncBufs {
  public:
    explicit AsyncBufs(cudaStream_t s) : s_(s) {}
    AsyncBufs(const AsyncBufs &) = delete;
    AsyncBufs &operator=(const AsyncBufs &) = delete;
    ~AsyncBufs() {
        for (int i = n_ - 1; i >= 0; i--) cudaFreeAsync(p_[i], s_);
    }
    template <class T>
    cudaError_t alloc(T **out, size_t bytes) {
        if (n_ == kMax) return cudaErrorMemoryAllocation;
        void *q = nullptr;
        const cudaError_t e = cudaMallocAsync(&q, bytes, s_);
        if (e == cudaSuccess) {
            p_[n_++] = q;
            *out = (T *)q;
        }
        return e;
    }

  private:
    static constexpr int kMax = 16;
    cudaStream_t s_;
    void *p_[kMax] = {};
    int n_ = 0;
};

#define ANN_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return ::ann::cuda_fail(_e, #call);       \
    } while (0)

#define ANN_ARG(cond, msg)                                               \
    do {                                                                 \
        if (!(cond)) return ::ann::fail(ANN_ERR_ARG, msg);               \
    } while (0)

constexpr int kMaxP = 4;
constexpr int kMaxN = 256;
constexpr int kMaxR = 32;
constexpr int kMaxB = 8;
constexpr int kMaxK = 128;
constexpr int kMaxT = 8192;

// ---------------------------------------------------------------------------
// index (device side)
// ---------------------------------------------------------------------------
// Bridge index layout.  Non-empty bridge vectors are kept sorted by bridge id
// (mixed radix of center ids, part 0 most significant).  The first PA parts
// (PA = min(2, P-1)) form the prefix "A" node a = c0*n + c1 (or c0), the
// remaining parts the suffix, packed as mixed radix `leaf`.  For every prefix
// node: a presence bit (bmA) and a CSR range [offA[a], offA[a+1]) of
// bridges; each bridge has b reference slots (-1 padded).  With two suffix
// parts (P = 4) and many bridges per prefix node, the bridges of a node are
// also grouped by their third center c2: groups [goff[a], goff[a+1]), group g
// holds c2 = gc2[g] and the bridges [gstart[g], gstart[g+1]), so a walk can
// bound a whole group by D0 + D1 + D2[c2] + min D3 before reading its leaves.
struct DevIndex {
    int dtype;
    int64_t N;
    int d, R, P, n, b, t;
    int PA;
    int64_t nA;          // n^PA
    int64_t M;           // non-empty bridges
    const void *X;       // N*d
    const int32_t *G;    // N*R
    const void *C;       // P*n*(d/P)
    const uint32_t *bmA; // ceil(nA/32) words
    const uint32_t *offA;// nA+1
    const uint32_t *leaf;// M
    const int32_t *brefs;// M*b
    int64_t ngroups;        // c2 groups (0: no group level)
    const uint32_t *goff;   // nA+1
    const uint32_t *gstart; // ngroups+1
    const uint8_t *gc2;     // ngroups
    // suffix-major copy (indexes without the group level): the same bridges
    // sorted by (suffix s, prefix a); per suffix node a presence bit (bmS)
    // and a CSR range (offS, nS + 1 entries); per bridge its prefix a (sleaf)
    // and its position in the prefix-major order (sidx).  nS = n^(P-PA);
    // sidx == nullptr when absent.
    int64_t nS;
    const uint32_t *bmS, *offS, *sleaf, *sidx;
};

}  // namespace ann

struct ann_index {
    int device;
    ann::DevIndex dev;
    // owned allocations
    void *X, *C;
    int32_t *G;
    uint32_t *bmA, *offA, *leaf;
    int32_t *brefs;
    uint32_t *goff, *gstart;
    uint8_t *gc2;
    uint32_t *bmS, *offS, *sleaf, *sidx;
    int64_t bridged_refs;
    // cached persistent-mode plans (see ann_search.cu)
    void *plans;
};

namespace ann {
// implemented in ann_search.cu
void free_plans(ann_index *ix);
// plain launch of Algorithm 1 sized for a budget capT known on the host (no sync)
int search_launch_plain(const ann_index *ix, const void *queries, int64_t nq, const int32_t *k, const int32_t *T,
                        int32_t kmax, int capT, int32_t *out_ids, void *out_keys, int32_t *out_status,
                        cudaStream_t stream);
// plain launch over the queries listed in list[0 .. count) (device), sized for capT
int search_launch_list(const ann_index *ix, const void *queries, int64_t nq, const int32_t *k, const int32_t *T,
                       int32_t kmax, int capT, const int32_t *list, int64_t count, int32_t *out_ids, void *out_keys,
                       int32_t *out_status, cudaStream_t stream);
// the persistent form's budget buckets: capacity 128 << b (capped at the largest budget)
int search_bucket_of(int32_t T);
int search_bucket_cap(int bucket);
int search_num_buckets();
// implemented in ann_knn_tc.cu: exact k-NN of uint8 rows on the tensor cores, d in {64, 128}, k <= 32
int knn_u8_tensor(const uint8_t *refs, int64_t N, const uint8_t *queries, int64_t nq, int d, int k,
                  int exclude_self, int32_t *out_ids, uint32_t *out_keys, cudaStream_t s);
bool knn_u8_tensor_fits(int d, int k);
// implemented in ann_index.cu
int build_bridge_index_from_host(ann_index *ix, int64_t M, const uint64_t *ids,
                                 const int64_t *offsets, const int32_t *refs);
}  // namespace ann
