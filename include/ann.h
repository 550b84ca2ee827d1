/*
 * ann.h -- C ABI of the GB300 (sm_103a) library for approximate nearest
 * neighbour search over the augmented neighbourhood graph of
 * "Fast Neighborhood Graph Search using Cartesian Concatenation"
 * (Wang, Wang, Zeng, Tu, Gan, Li; arXiv:1312.3062).
 *
 * Problem (Sec. 2): given reference vectors X (N x d, Euclidean), a query q,
 * a budget T (number of reference vectors examined: time-constrained search)
 * and k, return k reference ids with their distances.  The index (Sec. 4.1)
 * is an exact R-NN neighbourhood graph over X plus a bridge graph between the
 * Cartesian concatenation of P per-part center sets and X.  The search is
 * Algorithm 1 (Sec. 4.2).
 *
 * Conventions for every entry point:
 *  - Every call returns an ann_status; no C++ exception crosses the ABI.
 *    On failure ann_last_error() returns a thread-local message.
 *  - "device" pointers are CUDA device (or managed) pointers on the current
 *    device; "host" pointers are ordinary CPU memory.  The library never
 *    frees caller memory; handles own their own device memory.
 *  - Keys are SQUARED Euclidean distances: uint32 for ANN_U8 data (exact),
 *    float32 for ANN_F32 data (the float32 nearest to the exact value).
 *    Ties are broken by the smaller id everywhere.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *    take a stream are asynchronous unless stated otherwise; device-side
 *    failures are reported per query in out_status, never by a trap.
 *  - Limits: 2 <= P <= 4, n <= 256, d % P == 0, d % 16 == 0 (u8) or
 *    d % 4 == 0 (f32), n^P <= 2^32, R <= 32, b <= 8, k <= 128, T <= 8192.
 */
#ifndef ANN_H
#define ANN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { ANN_U8 = 0, ANN_F32 = 1 } ann_dtype;

typedef enum {
    ANN_OK = 0,
    ANN_PENDING = 1,       /* serve_poll: request still running */
    ANN_ERR_ARG = -1,      /* invalid argument (message says which) */
    ANN_ERR_OOM = -2,      /* device allocation failed / request never admissible */
    ANN_ERR_CAPACITY = -3, /* a per-query on-chip capacity was exceeded */
    ANN_ERR_TIMEOUT = -4,  /* a bounded device wait gave up */
    ANN_ERR_CUDA = -5,     /* a CUDA runtime call failed */
    ANN_ERR_FORMAT = -6    /* index file malformed */
} ann_status;

typedef struct ann_index ann_index;   /* opaque; owns device copies of all index arrays */
typedef struct ann_server ann_server; /* opaque; owns the serving loop, queues and scratch */

/* Thread-local description of the last failure in this thread. */
const char *ann_last_error(void);

/* ------------------------------------------------------------------------ */
/* Index construction                                                        */
/* ------------------------------------------------------------------------ */

/* Exact k nearest neighbours by linear scan (Sec. 2; the ground truth of
 * Sec. 5.1).  refs: device, N*d elements of dtype, row-major.  queries:
 * device, nq*d.  For each query, the k rows of refs with the smallest
 * (key, id), ascending.  exclude_self=1 requires queries == refs (nq == N)
 * and skips row i for query i: this is the exact R-NN neighbourhood graph of
 * Sec. 3.1 / Sec. 4.1.  Rows with fewer than k candidates are padded with
 * id -1 / key UINT32_MAX (u8) or +inf (f32).  out_ids: device int32[nq*k];
 * out_keys: device, optional (NULL), nq*k keys.  k <= 32. */
int ann_exact_knn(const void *refs, int64_t N, const void *queries, int64_t nq, int dtype,
                  int32_t d, int32_t k, int32_t exclude_self, int32_t *out_ids, void *out_keys,
                  void *stream);

/* Same computation and arguments as ann_exact_knn, but the call allocates
 * nothing: the uint8 row norms it needs live in a fixed array inside the
 * library (4 MiB, 1048576 rows), which every GPU that loads the library keeps
 * until the process exits.  The paper has no counterpart; it exists for
 * callers that cannot allocate device memory themselves (a host program
 * whose device memory belongs to another allocator, or a latency-critical
 * loop that cannot take an allocation's synchronisation and latency).
 * Limits: for ANN_U8, N plus nq (nq counts unless the queries are the first
 * nq rows of refs, i.e. queries == refs and nq <= N) must not exceed
 * 1048576, otherwise ANN_ERR_CAPACITY; ANN_F32 needs no scratch, but it
 * always runs the plain SIMT scan: at N >= 8192 and nq >= 256 it is about
 * 50x slower than ann_exact_knn, whose float32 tensor-core path needs
 * workspace.  The first call on a device looks up the array's device
 * address (once per device) and keeps it for the life of the process; make
 * that first call before any stream capture, and do not call this entry
 * point on a device after cudaDeviceReset.  Every call shares the one array,
 * so calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  Nothing in the array needs to start at zero -- each call
 * writes every norm it reads.  Asynchronous. */
int ann_exact_knn_static(const void *refs, int64_t N, const void *queries, int64_t nq, int dtype,
                         int32_t d, int32_t k, int32_t exclude_self, int32_t *out_ids,
                         void *out_keys, void *stream);

/* Exact R-NN neighbourhood graph of data (Sec. 3.1, Sec. 4.1): same as
 * ann_exact_knn(data, N, data, N, dtype, d, R, 1, ...). */
int ann_build_knn_graph(const void *data, int dtype, int64_t N, int32_t d, int32_t R,
                        int32_t *out_ids, void *out_keys, void *stream);

/* Approximate R-NN neighbourhood graph of uint8 data.  Sec. 5.3 builds its
 * graphs with an approximate construction (random divide-and-conquer, then
 * neighbourhood propagation; cost O(N log N), Sec. 5.5) and gives no steps;
 * this call fixes them:
 *  1. For each of `rounds` random partitions: positions [0, N) are halved
 *     recursively `levels` times (segment [lo, hi) has the children [lo, m)
 *     and [m, hi), m = lo + (hi - lo) / 2); starting from the identity
 *     order, at level l every segment s = 0 .. 2^l - 1 (left to right)
 *     reorders its members ascending by (<u, x>, id) with
 *     u = dirs[round][2^l - 1 + s].  The 2^levels final segments are leaves;
 *     every point is offered every other member of its leaf.
 *  2. `iters` propagation steps, each reading the rows of the step before:
 *     row i is offered every entry of its neighbours' rows (i excluded).
 * A row keeps the R smallest offered (key, id) pairs with distinct ids, so
 * the result is deterministic.  data: device N*d uint8, 16-byte aligned.
 * dirs: device int8[rounds][2^levels - 1][d], 16-byte aligned (random split
 * directions drawn by the caller; NULL allowed when levels == 0).  out_ids:
 * device int32[N*R]; out_keys: device uint32[N*R] or NULL.  Rows ascending
 * (key, id).  Requires dtype == ANN_U8, d % 16 == 0, R <= 32, every leaf
 * >= R + 1 points (floor(N / 2^levels) > R), and either d <= 128 (leaves of
 * any size; those beyond shared memory are streamed through it) or the
 * largest leaf, ceil(N / 2^levels) rows of d + 20 bytes, within one CTA's
 * shared memory; otherwise ANN_ERR_ARG.  Allocates its
 * scratch (16 N bytes of sort keys, 8 N R bytes per graph copy) with
 * cudaMallocAsync on `stream`.  Asynchronous. */
int ann_build_knn_graph_approx(const void *data, int dtype, int64_t N, int32_t d, int32_t R,
                               const int8_t *dirs, int32_t rounds, int32_t levels, int32_t iters,
                               int32_t *out_ids, void *out_keys, void *stream);

/* Graph-D-ADC (Sec. 5.4): the method as the coarse quantizer of an inverted
 * file whose residuals are product-quantized.  Precision: the paper fixes
 * none; codes and keys are decided in float32, every operation rounded (no
 * fused multiply-add), in this order: r_t = x_t - c_t; e = r_t - w_t; a
 * part's sum adds e * e for t ascending; a key adds the m parts ascending.
 *
 * ann_pq_encode: codes[i*m + j] = the codeword of part j (dims
 * [j*d/m, (j+1)*d/m)) nearest to the residual data[i] - centers[assign[i]],
 * ties to the lower codeword index.  data: device N*d elements of dtype;
 * centers: device float32 K*d coarse centers; assign: device int32[N], each
 * in [0, K) (an entry outside gets code 0); codebooks: device float32
 * m*ks*(d/m); codes: device uint8[N*m].  Limits: d % m == 0, d/m <= 32,
 * ks <= 256.  Asynchronous. */
int ann_pq_encode(const void *data, int dtype, int64_t N, int32_t d, const float *centers, int64_t K,
                  const int32_t *assign, int32_t m, int32_t ks, const float *codebooks, uint8_t *codes,
                  void *stream);

/* ann_adc_rerank: for each query q (device float32 nq*d), visit the lists
 * lists[q*w .. q*w + w) in that order (entries outside [0, K) are skipped),
 * members of list c being members[offsets[c] .. offsets[c+1]) (device;
 * offsets int64[K+1]; each list ascending by id); the first L members
 * overall are the candidates, keyed by the asymmetric distance
 * ||q - c - r^||^2 = sum over parts j of table_j[code_j], table_j[k] =
 * ||(q - c)^j - codeword(j, k)||^2.  out_ids: device int32[nq*T], the T
 * smallest (key, id) ascending, padded with -1; out_keys: device
 * float32[nq*T] or NULL (+inf padding); out_seen: device int64[nq] or NULL,
 * the candidates examined (min(L, members of the visited lists)).  Limits:
 * T <= 128, m <= 64, ks <= 256, m*ks*4 + 16384 bytes of shared memory.
 * Asynchronous. */
int ann_adc_rerank(const float *queries, int64_t nq, int32_t d, const int32_t *lists, int32_t w,
                   const int64_t *offsets, int64_t K, const int32_t *members, const float *centers,
                   const uint8_t *codes, int32_t m, int32_t ks, const float *codebooks, int64_t L, int32_t T,
                   int32_t *out_ids, float *out_keys, int64_t *out_seen, void *stream);

/* Per-part dictionaries for the bridge vectors (Sec. 4.1, "Computing bridge
 * vectors": product quantization, i.e. k-means on each of the P contiguous
 * parts of d/P dims).  Lloyd's algorithm in fp64: center j of every part
 * starts at training row init_rows[j] (host int64[n], distinct); assignment
 * ties go to the lower center; an empty cluster keeps its previous center.
 * train: device, ntrain*d elements.  out_centers: device, P*n*(d/P)
 * elements of dtype (u8: rounded half-to-even and clipped to [0,255]);
 * out_centers_f64: device, optional, the unrounded P*n*(d/P) doubles.
 * Synchronous. */
int ann_train_centers(const void *train, int dtype, int64_t ntrain, int32_t d, int32_t P,
                      int32_t n, int32_t iters, const int64_t *init_rows, void *out_centers,
                      double *out_centers_f64, void *stream);

/* Everything an index is made of.  data/graph/centers: device pointers (they
 * are copied).  If bridge_ids is NULL the bridge graph is built on the GPU
 * (Sec. 4.1: for each reference vector its top-t bridge vectors; for each
 * bridge vector the b nearest of those references).  Otherwise the caller
 * supplies it on the host: M ascending bridge ids (mixed radix of center ids,
 * part 0 most significant), CSR offsets int64[M+1] and reference ids, each
 * list ascending by (key to the bridge, id) and at most b long. */
typedef struct {
    int32_t dtype;
    int64_t N;
    int32_t d, R, P, n, t, b;
    const void *data;         /* device, N*d */
    const int32_t *graph;     /* device, N*R (-1 = no neighbour) */
    const void *centers;      /* device, P*n*(d/P) */
    int64_t M;                /* host bridge graph (optional) */
    const uint64_t *bridge_ids;
    const int64_t *bridge_offsets;
    const int32_t *bridge_refs;
} ann_index_desc;

/* Create an index on the current device.  Synchronous. */
int ann_index_create(const ann_index_desc *desc, ann_index **out);

/* Load an index written by ann_index_save onto `device` (-1 = current). */
int ann_index_load(const char *path, int device, ann_index **out);
int ann_index_save(const ann_index *index, const char *path);
int ann_index_free(ann_index *index);

/* Index statistics (Table 1: #reference and alpha). */
typedef struct {
    int64_t N, M;             /* references; non-empty bridge vectors */
    int32_t d, R, P, n, b, dtype;
    int64_t bridged_refs;     /* distinct references attached to some bridge */
    double alpha;             /* bridged_refs / n^P */
    int64_t bytes_vectors, bytes_graph, bytes_bridges;
    int64_t groups;   /* c2 groups of the prefix index (0: no group level; built for P = 4 when the
                         bridges average >= 32 per prefix node) */
} ann_index_info;
int ann_index_get_info(const ann_index *index, ann_index_info *out);

/* Copy the bridge graph back to the host: bridge ids (uint64[M], ascending)
 * and refs (int32[M*b], each list padded with -1). */
int ann_index_get_bridges(const ann_index *index, uint64_t *ids, int32_t *refs);

/* Reference lists of selected bridge ids (host arrays): refs (int32[nids*b])
 * receives each id's list (Sec. 4.1), ascending by (key to the bridge, id),
 * padded with -1; an id without references gets an all -1 row.  Reads only
 * the prefix offsets and the selected nodes' leaves, for indexes too large to
 * copy back whole.  ANN_ERR_ARG for an id >= n^P. */
int ann_index_lookup_bridges(const ann_index *index, const uint64_t *ids, int64_t nids, int32_t *refs);

/* ------------------------------------------------------------------------ */
/* Search: Algorithm 1 (Sec. 4.2)                                            */
/* ------------------------------------------------------------------------ */

enum { ANN_MODE_PLAIN = 0, ANN_MODE_PERSISTENT = 1 };

/* Per-query counters (out_stats, int64 each). */
enum {
    ANN_STAT_DISCOVERED = 0, /* t: reference vectors discovered (= distances computed) */
    ANN_STAT_REF_POPS,       /* reference vectors popped and expanded */
    ANN_STAT_BRIDGE_POPS,    /* non-empty bridge vectors popped */
    ANN_STAT_WALKS,          /* bridge-index walks (one per batch of bridges) */
    ANN_STAT_WALK_NODES,     /* prefix nodes read by those walks */
    ANN_STAT_WALK_LEAVES,    /* leaf entries read by those walks */
    ANN_STAT_MAX_Q,          /* largest main-queue length */
    ANN_STAT_PRELOADED,      /* reference pops whose kNN row was loaded during the previous step */
    ANN_NSTATS
};

/* Batched search.  queries: device, nq*d elements of the index dtype.
 * k, T: device int32[nq] per-query result counts and budgets, or NULL to use
 * k_all / T_all for every query.  kmax >= every k.  Outputs (device,
 * caller-owned): out_ids int32[nq*kmax] ascending by (key, id), padded with
 * -1; out_keys (optional) nq*kmax keys padded with UINT32_MAX / +inf;
 * out_status (optional) int32[nq], per query: ANN_OK; ANN_ERR_ARG for a
 * per-query k outside [0, kmax] or T outside [0, 8192] (that query's output
 * is all padding; the others are unaffected); ANN_ERR_CAPACITY if a bridge
 * window could not be split below its buffer, which a valid index never
 * causes (bridge ids are distinct, so every (key, rank tuple) composite
 * names one bridge and halving a window always separates them: the check
 * only guards against a corrupted index).
 * out_stats (optional) int64[nq*ANN_NSTATS].
 * mode ANN_MODE_PLAIN: one kernel launch for this batch on `stream`, sized
 * for the largest budget (per-query T costs one device max and a host sync).
 * mode ANN_MODE_PERSISTENT: queries are bucketed by budget (128 * 2^i) and
 * each bucket is run by a kernel sized for it, pulling queries from a device
 * ticket or taking fixed shares; the sequence is captured once per (index,
 * pointers, sizes, stream) into a CUDA graph and replayed (at most 32 plans
 * per index, least recently used evicted after its stream finished).  The
 * first call that meets a (budget bucket, kmax) measures candidate launch
 * shapes on the batch itself and keeps the fastest for the index; that call
 * synchronizes `stream` and runs the batch a few times.
 * Results are identical in both modes and for every launch shape.
 * Asynchronous except as stated. */
int ann_search_batch(const ann_index *index, const void *queries, int64_t nq, const int32_t *k,
                     const int32_t *T, int32_t k_all, int32_t T_all, int32_t kmax, int32_t mode,
                     int32_t *out_ids, void *out_keys, int32_t *out_status, int64_t *out_stats,
                     void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching with memory-based admission                  */
/* ------------------------------------------------------------------------ */

/* A server keeps the index resident, owns a pool of scratch_bytes of device
 * memory and a host thread that admits submitted requests whenever their
 * scratch fits, launching them on its own streams so requests overlap on the
 * GPU.  Results are identical to ann_search_batch for the same queries. */
int ann_server_create(const ann_index *index, size_t scratch_bytes, int32_t max_streams,
                      ann_server **out);
int ann_server_destroy(ann_server *server);

/* Submit nq queries (host memory, copied at once) with per-query k, T (host
 * int32[nq]).  *ticket identifies the request.  ANN_ERR_OOM if the request
 * could never fit in the scratch pool. */
int ann_serve_submit(ann_server *server, const void *host_queries, int32_t nq, const int32_t *k,
                     const int32_t *T, uint64_t *ticket);

/* Non-blocking.  ANN_PENDING while running; ANN_OK once done, after copying
 * ids (int32[nq*kmax_req]), keys (optional) and status (optional, int32[nq])
 * to the host buffers, where kmax_req is the request's largest k.  The
 * ticket is released by the successful poll. */
int ann_serve_poll(ann_server *server, uint64_t ticket, int32_t *host_ids, void *host_keys,
                   int32_t *host_status);

/* Submit-to-completion latency in seconds of a finished (polled) ticket's
 * request, measured by the server; -1 if unknown. */
double ann_serve_latency(ann_server *server, uint64_t ticket);

/* Load replay, a measurement tool with no counterpart in the paper.  Submits
 * nreq requests to the server from the calling thread, request r at
 * arrival_s[r] seconds after the call (non-decreasing), holding the size[r]
 * query rows starting at row first[r] of host_queries (host memory, the
 * index's dtype and d) with per-query k and T taken from the same rows of the
 * host arrays k and T; a second native thread collects every ticket (results
 * are discarded).  Writes each request's latency (submit -> completion,
 * seconds) to out_latency_s[nreq] and the time from the first arrival to the
 * last completion to *out_elapsed_s.  Returns ANN_OK or the first error of a
 * submission or a poll; all requests already submitted are collected before
 * it returns. */
int ann_serve_replay(ann_server *server, const void *host_queries, const int32_t *k, const int32_t *T,
                     int32_t nreq, const int64_t *first, const int32_t *size, const double *arrival_s,
                     double *out_latency_s, double *out_elapsed_s);

#ifdef __cplusplus
}
#endif
#endif /* ANN_H */
