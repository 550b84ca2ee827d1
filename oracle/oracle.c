/*
 * oracle.c -- CPU oracle for "Fast Neighborhood Graph Search using Cartesian
 * Concatenation" (Wang, Wang, Zeng, Tu, Gan, Li; arXiv:1312.3062).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may build, load or call it.  It
 * shares no code, header or table with the CUDA library.
 *
 * Conventions (the paper is silent on these; each reading is fixed here):
 *  - Every key is a SQUARED Euclidean distance (Sec. 2 defines dist as L2;
 *    Sec. 3.2 stores squared distances in the part tables; Sec. 4.2 sums
 *    squared part distances).  Squared keys order candidates exactly like
 *    dist() does, so Alg. 1's results are unchanged.
 *  - uint8 data: keys are exact integers.
 *  - float32 data: a key is computed in fp64 and then rounded to the nearest
 *    float32; every comparison is taken on that float32 value (the kernel's
 *    precision), so both implementations order candidates identically.
 *    A bridge key (Sec. 4.2: the sum over parts of the part distances) is
 *    the float32 nearest to the EXACT sum of the P float32 part keys, ties
 *    to even: one rounding, no grouping, and monotone in every part key, so
 *    the multi-sequence order of Sec. 3.3 holds for it.
 *  - Main queue order: (key, kind, id), kind ref = 0 < bridge = 1.
 *  - Result set: the k smallest by (key, id), returned ascending, padded with
 *    id -1 / key +inf when fewer than k points were discovered.
 *  - Budget: t counts discovered reference vectors; discovery stops the
 *    moment t reaches T, even inside an adjacency list, and the search ends.
 *  - Part p covers the contiguous dims [p*dp, (p+1)*dp), dp = d / P.
 *  - Part sort order: (part key, center id).  Bridge order in the
 *    multi-sequence: (bridge key, rank tuple compared lexicographically with
 *    part 0 first).  Bridge id: mixed radix of the ORIGINAL center ids with
 *    part 0 most significant.
 *  - Multi-sequence push rule: a tuple is pushed once all of its immediate
 *    predecessors (one rank lowered by one) have been POPPED.
 *  - kNN rows: ascending (key, id), self excluded.  Bridge lists: ascending
 *    (key to the bridge, ref id).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { DT_U8 = 0, DT_F32 = 1 };
#define MAXP_KEY 8 /* most parts a bridge key sums */

/* ------------------------------------------------------------------------ */
/* Distances (Sec. 2: dist(q, x) = ||q - x||_2; Sec. 3.2: squared tables)    */
/* ------------------------------------------------------------------------ */

/* Squared L2 between a[0..len) and b[0..len) of the given dtype.  uint8: the
   exact integer (each term is at most 255^2, so an int32 sum is exact up to
   33025 terms).  float32: an fp64 sum of the squared fp64 differences (four
   interleaved partial sums), rounded once to float32. */
static double sqdist(const void *a, const void *b, int len, int dtype) {
    if (dtype == DT_U8) {
        const uint8_t *x = (const uint8_t *)a, *y = (const uint8_t *)b;
        if (len <= 33025) {
            int32_t s = 0;
            for (int i = 0; i < len; i++) {
                int32_t t = (int32_t)x[i] - (int32_t)y[i];
                s += t * t;
            }
            return (double)s;
        }
        int64_t s = 0;
        for (int i = 0; i < len; i++) {
            int64_t t = (int64_t)x[i] - (int64_t)y[i];
            s += t * t;
        }
        return (double)s;
    } else {
        const float *x = (const float *)a, *y = (const float *)b;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int i = 0;
        for (; i + 4 <= len; i += 4) {
            double t0 = (double)x[i] - (double)y[i], t1 = (double)x[i + 1] - (double)y[i + 1];
            double t2 = (double)x[i + 2] - (double)y[i + 2], t3 = (double)x[i + 3] - (double)y[i + 3];
            s0 += t0 * t0;
            s1 += t1 * t1;
            s2 += t2 * t2;
            s3 += t3 * t3;
        }
        for (; i < len; i++) {
            double t = (double)x[i] - (double)y[i];
            s0 += t * t;
        }
        return (double)(float)((s0 + s1) + (s2 + s3)); /* decisions are taken at float32 */
    }
}

static const void *row_ptr(const void *base, int64_t row, int len, int dtype) {
    if (dtype == DT_U8) return (const uint8_t *)base + row * (int64_t)len;
    return (const float *)base + row * (int64_t)len;
}

/* The float32 nearest to the exact sum of n finite, non-negative float32
   values, ties to the even significand.  Every such value is an integer
   multiple of 2^-149 below 2^128, so the sum is held exactly as an integer
   count of 2^-149 in eleven 32-bit limbs (little end first) and rounded
   once to 24 significant bits at the end. */
static float f32_exact_sum(const float *v, int n) {
    uint32_t acc[11] = {0};
    for (int i = 0; i < n; i++) {
        uint32_t bits;
        memcpy(&bits, &v[i], sizeof bits);
        uint32_t ex = (bits >> 23) & 0xffu, man = bits & 0x7fffffu;
        /* normal: (2^23 + man) * 2^(ex - 150) = (2^23 + man) << (ex - 1) units;
           subnormal (ex = 0): man units */
        int sh = 0;
        if (ex) {
            man |= 0x800000u;
            sh = (int)ex - 1;
        }
        uint64_t part = (uint64_t)man << (sh % 32); /* < 2^55 */
        uint64_t carry = 0;
        for (int j = sh / 32; j < 11; j++) {
            uint64_t add = j == sh / 32 ? (part & 0xffffffffu) : (j == sh / 32 + 1 ? part >> 32 : 0);
            uint64_t t = (uint64_t)acc[j] + add + carry;
            acc[j] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    int top = -1; /* highest set bit */
    for (int j = 10; j >= 0 && top < 0; j--)
        for (int b = 31; b >= 0; b--)
            if ((acc[j] >> b) & 1u) {
                top = 32 * j + b;
                break;
            }
#define ACC_BIT(pos) ((acc[(pos) / 32] >> ((pos) % 32)) & 1u)
    if (top < 24) { /* below 2^24 units: exactly representable */
        uint32_t q = 0;
        for (int b = top; b >= 0; b--) q = (q << 1) | ACC_BIT(b);
        return ldexpf((float)q, -149);
    }
    int low = top - 23; /* the kept bits are [low, top] */
    uint32_t q = 0;
    for (int b = top; b >= low; b--) q = (q << 1) | ACC_BIT(b);
    uint32_t round = ACC_BIT(low - 1), sticky = 0;
    for (int b = low - 2; b >= 0 && !sticky; b--) sticky = ACC_BIT(b);
#undef ACC_BIT
    if (round && (sticky || (q & 1u))) q++;
    if (q == (1u << 24)) { /* carried into a new bit */
        q >>= 1;
        low++;
    }
    return ldexpf((float)q, low - 149);
}

/* Bridge key from P part keys (Sec. 4.2: dist^2(q, y) = sum_p dist^2(q^p, y^p)).
   uint8: the exact integer sum.  float32: the part keys are float32 values
   and the key is the float32 nearest to their exact sum (one rounding). */
static double bridge_key(const double *part_keys, int P, int dtype) {
    if (dtype == DT_U8) {
        double s = 0.0; /* integers far below 2^53: exact */
        for (int p = 0; p < P; p++) s += part_keys[p];
        return s;
    } else {
        float f[MAXP_KEY];
        for (int p = 0; p < P; p++) f[p] = (float)part_keys[p];
        return (double)f32_exact_sum(f, P);
    }
}

/* ------------------------------------------------------------------------ */
/* Top-k selection by (key, id)                                              */
/* ------------------------------------------------------------------------ */

static int pair_less(double ka, int64_t ia, double kb, int64_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

/* Insert (key, id) into the ascending list (keys, ids) of length *len, kept to
   at most cap entries. */
static void topk_insert(double *keys, int64_t *ids, int *len, int cap, double key, int64_t id) {
    int n = *len;
    if (n == cap) {
        if (!pair_less(key, id, keys[n - 1], ids[n - 1])) return;
        n--; /* drop the current largest */
    }
    int pos = n;
    while (pos > 0 && pair_less(key, id, keys[pos - 1], ids[pos - 1])) {
        keys[pos] = keys[pos - 1];
        ids[pos] = ids[pos - 1];
        pos--;
    }
    keys[pos] = key;
    ids[pos] = id;
    *len = n + 1;
}

/* ------------------------------------------------------------------------ */
/* Exact k nearest neighbours by linear scan (Sec. 2; Sec. 5.1 ground truth) */
/* and the exact R-NN neighbourhood graph (Sec. 3.1, Sec. 5.3).              */
/* ------------------------------------------------------------------------ */

/* For each query row i of Qs, the k nearest rows of X by (key, id).  When
   exclude_self is set, Qs must be X and row i is skipped for query i.
   Rows with fewer than k candidates are padded with id -1 / key +inf.
   Query rows are independent; nthreads > 1 splits them across threads. */
typedef struct {
    const void *X, *Qs;
    int64_t N, nq;
    int d, dtype, k, exclude_self;
    int32_t *out_ids;
    double *out_keys;
    int64_t next;
    pthread_mutex_t mu;
} knn_job_t;

static void knn_rows(knn_job_t *j, int64_t i) {
    double *keys = (double *)malloc(sizeof(double) * (size_t)j->k);
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)j->k);
    int len = 0;
    const void *q = row_ptr(j->Qs, i, j->d, j->dtype);
    for (int64_t r = 0; r < j->N; r++) {
        if (j->exclude_self && r == i) continue;
        double key = sqdist(q, row_ptr(j->X, r, j->d, j->dtype), j->d, j->dtype);
        topk_insert(keys, ids, &len, j->k, key, r);
    }
    for (int r = 0; r < j->k; r++) {
        j->out_ids[i * j->k + r] = r < len ? (int32_t)ids[r] : -1;
        j->out_keys[i * j->k + r] = r < len ? keys[r] : INFINITY;
    }
    free(keys);
    free(ids);
}

static void *knn_worker(void *arg) {
    knn_job_t *j = (knn_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->nq) break;
        knn_rows(j, i);
    }
    return NULL;
}

void oracle_exact_knn(const void *X, int64_t N, const void *Qs, int64_t nq, int d, int dtype,
                      int k, int exclude_self, int32_t *out_ids, double *out_keys, int nthreads) {
    knn_job_t job = {X, Qs, N, nq, d, dtype, k, exclude_self, out_ids, out_keys, 0,
                     PTHREAD_MUTEX_INITIALIZER};
    if (nthreads <= 1) {
        knn_worker(&job);
        return;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, knn_worker, &job);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
}

/* ------------------------------------------------------------------------ */
/* Subvector dictionaries: product-quantization k-means per part             */
/* (Sec. 3.2; Sec. 4.1 "Computing bridge vectors")                          */
/* ------------------------------------------------------------------------ */

/* Lloyd's algorithm in fp64 on each contiguous part independently.
   init_rows: n distinct training-row indices; center j of every part starts
   at row init_rows[j].  Assignment ties go to the lower center id; an empty
   cluster keeps its previous center.  centers: out, P*n*dp doubles. */
void oracle_kmeans(const void *X, int64_t N, int d, int dtype, int P, int n, int iters,
                   const int64_t *init_rows, double *centers) {
    int dp = d / P;
    double *sums = (double *)malloc(sizeof(double) * (size_t)n * dp);
    int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *assign = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *row = (double *)malloc(sizeof(double) * (size_t)dp);
    for (int p = 0; p < P; p++) {
        double *C = centers + (int64_t)p * n * dp;
        for (int j = 0; j < n; j++)
            for (int e = 0; e < dp; e++) {
                int64_t at = init_rows[j] * d + p * dp + e;
                C[j * dp + e] = dtype == DT_U8 ? (double)((const uint8_t *)X)[at]
                                               : (double)((const float *)X)[at];
            }
        for (int it = 0; it < iters; it++) {
            /* assignment step */
            for (int64_t i = 0; i < N; i++) {
                for (int e = 0; e < dp; e++) {
                    int64_t at = i * d + p * dp + e;
                    row[e] = dtype == DT_U8 ? (double)((const uint8_t *)X)[at]
                                            : (double)((const float *)X)[at];
                }
                double best = INFINITY;
                int arg = 0;
                for (int j = 0; j < n; j++) {
                    double s = 0.0;
                    for (int e = 0; e < dp; e++) {
                        double t = row[e] - C[j * dp + e];
                        s += t * t;
                    }
                    if (s < best) { best = s; arg = j; }
                }
                assign[i] = arg;
            }
            /* update step */
            memset(sums, 0, sizeof(double) * (size_t)n * dp);
            memset(counts, 0, sizeof(int64_t) * (size_t)n);
            for (int64_t i = 0; i < N; i++) {
                int j = assign[i];
                counts[j]++;
                for (int e = 0; e < dp; e++) {
                    int64_t at = i * d + p * dp + e;
                    sums[j * dp + e] += dtype == DT_U8 ? (double)((const uint8_t *)X)[at]
                                                       : (double)((const float *)X)[at];
                }
            }
            for (int j = 0; j < n; j++)
                if (counts[j] > 0)
                    for (int e = 0; e < dp; e++) C[j * dp + e] = sums[j * dp + e] / (double)counts[j];
        }
    }
    free(sums);
    free(counts);
    free(assign);
    free(row);
}

/* ------------------------------------------------------------------------ */
/* Per-part tables and their sort (Sec. 4.2, first step of the query)        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int P, n, dtype;
    double *key;    /* P*n part keys, unsorted: key[p*n + c] */
    double *skey;   /* P*n sorted part keys: skey[p*n + rank] */
    int32_t *scid;  /* P*n center id at each rank */
} tables_t;

typedef struct { double key; int32_t cid; } kc_t;

static int kc_cmp(const void *a, const void *b) {
    const kc_t *x = (const kc_t *)a, *y = (const kc_t *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->cid > y->cid) - (x->cid < y->cid);
}

/* Distances from the parts of vec to every center, then each part sorted by
   (key, center id). */
static void tables_build(tables_t *tb, const void *vec, int d, int dtype, int P, int n,
                         const void *centers) {
    int dp = d / P;
    tb->P = P;
    tb->n = n;
    tb->dtype = dtype;
    kc_t *tmp = (kc_t *)malloc(sizeof(kc_t) * (size_t)n);
    for (int p = 0; p < P; p++) {
        const void *qpart = dtype == DT_U8 ? (const void *)((const uint8_t *)vec + p * dp)
                                           : (const void *)((const float *)vec + p * dp);
        for (int c = 0; c < n; c++) {
            const void *cent = row_ptr(centers, (int64_t)p * n + c, dp, dtype);
            double k = sqdist(qpart, cent, dp, dtype);
            tb->key[p * n + c] = k;
            tmp[c].key = k;
            tmp[c].cid = c;
        }
        qsort(tmp, (size_t)n, sizeof(kc_t), kc_cmp);
        for (int r = 0; r < n; r++) {
            tb->skey[p * n + r] = tmp[r].key;
            tb->scid[p * n + r] = tmp[r].cid;
        }
    }
    free(tmp);
}

static tables_t tables_alloc(int P, int n) {
    tables_t tb;
    tb.key = (double *)malloc(sizeof(double) * (size_t)P * n);
    tb.skey = (double *)malloc(sizeof(double) * (size_t)P * n);
    tb.scid = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * n);
    tb.P = P;
    tb.n = n;
    tb.dtype = 0;
    return tb;
}

static void tables_free(tables_t *tb) {
    free(tb->key);
    free(tb->skey);
    free(tb->scid);
}

/* ------------------------------------------------------------------------ */
/* Multi-sequence enumeration (Sec. 3.3; ExtractNextNearestBridgeVector)     */
/* ------------------------------------------------------------------------ */

#define MAXP 8

typedef struct { double key; int32_t r[MAXP]; } ms_item;

typedef struct {
    const tables_t *tb;
    ms_item *heap;
    int64_t hlen, hcap;
    uint64_t *set; /* open-addressing set of popped rank codes (code + 1; 0 = empty) */
    int64_t scap, slen;
    int64_t max_frontier;
    int64_t npushed;
} mseq_t;

static int ms_less(const ms_item *a, const ms_item *b, int P) {
    if (a->key < b->key) return 1;
    if (a->key > b->key) return 0;
    for (int p = 0; p < P; p++) {
        if (a->r[p] < b->r[p]) return 1;
        if (a->r[p] > b->r[p]) return 0;
    }
    return 0;
}

static uint64_t ms_code(const int32_t *r, int P, int n) {
    uint64_t c = 0;
    for (int p = 0; p < P; p++) c = c * (uint64_t)n + (uint64_t)r[p];
    return c;
}

static uint64_t mix64(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

static int set_has(const mseq_t *m, uint64_t code) {
    uint64_t mask = (uint64_t)m->scap - 1, h = mix64(code) & mask;
    while (m->set[h]) {
        if (m->set[h] == code + 1) return 1;
        h = (h + 1) & mask;
    }
    return 0;
}

static void set_add(mseq_t *m, uint64_t code) {
    if (2 * (m->slen + 1) > m->scap) {
        uint64_t *old = m->set;
        int64_t oc = m->scap;
        m->scap *= 2;
        m->set = (uint64_t *)calloc((size_t)m->scap, sizeof(uint64_t));
        m->slen = 0;
        for (int64_t i = 0; i < oc; i++)
            if (old[i]) set_add(m, old[i] - 1);
        free(old);
    }
    uint64_t mask = (uint64_t)m->scap - 1, h = mix64(code) & mask;
    while (m->set[h]) {
        if (m->set[h] == code + 1) return;
        h = (h + 1) & mask;
    }
    m->set[h] = code + 1;
    m->slen++;
}

static void ms_push(mseq_t *m, const int32_t *r) {
    const tables_t *tb = m->tb;
    int P = tb->P;
    ms_item it;
    double parts[MAXP] = {0};
    for (int p = 0; p < P; p++) {
        it.r[p] = r[p];
        parts[p] = tb->skey[p * tb->n + r[p]];
    }
    it.key = bridge_key(parts, P, tb->dtype);
    if (m->hlen == m->hcap) {
        m->hcap *= 2;
        m->heap = (ms_item *)realloc(m->heap, sizeof(ms_item) * (size_t)m->hcap);
    }
    int64_t i = m->hlen++;
    m->heap[i] = it;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!ms_less(&m->heap[i], &m->heap[par], P)) break;
        ms_item t = m->heap[i]; m->heap[i] = m->heap[par]; m->heap[par] = t;
        i = par;
    }
    m->npushed++;
    if (m->hlen > m->max_frontier) m->max_frontier = m->hlen;
}

static void ms_init(mseq_t *m, const tables_t *tb) {
    m->tb = tb;
    m->hcap = 64;
    m->hlen = 0;
    m->heap = (ms_item *)malloc(sizeof(ms_item) * (size_t)m->hcap);
    m->scap = 64;
    m->slen = 0;
    m->set = (uint64_t *)calloc((size_t)m->scap, sizeof(uint64_t));
    m->max_frontier = 0;
    m->npushed = 0;
    int32_t zero[MAXP] = {0};
    ms_push(m, zero); /* start from the tuple of first ranks */
}

static void ms_free(mseq_t *m) {
    free(m->heap);
    free(m->set);
}

/* Pop the next tuple in (key, ranks) order.  Returns 0 when every tuple has
   been produced. */
static int ms_next(mseq_t *m, ms_item *out) {
    const tables_t *tb = m->tb;
    int P = tb->P, n = tb->n;
    if (m->hlen == 0) return 0;
    *out = m->heap[0];
    m->heap[0] = m->heap[--m->hlen];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < m->hlen && ms_less(&m->heap[l], &m->heap[s], P)) s = l;
        if (r < m->hlen && ms_less(&m->heap[r], &m->heap[s], P)) s = r;
        if (s == i) break;
        ms_item t = m->heap[i]; m->heap[i] = m->heap[s]; m->heap[s] = t;
        i = s;
    }
    set_add(m, ms_code(out->r, P, n));
    /* Successors: raise one rank by one; push once every predecessor of the
       successor (each of its nonzero ranks lowered by one) has been popped. */
    for (int b = 0; b < P; b++) {
        if (out->r[b] + 1 >= n) continue;
        int32_t v[MAXP];
        for (int p = 0; p < P; p++) v[p] = out->r[p];
        v[b]++;
        int ready = 1;
        for (int c = 0; c < P && ready; c++) {
            if (c == b || v[c] == 0) continue;
            v[c]--;
            if (!set_has(m, ms_code(v, P, n))) ready = 0;
            v[c]++;
        }
        if (ready) ms_push(m, v);
    }
    return 1;
}

static uint64_t bridge_id_of(const tables_t *tb, const int32_t *ranks) {
    uint64_t id = 0;
    for (int p = 0; p < tb->P; p++) id = id * (uint64_t)tb->n + (uint64_t)tb->scid[p * tb->n + ranks[p]];
    return id;
}

/* First m bridges of the multi-sequence for the unsorted part keys
   `part_keys` (P*n).  Writes bridge keys, bridge ids (center-id mixed radix)
   and rank tuples (m*P).  Returns how many were produced (< m only when all
   n^P were exhausted).  stats (optional, 2 values): max frontier, pushes. */
int64_t oracle_multiseq(const double *part_keys, int P, int n, int dtype, int64_t m,
                        double *out_keys, uint64_t *out_ids, int32_t *out_ranks, int64_t *stats) {
    tables_t tb = tables_alloc(P, n);
    tb.dtype = dtype;
    kc_t *tmp = (kc_t *)malloc(sizeof(kc_t) * (size_t)n);
    for (int p = 0; p < P; p++) {
        for (int c = 0; c < n; c++) {
            tb.key[p * n + c] = part_keys[p * n + c];
            tmp[c].key = part_keys[p * n + c];
            tmp[c].cid = c;
        }
        qsort(tmp, (size_t)n, sizeof(kc_t), kc_cmp);
        for (int r = 0; r < n; r++) {
            tb.skey[p * n + r] = tmp[r].key;
            tb.scid[p * n + r] = tmp[r].cid;
        }
    }
    free(tmp);
    mseq_t ms;
    ms_init(&ms, &tb);
    int64_t got = 0;
    ms_item it;
    while (got < m && ms_next(&ms, &it)) {
        out_keys[got] = it.key;
        out_ids[got] = bridge_id_of(&tb, it.r);
        for (int p = 0; p < P; p++) out_ranks[got * P + p] = it.r[p];
        got++;
    }
    if (stats) {
        stats[0] = ms.max_frontier;
        stats[1] = ms.npushed;
    }
    ms_free(&ms);
    tables_free(&tb);
    return got;
}

/* ------------------------------------------------------------------------ */
/* Bridge graph (Sec. 4.1 "Augmented neighborhood graph")                    */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t bridge; double key; int32_t ref; } triple_t;

static int triple_cmp(const void *a, const void *b) {
    const triple_t *x = (const triple_t *)a, *y = (const triple_t *)b;
    if (x->bridge != y->bridge) return x->bridge < y->bridge ? -1 : 1;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->ref > y->ref) - (x->ref < y->ref);
}

/* For each reference vector, its top-t bridges (in multi-sequence order);
   then for each bridge, the b nearest of the references that named it,
   ordered by (key, ref id).  Outputs (capacity N*t each):
     bridges[M]     ascending bridge ids that got at least one reference,
     offsets[M+1]   CSR offsets into refs/keys,
     refs, keys     the kept references and their keys to the bridge.
   Returns M. */
typedef struct {
    const void *X, *centers;
    int64_t N;
    int d, dtype, P, n, t;
    triple_t *all;
    int64_t *count; /* per reference: how many of its t slots are filled */
    int64_t next;
    pthread_mutex_t mu;
} bg_job_t;

static void *bg_worker(void *arg) {
    bg_job_t *j = (bg_job_t *)arg;
    tables_t tb = tables_alloc(j->P, j->n);
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->N) break;
        tables_build(&tb, row_ptr(j->X, i, j->d, j->dtype), j->d, j->dtype, j->P, j->n, j->centers);
        mseq_t ms;
        ms_init(&ms, &tb);
        ms_item it;
        int64_t c = 0;
        for (int s = 0; s < j->t && ms_next(&ms, &it); s++) {
            triple_t *o = &j->all[i * j->t + c++];
            o->bridge = bridge_id_of(&tb, it.r);
            o->key = it.key;
            o->ref = (int32_t)i;
        }
        j->count[i] = c;
        ms_free(&ms);
    }
    tables_free(&tb);
    return NULL;
}

int64_t oracle_bridge_graph(const void *X, int64_t N, int d, int dtype, int P, int n,
                            const void *centers, int t, int b, uint64_t *bridges,
                            int64_t *offsets, int32_t *refs, double *keys, int nthreads) {
    triple_t *all = (triple_t *)malloc(sizeof(triple_t) * (size_t)N * (size_t)t);
    int64_t *count = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    bg_job_t job = {X, centers, N, d, dtype, P, n, t, all, count, 0, PTHREAD_MUTEX_INITIALIZER};
    if (nthreads <= 1) {
        bg_worker(&job);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
        for (int q = 0; q < nthreads; q++) pthread_create(&th[q], NULL, bg_worker, &job);
        for (int q = 0; q < nthreads; q++) pthread_join(th[q], NULL);
        free(th);
    }
    /* compact (references with fewer than t bridges only when n^P < t) */
    int64_t cnt = 0;
    for (int64_t i = 0; i < N; i++)
        for (int64_t c = 0; c < count[i]; c++) all[cnt++] = all[i * t + c];
    free(count);
    qsort(all, (size_t)cnt, sizeof(triple_t), triple_cmp);
    int64_t M = 0, out = 0;
    for (int64_t s = 0; s < cnt;) {
        int64_t e = s;
        while (e < cnt && all[e].bridge == all[s].bridge) e++;
        bridges[M] = all[s].bridge;
        offsets[M] = out;
        for (int64_t j = s; j < e && j < s + b; j++) {
            refs[out] = all[j].ref;
            keys[out] = all[j].key;
            out++;
        }
        M++;
        s = e;
    }
    offsets[M] = out;
    free(all);
    return M;
}

/* Bridge lists of selected bridges only (Sec. 4.1, the same definition as
   oracle_bridge_graph, restricted to the ids in sel): every reference's top-t
   bridges are enumerated as above; a selected bridge keeps the b smallest
   (key, ref id) among the references that chose it.  For indexes whose full
   list of N*t triples is too large to sort in a test.
   sel: nsel strictly ascending bridge ids.  Outputs: counts[nsel] and, per
   selected bridge i, refs/keys[i*b .. i*b + counts[i]) ascending. */
typedef struct {
    const void *X, *centers;
    int64_t N;
    int d, dtype, P, n, t, b;
    const uint64_t *sel;
    int64_t nsel;
    int32_t *counts, *refs; /* shared result, guarded by mu */
    double *keys;
    int64_t next;
    pthread_mutex_t mu;
} bl_job_t;

static int64_t sel_find(const uint64_t *sel, int64_t nsel, uint64_t id) {
    int64_t lo = 0, hi = nsel;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (sel[mid] < id) lo = mid + 1;
        else hi = mid;
    }
    return lo < nsel && sel[lo] == id ? lo : -1;
}

static void *bl_worker(void *arg) {
    bl_job_t *j = (bl_job_t *)arg;
    tables_t tb = tables_alloc(j->P, j->n);
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->N) break;
        tables_build(&tb, row_ptr(j->X, i, j->d, j->dtype), j->d, j->dtype, j->P, j->n, j->centers);
        mseq_t ms;
        ms_init(&ms, &tb);
        ms_item it;
        for (int s = 0; s < j->t && ms_next(&ms, &it); s++) {
            int64_t w = sel_find(j->sel, j->nsel, bridge_id_of(&tb, it.r));
            if (w < 0) continue;
            pthread_mutex_lock(&j->mu);
            int len = j->counts[w];
            int64_t ids64[64];
            for (int q = 0; q < len; q++) ids64[q] = j->refs[w * j->b + q];
            topk_insert(j->keys + w * j->b, ids64, &len, j->b, it.key, i);
            for (int q = 0; q < len; q++) j->refs[w * j->b + q] = (int32_t)ids64[q];
            j->counts[w] = len;
            pthread_mutex_unlock(&j->mu);
        }
        ms_free(&ms);
    }
    tables_free(&tb);
    return NULL;
}

void oracle_bridge_lists(const void *X, int64_t N, int d, int dtype, int P, int n, const void *centers, int t,
                         int b, const uint64_t *sel, int64_t nsel, int32_t *counts, int32_t *refs, double *keys,
                         int nthreads) {
    bl_job_t job = {X, centers, N, d, dtype, P, n, t, b, sel, nsel, counts, refs, keys, 0,
                    PTHREAD_MUTEX_INITIALIZER};
    for (int64_t i = 0; i < nsel; i++) counts[i] = 0;
    if (nthreads <= 1) {
        bl_worker(&job);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
        for (int q = 0; q < nthreads; q++) pthread_create(&th[q], NULL, bl_worker, &job);
        for (int q = 0; q < nthreads; q++) pthread_join(th[q], NULL);
        free(th);
    }
}

/* The bridge graph restricted to the bridges some query can reach below its
   key limit (Sec. 4.1's definition, restricted): bridge y is kept when
   key(q, y) <= limit[q] for at least one query q (a bridge slightly above
   every limit may be kept too: the test only ever admits more), and it keeps
   the b smallest (key to y, ref id) among ALL references that chose it, so
   every kept list equals the full bridge graph's list.  Every bridge that is
   absent has either no reference or keys above every limit.  For indexes
   whose N*t triples are too many to sort at once.  Each thread keeps a hash
   map bridge id -> its b best so far; the maps are merged at the end.
   Outputs are allocated here (release each with oracle_free); returns M. */
typedef struct {
    uint64_t id; /* bridge id + 1; 0 = empty slot */
    int len;
    double keys[8];
    int64_t refs[8];
} near_slot_t;

typedef struct {
    near_slot_t *slot;
    int64_t cap, len;
} near_map_t;

static near_slot_t *near_get(near_map_t *m, uint64_t id) {
    if (2 * (m->len + 1) > m->cap) {
        near_slot_t *old = m->slot;
        int64_t oc = m->cap;
        m->cap = oc ? 2 * oc : 1024;
        m->slot = (near_slot_t *)calloc((size_t)m->cap, sizeof(near_slot_t));
        m->len = 0;
        for (int64_t i = 0; i < oc; i++)
            if (old[i].id) {
                near_slot_t *d = near_get(m, old[i].id - 1);
                *d = old[i];
            }
        free(old);
    }
    uint64_t mask = (uint64_t)m->cap - 1, h = mix64(id) & mask;
    while (m->slot[h].id && m->slot[h].id != id + 1) h = (h + 1) & mask;
    if (!m->slot[h].id) {
        m->slot[h].id = id + 1;
        m->slot[h].len = 0;
        m->len++;
    }
    return &m->slot[h];
}

typedef struct {
    const void *X, *centers;
    int64_t N;
    int d, dtype, P, n, t, b, nq;
    const double *qkeys;  /* nq * P * n part keys of the queries, unsorted */
    const double *limit;  /* nq */
    near_map_t *maps;     /* one per thread */
    int64_t next;
    pthread_mutex_t mu;
} near_job_t;

typedef struct { near_job_t *job; int th; } near_arg_t;

static void *near_worker(void *arg) {
    near_arg_t *a = (near_arg_t *)arg;
    near_job_t *j = a->job;
    near_map_t *map = &j->maps[a->th];
    tables_t tb = tables_alloc(j->P, j->n);
    int32_t cid[MAXP];
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->N) break;
        tables_build(&tb, row_ptr(j->X, i, j->d, j->dtype), j->d, j->dtype, j->P, j->n, j->centers);
        mseq_t ms;
        ms_init(&ms, &tb);
        ms_item it;
        for (int s = 0; s < j->t && ms_next(&ms, &it); s++) {
            for (int p = 0; p < j->P; p++) cid[p] = tb.scid[p * j->n + it.r[p]];
            int hit = 0;
            for (int q = 0; q < j->nq && !hit; q++) {
                /* the query's key to this bridge: exact for bytes; for float32 an
                   fp64 sum, admitted with a margin above the limit */
                double k = 0.0;
                for (int p = 0; p < j->P; p++) k += j->qkeys[((int64_t)q * j->P + p) * j->n + cid[p]];
                hit = j->dtype == DT_U8 ? k <= j->limit[q] : k <= j->limit[q] * (1.0 + 1e-5);
            }
            if (!hit) continue;
            near_slot_t *e = near_get(map, bridge_id_of(&tb, it.r));
            topk_insert(e->keys, e->refs, &e->len, j->b, it.key, i);
        }
        ms_free(&ms);
    }
    tables_free(&tb);
    return NULL;
}

static int u64_cmp(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

int64_t oracle_bridge_graph_near(const void *X, int64_t N, int d, int dtype, int P, int n, const void *centers,
                                 int t, int b, const void *queries, int nq, const double *limit,
                                 uint64_t **out_bridges, int64_t **out_offsets, int32_t **out_refs,
                                 double **out_keys, int nthreads) {
    if (b > 8 || P > MAXP) return -1;
    if (nthreads < 1) nthreads = 1;
    double *qkeys = (double *)malloc(sizeof(double) * (size_t)nq * P * n);
    tables_t tb = tables_alloc(P, n);
    for (int q = 0; q < nq; q++) {
        tables_build(&tb, row_ptr(queries, q, d, dtype), d, dtype, P, n, centers);
        memcpy(qkeys + (int64_t)q * P * n, tb.key, sizeof(double) * (size_t)P * n);
    }
    tables_free(&tb);
    near_job_t job = {X, centers, N, d, dtype, P, n, t, b, nq, qkeys, limit, NULL, 0, PTHREAD_MUTEX_INITIALIZER};
    job.maps = (near_map_t *)calloc((size_t)nthreads, sizeof(near_map_t));
    near_arg_t *args = (near_arg_t *)malloc(sizeof(near_arg_t) * (size_t)nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int q = 0; q < nthreads; q++) {
        args[q].job = &job;
        args[q].th = q;
        pthread_create(&th[q], NULL, near_worker, &args[q]);
    }
    for (int q = 0; q < nthreads; q++) pthread_join(th[q], NULL);
    /* merge: every thread's b best of a bridge, the b best overall */
    near_map_t all = {0};
    for (int q = 0; q < nthreads; q++) {
        near_map_t *m = &job.maps[q];
        for (int64_t i = 0; i < m->cap; i++) {
            near_slot_t *e = &m->slot[i];
            if (!e->id) continue;
            near_slot_t *g = near_get(&all, e->id - 1);
            for (int r = 0; r < e->len; r++) topk_insert(g->keys, g->refs, &g->len, b, e->keys[r], e->refs[r]);
        }
        free(m->slot);
    }
    int64_t M = all.len;
    uint64_t *ids = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(M > 0 ? M : 1));
    int64_t c = 0;
    for (int64_t i = 0; i < all.cap; i++)
        if (all.slot[i].id) ids[c++] = all.slot[i].id - 1;
    qsort(ids, (size_t)M, sizeof(uint64_t), u64_cmp);
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
    int32_t *refs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M * b + 1));
    double *keys = (double *)malloc(sizeof(double) * (size_t)(M * b + 1));
    int64_t o = 0;
    for (int64_t i = 0; i < M; i++) {
        near_slot_t *g = near_get(&all, ids[i]);
        offs[i] = o;
        for (int r = 0; r < g->len; r++) {
            refs[o] = (int32_t)g->refs[r];
            keys[o] = g->keys[r];
            o++;
        }
    }
    offs[M] = o;
    free(all.slot);
    free(job.maps);
    free(args);
    free(th);
    free(qkeys);
    *out_bridges = ids;
    *out_offsets = offs;
    *out_refs = refs;
    *out_keys = keys;
    return M;
}

void oracle_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Algorithm 1: ANN search over the augmented neighborhood graph (Sec. 4.2)  */
/* ------------------------------------------------------------------------ */

typedef struct { double key; int kind; int64_t id; } q_item; /* kind 0 = ref, 1 = bridge */

static int q_less(const q_item *a, const q_item *b) {
    if (a->key != b->key) return a->key < b->key;
    if (a->kind != b->kind) return a->kind < b->kind;
    return a->id < b->id;
}

typedef struct { q_item *h; int64_t len, cap; } pq_t;

static void pq_push(pq_t *q, q_item it) {
    if (q->len == q->cap) {
        q->cap = q->cap ? q->cap * 2 : 64;
        q->h = (q_item *)realloc(q->h, sizeof(q_item) * (size_t)q->cap);
    }
    int64_t i = q->len++;
    q->h[i] = it;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!q_less(&q->h[i], &q->h[p])) break;
        q_item t = q->h[i]; q->h[i] = q->h[p]; q->h[p] = t;
        i = p;
    }
}

static q_item pq_pop(pq_t *q) {
    q_item top = q->h[0];
    q->h[0] = q->h[--q->len];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < q->len && q_less(&q->h[l], &q->h[s])) s = l;
        if (r < q->len && q_less(&q->h[r], &q->h[s])) s = r;
        if (s == i) break;
        q_item t = q->h[i]; q->h[i] = q->h[s]; q->h[s] = t;
        i = s;
    }
    return top;
}

enum {
    ST_DISCOVERED = 0, /* t at the end: reference vectors discovered */
    ST_REF_POPS,       /* reference vectors popped (neighbourhoods expanded) */
    ST_BRIDGE_POPS,    /* bridge vectors popped */
    ST_NONEMPTY_POPS,  /* popped bridges with at least one reference */
    ST_MAX_Q,          /* largest main-queue length (refs + the bridge) */
    ST_MAX_FRONTIER,   /* largest multi-sequence queue length */
    ST_MS_PUSHES,      /* tuples pushed into the multi-sequence queue */
    ST_OVER_LIMIT,     /* 1 if a popped bridge's key exceeded the caller's limit (search stopped there) */
    ST_N
};

typedef struct {
    const void *X;
    int64_t N;
    int d, dtype;
    const int32_t *graph;
    int R;
    int P, n;
    const void *centers;
    int64_t M;
    const uint64_t *bridges;
    const int64_t *boff;
    const int32_t *brefs;
    int row_threads; /* threads that share one on-demand kNN row scan */
} index_t;

/* The R nearest other references of reference p by linear scan (Sec. 3.1:
   Adj[p] of the neighbourhood graph), ascending (key, id).  The scan over
   [0, N) is split into row_threads contiguous chunks; each chunk keeps its
   own R smallest, and the chunks' lists are merged by the same insertion,
   which gives the R smallest overall. */
typedef struct {
    const index_t *ix;
    int64_t p, lo, hi;
    double keys[64];
    int64_t ids[64];
    int len;
} rowscan_t;

static void *rowscan_worker(void *arg) {
    rowscan_t *c = (rowscan_t *)arg;
    const index_t *ix = c->ix;
    const void *xp = row_ptr(ix->X, c->p, ix->d, ix->dtype);
    c->len = 0;
    for (int64_t j = c->lo; j < c->hi; j++) {
        if (j == c->p) continue;
        double kj = sqdist(xp, row_ptr(ix->X, j, ix->d, ix->dtype), ix->d, ix->dtype);
        topk_insert(c->keys, c->ids, &c->len, ix->R, kj, j);
    }
    return NULL;
}

static void knn_row_scan(const index_t *ix, int64_t p, double *keys, int64_t *ids, int *len) {
    int nt = ix->row_threads < 1 ? 1 : (ix->row_threads > 16 ? 16 : ix->row_threads);
    rowscan_t c[16];
    pthread_t th[16];
    for (int t = 0; t < nt; t++) {
        c[t].ix = ix;
        c[t].p = p;
        c[t].lo = ix->N * t / nt;
        c[t].hi = ix->N * (t + 1) / nt;
        if (t > 0) pthread_create(&th[t], NULL, rowscan_worker, &c[t]);
    }
    rowscan_worker(&c[0]);
    for (int t = 1; t < nt; t++) pthread_join(th[t], NULL);
    *len = 0;
    for (int t = 0; t < nt; t++)
        for (int i = 0; i < c[t].len; i++) topk_insert(keys, ids, len, ix->R, c[t].keys[i], c[t].ids[i]);
}

/* Bridge id -> its reference list (binary search over the sorted ids). */
static int64_t bridge_lookup(const index_t *ix, uint64_t id, int64_t *len) {
    int64_t lo = 0, hi = ix->M;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ix->bridges[mid] < id) lo = mid + 1; else hi = mid;
    }
    if (lo < ix->M && ix->bridges[lo] == id) {
        *len = ix->boff[lo + 1] - ix->boff[lo];
        return ix->boff[lo];
    }
    *len = 0;
    return 0;
}

/* One query.  ids/keys: kmax outputs; stats: ST_N values. */
static void search_one(const index_t *ix, const void *q, int k, int T, int kmax, uint8_t *color,
                       int32_t *out_ids, double *out_keys, int64_t *stats, int32_t *disc,
                       int disc_cap, double bkey_limit) {
    int64_t st[ST_N] = {0};
    /* Mark each reference vector undiscovered. */
    memset(color, 0, (size_t)ix->N);
    /* Tables and per-part sort, then the nearest bridge vector. */
    tables_t tb = tables_alloc(ix->P, ix->n);
    tables_build(&tb, q, ix->d, ix->dtype, ix->P, ix->n, ix->centers);
    mseq_t ms;
    ms_init(&ms, &tb);
    pq_t Q = {0};
    double *rkeys = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    int64_t *rids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int rlen = 0;
    ms_item cur;
    int32_t cur_ranks[MAXP];
    if (ms_next(&ms, &cur)) {
        q_item it = {cur.key, 1, 0};
        memcpy(cur_ranks, cur.r, sizeof(cur_ranks));
        pq_push(&Q, it);
    }
    int64_t t = 0;
    int32_t rowbuf[64];
    double rowk[64];
    int64_t rowi[64];
    if (Q.len > st[ST_MAX_Q]) st[ST_MAX_Q] = Q.len;
    while (Q.len > 0 && t < T) {
        q_item p = pq_pop(&Q);
        const int32_t *adj;
        int64_t alen;
        if (p.kind == 0) {
            st[ST_REF_POPS]++;
            if (ix->graph) {
                adj = ix->graph + p.id * ix->R;
            } else {
                /* no stored graph: Adj[p] by its definition, the R nearest
                   other references by linear scan (Sec. 3.1) */
                int len = 0;
                knn_row_scan(ix, p.id, rowk, rowi, &len);
                for (int r = 0; r < ix->R; r++) rowbuf[r] = r < len ? (int32_t)rowi[r] : -1;
                adj = rowbuf;
            }
            alen = ix->R;
        } else {
            st[ST_BRIDGE_POPS]++;
            if (p.key > bkey_limit) {
                /* the caller's bridge lists are complete only up to this key */
                st[ST_OVER_LIMIT] = 1;
                break;
            }
            int64_t off = bridge_lookup(ix, bridge_id_of(&tb, cur_ranks), &alen);
            adj = ix->brefs + off;
            if (alen > 0) st[ST_NONEMPTY_POPS]++;
        }
        for (int64_t a = 0; a < alen && t < T; a++) {
            int32_t x = adj[a];
            if (x < 0) continue; /* padding in short kNN rows */
            if (color[x] == 0) {
                double D = sqdist(q, row_ptr(ix->X, x, ix->d, ix->dtype), ix->d, ix->dtype);
                q_item it = {D, 0, x};
                pq_push(&Q, it);
                color[x] = 1;
                if (k > 0) topk_insert(rkeys, rids, &rlen, k, D, x);
                if (disc && t < disc_cap) disc[t] = x;
                t++;
            }
        }
        if (p.kind == 1 && t < T) {
            if (ms_next(&ms, &cur)) {
                q_item it = {cur.key, 1, 0};
                memcpy(cur_ranks, cur.r, sizeof(cur_ranks));
                pq_push(&Q, it);
            }
        }
        if (Q.len > st[ST_MAX_Q]) st[ST_MAX_Q] = Q.len;
    }
    st[ST_DISCOVERED] = t;
    st[ST_MAX_FRONTIER] = ms.max_frontier;
    st[ST_MS_PUSHES] = ms.npushed;
    for (int r = 0; r < kmax; r++) {
        out_ids[r] = r < rlen ? (int32_t)rids[r] : -1;
        out_keys[r] = r < rlen ? rkeys[r] : INFINITY;
    }
    if (stats) memcpy(stats, st, sizeof(st));
    if (disc)
        for (int64_t i = t; i < disc_cap; i++) disc[i] = -1;
    free(rkeys);
    free(rids);
    free(Q.h);
    ms_free(&ms);
    tables_free(&tb);
}

typedef struct {
    const index_t *ix;
    const void *queries;
    int64_t nq;
    const int32_t *k, *T;
    int kmax;
    int32_t *out_ids;
    double *out_keys;
    int64_t *stats;
    int32_t *disc;
    int disc_cap;
    const double *bkey_limit;
    int64_t next;
    pthread_mutex_t mu;
} job_t;

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    const index_t *ix = j->ix;
    uint8_t *color = (uint8_t *)malloc((size_t)ix->N);
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->nq) break;
        search_one(ix, row_ptr(j->queries, i, ix->d, ix->dtype), j->k[i], j->T[i], j->kmax, color,
                   j->out_ids + i * j->kmax, j->out_keys + i * j->kmax,
                   j->stats ? j->stats + i * ST_N : NULL,
                   j->disc ? j->disc + i * (int64_t)j->disc_cap : NULL, j->disc_cap,
                   j->bkey_limit ? j->bkey_limit[i] : INFINITY);
    }
    free(color);
    return NULL;
}

/* Batched search: one query at a time per thread (nthreads >= 1).
   graph may be NULL: then each popped reference's R nearest neighbours are
   computed on demand by linear scan.
   k[i], T[i]: per-query result count (<= kmax) and budget.
   bridges/boff/brefs: the bridge graph as produced by oracle_bridge_graph.
   disc (optional, nq*disc_cap): discovered ids in discovery order, -1 after.
   bkey_limit (optional, nq): the bridge lists given are complete only for
   bridges with key <= bkey_limit[i]; a query that would pop a bridge above
   it stops there and reports ST_OVER_LIMIT. */
int oracle_search(const void *X, int64_t N, int d, int dtype, const int32_t *graph, int R, int P,
                  int n, const void *centers, int64_t M, const uint64_t *bridges,
                  const int64_t *boff, const int32_t *brefs, const void *queries, int64_t nq,
                  const int32_t *k, const int32_t *T, int kmax, int32_t *out_ids,
                  double *out_keys, int64_t *stats, int32_t *disc, int disc_cap, const double *bkey_limit,
                  int nthreads) {
    if (P > MAXP || P < 1 || d % P != 0 || R > 64) return -1;
    /* threads left over when there are fewer queries than threads share the
       on-demand kNN row scans of each query */
    int row_threads = nq > 0 && nthreads > nq ? (int)(nthreads / nq) : 1;
    index_t ix = {X, N, d, dtype, graph, R, P, n, centers, M, bridges, boff, brefs, row_threads};
    job_t job = {&ix, queries, nq, k, T, kmax, out_ids, out_keys, stats, disc, disc_cap, bkey_limit, 0,
                 PTHREAD_MUTEX_INITIALIZER};
    if (nthreads <= 1) {
        worker(&job);
        return 0;
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, worker, &job);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

int oracle_num_stats(void) { return ST_N; }

/* ------------------------------------------------------------------------ */
/* Approximate R-NN neighbourhood graph.  Sec. 5.3 builds the neighbourhood */
/* graph approximately with the construction of its reference [WangWZTGL12] */
/* (random divide-and-conquer, then neighbourhood propagation) and Sec. 5.5 */
/* puts its cost at O(N log N); the paper gives no steps.  The reading      */
/* fixed here, for uint8 data:                                              */
/*  - `rounds` random partitions.  Positions [0, N) are halved recursively  */
/*    `levels` times: segment [lo, hi) has the children [lo, m) and         */
/*    [m, hi), m = lo + (hi - lo) / 2 (integer division).  Level l holds     */
/*    the 2^l segments s = 0 .. 2^l - 1, left to right.  Starting from the  */
/*    identity order, at each level l every segment s reorders its members  */
/*    ascending by (<u, x>, id), u = dirs[round][2^l - 1 + s] (d int8       */
/*    entries, a random direction drawn by the caller).  The 2^levels       */
/*    segments below the last level are the leaves.                         */
/*  - Leaf step: every point is offered every other member of its leaf, in  */
/*    every round.                                                          */
/*  - `iters` propagation steps, each from the rows of the step before:     */
/*    row i is offered every entry of the rows of its neighbours (i itself  */
/*    excluded).                                                            */
/* Offering (key, id) keeps the R smallest (key, id) pairs with distinct    */
/* ids, so a row is the R best of every candidate offered, in any order.    */
/* ------------------------------------------------------------------------ */

/* The range [lo, hi) of segment s at level l of the recursive halving. */
static void seg_range(int64_t N, int l, int64_t s, int64_t *lo, int64_t *hi) {
    int64_t a = 0, b = N;
    for (int bit = l - 1; bit >= 0; bit--) {
        int64_t m = a + (b - a) / 2;
        if ((s >> bit) & 1) a = m;
        else b = m;
    }
    *lo = a;
    *hi = b;
}

typedef struct {
    int64_t proj, id;
} proj_id_t;

static int proj_id_cmp(const void *a, const void *b) {
    const proj_id_t *x = (const proj_id_t *)a, *y = (const proj_id_t *)b;
    if (x->proj != y->proj) return x->proj < y->proj ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* One random partition: perm[p] = the point at position p after `levels`
   levels of median splits along the directions dirs[(2^l - 1 + s) * d]. */
void oracle_rp_partition(const uint8_t *X, int64_t N, int d, const int8_t *dirs, int levels, int32_t *perm) {
    for (int64_t i = 0; i < N; i++) perm[i] = (int32_t)i;
    proj_id_t *buf = (proj_id_t *)malloc(sizeof(proj_id_t) * (size_t)(N > 0 ? N : 1));
    for (int l = 0; l < levels; l++) {
        for (int64_t s = 0; s < ((int64_t)1 << l); s++) {
            int64_t lo, hi;
            seg_range(N, l, s, &lo, &hi);
            const int8_t *u = dirs + ((((int64_t)1 << l) - 1) + s) * d;
            for (int64_t p = lo; p < hi; p++) {
                const uint8_t *x = X + (int64_t)perm[p] * d;
                int64_t acc = 0;
                for (int w = 0; w < d; w++) acc += (int64_t)u[w] * (int64_t)x[w];
                buf[p - lo].proj = acc;
                buf[p - lo].id = perm[p];
            }
            qsort(buf, (size_t)(hi - lo), sizeof(proj_id_t), proj_id_cmp);
            for (int64_t p = lo; p < hi; p++) perm[p] = (int32_t)buf[p - lo].id;
        }
    }
    free(buf);
}

/* offer (key, id) to a row: keep the cap smallest pairs, ids distinct */
static void offer_distinct(double *keys, int64_t *ids, int *len, int cap, double key, int64_t id) {
    for (int r = 0; r < *len; r++)
        if (ids[r] == id) return;
    topk_insert(keys, ids, len, cap, key, id);
}

/* Rows of every propagation step, computed on demand and kept. */
typedef struct {
    int64_t cap, used;
    int32_t *slot;  /* N entries: index into the pool, -1 if not computed */
    int64_t *ids;   /* pool, cap * R */
    double *keys;
    int *len;
} row_store_t;

typedef struct {
    const uint8_t *X;
    int64_t N;
    int d, R, rounds, levels;
    int32_t *perm; /* rounds * N: point at each position */
    int32_t *pos;  /* rounds * N: position of each point */
    row_store_t *st; /* iters + 1 stores */
} approx_t;

static int64_t store_new(row_store_t *s, int R) {
    if (s->used == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 1024;
        s->ids = (int64_t *)realloc(s->ids, sizeof(int64_t) * (size_t)(s->cap * R));
        s->keys = (double *)realloc(s->keys, sizeof(double) * (size_t)(s->cap * R));
        s->len = (int *)realloc(s->len, sizeof(int) * (size_t)s->cap);
    }
    return s->used++;
}

/* Row of point i after step it (0 = leaf step); copies it to keys/ids/len. */
static void approx_row(approx_t *g, int it, int64_t i, double *keys, int64_t *ids, int *len) {
    row_store_t *s = &g->st[it];
    const int R = g->R;
    if (s->slot[i] < 0) {
        double k0[64];
        int64_t i0[64];
        int n0 = 0;
        const uint8_t *xi = g->X + i * g->d;
        if (it == 0) {
            for (int r = 0; r < g->rounds; r++) {
                int64_t p = g->pos[(int64_t)r * g->N + i], lo = 0, hi = g->N;
                for (int l = 0; l < g->levels; l++) {
                    int64_t m = lo + (hi - lo) / 2;
                    if (p >= m) lo = m;
                    else hi = m;
                }
                for (int64_t q = lo; q < hi; q++) {
                    int64_t j = g->perm[(int64_t)r * g->N + q];
                    if (j == i) continue;
                    offer_distinct(k0, i0, &n0, R, sqdist(xi, g->X + j * g->d, g->d, DT_U8), j);
                }
            }
        } else {
            double kb[64];
            int64_t ib[64];
            int nb = 0;
            approx_row(g, it - 1, i, kb, ib, &nb);
            for (int r = 0; r < nb; r++) offer_distinct(k0, i0, &n0, R, kb[r], ib[r]);
            for (int r = 0; r < nb; r++) {
                double kj[64];
                int64_t ij[64];
                int nj = 0;
                approx_row(g, it - 1, ib[r], kj, ij, &nj);
                for (int c = 0; c < nj; c++) {
                    if (ij[c] == i) continue;
                    offer_distinct(k0, i0, &n0, R, sqdist(xi, g->X + ij[c] * g->d, g->d, DT_U8), ij[c]);
                }
            }
        }
        int64_t at = store_new(s, R);
        memcpy(s->keys + at * R, k0, sizeof(double) * (size_t)n0);
        memcpy(s->ids + at * R, i0, sizeof(int64_t) * (size_t)n0);
        s->len[at] = n0;
        s->slot[i] = (int32_t)at;
    }
    int64_t at = s->slot[i];
    *len = s->len[at];
    memcpy(keys, s->keys + at * R, sizeof(double) * (size_t)*len);
    memcpy(ids, s->ids + at * R, sizeof(int64_t) * (size_t)*len);
}

/* Approximate R-NN graph rows (the reading above).  dirs: rounds *
   (2^levels - 1) * d int8.  rows: the points whose rows are wanted (NULL =
   all N, in order); out: nrows * R ids / keys, ascending (key, id), padded
   with -1 / +inf.  Rows are evaluated on demand, so a few sampled rows of a
   large set cost only their own dependencies.  R <= 64. */
void oracle_knn_graph_approx(const uint8_t *X, int64_t N, int d, int R, const int8_t *dirs, int rounds,
                             int levels, int iters, const int64_t *rows, int64_t nrows, int32_t *out_ids,
                             double *out_keys) {
    approx_t g = {X, N, d, R, rounds, levels, NULL, NULL, NULL};
    g.perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rounds * N));
    g.pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rounds * N));
    const int64_t nseg = ((int64_t)1 << levels) - 1;
    for (int r = 0; r < rounds; r++) {
        int32_t *pm = g.perm + (int64_t)r * N;
        oracle_rp_partition(X, N, d, dirs + (int64_t)r * nseg * d, levels, pm);
        for (int64_t p = 0; p < N; p++) g.pos[(int64_t)r * N + pm[p]] = (int32_t)p;
    }
    g.st = (row_store_t *)calloc((size_t)iters + 1, sizeof(row_store_t));
    for (int it = 0; it <= iters; it++) {
        g.st[it].slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
        for (int64_t i = 0; i < N; i++) g.st[it].slot[i] = -1;
    }
    if (!rows) nrows = N;
    for (int64_t q = 0; q < nrows; q++) {
        int64_t i = rows ? rows[q] : q;
        double k[64];
        int64_t id[64];
        int n = 0;
        approx_row(&g, iters, i, k, id, &n);
        for (int r = 0; r < R; r++) {
            out_ids[q * R + r] = r < n ? (int32_t)id[r] : -1;
            out_keys[q * R + r] = r < n ? k[r] : INFINITY;
        }
    }
    for (int it = 0; it <= iters; it++) {
        free(g.st[it].slot);
        free(g.st[it].ids);
        free(g.st[it].keys);
        free(g.st[it].len);
    }
    free(g.st);
    free(g.perm);
    free(g.pos);
}

/* ------------------------------------------------------------------------ */
/* Graph-D-ADC (Sec. 5.4): the method as the coarse quantizer of an inverted */
/* file with product-quantized residuals.  Each reference x is listed under  */
/* its assigned coarse center c(x); its residual r = x - c(x) is encoded by  */
/* m sub-quantizers of ks codewords over contiguous parts of d / m dims.    */
/* A query visits the lists of its nearest centers (found by Alg. 1 over an */
/* index of the centers) and re-ranks their members by the asymmetric       */
/* distance ||q - c - r^||^2, r^ the concatenated codewords of x's code.    */
/* Readings fixed here: codes take the nearest codeword of each part, ties  */
/* to the lower codeword index; lists are visited in the order given        */
/* (ascending coarse key), members of a list ascending by id, and the first */
/* L members overall are the candidates; the top T candidates by (ADC key, */
/* id) are returned.                                                        */
/* Precision: the paper fixes none.  Both distances are real-valued        */
/* squared distances of Sec. 5.4 (nearest codeword; asymmetric distance     */
/* between the query and the reconstruction c + r^), taken here in fp64 on  */
/* the float32 inputs, so a code or a rank differs from the real one only   */
/* where two candidates lie within fp64 rounding of each other.             */
/* ------------------------------------------------------------------------ */

/* codes[i*m + j] = the codeword of part j nearest to the residual of X[i]
   (X: N*d, centers: K*d, assign: N coarse ids, codebooks: m*ks*(d/m)). */
void oracle_pq_encode(const float *X, int64_t N, int d, const float *centers, const int32_t *assign, int m, int ks,
                      const float *codebooks, uint8_t *codes) {
    const int dp = d / m;
    for (int64_t i = 0; i < N; i++) {
        const float *x = X + i * d;
        const float *c = centers + (int64_t)assign[i] * d;
        for (int j = 0; j < m; j++) {
            double best = INFINITY;
            int arg = 0;
            for (int k = 0; k < ks; k++) {
                const float *w = codebooks + ((int64_t)j * ks + k) * dp;
                double sum = 0.0;
                for (int t = 0; t < dp; t++) {
                    double e = ((double)x[j * dp + t] - (double)c[j * dp + t]) - (double)w[t];
                    sum += e * e;
                }
                if (sum < best) { /* strict: ties keep the lower codeword */
                    best = sum;
                    arg = k;
                }
            }
            codes[i * m + j] = (uint8_t)arg;
        }
    }
}

/* The asymmetric distance of one candidate x listed under center c:
   sum over parts j of || (q - c)^j - codeword(j, code_j(x)) ||^2. */
static double adc_key(const float *q, const float *cv, const uint8_t *code, int m, int ks, int dp,
                      const float *codebooks) {
    double key = 0.0;
    for (int j = 0; j < m; j++) {
        const float *w = codebooks + ((int64_t)j * ks + code[j]) * dp;
        for (int t = 0; t < dp; t++) {
            double e = ((double)q[j * dp + t] - (double)cv[j * dp + t]) - (double)w[t];
            key += e * e;
        }
    }
    return key;
}

/* Re-rank one query.  lists: the nlists coarse centers to visit, in order
   (negative entries skipped); offsets/members: inverted lists (members
   ascending by id within a list); centers: K*d coarse centers.  Out: the T
   best (key, id), padded -1/+inf.  Returns the number of candidates
   examined (<= L). */
int64_t oracle_adc_rerank(const float *q, int d, const int32_t *lists, int nlists, const int64_t *offsets,
                          const int32_t *members, const float *centers, const uint8_t *codes, int m, int ks,
                          const float *codebooks, int64_t L, int T, int32_t *out_ids, double *out_keys) {
    const int dp = d / m;
    double *keys = (double *)malloc(sizeof(double) * (size_t)T);
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)T);
    int len = 0;
    int64_t seen = 0;
    for (int li = 0; li < nlists && seen < L; li++) {
        const int32_t c = lists[li];
        if (c < 0) continue;
        const float *cv = centers + (int64_t)c * d;
        for (int64_t p = offsets[c]; p < offsets[c + 1] && seen < L; p++, seen++) {
            const int32_t x = members[p];
            topk_insert(keys, ids, &len, T, adc_key(q, cv, codes + (int64_t)x * m, m, ks, dp, codebooks), x);
        }
    }
    for (int r = 0; r < T; r++) {
        out_ids[r] = r < len ? (int32_t)ids[r] : -1;
        out_keys[r] = r < len ? keys[r] : INFINITY;
    }
    free(keys);
    free(ids);
    return seen;
}

/* The asymmetric distances of n given candidates to one query (x's list is
   assign[x]), for comparing any candidate a caller holds. */
void oracle_adc_keys(const float *q, int d, const int32_t *cand, int64_t n, const int32_t *assign,
                     const float *centers, const uint8_t *codes, int m, int ks, const float *codebooks,
                     double *out_keys) {
    const int dp = d / m;
    for (int64_t i = 0; i < n; i++) {
        const int32_t x = cand[i];
        out_keys[i] = adc_key(q, centers + (int64_t)assign[x] * d, codes + (int64_t)x * m, m, ks, dp, codebooks);
    }
}
