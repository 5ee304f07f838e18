/*
 * hamming_oracle.c -- CPU oracle for exact search in Hamming space.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load it; the library never does,
 * and it shares no code, header or table with the CUDA sources.
 *
 * Paper: M. Norouzi, A. Punjani, D. J. Fleet, "Fast Exact Search in Hamming
 * Space with Multi-Index Hashing" (arXiv:1307.2982).
 *
 * Conventions (the paper leaves bit order open; see the readings below):
 *   - a code of q bits is stored as W = ceil(q/64) little-endian uint64
 *     words; code bit b is bit (b % 64) of word (b / 64); bits >= q are 0;
 *   - substring j covers code bits [off_j, off_j + len_j) and its key has
 *     key bit t = code bit off_j + t;
 *   - results are ordered by (distance, id) ascending, which makes the
 *     k-NN answer unique (the paper allows any choice among equidistant
 *     codes, Sec. 5.2).
 *
 * Contents:
 *   orc_hamming          Sec. 1.1 (Hamming distance), Sec. 6 "Hamming Distance"
 *   orc_substring_layout Sec. 2.1 and its footnote (substring lengths)
 *   orc_substring_keys   Sec. 2.1 (contiguous substrings), bit by bit
 *   orc_knn              Sec. 1.1 (k-NN problem), by definition
 *   orc_rnear_count/fill Sec. 1.1 (r-neighbour problem), by definition
 *   orc_table_build      Algorithm 1 (one table per substring)
 *   orc_ring             Algorithm 3 (buckets at exactly r' bits), brute force
 *   orc_mih_rnear        Algorithm 2 (r-neighbour search by MIH)
 *   orc_mih_knn          Algorithm 3 (k-NN search by MIH, growing radius)
 *   orc_rerank_asym      Sec. 5.1 / Conclusion: candidates re-ranked by an
 *                        asymmetric Hamming distance (reading c17)
 *
 * Parity is pinned by tests/test_oracle_pins.py against brute force in numpy,
 * closed forms (Eq. 1), Propositions 1 and 2, and special cases.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ 256
#define ORC_PAD_ID 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Sec. 1.1: ||h - g||_H is the number of bit positions in which h and g differ.
 * Sec. 6 "Hamming Distance": one xor per 64 bits and a population count. */
int orc_hamming(const uint64_t *a, const uint64_t *b, int W)
{
    int d = 0;
    for (int w = 0; w < W; ++w)
        d += __builtin_popcountll(a[w] ^ b[w]);
    return d;
}

static int code_bit(const uint64_t *code, int b)
{
    return (int)((code[b >> 6] >> (b & 63)) & 1u);
}

/* Sec. 2.1 and its footnote: m disjoint substrings of contiguous bits, each
 * floor(q/m) or ceil(q/m) bits long.  Reading: the first m - (q mod m)
 * substrings take floor(q/m) bits and the last (q mod m) take ceil(q/m). */
void orc_substring_layout(int q, int m, int *off, int *len)
{
    int shortl = q / m, nlong = q % m, o = 0;
    for (int j = 0; j < m; ++j) {
        len[j] = shortl + (j >= m - nlong ? 1 : 0);
        off[j] = o;
        o += len[j];
    }
}

/* Key of one substring, built one bit at a time: key bit t = code bit off+t. */
uint64_t orc_substring_key(const uint64_t *code, int off, int len)
{
    uint64_t key = 0;
    for (int t = 0; t < len; ++t)
        key |= (uint64_t)code_bit(code, off + t) << t;
    return key;
}

void orc_substring_keys(const uint64_t *codes, uint64_t n, int W, int off,
                        int len, uint64_t *keys)
{
    for (uint64_t i = 0; i < n; ++i)
        keys[i] = orc_substring_key(codes + i * W, off, len);
}

/* ------------------------------------------------------------------------ */
/* Threading over queries: each worker takes queries i = tid, tid+T, ... */
typedef struct {
    const uint64_t *codes;
    uint64_t n;
    int W;
    const uint64_t *queries;
    uint64_t nq;
    const uint32_t *k;        /* k-NN: per-query k */
    const uint64_t *out_off;  /* k-NN / rnear fill: per-query output offset */
    int r;                    /* rnear radius */
    uint64_t *counts;         /* rnear count */
    uint32_t *out_ids;
    int32_t *out_dist;
    int tid, nthreads;
    int status;
} orc_job;

static int run_threads(orc_job *proto, int nthreads, void *(*fn)(void *))
{
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > proto->nq && proto->nq > 0) nthreads = (int)proto->nq;
    orc_job *jobs = (orc_job *)calloc((size_t)nthreads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    int status = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nthreads;
        jobs[t].status = 0;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) { jobs[t].status = -1; th[t] = 0; }
    fn(&jobs[0]);
    for (int t = 1; t < nthreads; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status) status = jobs[t].status;
    free(jobs);
    free(th);
    return status;
}

/* Sec. 1.1, k-NN problem: the k codes closest to g.  With the (distance, id)
 * order the answer is the first min(k, n) entries of the list of all
 * (||h_i - g||_H, i), sorted lexicographically.  Distances are integers in
 * 0..q, so the list is laid out by a counting sort over the distance that is
 * stable in i: one pass counts the codes at each distance, a second pass
 * visits the ids in increasing order and places each at the next slot of its
 * distance.  Slots past n are padded with id 0xFFFFFFFF and distance -1. */
static void *knn_worker(void *arg)
{
    orc_job *J = (orc_job *)arg;
    for (uint64_t qi = (uint64_t)J->tid; qi < J->nq; qi += (uint64_t)J->nthreads) {
        const uint64_t *g = J->queries + qi * J->W;
        uint64_t hist[ORC_MAXQ + 2];
        memset(hist, 0, sizeof(hist));
        for (uint64_t i = 0; i < J->n; ++i)
            hist[orc_hamming(J->codes + i * J->W, g, J->W)]++;
        uint64_t k = J->k[qi];
        uint64_t kk = k < J->n ? k : J->n;
        /* start[d] = number of codes closer than d = first sorted slot of d */
        uint64_t start[ORC_MAXQ + 2], acc = 0;
        int dmax = -1;                        /* last distance that reaches a slot < kk */
        for (int d = 0; d <= ORC_MAXQ; ++d) {
            start[d] = acc;
            if (acc < kk) dmax = d;
            acc += hist[d];
        }
        uint32_t *oid = J->out_ids + J->out_off[qi];
        int32_t *odist = J->out_dist + J->out_off[qi];
        for (uint64_t i = 0; i < J->n; ++i) {
            int d = orc_hamming(J->codes + i * J->W, g, J->W);
            if (d > dmax) continue;
            uint64_t p = start[d]++;
            if (p < kk) { oid[p] = (uint32_t)i; odist[p] = d; }
        }
        for (uint64_t p = kk; p < k; ++p) { oid[p] = ORC_PAD_ID; odist[p] = -1; }
    }
    return NULL;
}

int orc_knn(const uint64_t *codes, uint64_t n, int W, const uint64_t *queries,
            uint64_t nq, const uint32_t *k, const uint64_t *out_off,
            uint32_t *out_ids, int32_t *out_dist, int nthreads)
{
    orc_job J;
    memset(&J, 0, sizeof(J));
    J.codes = codes; J.n = n; J.W = W; J.queries = queries; J.nq = nq;
    J.k = k; J.out_off = out_off; J.out_ids = out_ids; J.out_dist = out_dist;
    return run_threads(&J, nthreads, knn_worker);
}

/* Sec. 1.1, r-neighbour problem: every code within r bits of g, listed in
 * (distance, id) order.  Two calls: count, then fill at caller offsets. */
static void *rnear_count_worker(void *arg)
{
    orc_job *J = (orc_job *)arg;
    for (uint64_t qi = (uint64_t)J->tid; qi < J->nq; qi += (uint64_t)J->nthreads) {
        const uint64_t *g = J->queries + qi * J->W;
        uint64_t c = 0;
        for (uint64_t i = 0; i < J->n; ++i)
            if (orc_hamming(J->codes + i * J->W, g, J->W) <= J->r) ++c;
        J->counts[qi] = c;
    }
    return NULL;
}

static void *rnear_fill_worker(void *arg)
{
    orc_job *J = (orc_job *)arg;
    for (uint64_t qi = (uint64_t)J->tid; qi < J->nq; qi += (uint64_t)J->nthreads) {
        const uint64_t *g = J->queries + qi * J->W;
        uint64_t slot[ORC_MAXQ + 2];
        memset(slot, 0, sizeof(slot));
        for (uint64_t i = 0; i < J->n; ++i) {
            int d = orc_hamming(J->codes + i * J->W, g, J->W);
            if (d <= J->r) slot[d + 1]++;
        }
        for (int d = 1; d <= ORC_MAXQ + 1; ++d) slot[d] += slot[d - 1];
        uint32_t *oid = J->out_ids + J->out_off[qi];
        int32_t *odist = J->out_dist + J->out_off[qi];
        for (uint64_t i = 0; i < J->n; ++i) {
            int d = orc_hamming(J->codes + i * J->W, g, J->W);
            if (d <= J->r) { uint64_t p = slot[d]++; oid[p] = (uint32_t)i; odist[p] = d; }
        }
    }
    return NULL;
}

int orc_rnear_count(const uint64_t *codes, uint64_t n, int W, const uint64_t *queries,
                    uint64_t nq, int r, uint64_t *counts, int nthreads)
{
    orc_job J;
    memset(&J, 0, sizeof(J));
    J.codes = codes; J.n = n; J.W = W; J.queries = queries; J.nq = nq; J.r = r;
    J.counts = counts;
    return run_threads(&J, nthreads, rnear_count_worker);
}

int orc_rnear_fill(const uint64_t *codes, uint64_t n, int W, const uint64_t *queries,
                   uint64_t nq, int r, const uint64_t *out_off, uint32_t *out_ids,
                   int32_t *out_dist, int nthreads)
{
    orc_job J;
    memset(&J, 0, sizeof(J));
    J.codes = codes; J.n = n; J.W = W; J.queries = queries; J.nq = nq; J.r = r;
    J.out_off = out_off; J.out_ids = out_ids; J.out_dist = out_dist;
    return run_threads(&J, nthreads, rnear_fill_worker);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: insert every code's j-th substring into the j-th table.  A
 * table is written out as its (key, id) pairs ordered by key and, within a
 * bucket, by id; bucket b is the run of pairs with key b. */
typedef struct { uint64_t key; uint32_t id; } orc_pair;

static int pair_cmp(const void *a, const void *b)
{
    const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

int orc_table_build(const uint64_t *codes, uint64_t n, int W, int off, int len,
                    uint64_t *sorted_keys, uint32_t *ids)
{
    orc_pair *p = (orc_pair *)malloc((n ? n : 1) * sizeof(orc_pair));
    if (!p) return -1;
    for (uint64_t i = 0; i < n; ++i) {
        p[i].key = orc_substring_key(codes + i * W, off, len);
        p[i].id = (uint32_t)i;
    }
    qsort(p, (size_t)n, sizeof(orc_pair), pair_cmp);
    for (uint64_t i = 0; i < n; ++i) { sorted_keys[i] = p[i].key; ids[i] = p[i].id; }
    free(p);
    return 0;
}

/* Algorithm 3: the buckets of an s-bit table that differ from a key in exactly
 * rho bits are key ^ x for every x < 2^s with popcount(x) = rho.  Brute
 * force over all x (s <= 30), in increasing order of x.  Returns the count;
 * writes at most cap values. */
uint64_t orc_ring(int s, int rho, uint64_t *out, uint64_t cap)
{
    uint64_t c = 0;
    for (uint64_t x = 0; x < ((uint64_t)1 << s); ++x)
        if (__builtin_popcountll(x) == rho) {
            if (c < cap) out[c] = x;
            ++c;
        }
    return c;
}

/* ------------------------------------------------------------------------ */
/* Multi-index hashing on the CPU, following Algorithms 2 and 3 step by step.
 * The tables are those of orc_table_build, looked up by binary search. */
typedef struct {
    int q, m, W;
    const uint64_t *codes;
    uint64_t n;
    const int *off, *len;
    const uint64_t *const *keys;   /* m sorted key arrays, n each */
    const uint32_t *const *ids;    /* m id arrays, n each */
} orc_mih;

/* counters: [0] lookups (buckets examined), [1] raw candidates (bucket
 * entries read), [2] unique candidates, [3] last step executed. */
enum { C_LOOKUPS = 0, C_RAW = 1, C_UNIQUE = 2, C_LAST_STEP = 3 };

typedef struct {
    const orc_mih *X;
    const uint64_t *g;
    uint8_t *seen;            /* duplicate bit-string (one byte per code here) */
    uint64_t *hist;           /* |N_d| */
    uint32_t **nd_ids;        /* N_d members */
    uint64_t *nd_cap;
    int64_t *cnt;
    int collect_le;           /* rnear: keep only d <= collect_le */
    int status;
} orc_search;

static void bucket_range(const uint64_t *keys, uint64_t n, uint64_t key,
                         uint64_t *lo_out, uint64_t *hi_out)
{
    uint64_t lo = 0, hi = n;                 /* first index with keys[i] >= key */
    while (lo < hi) { uint64_t mid = lo + (hi - lo) / 2; if (keys[mid] < key) lo = mid + 1; else hi = mid; }
    uint64_t b = lo;
    hi = n;                                   /* first index with keys[i] > key */
    while (lo < hi) { uint64_t mid = lo + (hi - lo) / 2; if (keys[mid] <= key) lo = mid + 1; else hi = mid; }
    *lo_out = b;
    *hi_out = lo;
}

/* One bucket lookup: every id in the bucket is a candidate; a candidate seen
 * before is discarded (Sec. 6 "Duplicate Candidates"), the others are
 * measured on the full code and added to N_d. */
static void visit_bucket(orc_search *S, int j, uint64_t key)
{
    const orc_mih *X = S->X;
    uint64_t lo, hi;
    S->cnt[C_LOOKUPS]++;
    bucket_range(X->keys[j], X->n, key, &lo, &hi);
    for (uint64_t p = lo; p < hi; ++p) {
        uint32_t id = X->ids[j][p];
        S->cnt[C_RAW]++;
        if (S->seen[id]) continue;
        S->seen[id] = 1;
        S->cnt[C_UNIQUE]++;
        int d = orc_hamming(X->codes + (uint64_t)id * X->W, S->g, X->W);
        if (S->collect_le >= 0 && d > S->collect_le) continue;
        if (S->hist[d] == S->nd_cap[d]) {
            uint64_t nc = S->nd_cap[d] ? 2 * S->nd_cap[d] : 16;
            uint32_t *nb = (uint32_t *)realloc(S->nd_ids[d], nc * sizeof(uint32_t));
            if (!nb) { S->status = -1; return; }
            S->nd_ids[d] = nb;
            S->nd_cap[d] = nc;
        }
        S->nd_ids[d][S->hist[d]++] = id;
    }
}

/* All keys at exactly rho bits from `key` within `len` bits: choose the
 * flipped positions recursively, lowest position first. */
static void flip_bits(orc_search *S, int j, uint64_t key, int len, int first, int rho)
{
    if (rho == 0) { visit_bucket(S, j, key); return; }
    for (int b = first; b <= len - rho; ++b)
        flip_bits(S, j, key ^ ((uint64_t)1 << b), len, b + 1, rho - 1);
}

/* One step of Algorithm 3: the ring of radius rho in table j. */
static void search_ring(orc_search *S, int j, int rho)
{
    const orc_mih *X = S->X;
    if (rho > X->len[j]) return;           /* no bucket lies rho > s bits away */
    uint64_t gkey = orc_substring_key(S->g, X->off[j], X->len[j]);
    flip_bits(S, j, gkey, X->len[j], 0, rho);
}

static int search_init(orc_search *S, const orc_mih *X, const uint64_t *g, int64_t *cnt)
{
    memset(S, 0, sizeof(*S));
    S->X = X; S->g = g; S->cnt = cnt;
    S->seen = (uint8_t *)calloc(X->n ? X->n : 1, 1);
    S->hist = (uint64_t *)calloc(ORC_MAXQ + 1, sizeof(uint64_t));
    S->nd_ids = (uint32_t **)calloc(ORC_MAXQ + 1, sizeof(uint32_t *));
    S->nd_cap = (uint64_t *)calloc(ORC_MAXQ + 1, sizeof(uint64_t));
    S->collect_le = -1;
    for (int c = 0; c < 4; ++c) cnt[c] = 0;
    return (S->seen && S->hist && S->nd_ids && S->nd_cap) ? 0 : -1;
}

static void search_free(orc_search *S)
{
    if (S->nd_ids)
        for (int d = 0; d <= ORC_MAXQ; ++d) free(S->nd_ids[d]);
    free(S->nd_ids); free(S->nd_cap); free(S->hist); free(S->seen);
}

static int u32_cmp(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Algorithm 3 for one query.  Step t searches ring r' = floor(t/m) of table
 * a+1 = (t mod m)+1; after step t the loop ends once sum_{d<=t} |N_d| >=
 * min(k, n) (Alg. 3's test after r has been incremented to t+1).  Rings
 * wider than a substring are empty.  The answer is N_0, N_1, ... with each
 * N_d in increasing id order, cut at min(k, n) and padded to k. */
int orc_mih_knn(const orc_mih *X, const uint64_t *g, uint32_t k,
                uint32_t *out_ids, int32_t *out_dist, int64_t *cnt)
{
    orc_search S;
    if (search_init(&S, X, g, cnt)) { search_free(&S); return -1; }
    uint64_t kk = (uint64_t)k < X->n ? (uint64_t)k : X->n;
    int rp = 0, a = 0, r = 0;                 /* Alg. 3: r' = 0, a = 0, r = 0 */
    for (;;) {
        search_ring(&S, a, rp);
        if (S.status) break;
        cnt[C_LAST_STEP] = r;
        a++;
        if (a >= X->m) { a = 0; rp++; }
        r++;
        uint64_t found = 0;
        for (int d = 0; d <= r - 1 && d <= X->q; ++d) found += S.hist[d];
        if (found >= kk) break;
        if (r > X->q) break;                  /* unreachable: all codes lie within q */
    }
    uint64_t p = 0;
    for (int d = 0; d <= X->q && p < kk; ++d) {
        qsort(S.nd_ids[d], (size_t)S.hist[d], sizeof(uint32_t), u32_cmp);
        for (uint64_t e = 0; e < S.hist[d] && p < kk; ++e, ++p) {
            out_ids[p] = S.nd_ids[d][e];
            out_dist[p] = d;
        }
    }
    for (; p < k; ++p) { out_ids[p] = ORC_PAD_ID; out_dist[p] = -1; }
    int st = S.status;
    search_free(&S);
    return st;
}

/* Algorithm 2 for one query: with r = m r' + a, tables 1..a+1 are searched to
 * radius r' and tables a+2..m to radius r'-1 (none when r' = 0); the union of
 * the buckets is culled to the codes within r.  Returns the number of
 * r-neighbours; writes at most cap of them in (distance, id) order. */
int64_t orc_mih_rnear(const orc_mih *X, const uint64_t *g, int r, uint64_t cap,
                      uint32_t *out_ids, int32_t *out_dist, int64_t *cnt)
{
    orc_search S;
    if (search_init(&S, X, g, cnt)) { search_free(&S); return -1; }
    S.collect_le = r;
    int rp = r / X->m, a = r - X->m * rp;
    for (int j = 0; j < X->m; ++j) {
        int radius = j <= a ? rp : rp - 1;
        for (int rho = 0; rho <= radius; ++rho) search_ring(&S, j, rho);
    }
    cnt[C_LAST_STEP] = r;
    uint64_t p = 0;
    for (int d = 0; d <= X->q && d <= r; ++d) {
        qsort(S.nd_ids[d], (size_t)S.hist[d], sizeof(uint32_t), u32_cmp);
        for (uint64_t e = 0; e < S.hist[d]; ++e, ++p)
            if (p < cap) { out_ids[p] = S.nd_ids[d][e]; out_dist[p] = d; }
    }
    int st = S.status;
    search_free(&S);
    return st ? -1 : (int64_t)p;
}

/* Flat entry points for ctypes: the tables are passed as m pointers each. */
int orc_mih_knn_flat(int q, int m, const uint64_t *codes, uint64_t n, int W,
                     const int *off, const int *len, const uint64_t *const *keys,
                     const uint32_t *const *ids, const uint64_t *g, uint32_t k,
                     uint32_t *out_ids, int32_t *out_dist, int64_t *cnt)
{
    orc_mih X = {q, m, W, codes, n, off, len, keys, ids};
    return orc_mih_knn(&X, g, k, out_ids, out_dist, cnt);
}

int64_t orc_mih_rnear_flat(int q, int m, const uint64_t *codes, uint64_t n, int W,
                           const int *off, const int *len, const uint64_t *const *keys,
                           const uint32_t *const *ids, const uint64_t *g, int r,
                           uint64_t cap, uint32_t *out_ids, int32_t *out_dist, int64_t *cnt)
{
    orc_mih X = {q, m, W, codes, n, off, len, keys, ids};
    return orc_mih_rnear(&X, g, r, cap, out_ids, out_dist, cnt);
}

/* ------------------------------------------------------------------------ */
/* Re-ranking by an asymmetric Hamming distance.  Sec. 5.1 notes that Hamming
 * distance cannot order codes at equal distance and that a re-ranking phase
 * with an asymmetric Hamming distance helps in practice; the Conclusion
 * describes the asymmetric form: the query stays real-valued (no quantisation
 * of the query), and multi-index hashing supplies the candidates that the
 * asymmetric distance then culls.  The paper gives no formula.  Reading c17:
 * the query is the q real values y_b whose signs give its code (bit b is set
 * when y_b > 0), and the distance to a database code h is
 *     a(y, h) = sum of |y_b| over the bits b where h_b != [y_b > 0],
 * every disagreeing bit weighted by the query's margin from that bit's
 * threshold.  The sum is exact on a fixed-point grid: with M the largest
 * |y_b| of the query and E its binary exponent (2^E <= M < 2^(E+1)), the
 * weights are w_b = floor(|y_b| 2^s) with s = 53 - E (each below 2^54), their
 * sum over the disagreeing bits is an exact integer (below 2^62, any order),
 * and a = that integer rounded to double, times 2^-s.  Each query's candidate
 * list is ordered by (integer sum, id) and its first k entries are returned;
 * candidate id 0xFFFFFFFF is padding and is skipped, and result slots past
 * the candidates are padded with id 0xFFFFFFFF and a = -1.
 * Returns 0, -1 when out of memory, -2 when a candidate id is >= n. */
typedef struct {
    uint64_t a;
    uint32_t id;
} orc_scored;

static int scored_cmp(const void *x, const void *y)
{
    const orc_scored *u = (const orc_scored *)x, *v = (const orc_scored *)y;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    return (u->id > v->id) - (u->id < v->id);
}

int orc_rerank_asym(const uint64_t *codes, uint64_t n, int q, const float *proj,
                    uint64_t nq, const uint32_t *ids, uint32_t k_in, uint32_t k,
                    uint32_t *out_ids, double *out_a)
{
    const int W = q / 64;
    orc_scored *list = (orc_scored *)malloc(sizeof(orc_scored) * (k_in ? k_in : 1));
    if (!list) return -1;
    for (uint64_t qi = 0; qi < nq; ++qi) {
        const float *y = proj + qi * (uint64_t)q;
        /* the grid: s = 53 - E for the largest magnitude M = m 2^e, m in [0.5, 1) */
        double M = 0.0;
        for (int b = 0; b < q; ++b)
            if (fabs((double)y[b]) > M) M = fabs((double)y[b]);
        int s = 0;
        if (M > 0.0) {
            int e;
            frexp(M, &e);
            s = 53 - (e - 1);
        }
        uint64_t w[ORC_MAXQ];
        for (int b = 0; b < q; ++b)
            w[b] = (uint64_t)floor(ldexp(fabs((double)y[b]), s));
        uint32_t cnt = 0;
        for (uint32_t i = 0; i < k_in; ++i) {
            uint32_t id = ids[qi * k_in + i];
            if (id == ORC_PAD_ID) continue;
            if ((uint64_t)id >= n) { free(list); return -2; }
            const uint64_t *h = codes + (uint64_t)id * W;
            uint64_t a = 0;
            for (int b = 0; b < q; ++b) {
                int query_bit = y[b] > 0.0f;
                if (code_bit(h, b) != query_bit) a += w[b];
            }
            list[cnt].a = a;
            list[cnt].id = id;
            ++cnt;
        }
        qsort(list, cnt, sizeof(orc_scored), scored_cmp);
        for (uint32_t p = 0; p < k; ++p) {
            out_ids[qi * k + p] = p < cnt ? list[p].id : ORC_PAD_ID;
            out_a[qi * k + p] = p < cnt ? ldexp((double)list[p].a, -s) : -1.0;
        }
    }
    free(list);
    return 0;
}
