/*
 * mih.h -- exact k-nearest-neighbour and r-neighbour search in Hamming space
 * by multi-index hashing (MIH) on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: M. Norouzi, A. Punjani, D. J. Fleet, "Fast Exact Search in Hamming
 * Space with Multi-Index Hashing" (arXiv:1307.2982).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Codes.   A database or query code of q bits (q in {64, 128, 256}) is stored
 *          as W = q/64 consecutive uint64 words, row-major: code i occupies
 *          words [i*W, (i+1)*W).  Bit b of a code is bit (b % 64) of word
 *          (b / 64).  Ids are the row numbers 0..n-1 as uint32 (n < 2^32 - 1;
 *          4-byte ids as in Sec. 6 "Memory Requirements").
 * Order.   Results are ordered by (Hamming distance, id) ascending.  The paper
 *          allows any choice among equidistant codes (Sec. 5.2); the id
 *          tie-break makes every answer unique and schedule-independent.
 * Memory.  Unless a parameter says "host", a pointer is a CUDA device pointer
 *          on the current device.  The library never takes ownership of a
 *          caller pointer; outputs are written into caller-allocated buffers.
 *          Scratch memory comes from a stream-ordered pool owned by the
 *          library (cudaMallocAsync on a private pool of the current device).
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *          default stream).  Work is enqueued on it; entry points that must
 *          read sizes back (build, knn, rnear) synchronise that stream before
 *          returning.  Inputs must stay unchanged until the call returns.
 * Errors.  Every entry point returns a status; no exception, abort or device
 *          trap crosses the boundary.  mih_last_error() gives a detail string
 *          for the calling host thread.  After MIH_ECUDA the CUDA context
 *          may be unusable (e.g. a caller pointer that is not device memory).
 */
#ifndef MIH_H_
#define MIH_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MIH_API __attribute__((visibility("default")))
#else
#define MIH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MIH_OK = 0,
    MIH_EINVAL = 1,      /* invalid argument (size, q, m, k, r, null pointer) */
    MIH_ENOMEM = 2,      /* device scratch or index allocation failed */
    MIH_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    MIH_EOVERFLOW = 4,   /* mih_rnear: results exceed `capacity` (sizes returned) */
    MIH_ETIMEOUT = 5,    /* a bounded device wait gave up */
    MIH_EINTERNAL = 6    /* an internal consistency check failed */
} mih_status;

/* Opaque index: m substring hash tables over a borrowed code array. */
typedef struct mih_index mih_index;

/* Table representation per substring (Sec. 6 "Implementation details"). */
enum {
    MIH_TABLE_AUTO = 0,    /* direct for s <= 24 bits, sparse above */
    MIH_TABLE_DIRECT = 1,  /* CSR over all 2^s buckets: offsets[2^s + 1] */
    MIH_TABLE_SPARSE = 2   /* sorted non-empty keys + open-addressing index */
};

typedef struct {
    int32_t table_kind;    /* MIH_TABLE_*; DIRECT requires s <= 28 */
    int32_t scan_factor;   /* A query whose lookups would exceed scan_factor * n
                              switches to one verification pass over all codes
                              (results unchanged; lookups are as costly as
                              candidate tests, Sec. 3).  0 = default (4);
                              negative = never, which reproduces the lookup
                              and candidate counts of Algorithms 2 and 3. */
    int32_t inline_codes;  /* Keep a copy of the codes in each table's bucket order
                              (m * n * q/8 extra bytes) so that a bucket's
                              candidates are one contiguous read.  0 = auto (when
                              ids and inline codes fit in 60% of the free
                              device memory), 1 = always, negative = never. */
    int32_t probe;         /* Before the first step, measure up to `probe` entries
                              of each query's own bucket in every table to get a
                              first bound on its k-th distance (results
                              unchanged).  0 = default (4096), negative = off. */
    int32_t executor;      /* How mih_knn runs its waves of Alg. 3 steps (results
                              unchanged): MIH_EXEC_GRAPH = one CUDA graph whose
                              while-loop node repeats the wave and its stopping
                              test on the device, with no host round trip between
                              waves; MIH_EXEC_HOST = a host loop that reads the
                              number of active queries after every wave.
                              0 = MIH_EXEC_AUTO (the graph). */
    int32_t tail_from;     /* Step from which a k-NN query runs two Alg. 3 steps
                              per wave instead of one (results unchanged: after
                              steps 0..t every code within t bits is found,
                              Prop. 2, so the stopping test after a wave stays
                              exact; a query may do one step more than Alg. 3).
                              Saves waves when few slow queries remain, at the
                              price of the extra steps' work: whether it pays
                              depends on the workload (mih_tune_search times it).
                              0 = default (never), negative = never.  Never with
                              per-query counters requested (they are Alg. 3's). */
    const int32_t *bit_order; /* Sec. 5.5 "Substring Optimization": NULL = the
                              consecutive substrings of Sec. 2.1.  Otherwise a
                              host array of q distinct bit indices, read during
                              mih_build only: bit p of the code the tables see is
                              bit bit_order[p] of the stored code, so substring j
                              takes bits bit_order[o_j .. o_j + s_j - 1] (o_j, s_j
                              of mih_substring_layout).  Results are unchanged
                              (a common permutation of the bits keeps every
                              Hamming distance); the index then holds a permuted
                              copy of the codes (n * q/8 bytes) and permutes each
                              batch of queries.  mih_greedy_substrings computes
                              the paper's greedy order. */
    const int32_t *substring_length; /* Per-table substring lengths (the Conclusion,
                              Sec. 8, leaves them open): NULL = the floor/ceil
                              layout of Sec. 2.1.  Otherwise a host array of m
                              lengths, each 1..32, summing to q, read during
                              mih_build only: table j takes the contiguous bits
                              [o_j, o_j + length[j]) with o_j the sum of the
                              lengths before it.  Results are unchanged (Props. 1
                              and 2 hold for any partition into m disjoint
                              substrings); only the work per step changes.
                              mih_cost_layout proposes lengths. */
    int32_t slice_shape;   /* Shape of the kernel that streams big buckets in the
                              k-NN waves (a launch choice; results unchanged):
                              MIH_SLICE_SHAPE_3K_8W (default) 3 KB stages, 8 warps
                              per CTA, 2 stages in flight per warp (4 CTAs per SM);
                              MIH_SLICE_SHAPE_8K_4W 8 KB stages, 4 warps;
                              MIH_SLICE_SHAPE_4K_8W 4 KB stages, 8 warps (3 CTAs
                              per SM).  mih_tune_search picks one by timing. */
    int32_t reserved[5];   /* must be zero */
} mih_params;

/* mih_params.slice_shape values. */
enum { MIH_SLICE_SHAPE_3K_8W = 0, MIH_SLICE_SHAPE_8K_4W = 1, MIH_SLICE_SHAPE_4K_8W = 2 };

/* mih_params.executor (not part of the paper: a launch strategy). */
enum {
    MIH_EXEC_AUTO = 0,
    MIH_EXEC_HOST = 1,
    MIH_EXEC_GRAPH = 2
};

/* Aggregate work counters of one mih_knn / mih_rnear call (host struct). */
typedef struct {
    uint64_t lookups;            /* buckets examined (Sec. 3, "lookups") */
    uint64_t candidates_raw;     /* bucket entries read */
    uint64_t candidates_unique;  /* candidates left after duplicate removal; counted
                                    only when query_stats is requested (else 0): without
                                    it candidates beyond a query's bound are dropped
                                    before the duplicate test */
    uint64_t steps;              /* Alg. 3 steps executed, summed over queries */
    uint64_t phase2_queries;     /* k-NN queries re-collected in a second pass */
    uint64_t waves;              /* search waves launched */
    uint64_t candidates_sliced;  /* of candidates_raw: entries of big buckets, which the
                                    slice kernel streams (the rest the chunk kernel reads) */
} mih_stats;

typedef struct {
    int32_t q, m, W;
    int32_t substring_offset[256];  /* first code bit of substring j */
    int32_t substring_length[256];  /* s_j */
    int32_t table_kind[256];        /* MIH_TABLE_DIRECT or MIH_TABLE_SPARSE */
    uint64_t n;
    uint64_t distinct_keys[256];    /* non-empty buckets of table j */
    uint64_t max_bucket[256];       /* largest bucket of table j */
    uint64_t index_bytes;           /* device bytes owned by the index */
    int32_t inline_codes;           /* 1 if the tables hold codes in bucket order */
} mih_index_info;

/* ------------------------------------------------------------------------
 * mih_build -- Algorithm 1 (Sec. 2.2): build one hash table per substring.
 *
 * codes   device, uint64[n][q/64], borrowed: the index keeps this pointer
 *         and reads it during every search; the caller keeps the memory
 *         alive and unchanged until mih_free.
 * n       number of codes, 0 <= n < 2^32 - 1.
 * q       code length in bits: 64, 128 or 256.
 * m       number of substrings, 1 <= m <= q, with every substring at most 32
 *         bits (m >= q/32).  Substring j covers contiguous bits; the first
 *         m - (q mod m) substrings have floor(q/m) bits and the rest
 *         ceil(q/m) bits (Sec. 2.1 footnote).
 * params  host, nullable (NULL = defaults).
 * out     host; receives the index on MIH_OK, NULL otherwise.
 * Each table is a stable radix sort of (substring key, id), written as CSR
 * buckets: direct-addressed offsets for short substrings, sorted distinct
 * keys plus an open-addressing key index for long ones.  Synchronises
 * `stream`.
 * Errors: MIH_EINVAL (q, m, n, pointers), MIH_ENOMEM, MIH_ECUDA.
 */
MIH_API mih_status mih_build(const uint64_t *codes, uint64_t n, int q, int m,
                     const mih_params *params, void *stream, mih_index **out);

/* Release an index and the device memory it owns (not the codes).  NULL ok. */
MIH_API void mih_free(mih_index *index);

/* Fill `info` (host) with the index layout and sizes. */
MIH_API mih_status mih_index_get_info(const mih_index *index, mih_index_info *info);

/* ------------------------------------------------------------------------
 * mih_knn -- Algorithm 3 (Sec. 4): exact k-NN of each query by multi-index
 * hashing with a growing search radius.
 *
 * queries      device, uint64[nq][q/64].
 * nq           number of queries, 0 <= nq <= 2^23.
 * k            device uint32[nq] per-query k, or NULL to use k_uniform.
 * k_uniform    k for every query when `k` is NULL.
 * out_offsets  device uint64[nq+1] CSR offsets of each query's results when
 *              `k` is given (out_offsets[i+1] - out_offsets[i] = k[i]); NULL
 *              when k is uniform (query i then writes at i * k_uniform).
 * out_ids      device uint32, per query min(k, n) ids in (distance, id)
 *              order, then 0xFFFFFFFF padding up to k.
 * out_dist     device int32, the matching distances, -1 for padding.
 * query_stats  device uint64[nq][4] or NULL: per query lookups, raw
 *              candidates, unique candidates, last step executed.  In the
 *              paper's stopping rule the last step equals the k-th distance.
 *              Requesting it makes every candidate pass the duplicate test
 *              (slower); results are the same either way.
 * stats        host, nullable: aggregate counters of this call.
 * Every k must satisfy 1 <= k <= MIH_MAX_K.  Synchronises `stream`.
 * Step t searches ring floor(t/m) of table (t mod m); a query stops after
 * the first step t at which at least min(k, n) codes within t bits were
 * found (Alg. 3; all codes within t bits are found by then, Prop. 2).
 * Errors: MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA, MIH_EINTERNAL.
 */
#define MIH_MAX_K 8192u

MIH_API mih_status mih_knn(const mih_index *index, const uint64_t *queries, uint32_t nq,
                   const uint32_t *k, uint32_t k_uniform, const uint64_t *out_offsets,
                   uint32_t *out_ids, int32_t *out_dist, uint64_t *query_stats,
                   mih_stats *stats, void *stream);

/* CSR offsets for per-query k (the out_offsets of mih_knn / linscan_knn),
 * computed on the device: out_offsets[i] = k[0] + ... + k[i-1] for
 * i = 0..nq, so out_offsets[nq] is the total.  k: device uint32[nq];
 * out_offsets: device uint64[nq + 1].  Stream-ordered (does not synchronise).
 * Errors: MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA. */
MIH_API mih_status mih_k_offsets(const uint32_t *k, uint32_t nq, uint64_t *out_offsets, void *stream);

/* ------------------------------------------------------------------------
 * mih_rnear -- Algorithm 2 (Sec. 2.2): all codes within r bits of each query.
 *
 * With r = m r' + a, tables 1..a+1 are searched to radius r' and the others
 * to r' - 1; the union is culled by the full-code distance.
 * r            0 <= r; r >= q returns the whole database.
 * capacity     number of (id, dist) slots in out_ids / out_dist.
 * out_offsets  device uint64[nq+1]: CSR offsets of the results, always
 *              written (also on MIH_EOVERFLOW, so the caller can allocate
 *              out_offsets[nq] slots and call again).
 * out_ids, out_dist  device, `capacity` slots, may be NULL when capacity is 0.
 * total        host, nullable: total number of results.
 * query_stats, stats  as in mih_knn (last step = r).
 * Synchronises `stream`.
 * Errors: MIH_EOVERFLOW when the total exceeds capacity (nothing written to
 * out_ids / out_dist), MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA.
 */
MIH_API mih_status mih_rnear(const mih_index *index, const uint64_t *queries, uint32_t nq, int r,
                     uint64_t capacity, uint64_t *out_offsets, uint32_t *out_ids,
                     int32_t *out_dist, uint64_t *total, uint64_t *query_stats,
                     mih_stats *stats, void *stream);

/* ------------------------------------------------------------------------
 * linscan_knn -- the linear-scan baseline (Sec. 5.2): exact k-NN of each
 * query by computing the Hamming distance to every code (one xor per 64 bits
 * and a population count, Sec. 6 "Hamming Distance").
 *
 * Arguments as in mih_build (codes, n, q) and mih_knn (queries ... out_dist);
 * the codes are only read during the call.  Synchronises `stream`.
 * Errors: MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA.
 */
MIH_API mih_status linscan_knn(const uint64_t *codes, uint64_t n, int q, const uint64_t *queries,
                       uint32_t nq, const uint32_t *k, uint32_t k_uniform,
                       const uint64_t *out_offsets, uint32_t *out_ids, int32_t *out_dist,
                       void *stream);

/* ------------------------------------------------------------------------
 * mih_merge_topk -- exact k-NN over a database split into id ranges (one
 * index per range, e.g. one per GPU): merges the ranges' answers.  By the
 * k-NN definition (Sec. 1.1) the k nearest codes of the whole database are
 * the k smallest (distance, global id) pairs among the ranges' own k nearest,
 * since the ranges partition the database and (distance, id) is a total order.
 *
 * ids, dist   device, [parts][nq][k_in]: part p's answers for every query,
 *             each row in (distance, id) order with ids relative to the part
 *             (as mih_knn / linscan_knn give them for a uniform k_in, padding
 *             id 0xFFFFFFFF / distance -1 last).
 * id_base     host, parts entries, non-decreasing: the global id of each
 *             part's id 0 (global ids must stay below 2^32 - 1).
 * k           results per query, 1 <= k <= MIH_MAX_K; out_ids / out_dist:
 *             device [nq][k], (distance, global id) order, padded as mih_knn.
 * 1 <= parts <= 64, 1 <= k_in <= MIH_MAX_K.  Synchronises `stream`.
 * Errors: MIH_EINVAL, MIH_ECUDA.
 */
MIH_API mih_status mih_merge_topk(const uint32_t *ids, const int32_t *dist, uint32_t parts, uint32_t nq,
                                  uint32_t k_in, const uint32_t *id_base, uint32_t k, uint32_t *out_ids,
                                  int32_t *out_dist, void *stream);

/* ------------------------------------------------------------------------
 * mih_rerank_asym -- the re-ranking phase of Sec. 5.1 with an asymmetric
 * Hamming distance (the Conclusion: the query stays real-valued; multi-index
 * hashing finds the candidates, the asymmetric distance culls them).  For
 * query row i with real projections y = proj[i] (its code is their signs:
 * bit b set where y_b > 0) and database code h,
 *     a(y, h) = sum of |y_b| over the bits b where h_b != [y_b > 0],
 * summed exactly on a fixed-point grid: with 2^E <= max_b |y_b| < 2^(E+1),
 * w_b = floor(|y_b| 2^(53-E)), the integer sum of the w_b over the
 * disagreeing bits (below 2^62) is exact, and a = that sum rounded to double
 * times 2^-(53-E).  Row i's candidates are ordered by (integer sum, id) and
 * the first k kept.
 * Leaves the exact-Hamming contract of mih_knn: with every |y_b| equal it
 * orders by Hamming distance, otherwise by the weighted form.
 *
 * codes      device, uint64[n][q/64] (as mih_build), read by candidate id;
 *            16-byte aligned for q >= 128.
 * n          number of codes, n < 2^32 - 1.  q: 64, 128 or 256.
 * proj       device, float32[nq][q], row-major; finite values.
 * ids        device, uint32[nq][k_in]: each row's candidates (e.g. mih_knn's
 *            out_ids for k_uniform = k_in); 0xFFFFFFFF is padding and is
 *            skipped; a row may hold any ids below n (duplicates are scored
 *            as given).
 * k_in, k    1 <= k_in, k <= MIH_MAX_K.
 * out_ids    device, uint32[nq][k]: the ids in (a, id) order, then
 *            0xFFFFFFFF padding when a row has fewer than k candidates.
 * out_a      device, double[nq][k]: the matching a, -1 for padding.
 * Synchronises `stream`.
 * Errors: MIH_EINVAL (sizes, pointers, a candidate id >= n that is not
 * padding: out_ids / out_a are then unspecified), MIH_ENOMEM, MIH_ECUDA.
 */
MIH_API mih_status mih_rerank_asym(const uint64_t *codes, uint64_t n, int q, const float *proj, uint32_t nq,
                                   const uint32_t *ids, uint32_t k_in, uint32_t k, uint32_t *out_ids,
                                   double *out_a, void *stream);

/* mih_rerank_asym for rows of different lengths (e.g. mih_knn's answers
 * for a per-query k, with their CSR offsets): row i's candidates are
 * ids[in_offsets[i] .. in_offsets[i+1]) and its results go to
 * out_ids / out_a [out_offsets[i] .. out_offsets[i+1]), the first
 * out_offsets[i+1] - out_offsets[i] entries of the row in (a, id) order,
 * padded as in mih_rerank_asym.  in_offsets, out_offsets: device
 * uint64[nq + 1], non-decreasing.  k_in_max: the longest candidate row,
 * 1 <= k_in_max <= MIH_MAX_K (it sizes the sort); every result row at most
 * MIH_MAX_K.  Other arguments, the distance and the synchronisation as in
 * mih_rerank_asym.
 * Errors: MIH_EINVAL (as mih_rerank_asym, and a row longer than k_in_max or
 * MIH_MAX_K, or decreasing offsets: the outputs are then unspecified),
 * MIH_ENOMEM, MIH_ECUDA.
 */
MIH_API mih_status mih_rerank_asym_csr(const uint64_t *codes, uint64_t n, int q, const float *proj, uint32_t nq,
                                       const uint32_t *ids, const uint64_t *in_offsets, uint32_t k_in_max,
                                       const uint64_t *out_offsets, uint32_t *out_ids, double *out_a,
                                       void *stream);

/* ------------------------------------------------------------------------
 * mih_set_scan_kernel -- which kernel linscan_knn uses for calls from the
 * calling host thread (results are identical):
 *   MIH_SCAN_POPC    xor and population count per 32-bit word (Sec. 6
 *                    "Hamming Distance"), with an OR lower bound that settles
 *                    most pairs in one popcount;
 *   MIH_SCAN_TENSOR  fp8 tensor-core products: bits as +-1 e4m3 values, so the
 *                    dot product of two codes is q - 2 d (exact in f32);
 *   MIH_SCAN_AUTO    the popcount form (measured faster on GB300 at 1e9 x
 *                    128-bit codes and 10^4 queries).
 * Errors: MIH_EINVAL for an unknown kind. */
enum { MIH_SCAN_AUTO = 0, MIH_SCAN_POPC = 1, MIH_SCAN_TENSOR = 2 };
MIH_API mih_status mih_set_scan_kernel(int kind);

/* ------------------------------------------------------------------------
 * mih_autotune -- choose the number of substrings m by timing the search on
 * a hold-out set of queries (Sec. 6 "Number of Substrings": estimate the
 * run time for m near q / log2(n) and keep the fastest; Table 4).
 *
 * codes, n, q   as in mih_build (device, borrowed only during the call).
 * queries, nq   device, hold-out queries (1 <= nq <= 2^23).
 * k             1 <= k <= MIH_MAX_K.
 * candidates    host int[n_candidates] values of m to try, or NULL to try
 *               mih_suggest_m(q, n) and its neighbours (invalid values are
 *               skipped: m < 1, m > q or substrings above 32 bits).
 * params        host, nullable: build parameters used for every candidate.
 * best_m        host out: the fastest m.
 * ms_per_query  host out, nullable: double[n_candidates] (3 when
 *               candidates is NULL): mean search time per query of each
 *               candidate, -1 for skipped ones.
 * Each candidate builds an index, runs one untimed and one timed mih_knn
 * over the hold-out queries, and frees the index, so at most one index
 * exists at a time.  Synchronises `stream`.
 * Errors: MIH_EINVAL (no valid candidate, sizes), then as mih_build and
 * mih_knn.
 */
MIH_API mih_status mih_autotune(const uint64_t *codes, uint64_t n, int q, const uint64_t *queries,
                                uint32_t nq, uint32_t k, const int *candidates, int n_candidates,
                                const mih_params *params, void *stream, int *best_m,
                                double *ms_per_query);

/* ------------------------------------------------------------------------
 * mih_tune_search -- the launch choices of an index's k-NN waves, picked by
 * timing on hold-out queries (the selection by validation of Sec. 6, applied
 * to the launch shapes; results do not depend on them): every combination of
 * the slice kernel's shape (mih_params.slice_shape) and the step from which
 * queries run two steps per wave (mih_params.tail_from: 2m, m, never) runs
 * one untimed and one timed mih_knn of the hold-out queries with k; the
 * fastest is kept in the index.  Do not search the index from other threads
 * during the call.
 * queries, nq   device, hold-out queries (1 <= nq <= 2^23); k in 1..MIH_MAX_K.
 * best          host out, nullable: {slice_shape, tail_from} chosen.
 * ms_per_query  host out, nullable, double[3 * 3]: entry [shape * 3 + tail],
 *               tail 0 = from step 2m, 1 = from step m, 2 = never.
 * Synchronises `stream`.  Errors: as mih_knn.
 */
typedef struct {
    int32_t slice_shape;
    int32_t tail_from;
} mih_search_tuning;

MIH_API mih_status mih_tune_search(mih_index *index, const uint64_t *queries, uint32_t nq, uint32_t k,
                                   void *stream, mih_search_tuning *best, double *ms_per_query);

/* ------------------------------------------------------------------------
 * linscan_knn_noalloc -- linscan_knn for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a service of the library.
 *
 * Some callers must not call cudaMalloc or cudaFree while they search: a
 * process whose memory allocator has already reserved (nearly) all device
 * memory, so a fresh allocation fails; a latency-bound serving thread, where
 * cudaFree (and often cudaMalloc) synchronises the whole device and stalls
 * the work of other streams; code held to a fixed device-memory budget.
 * This entry point allocates nothing.  Its scratch is one array of about
 * 16.3 MiB compiled into the library (a static __device__ array), which every
 * GPU that loads the library holds until the process exits.  The caller
 * still passes the inputs and the outputs.
 *
 * Results equal linscan_knn's with a uniform k (out_ids / out_dist hold
 * nq * k entries).  Limits: nq <= 256 and 1 <= k <= 256, else MIH_EINVAL;
 * when ties at the k-th distance need more than 2^20 second-pass slots in
 * one call it returns MIH_ENOMEM (use linscan_knn then).
 * Set-up: the first call on each device looks up the array's device address
 * with cudaGetSymbolAddress (that device current); make this first call on a
 * device before capturing any stream.  The address is kept for the life of
 * the process: after cudaDeviceReset on a device, do not call this entry
 * point on that device again in the same process.
 * Cost: each query has 4096 first-pass slots (16 times the largest k, 256);
 * queries whose candidates within the running bound exceed them (many ties
 * at the k-th distance) are collected by a second scan of the database, so
 * such calls read the codes twice.
 * Concurrency: all calls on a device share the one array, and each call clears
 * what must start at zero when it begins; calls that overlap on the GPU (from
 * other streams or host threads) race and corrupt each other's results.
 * Synchronises `stream`.
 * Errors: MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA, MIH_EINTERNAL.
 */
MIH_API mih_status linscan_knn_noalloc(const uint64_t *codes, uint64_t n, int q,
                                       const uint64_t *queries, uint32_t nq, uint32_t k,
                                       uint32_t *out_ids, int32_t *out_dist, void *stream);

/* ------------------------------------------------------------------------
 * Host-only helpers (no GPU needed).
 */

/* Substring layout of Sec. 2.1 (footnote): writes m offsets and lengths
 * (host arrays).  Errors: MIH_EINVAL when q < 1, m < 1 or m > q. */
MIH_API mih_status mih_substring_layout(int q, int m, int32_t *offset, int32_t *length);

/* Cost model of Eq. 7 (Sec. 3.1) in units of one lookup, for q-bit uniform
 * codes, n codes, substring length s and search radius r:
 * (1 + n / 2^s) (q / s) sum_{z <= floor(s r / q)} C(s, z). */
MIH_API double mih_cost_model(int q, uint64_t n, int s, int r);

/* Per-table substring lengths for m tables that minimise the cost model of
 * Eq. 7 (Sec. 3.1) applied table by table to Algorithm 3.  A query that stops
 * after step t has searched rings 0..floor((t - j) / m) of table j (none when
 * t < j), and a ring rho of a table of s bits costs C(s, rho) lookups plus
 * n / 2^s candidates per lookup (uniform codes; Sec. 3 counts a candidate
 * check as about one lookup).  With weight w[t] on stop step t
 * (t = 0 .. n_steps - 1, e.g. a histogram of measured stop steps) the cost is
 *   sum_t w[t] sum_j (1 + n / 2^s_j) sum_{rho <= floor((t - j)/m)} C(s_j, rho),
 * minimised exactly (dynamic programming over the tables) over lengths
 * s_j in 1..32 with sum q; among layouts of equal cost the one closest to
 * q/m per table is taken.  Writes `length` (host, m entries) and returns the
 * cost, or -1 for invalid arguments (q < 1, m < 1, m > q, q > 32 m,
 * n_steps < 1, negative weights, NULL pointers). */
MIH_API double mih_cost_layout(int q, uint64_t n, int m, const double *step_weight, int n_steps,
                               int32_t *length);

/* ------------------------------------------------------------------------
 * mih_autotune_layout -- per-table substring lengths for a given m, chosen
 * by timing on hold-out queries (the selection by validation of Sec. 6,
 * applied to the lengths the Conclusion leaves open).  Runs the hold-out
 * queries once on the Sec. 2.1 layout with per-query counters to measure
 * their stop steps, proposes mih_cost_layout's lengths for that histogram,
 * then times one mih_knn of each layout (after an untimed one) and writes
 * the faster layout's lengths.
 * codes, n, q, queries, nq, k, params  as in mih_autotune (params must not
 *               set substring_length).
 * m            number of tables (substrings of at most 32 bits).
 * best_length  host out, m entries.
 * ms_per_query host out, nullable, double[2]: the Sec. 2.1 layout, the
 *              cost-model layout (the same figure when both are equal).
 * Synchronises `stream`.  Errors as mih_autotune.
 */
MIH_API mih_status mih_autotune_layout(const uint64_t *codes, uint64_t n, int q, const uint64_t *queries,
                                       uint32_t nq, uint32_t k, int m, const mih_params *params, void *stream,
                                       int32_t *best_length, double *ms_per_query);

/* Number of substrings suggested by Sec. 3.1 / Table 4: the integer closest
 * to q / log2(n), clamped so that no substring exceeds 32 bits and m <= q. */
MIH_API int mih_suggest_m(int q, uint64_t n);

/* Greedy assignment of bits to substrings from their correlation (Sec. 5.5
 * "Substring Optimization").  corr: host double[q][q], row-major, the
 * correlation between bits a and b (mih_bit_correlation; only |corr| is
 * used).  The first substring takes bit (seed mod q); substring j = 1..m-1
 * then takes the unused bit most correlated with the bit substring j-1 took.
 * Then, visiting the substrings in turn and skipping full ones, substring j
 * takes the unused bit whose largest correlation with the bits it already
 * holds is smallest.  Ties go to the lower bit index.  Substring sizes are
 * those of mih_substring_layout.  Writes bit_order[q] (host) in the format
 * of mih_params.bit_order: the bits of substring j in the order taken.
 * Errors: MIH_EINVAL for q not in {64, 128, 256}, m < 1, m > q, NULL
 * pointers. */
MIH_API mih_status mih_greedy_substrings(const double *corr, int q, int m, uint64_t seed, int32_t *bit_order);

/* ------------------------------------------------------------------------
 * mih_bit_correlation -- the correlation between every pair of the q bits
 * over n sample codes (Sec. 5.5 uses 10M codes), computed on the GPU from
 * bit-plane AND-popcounts: corr[a][b] = (n c_ab - c_a c_b) /
 * sqrt(c_a (n - c_a) c_b (n - c_b)), where c_a counts the codes with bit a
 * set and c_ab those with both; 0 where a bit is constant.  The diagonal
 * is 1 (0 for a constant bit).
 *
 * codes   device, uint64[n][q/64], 16-byte aligned for q >= 128; 1 <= n <= 2^32 - 1.
 * corr    host, double[q][q], written before return (the call synchronises
 *         its stream).
 * Errors: MIH_EINVAL (q, n, pointers), MIH_ENOMEM, MIH_ECUDA. */
MIH_API mih_status mih_bit_correlation(const uint64_t *codes, uint64_t n, int q, double *corr, void *stream);

/* ------------------------------------------------------------------------
 * Per-call profile of the calling host thread (not part of the paper).
 * With timing enabled, mih_knn, mih_rnear, linscan_knn and mih_rerank_asym
 * record CUDA events on their stream around their main kernels (the fused
 * search kernels, the linear-scan kernel, the re-ranking kernel) and around
 * the whole call.  With per-kernel timing
 * (level 2) they also record an event pair around every launch of the kinds
 * below, and mih_knn runs its waves from a host loop (MIH_EXEC_HOST: the
 * same kernels and results, but each launch can be bracketed by events).
 */
enum {
    MIH_PROF_CHUNK = 0,     /* search_kernel: ring chunks (lookups, small buckets) */
    MIH_PROF_SLICE = 1,     /* search_stream_kernel / search_big_kernel: big-bucket slices */
    MIH_PROF_PROBE = 2,     /* bound_probe_kernel */
    MIH_PROF_PLAN = 3,      /* per-wave chunk planning (counts and their scan) */
    MIH_PROF_STOP = 4,      /* knn_stop_kernel: the stopping test of Alg. 3 */
    MIH_PROF_SELECT = 5,    /* select_kernel (with the ids of table positions) */
    MIH_PROF_SCAN = 6,      /* linscan_kernel */
    MIH_PROF_RERANK = 7,    /* rerank_asym_kernel */
    MIH_PROF_KINDS = 8
};

typedef struct {
    uint64_t launches;       /* kernel launches issued by the last call */
    uint64_t main_launches;  /* launches of the main kernels */
    double main_ms;          /* summed device time of the main kernels (timing on) */
    double call_ms;          /* device time from first to last launch (timing on) */
    double kernel_ms[MIH_PROF_KINDS];         /* per kind, summed (timing level 2) */
    uint64_t kernel_launches[MIH_PROF_KINDS]; /* per kind, launches timed (level 2) */
} mih_profile;

/* Timing for calls from this host thread: 0 off, 1 main kernels and the
 * call, 2 also every kernel kind above (and host-loop waves in mih_knn). */
MIH_API void mih_set_timing(int level);

/* Profile of this thread's last mih_knn / mih_rnear / linscan_knn /
 * mih_rerank_asym call. */
MIH_API mih_status mih_last_profile(mih_profile *out);

/* ------------------------------------------------------------------------
 * mih_measure_ceilings -- throughput ceilings of the current GPU that the
 * kernels' rooflines are quoted against (not part of the paper).  Each figure
 * is one timed launch (after an untimed one) that keeps independent chains of
 * the operation in flight on every SM:
 *   popc_per_s              32-bit population counts per second (the linear
 *                           scan computes the distance of Sec. 6 with them);
 *   b1_mma_pairs128_per_s   (row, column) pairs of 128-bit operands per second
 *                           of mma.sync m16n8k128 b1 AND-popcount, from which
 *                           popc(a xor b) = popc a + popc b - 2 popc(a and b);
 *   fp8_mma_tflops          mma.sync m16n8k32 e4m3 -> f32, and the pairs of
 *                           128 +-1 elements per second it gives (Hamming
 *                           distance = (q - <a, b>) / 2, exact in f32);
 *   gather32_gbs            bytes per second of reads of random 32-byte
 *                           sectors of a buffer of gather_bytes (at least
 *                           64 MiB; use one far larger than L2).
 * Synchronises `stream`.  Errors: MIH_EINVAL, MIH_ENOMEM, MIH_ECUDA. */
typedef struct {
    double popc_per_s;
    double b1_mma_pairs128_per_s;
    double fp8_mma_tflops;
    double fp8_mma_pairs128_per_s;
    double gather32_gbs;
    int32_t sms;
    double sm_clock_mhz;   /* the device's maximum SM clock */
} mih_ceilings;

MIH_API mih_status mih_measure_ceilings(mih_ceilings *out, uint64_t gather_bytes, void *stream);

/* ------------------------------------------------------------------------
 * mih_set_wait_limit -- bounded device waits (not part of the paper).
 * The slice kernel of mih_knn / mih_rnear waits on its bulk copies into
 * shared memory; a wait that runs past `limit_us` microseconds (0 = the
 * default of one second) gives up, the kernel drains the copies it still has
 * in flight (each with the one-second limit) and the call returns
 * MIH_ETIMEOUT.  expire_first_wait = 1 is for testing that path: the first
 * wait of each warp of the slice kernel is made on a barrier that no copy
 * completes, so every call that streams a big bucket returns MIH_ETIMEOUT
 * after about `limit_us`; 0 restores normal waits.  Applies to calls from the
 * calling host thread.  Errors: MIH_EINVAL when limit_us exceeds 60 s.
 */
MIH_API mih_status mih_set_wait_limit(uint32_t limit_us, int expire_first_wait);

/* Static text of a status code. */
MIH_API const char *mih_status_str(mih_status s);

/* Detail of the last error raised on the calling host thread ("" if none). */
MIH_API const char *mih_last_error(void);

/* Library version string. */
MIH_API const char *mih_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MIH_H_ */
