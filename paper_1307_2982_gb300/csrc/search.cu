// search.cu -- multi-index hashing search on the GPU: Algorithm 3 (k-NN,
// mih_knn) and Algorithm 2 (r-neighbours, mih_rnear), plus the k-selection
// shared with the linear scan.
//
// Work model.  Step t of a query searches ring rho = floor(t/m) of table
// j = t mod m: the C(s_j, rho) buckets whose key differs from the query's
// j-th substring in exactly rho bits.  All codes within t bits of the query
// have been found once steps 0..t are done (Prop. 2), so Alg. 2 at radius r
// is steps 0..r and Alg. 3 stops after the first step t with at least
// min(k, n) codes within t bits.  A query's pending steps are cut into chunks
// of 256 ring keys; one warp takes one chunk: each lane unranks its first key
// (combinatorial number system) and walks 8 keys by Gosper steps, looks the
// buckets up, and the warp then shares out the union of the 32 buckets'
// entries, verifies each candidate on the full code and bins it by
// distance.  Buckets above 64 entries are cut into slices of at most 1024
// that a second kernel spreads over all warps (streamed through shared memory
// when the tables keep their codes inline).  Before the first step a probe
// of each query's own buckets gives a first bound on its k-th distance.
//
// Duplicates (Sec. 6 "Duplicate Candidates") are removed without an n-bit
// set: a code reached at step t = m rho + j is kept only if t is the first
// step that reaches it, i.e. no table j' < j has substring distance <= rho
// and no table j' > j has substring distance < rho.  The substring distances
// come from the full code that verification loads anyway.  The rule depends
// only on (query, code), so results do not depend on batching or order.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "index.h"
#include "launch.h"
#include "search.h"
#include "substrings.h"

namespace mih {
namespace {

constexpr int kSearchThreads = 256;
constexpr uint32_t kSliceEntries = 1024;   // big-bucket slice of whole codes
#ifndef MIH_STAGE_BYTES
#define MIH_STAGE_BYTES 3072
#endif
constexpr uint32_t kDefaultStageBytes = MIH_STAGE_BYTES;   // one shared-memory stage of the slice kernel

// Entries per stage of the slice kernel: whole codes (W uint64 words), or
// records of 2W - 1 uint32 words (inline records, every substring one 32-bit
// word).  A stage of records is read in groups of four records (16 (2W - 1)
// bytes, 16-byte aligned) that start at a multiple of four, and its copy
// starts up to three records early: it holds the whole groups that fit in
// SB stage bytes, less those three records.
template <int W, bool REDUCED, uint32_t SB = kDefaultStageBytes>
__host__ __device__ constexpr uint32_t stage_entries() {
    return REDUCED ? 4u * (SB / (16u * (2 * W - 1))) - 3u : SB / (8 * W);
}

// Entries per big-bucket slice: 1024 whole codes, or MIH_SLICE_STAGES (6)
// full stages of records, so that no slice ends in a nearly empty stage.
// (3, 4, 6 and 8 stages of 3 KB: 6.21, 6.11, 6.08 and 6.14 ms per 1e9 x
// 128-bit batch: longer slices mean fewer descriptors for the chunk kernel
// to write, shorter ones a better balanced end of each wave.)
#ifndef MIH_SLICE_STAGES
#define MIH_SLICE_STAGES 6
#endif
template <int W, bool ALIGNED, uint32_t SB = kDefaultStageBytes>
__host__ __device__ constexpr uint32_t slice_entries() {
    return ALIGNED ? static_cast<uint32_t>(MIH_SLICE_STAGES) * stage_entries<W, true, SB>() : kSliceEntries;
}
constexpr uint32_t kScanChunk = 4096;      // codes per chunk of a full verification pass
constexpr int kQueryShift = 41;            // composite entry: q << 41 | d << 32 | id
constexpr uint64_t kEntryMask = (1ull << kQueryShift) - 1ull;

struct BigSlice {
    uint32_t q;
    int32_t t;
    uint32_t begin;
    uint32_t end;
};

enum Mode { kModeKnn = 0, kModeCollect = 1, kModeCount = 2 };

struct SearchArgs {
    const TableDesc* tables;
    int m, q;
    const uint64_t* codes;
    const uint64_t* queries;
    uint32_t nq;
    const int32_t* t_lo;               // per query first step of this launch
    const int32_t* t_hi;               // per query last step (inclusive); < t_lo = idle
    const uint64_t* chunk_off;         // [nq + 1]
    unsigned long long* chunk_next;    // work counter
    uint32_t* hist;                    // knn: [nq][q+1]
    const int32_t* bound;              // knn: store if d <= bound; collect/count: keep if d <= bound
    uint64_t* buf;                     // knn: [nq][cap]; collect: entries
    uint32_t cap;                      // knn: slots per query
    uint32_t* cnt;                     // knn: stored count; collect: cursor; count: count
    const uint64_t* out_base;          // collect: first slot of each query, [nq + 1]
    int* err;                          // collect: set if a query writes past its range
    unsigned long long* qstats;        // [nq][4]: lookups, raw, unique, last step
    BigSlice* big;
    uint32_t big_cap;
    unsigned int* big_count;
    unsigned int* big_next;
    const uint8_t* exh;                // per query: verify every code this launch
    const int32_t* hist_done;          // knn: last step already in the histogram (-1: none)
    uint64_t n;
    int inline_codes;                  // tables keep codes in bucket order
    int* timeout;                      // set when a bounded wait gives up
    int exact_stats;                   // count every unique candidate (per-query counters requested)
    uint64_t wait_ns;                  // limit of a bounded wait on stage data
    int wait_test;                     // timeout test: each warp's first wait runs out
    unsigned long long* sliced;        // raw candidates queued as big-bucket slices (nullable)
    uint32_t slice_entries;            // entries per big-bucket slice (set for the slice kernel's shape)
    int variant;                       // slice kernel shape (k-NN waves; see kStreamVariants)
};

// Chunks of step t for a query: ceil(C(s_j, rho) / 256), 0 if rho > s_j.
__device__ __forceinline__ uint64_t step_chunks(const int* s_len, int m, int t) {
    const int j = t % m, rho = t / m;
    const uint64_t keys = binom(s_len[j], rho);
    return (keys + kChunkKeys - 1) / kChunkKeys;
}

template <int W>
__device__ __forceinline__ Code<W> load_query(const uint64_t* __restrict__ queries, uint32_t q) {
    Code<W> g;
#pragma unroll
    for (int w = 0; w < W; ++w) g.w[w] = __ldg(queries + static_cast<uint64_t>(q) * W + w);
    return g;
}

// Substring layout as the kernels see it: for table j, s_mask[j * 2W + i] is
// the part of 32-bit word i of a code that belongs to substring j, so the
// substring distance is sum_i popc(x_i & mask) for x = code xor query.  When
// every substring is one whole 32-bit word (m = 2W, the ALIGNED layout) the
// substring distances are the per-word popcounts that the full distance sums
// anyway.
struct Layout {
    const int* len;         // s_j
    const uint32_t* mask;   // [m][2W]
};

__device__ __forceinline__ void build_layout(const TableDesc* tables, int m, int W, int* s_len, uint32_t* s_mask) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const int off = tables[j].off, len = tables[j].len;
        s_len[j] = len;
        for (int i = 0; i < 2 * W; ++i) {
            const int lo = max(off, 32 * i), hi = min(off + len, 32 * i + 32);
            uint32_t mk = 0;
            if (hi > lo) {
                const int nb = hi - lo, sh = lo - 32 * i;
                mk = (nb >= 32 ? 0xFFFFFFFFu : ((1u << nb) - 1u)) << sh;
            }
            s_mask[j * 2 * W + i] = mk;
        }
    }
}

// Distance of one candidate and its duplicate test.
//
// A candidate farther than `far` is dropped right after its distance: with a
// bound U on the k-th distance (far = U) such a code is never stored, and
// every later stop test only counts distances below the step index, which
// stays below U while the query runs.  far is "no limit" while the query has
// no bound yet and when exact per-query counters were requested.
//
// Ring mode (j >= 0): the code was reached at step t = m rho + j and is kept
// only if t is its first step (no table j' < j within rho bits, none j' > j
// within rho - 1).  Full-pass mode (j < 0): every code is visited once and
// kept if its first step, min_j' (m d_j' + j'), is after t_done.  Either way
// a kept code enters the histogram and the counters only if its first step is
// after hist_done (steps up to hist_done were counted before and are revisited
// only to store their codes under a bound found later).
template <int W, bool ALIGNED>
__device__ __forceinline__ void eval_candidate(int m, const Layout& L, int j, int rho, int t_done, int hist_done,
                                               int far, const Code<W>& g, const Code<W>& c, int& d, bool& keep,
                                               bool& count) {
    constexpr int NW = 2 * W;
    uint32_t x[NW];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint64_t v = c.w[w] ^ g.w[w];
        x[2 * w] = static_cast<uint32_t>(v);
        x[2 * w + 1] = static_cast<uint32_t>(v >> 32);
    }
    int pc[NW];
    d = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        pc[i] = __popc(x[i]);
        d += pc[i];
    }
    if (d > far) {
        // beyond the query's bound: never stored and never inside a stop test
        keep = count = false;
        return;
    }
    if constexpr (ALIGNED) {
        if (j >= 0) {
            keep = true;
#pragma unroll
            for (int jj = 0; jj < NW; ++jj)
                if (jj != j && (jj < j ? (pc[jj] <= rho) : (pc[jj] < rho))) keep = false;
            count = NW * rho + j > hist_done;
        } else {
            int first = 0x7FFFFFFF;
#pragma unroll
            for (int jj = 0; jj < NW; ++jj) first = min(first, NW * pc[jj] + jj);
            keep = first > t_done;
            count = first > hist_done;
        }
    } else {
        if (j >= 0) {
            keep = true;
            for (int jj = 0; jj < m; ++jj) {
                if (jj == j) continue;
                int dj = 0;
#pragma unroll
                for (int i = 0; i < NW; ++i) dj += __popc(x[i] & L.mask[jj * NW + i]);
                if (jj < j ? (dj <= rho) : (dj < rho)) {
                    keep = false;
                    break;
                }
            }
            count = m * rho + j > hist_done;
        } else {
            int first = 0x7FFFFFFF;
            for (int jj = 0; jj < m; ++jj) {
                int dj = 0;
#pragma unroll
                for (int i = 0; i < NW; ++i) dj += __popc(x[i] & L.mask[jj * NW + i]);
                first = min(first, m * dj + jj);
            }
            keep = first > t_done;
            count = first > hist_done;
        }
    }
}

// Where a batch of candidates lives.  Candidate positions index either a
// table's entries (its ids, and its codes in bucket order when the index keeps
// them inline) or, for a full pass, the code array itself (id = position).
struct CandSource {
    const uint64_t* codes;  // codes by position (inline) or by id (base array)
    const uint32_t* ids;    // ids by position, or null when id = position
    bool by_id;             // codes are indexed by id: load the id first
};

template <int W, int MODE, bool ALIGNED, int B>
__device__ __forceinline__ void process_loaded(const SearchArgs& a, const Layout& L, uint32_t* whist, uint32_t q,
                                               int j, int rho, int t_done, int hist_done, int bnd, const Code<W>& g,
                                               const CandSource& src, const uint32_t (&pos)[B],
                                               const bool (&valid)[B], const Code<W> (&c)[B],
                                               const uint32_t (&id)[B], uint32_t& unique_acc, uint32_t& raw_acc);

// B candidates per lane, warp-synchronous (all 32 lanes call together; every
// valid candidate belongs to query q).  All B loads of a kind are issued
// before any is used, so each lane keeps B gathers in flight.  With inline
// codes the id is read only for candidates that are stored.  Kept distances
// go to the warp's shared-memory histogram `whist` (flushed by flush_hist).
template <int W, int MODE, bool ALIGNED, int B>
__device__ __forceinline__ void handle_batch(const SearchArgs& a, const Layout& L,
                                             uint32_t* whist, uint32_t q, int j, int rho, int t_done, int hist_done,
                                             int bnd, const Code<W>& g, const CandSource& src,
                                             const uint32_t (&pos)[B], const bool (&valid)[B],
                                             uint32_t& unique_acc, uint32_t& raw_acc) {
    Code<W> c[B];
    uint32_t id[B];
    if (src.by_id) {
#pragma unroll
        for (int b = 0; b < B; ++b) id[b] = valid[b] ? __ldg(src.ids + pos[b]) : 0u;
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (valid[b]) c[b] = load_code<W>(src.codes, id[b]);
            else
#pragma unroll
                for (int w = 0; w < W; ++w) c[b].w[w] = 0ull;
        }
    } else {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            id[b] = pos[b];
            if (valid[b]) c[b] = load_code<W>(src.codes, pos[b]);
            else
#pragma unroll
                for (int w = 0; w < W; ++w) c[b].w[w] = 0ull;
        }
    }
    process_loaded<W, MODE, ALIGNED, B>(a, L, whist, q, j, rho, t_done, hist_done, bnd, g, src, pos, valid, c, id,
                                        unique_acc, raw_acc);
}

// Stores (k-NN), collects or counts the taken candidates of a warp batch:
// bit b of take_mask marks candidate b of the lane.  One atomic reserves the
// slots of the whole warp batch.  With lazy ids (inline codes) a k-NN entry
// keeps the table position and the table (j + 1 in bits 41..49).
template <int MODE, int B>
__device__ __forceinline__ void store_batch(const SearchArgs& a, uint32_t q, int j, bool lazy_id,
                                            const uint32_t* ids, const uint32_t (&pos)[B], const uint32_t (&id)[B],
                                            const int (&dist)[B], uint32_t take_mask) {
    const uint32_t lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;
    if constexpr (MODE == kModeCount) {
        const uint32_t mine = __popc(take_mask);
        const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, mine);
        if (total != 0 && lane == 0) atomicAdd(&a.cnt[q], total);
        return;
    }
    if (!__any_sync(0xFFFFFFFFu, take_mask != 0)) return;
    // lane offsets within the batch: candidates ordered by (b, lane)
    uint32_t before[B];
    uint32_t total = 0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (take_mask >> b) & 1u);
        before[b] = total + __popc(bal & lt);
        total += __popc(bal);
    }
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.cnt[q], total);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (!((take_mask >> b) & 1u)) continue;
        if constexpr (MODE == kModeKnn) {
            // With inline codes the entry keeps the table position and the
            // table (j + 1 in bits 41..49); the selection turns the entries
            // within d_k into ids after the search, off this kernel's
            // critical path.
            const uint32_t p = base + before[b];
            const uint64_t e = lazy_id ? (static_cast<uint64_t>(j + 1) << kQueryShift) | pack_entry(dist[b], pos[b])
                                       : pack_entry(dist[b], id[b]);
            if (p < a.cap) a.buf[static_cast<uint64_t>(q) * a.cap + p] = e;
        } else {
            const uint32_t cid = lazy_id ? __ldg(ids + pos[b]) : id[b];
            const uint64_t p = __ldg(a.out_base + q) + base + before[b];
            if (p < __ldg(a.out_base + q + 1))
                a.buf[p] = (static_cast<uint64_t>(q) << kQueryShift) | pack_entry(dist[b], cid);
            else
                atomicExch(a.err, 1);
        }
    }
}


// The second half of handle_batch, for codes already in registers (from
// global memory or from a shared-memory stage).  id[b] is the candidate's id
// unless the source keeps codes inline (then ids are read only when stored).
template <int W, int MODE, bool ALIGNED, int B>
__device__ __forceinline__ void process_loaded(const SearchArgs& a, const Layout& L, uint32_t* whist, uint32_t q,
                                               int j, int rho, int t_done, int hist_done, int bnd, const Code<W>& g,
                                               const CandSource& src, const uint32_t (&pos)[B],
                                               const bool (&valid)[B], const Code<W> (&c)[B],
                                               const uint32_t (&id)[B], uint32_t& unique_acc, uint32_t& raw_acc) {
    const bool lazy_id = !src.by_id && src.ids != nullptr;
    const int far = (bnd < 0 || a.exact_stats) ? 0x7FFFFFFF : bnd;
    // Distances and tests of all B candidates first; the kept entries of the
    // batch then take one slot reservation (a single atomic) for the warp.
    int dist[B];
    uint32_t take_mask = 0;   // bit b: candidate b is stored / collected
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int d = 0;
        bool keep = false, count = false;
        if (valid[b]) eval_candidate<W, ALIGNED>(a.m, L, j, rho, t_done, hist_done, far, g, c[b], d, keep, count);
        dist[b] = d;
        if (j < 0) raw_acc += (valid[b] && count) ? 1u : 0u;
        if constexpr (MODE == kModeKnn) {
            if (keep && count) {
                atomicAdd(&whist[d], 1u);
                ++unique_acc;
            }
        } else {
            unique_acc += keep ? 1u : 0u;
        }
        if (keep && d <= bnd) take_mask |= 1u << b;
    }
    store_batch<MODE, B>(a, q, j, lazy_id, src.ids, pos, id, dist, take_mask);
}

// process_loaded for inline records without the table's own word (every
// substring one 32-bit word): record word i is code word i (i < j) or i + 1
// (i >= j), gq holds the query's words in the same order, and the table's own
// word differs from the query's in exactly rho bits (the ring).  The
// first-discoverer test (reading c8) keeps the code when no earlier table is
// within rho bits and no later one within rho - 1: word i needs at least
// th[i] = rho + (i < j) differing bits.
template <int R, int MODE, int B>
__device__ __forceinline__ void process_records(const SearchArgs& a, uint32_t* whist, uint32_t q, int j, int rho,
                                                int bnd, bool count_new, const uint32_t (&gq)[R],
                                                const uint32_t (&th)[R], const uint32_t* ids,
                                                const uint32_t (&pos)[B], const bool (&valid)[B],
                                                const uint32_t (&rec)[B][R], uint32_t& unique_acc) {
    const int far = (bnd < 0 || a.exact_stats) ? 0x7FFFFFFF : bnd;
    int dist[B];
    uint32_t take_mask = 0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int d = rho;
        int pc[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            pc[i] = __popc(rec[b][i] ^ gq[i]);
            d += pc[i];
        }
        dist[b] = d;
        if (valid[b] && d <= far) {
            bool keep = true;
#pragma unroll
            for (int i = 0; i < R; ++i) keep = keep && static_cast<uint32_t>(pc[i]) >= th[i];
            if constexpr (MODE == kModeKnn) {
                if (keep && count_new) {
                    atomicAdd(&whist[d], 1u);
                    ++unique_acc;
                }
            } else {
                unique_acc += keep ? 1u : 0u;
            }
            if (keep && d <= bnd) take_mask |= 1u << b;
        }
    }
    store_batch<MODE, B>(a, q, j, true, ids, pos, pos, dist, take_mask);
}

// Add the warp's histogram to query q's global histogram and clear it.
__device__ __forceinline__ void flush_hist(uint32_t* whist, uint32_t* ghist, int qbits) {
    __syncwarp();
    for (int d = lane_id(); d <= qbits; d += 32) {
        const uint32_t v = whist[d];
        if (v) {
            atomicAdd(ghist + d, v);
            whist[d] = 0;
        }
    }
    __syncwarp();
}

// Buckets of R keys of one lane, with every table read of the R lookups in
// flight together: the first slot group of each key's probe sequence, then
// the bucket bounds.  A key whose first group neither holds it nor ends its
// probe sequence (rare at the tables' load factor) takes the full lookup.
template <int R>
__device__ __forceinline__ void lookup_buckets(const TableDesc& t, const uint32_t (&key)[R], int mine,
                                               uint32_t (&b)[R], uint32_t (&e)[R]) {
    if (t.kind == MIH_TABLE_DIRECT) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            b[r] = r < mine ? __ldg(t.offsets + key[r]) : 0u;
            e[r] = r < mine ? __ldg(t.offsets + key[r] + 1) : 0u;
        }
        return;
    }
    uint32_t rank[R];
    bool open[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint4 s01 = make_uint4(0u, kEmptySlot, 0u, kEmptySlot);
        uint4 s23 = s01;
        if (r < mine) {
            const uint4* s4 = reinterpret_cast<const uint4*>(t.slots + 4 * (hash_key(key[r]) & t.bucket_mask));
            s01 = __ldg(s4);
            s23 = __ldg(s4 + 1);
        }
        // first match or first empty slot of the group decides
        uint32_t rk = kEmptySlot;
        bool op = false;
        if (s01.y == kEmptySlot) op = true;
        else if (s01.x == key[r]) rk = s01.y;
        else if (s01.w == kEmptySlot) op = true;
        else if (s01.z == key[r]) rk = s01.w;
        else if (s23.y == kEmptySlot) op = true;
        else if (s23.x == key[r]) rk = s23.y;
        else if (s23.w == kEmptySlot) op = true;
        else if (s23.z == key[r]) rk = s23.w;
        rank[r] = rk;
        open[r] = op || r >= mine;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        b[r] = e[r] = 0u;
        if (rank[r] != kEmptySlot) {
            b[r] = __ldg(t.offsets + rank[r]);
            e[r] = __ldg(t.offsets + rank[r] + 1);
        } else if (!open[r]) {
            lookup_bucket(t, key[r], b[r], e[r]);   // group full of other keys: keep probing
        }
    }
}

constexpr int kBatch = 4;      // candidates in flight per lane, bucket unions
#ifndef MIH_BIG_BATCH
#define MIH_BIG_BATCH 8
#endif
constexpr int kBigBatch = MIH_BIG_BATCH;   // candidates in flight per lane, big-bucket slices
constexpr int kWarps = kSearchThreads / 32;
constexpr int kHistBins = 257; // distances 0..256

// resident CTAs per SM asked of the chunk kernel (its chunks are latency-bound:
// more warps in flight, more chunks per second)
#ifndef MIH_SEARCH_MIN_BLOCKS
#define MIH_SEARCH_MIN_BLOCKS 4
#endif

template <int W, int MODE, bool ALIGNED>
__global__ void __launch_bounds__(kSearchThreads, MIH_SEARCH_MIN_BLOCKS) search_kernel(SearchArgs a) {
    __shared__ int s_off[kMaxTables];
    __shared__ int s_len[kMaxTables];
    __shared__ uint32_t s_mask[kMaxTables * 2 * W];
    __shared__ uint32_t s_hist[kWarps][kHistBins];
    __shared__ uint2 s_list[kWarps][kChunkKeys];   // a chunk's nonempty buckets: {begin, first union index}
    for (int j = threadIdx.x; j < a.m; j += blockDim.x) s_off[j] = a.tables[j].off;
    build_layout(a.tables, a.m, W, s_len, s_mask);
    for (int i = threadIdx.x; i < kWarps * kHistBins; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const Layout L{s_len, s_mask};
    const uint32_t lane = lane_id();
    uint32_t* whist = s_hist[threadIdx.x >> 5];
    const unsigned long long total_chunks = a.chunk_off[a.nq];
    const uint32_t kSlice = a.slice_entries;
    // Chunk indices: the warp's own index first (no atomic), then nwarps plus
    // the values of a shared counter.  Lane 0 grabs the next index before the
    // current chunk runs and the warp reads it afterwards, so the atomic's round
    // trip is off the critical path.  An index a warp grabbed but does not run
    // lies at or beyond total_chunks (the counter only grows).
    const unsigned long long nwarps = static_cast<unsigned long long>(gridDim.x) * (blockDim.x >> 5);
    unsigned long long c = static_cast<unsigned long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    unsigned long long pending = 0;
    if (lane == 0) pending = atomicAdd(a.chunk_next, 1ull);
    for (;; c = nwarps + __shfl_sync(0xFFFFFFFFu, pending, 0), pending = lane == 0 ? atomicAdd(a.chunk_next, 1ull)
                                                                                   : 0ull) {
        if (c >= total_chunks) break;
        // query owning chunk c: the last q with chunk_off[q] <= c, by a 32-ary
        // search (every lane probes one point per round; chunk_off[lo] <= c <
        // chunk_off[hi] throughout)
        uint32_t lo = 0, hi = a.nq;
        for (;;) {
            const uint32_t step = hi - lo > 32 ? (hi - lo + 31) / 32 : 1;
            const uint32_t probe = lo + lane * step;
            const bool le = probe < hi && __ldg(a.chunk_off + probe) <= c;
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, le);   // lane 0 always (probe = lo)
            lo += (31u - static_cast<uint32_t>(__clz(bal))) * step;
            if (step == 1) break;
            hi = min(hi, lo + step);
        }
        const uint32_t q = lo;
        uint64_t lc = c - __ldg(a.chunk_off + q);
        int t = __ldg(a.t_lo + q);
        const int hd = a.hist_done ? __ldg(a.hist_done + q) : -1;
        const int bnd = __ldg(a.bound + q);
        uint32_t* ghist = (MODE == kModeKnn) ? a.hist + static_cast<uint64_t>(q) * (a.q + 1) : nullptr;
        if (a.exh && a.exh[q]) {
            // Verify codes [lc * kScanChunk, ...) against the query once.
            const uint64_t base = lc * kScanChunk;
            const uint64_t end = min(a.n, base + kScanChunk);
            const Code<W> g = load_query<W>(a.queries, q);
            uint32_t unique = 0, raw = 0;
            const CandSource src{a.codes, nullptr, false};
            for (uint64_t p = base; p < end; p += 32 * kBigBatch) {
                uint32_t pos[kBigBatch];
                bool valid[kBigBatch];
#pragma unroll
                for (int k = 0; k < kBigBatch; ++k) {
                    const uint64_t i = p + k * 32 + lane;
                    valid[k] = i < end;
                    pos[k] = static_cast<uint32_t>(i);
                }
                handle_batch<W, MODE, ALIGNED, kBigBatch>(a, L, whist, q, -1, 0, t - 1, hd, bnd, g, src, pos,
                                                          valid, unique, raw);
            }
            if (MODE == kModeKnn) flush_hist(whist, ghist, a.q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unique += __shfl_down_sync(0xFFFFFFFFu, unique, o);
                raw += __shfl_down_sync(0xFFFFFFFFu, raw, o);
            }
            if (lane == 0 && a.qstats) {
                atomicAdd(&a.qstats[4ull * q + 1], static_cast<unsigned long long>(raw));
                atomicAdd(&a.qstats[4ull * q + 2], static_cast<unsigned long long>(unique));
            }
            continue;
        }
        for (;;) {
            const uint64_t nch = step_chunks(s_len, a.m, t);
            if (lc < nch) break;
            lc -= nch;
            ++t;
        }
        const int j = t % a.m, rho = t / a.m, s = s_len[j];
        const uint64_t nkeys = binom(s, rho);
        const uint64_t first = lc * kChunkKeys + static_cast<uint64_t>(lane) * kKeysPerLane;
        const uint64_t left = first < nkeys ? nkeys - first : 0ull;
        const int mine = left < static_cast<uint64_t>(kKeysPerLane) ? static_cast<int>(left) : kKeysPerLane;
        const Code<W> g = load_query<W>(a.queries, q);
        const uint32_t gkey = substring_bits<W>(g, s_off[j], s);
        const TableDesc& tab = a.tables[j];
        // whole inline codes, else (no inline codes, or records) the codes by id
        const CandSource src = (tab.codes && tab.rec_words == 0) ? CandSource{tab.codes, tab.ids, false}
                                                                 : CandSource{a.codes, tab.ids, true};
        uint64_t x = mine > 0 ? unrank_subset(first, s, rho) : 0ull;
        uint32_t key[kKeysPerLane], bb[kKeysPerLane], ee[kKeysPerLane];
#pragma unroll
        for (int r = 0; r < kKeysPerLane; ++r) {
            key[r] = gkey ^ static_cast<uint32_t>(x);
            if (rho > 0 && r + 1 < mine) x = next_subset(x);
        }
        lookup_buckets<kKeysPerLane>(tab, key, mine, bb, ee);
        uint32_t raw = 0, unique = 0;
        // Big buckets go to the slice kernel.  The warp reserves the slices of
        // all its big buckets with one atomic; if the list is full the
        // reserved slots are marked empty and the warp scans those buckets here.
        uint32_t ns_lane = 0;
#pragma unroll
        for (int r = 0; r < kKeysPerLane; ++r) {
            const uint32_t sz = ee[r] - bb[r];
            if (sz > kBigBucket) ns_lane += (sz + kSlice - 1) / kSlice;
        }
        const uint32_t ns_incl = warp_inclusive_scan(ns_lane);
        const uint32_t ns_total = __shfl_sync(0xFFFFFFFFu, ns_incl, 31);
        uint32_t at = 0;
        bool fits = true;
        if (ns_total != 0) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(a.big_count, ns_total);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            at = base + ns_incl - ns_lane;
            fits = static_cast<uint64_t>(base) + ns_total <= a.big_cap;
        }
        int nz = 0;
        uint32_t tot = 0, sliced = 0;
#pragma unroll
        for (int r = 0; r < kKeysPerLane; ++r) {
            uint32_t sz = ee[r] - bb[r];
            if (sz > kBigBucket) {
                const uint32_t ns = (sz + kSlice - 1) / kSlice;
                for (uint32_t i = 0; i < ns; ++i, ++at) {
                    if (at >= a.big_cap) continue;
                    BigSlice bs;
                    bs.q = fits ? q : kPadId;
                    bs.t = t;
                    bs.begin = bb[r] + i * kSlice;
                    bs.end = min(ee[r], bs.begin + kSlice);
                    a.big[at] = bs;
                }
                if (fits) {
                    raw += sz;
                    sliced += sz;
                    sz = 0;
                }
            }
            raw += sz;
            ee[r] = sz;   // from here on: entries this warp scans itself
            nz += sz != 0 ? 1 : 0;
            tot += sz;
        }
        // The warp scans the union of its nonempty small buckets, 32 * kBatch
        // entries per round: list them (begin, first union index) in shared
        // memory, and map a union index to its bucket by binary search.
        const uint32_t nz_incl = warp_inclusive_scan(static_cast<uint32_t>(nz));
        const uint32_t tot_incl = warp_inclusive_scan(tot);
        const uint32_t n_list = __shfl_sync(0xFFFFFFFFu, nz_incl, 31);
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, tot_incl, 31);
        if (total > 0) {
            uint2* list = s_list[threadIdx.x >> 5];
            uint32_t at = nz_incl - nz, run = tot_incl - tot;
#pragma unroll
            for (int r = 0; r < kKeysPerLane; ++r)
                if (ee[r] != 0) {
                    list[at++] = make_uint2(bb[r], run);
                    run += ee[r];
                }
            __syncwarp();
            for (uint32_t base = 0; base < total; base += 32 * kBatch) {
                uint32_t pos[kBatch];
                bool valid[kBatch];
#pragma unroll
                for (int k = 0; k < kBatch; ++k) {
                    const uint32_t idx = base + k * 32 + lane;
                    uint32_t lo = 0, hi = n_list;   // last entry whose first index <= idx
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (list[mid].y <= idx) lo = mid; else hi = mid;
                    }
                    const uint2 ent = list[lo];
                    valid[k] = idx < total;
                    pos[k] = valid[k] ? ent.x + (idx - ent.y) : 0u;
                }
                if constexpr (ALIGNED) {
                    if (tab.rec_words != 0) {
                        // inline records of this table: R consecutive words at
                        // each position, read in place (no id, no gather)
                        constexpr int R = 2 * W - 1;
                        const uint32_t* recs = reinterpret_cast<const uint32_t*>(tab.codes);
                        uint32_t g32[2 * W], gq[R], th[R];
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            g32[2 * w] = static_cast<uint32_t>(g.w[w]);
                            g32[2 * w + 1] = static_cast<uint32_t>(g.w[w] >> 32);
                        }
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            gq[i] = i < j ? g32[i] : g32[i + 1];
                            th[i] = static_cast<uint32_t>(rho) + (i < j ? 1u : 0u);
                        }
                        uint32_t rec[kBatch][R];
#pragma unroll
                        for (int k = 0; k < kBatch; ++k)
#pragma unroll
                            for (int i = 0; i < R; ++i)
                                rec[k][i] = valid[k] ? __ldg(recs + static_cast<uint64_t>(pos[k]) * R + i) : 0u;
                        process_records<R, MODE, kBatch>(a, whist, q, j, rho, bnd, a.m * rho + j > hd, gq, th,
                                                         tab.ids, pos, valid, rec, unique);
                        continue;
                    }
                }
                uint32_t unused = 0;
                handle_batch<W, MODE, ALIGNED, kBatch>(a, L, whist, q, j, rho, -1, hd, bnd, g, src, pos, valid,
                                                       unique, unused);
            }
            __syncwarp();
        }
        if (MODE == kModeKnn) flush_hist(whist, ghist, a.q);
        // per-query counters (lookups, raw candidates, unique candidates) of
        // steps not counted before
        const bool counting = t > hd;
        uint32_t lk = counting ? static_cast<uint32_t>(mine) : 0u;
        if (!counting) raw = sliced = 0;
        if (a.sliced) {
            const uint32_t ws = __reduce_add_sync(0xFFFFFFFFu, sliced);
            if (lane == 0 && ws != 0) atomicAdd(a.sliced, static_cast<unsigned long long>(ws));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lk += __shfl_down_sync(0xFFFFFFFFu, lk, o);
            raw += __shfl_down_sync(0xFFFFFFFFu, raw, o);
            unique += __shfl_down_sync(0xFFFFFFFFu, unique, o);
        }
        if (lane == 0 && a.qstats) {
            atomicAdd(&a.qstats[4ull * q + 0], static_cast<unsigned long long>(lk));
            atomicAdd(&a.qstats[4ull * q + 1], static_cast<unsigned long long>(raw));
            atomicAdd(&a.qstats[4ull * q + 2], static_cast<unsigned long long>(unique));
        }
    }
}

// Slices are taken from the wave's list through a shared counter.  To keep
// that round trip off the critical path each warp holds the index of its next
// slice (fetched one slice ahead) and that slice's descriptor (loaded one
// slice ahead): starting a slice uses only values already in registers.
struct SliceFeed {
    uint32_t grab;       // lane 0: first index of the pending grab (its atomic was
                         // issued at least one slice ago; other lanes: unused)
    uint32_t next_idx;   // first index of the current grab not yet loaded (warp-uniform)
    uint32_t left;       // indices of the current grab not yet loaded (>= 1)
    BigSlice ahead;      // descriptor of the slice the warp starts next (t < 0 past the end)
};

// Slice indices are taken kSliceGrab at a time, so the shared counter sees a
// fraction of the warps' requests.
#ifndef MIH_SLICE_GRAB
#define MIH_SLICE_GRAB 2
#endif
constexpr uint32_t kSliceGrab = MIH_SLICE_GRAB;

__device__ __forceinline__ BigSlice load_slice(const SearchArgs& a, uint32_t i, unsigned int count) {
    BigSlice bs;
    bs.q = kPadId;
    bs.t = -1;
    bs.begin = bs.end = 0;
    if (i < count) bs = a.big[i];
    return bs;
}

// Lane 0 starts the next grab; its result is read (broadcast) only when the
// warp needs it, a slice later, so the atomic's latency stays hidden.
__device__ __forceinline__ void start_grab(const SearchArgs& a, SliceFeed& feed) {
    if (lane_id() == 0) feed.grab = atomicAdd(a.big_next, kSliceGrab);
}

__device__ __forceinline__ void take_grab(SliceFeed& feed) {
    feed.next_idx = __shfl_sync(0xFFFFFFFFu, feed.grab, 0);
    feed.left = kSliceGrab;
}

// Moves the feed one slice on: loads the descriptor of next_idx into `ahead`;
// when the current grab runs out the pending grab becomes current and the
// next one is started.  One grab is always pending.
__device__ __forceinline__ void advance_feed(const SearchArgs& a, SliceFeed& feed, unsigned int count) {
    feed.ahead = load_slice(a, feed.next_idx, count);
    ++feed.next_idx;
    if (--feed.left == 0) {
        take_grab(feed);
        start_grab(a, feed);
    }
}

// Slices of large buckets, one warp per slice, 32 * kBigBatch entries per round.
#ifndef MIH_BIG_MIN_BLOCKS
#define MIH_BIG_MIN_BLOCKS 1
#endif

template <int W, int MODE, bool ALIGNED>
__global__ void __launch_bounds__(kSearchThreads, MIH_BIG_MIN_BLOCKS) search_big_kernel(SearchArgs a) {
    __shared__ int s_len[kMaxTables];
    __shared__ uint32_t s_mask[kMaxTables * 2 * W];
    __shared__ uint32_t s_hist[kWarps][kHistBins];
    build_layout(a.tables, a.m, W, s_len, s_mask);
    for (int i = threadIdx.x; i < kWarps * kHistBins; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const Layout L{s_len, s_mask};
    const uint32_t lane = lane_id();
    uint32_t* whist = s_hist[threadIdx.x >> 5];
    const unsigned int count = min(*a.big_count, a.big_cap);
    SliceFeed feed;
    feed.grab = 0;
    start_grab(a, feed);
    take_grab(feed);        // the first grab is waited for
    start_grab(a, feed);    // the pending one
    advance_feed(a, feed, count);
    for (;;) {
        const BigSlice bs = feed.ahead;
        if (bs.t < 0) break;              // the list is exhausted
        advance_feed(a, feed, count);     // the next descriptor loads while this slice runs
        if (bs.q == kPadId) continue;
        const int j = bs.t % a.m, rho = bs.t / a.m;
        const Code<W> g = load_query<W>(a.queries, bs.q);
        const TableDesc& tab = a.tables[j];
        const CandSource src = (tab.codes && tab.rec_words == 0) ? CandSource{tab.codes, tab.ids, false}
                                                                 : CandSource{a.codes, tab.ids, true};
        const int hd = a.hist_done ? __ldg(a.hist_done + bs.q) : -1;
        const int bnd = __ldg(a.bound + bs.q);
        uint32_t unique = 0, unused = 0;
        for (uint32_t p = bs.begin; p < bs.end; p += 32 * kBigBatch) {
            uint32_t pos[kBigBatch];
            bool valid[kBigBatch];
#pragma unroll
            for (int k = 0; k < kBigBatch; ++k) {
                const uint32_t e = p + k * 32 + lane;
                valid[k] = e < bs.end;
                pos[k] = e;
            }
            handle_batch<W, MODE, ALIGNED, kBigBatch>(a, L, whist, bs.q, j, rho, -1, hd, bnd, g, src, pos, valid,
                                                      unique, unused);
        }
        if (MODE == kModeKnn) flush_hist(whist, a.hist + static_cast<uint64_t>(bs.q) * (a.q + 1), a.q);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) unique += __shfl_down_sync(0xFFFFFFFFu, unique, o);
        if (lane == 0 && a.qstats) atomicAdd(&a.qstats[4ull * bs.q + 2], static_cast<unsigned long long>(unique));
    }
}

// ------------------------------------------------------- streamed slices
// With inline codes every big-bucket slice is one contiguous run of codes.
// Each warp streams its slices through a ring of kStages shared-memory stages
// (3 KB in the default shape): lane 0 keeps bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier per stage) of the next
// kStages - 1 stages in flight
// while the warp verifies the current one.  Every wait on an mbarrier is
// bounded; on expiry the kernel raises a.timeout, waits (bounded) for its own
// copies still in flight and leaves.
// Shapes of the slice kernel: stage bytes, warps per CTA, stages in flight
// per warp.  The k-NN waves run any of them (mih_tune_search times them on
// hold-out queries); the collect and count passes run the first.
template <uint32_t SB, int NW, int NS>
struct StreamShape {
    static constexpr uint32_t kStageBytes = SB;
    static constexpr int kWarps = NW;
    static constexpr int kStages = NS;
    static constexpr uint32_t kSlot = SB + 16;   // + one 8-byte code of realignment (W = 1)
    static constexpr size_t kSmem = static_cast<size_t>(NW) * NS * kSlot;
    static_assert(NS >= 2 && NS <= 4, "stage ring of 2 to 4 slots");
};

// Static shared memory of the slice kernel for W-word codes: a histogram of
// distances 0..64 W per warp, the barriers, and (whole codes only: records
// never read them) the substring layout of up to 64 W tables.
template <class Shape, int W, bool REDUCED>
constexpr size_t stream_static_smem() {
    return static_cast<size_t>(Shape::kWarps) * (64 * W + 1) * 4 + static_cast<size_t>(Shape::kWarps) * Shape::kStages * 8 +
           16 + (REDUCED ? 8 : static_cast<size_t>(64 * W) * 4 * (1 + 2 * W));
}
// Resident CTAs per SM that shared memory allows (228 KB per SM, 1 KB of it
// reserved per CTA); sets the kernel's register budget.
template <class Shape, int W, bool REDUCED>
constexpr int stream_min_blocks() {
    constexpr size_t per = Shape::kSmem + stream_static_smem<Shape, W, REDUCED>() + 1024;
    return (228 * 1024) / per > 0 ? static_cast<int>((228 * 1024) / per) : 1;
}
#ifndef MIH_STREAM_STAGES
#define MIH_STREAM_STAGES 2
#endif
#ifndef MIH_STREAM_WARPS
#define MIH_STREAM_WARPS 8
#endif
// The default: 3 KB stages leave room for 4 CTAs (32 warps) per SM.
using Shape0 = StreamShape<kDefaultStageBytes, MIH_STREAM_WARPS, MIH_STREAM_STAGES>;
using Shape1 = StreamShape<8192, 4, 2>;   // larger stages, fewer warps
using Shape2 = StreamShape<4096, 8, 2>;   // 4 KB stages, 3 CTAs per SM
constexpr int kStreamVariants = 3;

// Largest bulk copy issue_stage makes for one stage: records start up to three
// entries early (16-byte aligned groups of four), W = 1 codes up to one, and
// both round the size up to 16 bytes.  Every layout must fit its slot.
template <int W, bool REDUCED, uint32_t SB>
constexpr uint32_t max_stage_copy() {
    return REDUCED ? (((stage_entries<W, true, SB>() + 3u) * 4u * (2 * W - 1) + 15u) & ~15u)
                   : (W == 1 ? (((stage_entries<1, false, SB>() + 1u) * 8u + 15u) & ~15u)
                             : stage_entries<W, false, SB>() * 8u * W);
}
// Groups of four records read by one lane (16-byte shared loads), and the
// groups a stage can span; every group a lane reads lies inside its slot.
template <int W, uint32_t SB>
constexpr uint32_t stage_groups() {
    return (3u + stage_entries<W, true, SB>() + 3u) / 4u;
}
template <uint32_t SB>
constexpr bool stage_fits_slot() {
    constexpr uint32_t slot = SB + 16;
    return max_stage_copy<1, false, SB>() <= slot && max_stage_copy<2, false, SB>() <= slot &&
           max_stage_copy<4, false, SB>() <= slot && max_stage_copy<1, true, SB>() <= slot &&
           max_stage_copy<2, true, SB>() <= slot && max_stage_copy<4, true, SB>() <= slot &&
           stage_groups<1, SB>() * 16u * 1u <= slot && stage_groups<2, SB>() * 16u * 3u <= slot &&
           stage_groups<4, SB>() * 16u * 7u <= slot && stage_entries<1, true, SB>() >= 32 &&
           stage_entries<2, true, SB>() >= 32 && stage_entries<4, true, SB>() >= 32 &&
           stage_entries<4, false, SB>() % 32 == 0;
}
static_assert(stage_fits_slot<Shape0::kStageBytes>() && stage_fits_slot<Shape1::kStageBytes>() &&
                  stage_fits_slot<Shape2::kStageBytes>(),
              "a stage's copy or its record groups overrun the shared-memory slot");

// One stage: entries [pos, pos + cnt) of a slice ending at `end`, all of
// query q at step t, with the query's state for verifying them (loaded when
// the slice's first stage is issued, two stages before it is verified).
// Warp-uniform.
template <int W>
struct Stage {
    uint32_t q;
    int t;
    uint32_t pos, cnt, end;
    bool valid;
    int bnd, hd;
    uint32_t shift;   // code offset of the stage inside its slot (W = 1 realigns to 16 bytes)
    Code<W> g;
};

template <int W, bool REDUCED, uint32_t SB>
__device__ __forceinline__ Stage<W> next_stage(const SearchArgs& a, const Stage<W>& st, unsigned int count,
                                               SliceFeed& feed) {
    constexpr uint32_t kPer = stage_entries<W, REDUCED, SB>();
    Stage<W> r = st;
    if (!st.valid) return r;
    if (st.pos + st.cnt < st.end) {
        r.pos = st.pos + st.cnt;
        r.cnt = min(kPer, st.end - r.pos);
        return r;
    }
    for (;;) {
        const BigSlice bs = feed.ahead;
        if (bs.t < 0) {   // the list is exhausted
            r.valid = false;
            return r;
        }
        // refill the feed: the descriptor of the index known since the last
        // slice (its load completes while this slice is verified)
        advance_feed(a, feed, count);
        if (bs.q == kPadId) continue;   // reserved but never filled
        r.q = bs.q;
        r.t = bs.t;
        r.pos = bs.begin;
        r.end = bs.end;
        r.cnt = min(kPer, bs.end - bs.begin);
        r.bnd = __ldg(a.bound + bs.q);
        r.hd = a.hist_done ? __ldg(a.hist_done + bs.q) : -1;
        r.g = load_query<W>(a.queries, bs.q);
        return r;
    }
}

// Lane 0 starts the copy of stage st into slot `buf`; returns the entry
// offset of the stage inside the slot: the copy starts on a 16-byte boundary,
// so W = 1 codes realign by up to one code and REDUCED records by up to three.
template <int W, bool REDUCED>
__device__ __forceinline__ uint32_t issue_stage(const SearchArgs& a, const Stage<W>& st, unsigned char* buf,
                                                uint64_t* bar) {
    const unsigned char* base = reinterpret_cast<const unsigned char*>(a.tables[st.t % a.m].codes);
    uint32_t lo = st.pos, shift = 0, bytes = st.cnt * 8u * W;
    uint64_t src_off = static_cast<uint64_t>(st.pos) * 8u * W;
    if constexpr (REDUCED) {
        constexpr uint32_t rb = 4u * (2 * W - 1);   // record bytes; 4 records are 16 R bytes
        lo = st.pos & ~3u;
        shift = st.pos - lo;
        bytes = ((st.cnt + shift) * rb + 15u) & ~15u;   // the table keeps 16 bytes of padding
        src_off = static_cast<uint64_t>(lo) * rb;
    } else if constexpr (W == 1) {
        lo = st.pos & ~1u;
        shift = st.pos - lo;
        bytes = ((st.cnt + shift) * 8u + 15u) & ~15u;   // the table keeps 16 bytes of padding
        src_off = static_cast<uint64_t>(lo) * 8u;
    }
    if (lane_id() == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads of the slot are done
        bulk_copy_to_smem(buf, base + src_off, bytes, bar);
    }
    return shift;
}

template <int W, int MODE, bool ALIGNED, class Shape>
__global__ void __launch_bounds__(Shape::kWarps * 32, (stream_min_blocks<Shape, W, ALIGNED>()))
    search_stream_kernel(SearchArgs a) {
    constexpr int kStreamWarps = Shape::kWarps;
    constexpr int kStages = Shape::kStages;
    constexpr uint32_t kStageSlot = Shape::kSlot;
    constexpr uint32_t SB = Shape::kStageBytes;
    // aligned tables (every substring one 32-bit word) keep inline records
    // without their own word; the others keep whole codes
    constexpr bool REDUCED = ALIGNED;
    // distances 0..64 W; up to 64 W tables (m <= q), whose layout only
    // whole codes read
    constexpr int kBins = 64 * W + 1;
    constexpr int kTabs = REDUCED ? 1 : 64 * W;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ int s_len[kTabs];
    __shared__ uint32_t s_mask[kTabs * 2 * W];
    __shared__ uint32_t s_hist[kStreamWarps][kBins];
    __shared__ __align__(8) uint64_t s_bar[kStreamWarps][kStages];
    __shared__ __align__(8) uint64_t s_never;   // a barrier no copy completes (timeout test)
    if constexpr (!REDUCED) build_layout(a.tables, a.m, W, s_len, s_mask);
    for (int i = threadIdx.x; i < kStreamWarps * kBins; i += blockDim.x) (&s_hist[0][0])[i] = 0;
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    if (lane == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&s_bar[warp][i], 1);
        if (warp == 0) mbar_init(&s_never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const Layout L{s_len, s_mask};
    uint32_t* whist = s_hist[warp];
    // slot/barrier i of this warp, selected by arithmetic (no register arrays
    // indexed at run time, which would live in local memory)
    unsigned char* const slot0 = dsm + warp * kStages * kStageSlot;
    uint64_t* const bar0 = &s_bar[warp][0];
    uint32_t parities = 0u;   // bit i: phase parity of barrier i
    const unsigned int count = min(*a.big_count, a.big_cap);

    SliceFeed feed;
    feed.grab = 0;
    start_grab(a, feed);
    take_grab(feed);        // the first grab is waited for
    start_grab(a, feed);    // the pending one
    advance_feed(a, feed, count);
    Stage<W> none;
    none.valid = true;
    none.pos = none.cnt = none.end = 0;
    none.q = 0;
    none.t = 0;
    none.bnd = none.hd = 0;
    none.shift = 0;
    // the ring: cur (slot b), then up to kStages - 1 stages already issued
    Stage<W> cur = next_stage<W, REDUCED, SB>(a, none, count, feed);
    if (!cur.valid) return;
    cur.shift = issue_stage<W, REDUCED>(a, cur, slot0, bar0);
    Stage<W> n1 = next_stage<W, REDUCED, SB>(a, cur, count, feed);
    if (n1.valid) n1.shift = issue_stage<W, REDUCED>(a, n1, slot0 + kStageSlot, bar0 + 1);
    Stage<W> n2 = n1;
    if constexpr (kStages >= 3) {
        n2 = next_stage<W, REDUCED, SB>(a, n1, count, feed);
        if (n2.valid) n2.shift = issue_stage<W, REDUCED>(a, n2, slot0 + 2 * kStageSlot, bar0 + 2);
    }
    Stage<W> n3 = n2;
    if constexpr (kStages >= 4) {
        n3 = next_stage<W, REDUCED, SB>(a, n2, count, feed);
        if (n3.valid) n3.shift = issue_stage<W, REDUCED>(a, n3, slot0 + 3 * kStageSlot, bar0 + 3);
    }
    // entries per lane and batch: whole codes, B of them per lane at a time
    // (up to 32 * 4 codes per batch), or records
    constexpr int kPer = static_cast<int>(stage_entries<W, REDUCED, SB>());
    constexpr int B = kPer / 32 < 4 ? kPer / 32 : 4;
    constexpr int R = 2 * W - 1;
    int b = 0;
    uint32_t unique = 0;
    bool first_wait = true;
    while (cur.valid) {
        unsigned char* const slot_b = slot0 + b * kStageSlot;
        uint64_t* const bar_b = bar0 + b;
        // With the timeout test on, the warp's first wait is on a barrier that
        // no copy completes, so it runs out after a.wait_ns (its copies stay
        // issued and are drained below).  The decision is warp-uniform.
        const bool ok_lane = (a.wait_test && first_wait) ? mbar_wait_bounded(&s_never, 0u, a.wait_ns)
                                                          : mbar_wait_bounded(bar_b, (parities >> b) & 1u, a.wait_ns);
        first_wait = false;
        if (!__all_sync(0xFFFFFFFFu, ok_lane)) {
            if (lane == 0) atomicExch(a.timeout, 1);
            // every copy this warp issued (slot b's and the stages after it)
            // lands before the warp leaves, each waited for with the full limit
            mbar_wait_bounded(bar_b, (parities >> b) & 1u, kWaitNs);
            for (int i = 1; i < kStages; ++i) {
                const bool issued = i == 1 ? n1.valid : (i == 2 ? n2.valid : n3.valid);
                const int bi = (b + i) % kStages;
                if (issued) mbar_wait_bounded(bar0 + bi, (parities >> bi) & 1u, kWaitNs);
            }
            __syncwarp();
            return;
        }
        parities ^= 1u << b;
        // verify the stage out of shared memory
        const int j = cur.t % a.m, rho = cur.t / a.m;
        if constexpr (REDUCED) {
            uint32_t g32[2 * W], gq[R], th[R];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                g32[2 * w] = static_cast<uint32_t>(cur.g.w[w]);
                g32[2 * w + 1] = static_cast<uint32_t>(cur.g.w[w] >> 32);
            }
#pragma unroll
            for (int i = 0; i < R; ++i) {
                gq[i] = i < j ? g32[i] : g32[i + 1];
                th[i] = static_cast<uint32_t>(rho) + (i < j ? 1u : 0u);
            }
            const bool count_new = 2 * W * rho + j > cur.hd;
            const uint32_t* ids = a.tables[j].ids;
            const int far = (cur.bnd < 0 || a.exact_stats) ? 0x7FFFFFFF : cur.bnd;
            // The slot holds records [0, shift + cnt) of the copy, the stage's
            // own from `shift` on.  Lane l reads group g = l, l + 32, ... of
            // four records with R 16-byte loads; only groups that hold a
            // stage record are read.
            const uint4* sg = reinterpret_cast<const uint4*>(slot_b);
            const uint32_t r_lo = cur.shift, r_hi = cur.shift + cur.cnt;
            const uint32_t ngroups = (r_hi + 3u) / 4u;
            for (uint32_t g0 = 0; g0 < ngroups; g0 += 32) {
                const uint32_t g = g0 + lane;
                uint32_t wv[4 * R];
                if (g < ngroups) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const uint4 v = sg[g * R + r];
                        wv[4 * r] = v.x;
                        wv[4 * r + 1] = v.y;
                        wv[4 * r + 2] = v.z;
                        wv[4 * r + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 4 * R; ++r) wv[r] = 0u;
                }
                // Distances first: a record farther than the query's bound is
                // never stored nor counted (far = no limit without a bound),
                // and nearly every record is, so the warp goes on to the
                // duplicate test and the stores only when a lane has a near one.
                bool valid[4];
                uint32_t near = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t ri = 4u * g + k;
                    valid[k] = ri >= r_lo && ri < r_hi;
                    int d = rho;
#pragma unroll
                    for (int i = 0; i < R; ++i) d += __popc(wv[k * R + i] ^ gq[i]);
                    near |= (valid[k] && d <= far) ? (1u << k) : 0u;
                }
                if (!__any_sync(0xFFFFFFFFu, near != 0u)) continue;
                uint32_t pos[4];
                uint32_t rec[4][R];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    pos[k] = cur.pos + (4u * g + k - r_lo);
#pragma unroll
                    for (int i = 0; i < R; ++i) rec[k][i] = wv[k * R + i];
                }
                process_records<R, MODE, 4>(a, whist, cur.q, j, rho, cur.bnd, count_new, gq, th, ids, pos, valid,
                                            rec, unique);
            }
        } else {
        const CandSource src{nullptr, a.tables[j].ids, false};
        const Code<W>* sc = reinterpret_cast<const Code<W>*>(slot_b) + cur.shift;
        uint32_t unused = 0;
        for (uint32_t base = 0; base < cur.cnt; base += 32 * B) {
            uint32_t pos[B], id[B];
            bool valid[B];
            Code<W> c[B];
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const uint32_t i = base + k * 32 + lane;
                valid[k] = i < cur.cnt;
                pos[k] = cur.pos + i;
                id[k] = pos[k];
                if (valid[k]) c[k] = sc[i];
                else
#pragma unroll
                    for (int w = 0; w < W; ++w) c[k].w[w] = 0ull;
            }
            process_loaded<W, MODE, ALIGNED, B>(a, L, whist, cur.q, j, rho, -1, cur.hd, cur.bnd, cur.g, src, pos,
                                                valid, c, id, unique, unused);
        }
        }
        __syncwarp();
        // the slot just read takes the stage kStages after cur
        const Stage<W>& last = kStages == 2 ? n1 : (kStages == 3 ? n2 : n3);
        Stage<W> nn = next_stage<W, REDUCED, SB>(a, last, count, feed);
        if (nn.valid) nn.shift = issue_stage<W, REDUCED>(a, nn, slot_b, bar_b);
        // histogram and counters go out once the warp leaves this query
        if (!n1.valid || n1.q != cur.q) {
            if (MODE == kModeKnn) flush_hist(whist, a.hist + static_cast<uint64_t>(cur.q) * (a.q + 1), a.q);
            if (a.qstats) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) unique += __shfl_down_sync(0xFFFFFFFFu, unique, o);
                if (lane == 0) atomicAdd(&a.qstats[4ull * cur.q + 2], static_cast<unsigned long long>(unique));
            }
            unique = 0;
        }
        cur = n1;
        if constexpr (kStages == 2) {
            n1 = nn;
        } else if constexpr (kStages == 3) {
            n1 = n2;
            n2 = nn;
        } else {
            n1 = n2;
            n2 = n3;
            n3 = nn;
        }
        b = (b + 1 == kStages) ? 0 : b + 1;
    }
}

// Entries per big-bucket slice and launch shape of each slice-kernel variant.
template <int W, bool ALIGNED>
uint32_t variant_slice_entries(int v) {
    if (v == 1) return slice_entries<W, ALIGNED, Shape1::kStageBytes>();
    if (v == 2) return slice_entries<W, ALIGNED, Shape2::kStageBytes>();
    return slice_entries<W, ALIGNED, Shape0::kStageBytes>();
}

// ------------------------------------------------------------ planning
// Chunk count of each query's step range [t_lo, t_hi].
__global__ void plan_chunks_kernel(const TableDesc* __restrict__ tables, int m, uint32_t nq, uint64_t n,
                                   const int32_t* __restrict__ t_lo, const int32_t* __restrict__ t_hi,
                                   const uint8_t* __restrict__ exh, uint64_t* __restrict__ chunks /* [nq + 1] */) {
    __shared__ int s_len[kMaxTables];
    for (int j = threadIdx.x; j < m; j += blockDim.x) s_len[j] = tables[j].len;
    __syncthreads();
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x) {
        uint64_t c = 0;
        if (q < nq && t_lo[q] <= t_hi[q]) {
            if (exh && exh[q]) c = (n + kScanChunk - 1) / kScanChunk;
            else
                for (int t = t_lo[q]; t <= t_hi[q]; ++t) c += step_chunks(s_len, m, t);
        }
        chunks[q] = c;
    }
}

// Chunks of query q's step range (0 when idle), as plan_chunks_kernel counts them.
__device__ __forceinline__ uint64_t query_chunks(const int* s_len, int m, uint64_t n, const int32_t* t_lo,
                                                 const int32_t* t_hi, const uint8_t* exh, uint32_t q) {
    uint64_t c = 0;
    if (t_lo[q] <= t_hi[q]) {
        if (exh && exh[q]) c = (n + kScanChunk - 1) / kScanChunk;
        else
            for (int t = t_lo[q]; t <= t_hi[q]; ++t) c += step_chunks(s_len, m, t);
    }
    return c;
}

// One CTA plans a whole wave when nq is small enough: chunk counts, their
// exclusive scan into chunk_off[0..nq] and the zeroed work counters, in one
// launch instead of a count kernel, a multi-kernel scan and a memset.
constexpr int kPlanThreads = 1024;
constexpr uint32_t kPlanOneBlockMax = 64u * kPlanThreads;   // nq + 1 entries at most

__global__ void __launch_bounds__(kPlanThreads) plan_scan_kernel(const TableDesc* __restrict__ tables, int m,
                                                                 uint32_t nq, uint64_t n,
                                                                 const int32_t* __restrict__ t_lo,
                                                                 const int32_t* __restrict__ t_hi,
                                                                 const uint8_t* __restrict__ exh,
                                                                 uint64_t* __restrict__ chunk_off,
                                                                 unsigned long long* __restrict__ counters) {
    __shared__ int s_len[kMaxTables];
    __shared__ unsigned long long s_warp[kPlanThreads / 32];
    for (int j = threadIdx.x; j < m; j += blockDim.x) s_len[j] = tables[j].len;
    if (threadIdx.x < 2) counters[threadIdx.x] = 0ull;
    __syncthreads();
    // thread i owns queries [i * per, (i + 1) * per)
    const uint32_t per = (nq + kPlanThreads - 1) / kPlanThreads;
    const uint32_t q0 = threadIdx.x * per;
    const uint32_t q1 = min(nq, q0 + per);
    unsigned long long sum = 0;
    for (uint32_t q = q0; q < q1; ++q) sum += query_chunks(s_len, m, n, t_lo, t_hi, exh, q);
    // block exclusive scan of the per-thread sums
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (static_cast<int>(lane) >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (static_cast<int>(lane) >= o) w += v;
        }
        s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    unsigned long long run = (warp > 0 ? s_warp[warp - 1] : 0ull) + incl - sum;
    for (uint32_t q = q0; q < q1; ++q) {
        chunk_off[q] = run;
        run += query_chunks(s_len, m, n, t_lo, t_hi, exh, q);
    }
    if (threadIdx.x == kPlanThreads - 1) chunk_off[nq] = s_warp[kPlanThreads / 32 - 1];
}

// The same planning from per-query chunk counts that the stopping test wrote
// for this wave: an exclusive scan of `counts` into chunk_off[0..nq], in
// tiles of sixteen counts per thread, and the zeroed work counters.  One CTA.
__global__ void __launch_bounds__(kPlanThreads) plan_counts_kernel(const uint32_t* __restrict__ counts, uint32_t nq,
                                                                   uint64_t* __restrict__ chunk_off,
                                                                   unsigned long long* __restrict__ counters) {
    __shared__ unsigned long long s_warp[kPlanThreads / 32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x < 2) counters[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) s_carry = 0ull;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    // kPer counts per thread: up to 16K queries are one tile, every load in
    // flight at once (16-byte loads where the counts are 16-byte aligned)
    constexpr int kPer = 16;
    constexpr uint32_t kTile = kPer * kPlanThreads;
    const bool vec = (reinterpret_cast<uintptr_t>(counts) & 15u) == 0;
    for (uint32_t base = 0; base < nq; base += kTile) {
        const uint32_t i0 = base + kPer * threadIdx.x;
        uint32_t c[kPer];
        if (vec && i0 + kPer <= nq) {
#pragma unroll
            for (int r = 0; r < kPer; r += 4) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(counts + i0 + r));
                c[r] = v.x;
                c[r + 1] = v.y;
                c[r + 2] = v.z;
                c[r + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int r = 0; r < kPer; ++r) c[r] = i0 + r < nq ? __ldg(counts + i0 + r) : 0u;
        }
        unsigned long long sum = 0;
#pragma unroll
        for (int r = 0; r < kPer; ++r) sum += c[r];
        unsigned long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (static_cast<int>(lane) >= o) incl += v;
        }
        __syncthreads();   // the previous tile is done with s_warp and s_carry
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (static_cast<int>(lane) >= o) w += v;
            }
            s_warp[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        unsigned long long run = s_carry + (warp > 0 ? s_warp[warp - 1] : 0ull) + incl - sum;
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            if (i0 + r < nq) chunk_off[i0 + r] = run;
            run += c[r];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_warp[kPlanThreads / 32 - 1];
    }
    __syncthreads();
    if (threadIdx.x == 0) chunk_off[nq] = s_carry;
}

// Lookups of steps t0..t1 (sum of ring sizes, Eq. 1 per table).
__device__ __forceinline__ uint64_t steps_lookups(const int* s_len, int m, int t0, int t1) {
    uint64_t l = 0;
    for (int t = t0; t <= t1; ++t) l += binom(s_len[t % m], t / m);
    return l;
}

__device__ __forceinline__ uint32_t kk_of(const uint32_t* kq, uint32_t k_uniform, uint32_t q, uint64_t n) {
    const uint64_t k = kq ? kq[q] : k_uniform;
    return static_cast<uint32_t>(k < n ? k : n);
}

// Alg. 3 stopping test after step t_hi[q]; advances or retires each query.
//
// A query starts with bound = -1: its steps only fill the histogram.  Once
// min(k, n) codes are known the bound (an upper bound on the k-th distance)
// exists; the next launch then revisits steps 0..t to store the codes within
// the bound (without counting them again) together with step t+1.
__global__ void knn_stop_kernel(uint32_t nq, int qbits, uint64_t n, const uint32_t* __restrict__ kq,
                                uint32_t k_uniform, const uint32_t* __restrict__ hist, int32_t* __restrict__ t_lo,
                                int32_t* __restrict__ t_hi, int32_t* __restrict__ bound, int32_t* __restrict__ dk,
                                int32_t* __restrict__ hist_done, uint32_t* __restrict__ cnt1, uint32_t cap,
                                unsigned long long* __restrict__ qstats, unsigned int* __restrict__ active,
                                const TableDesc* __restrict__ tables, int m, uint8_t* __restrict__ exh,
                                long long scan_budget, uint32_t* __restrict__ next_chunks, int tail_from) {
    __shared__ int s_len[kMaxTables];
    for (int j = threadIdx.x; j < m; j += blockDim.x) s_len[j] = tables[j].len;
    __syncthreads();
    // one warp per query: lane l sums bins [l * per, (l + 1) * per)
    const uint32_t lane = lane_id();
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const int per = (qbits + 1 + 31) / 32;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const int t = t_hi[q];
        if (t < t_lo[q]) continue;  // retired earlier (warp-uniform)
        const uint32_t kk = kk_of(kq, k_uniform, q, n);
        const uint32_t* h = hist + static_cast<uint64_t>(q) * (qbits + 1);
        const int d0 = static_cast<int>(lane) * per;
        uint32_t part = 0;
        for (int i = 0; i < per; ++i)
            if (d0 + i <= qbits) part += h[d0 + i];
        const uint32_t incl = warp_inclusive_scan(part);   // codes at distances < (lane + 1) * per
        // first distance at which the cumulative count reaches min(k, n)
        int reach = -1;
        if (incl >= kk && incl - part < kk) {
            uint32_t cum = incl - part;
            for (int i = 0; i < per && reach < 0; ++i) {
                cum += h[d0 + i];
                if (cum >= kk) reach = d0 + i;
            }
        }
        const uint32_t who = __ballot_sync(0xFFFFFFFFu, reach >= 0);
        const int first_reach = who ? __shfl_sync(0xFFFFFFFFu, reach, __ffs(who) - 1) : -1;
        if (lane != 0) continue;
        const bool full = exh[q] != 0;  // this launch verified every remaining code
        if (first_reach >= 0 && (first_reach <= t || full)) {
            dk[q] = first_reach;            // every code within t bits (or all codes) is known
            t_lo[q] = t + 1;
            qstats[4ull * q + 3] = static_cast<unsigned long long>(t);
            if (bound[q] < 0) cnt1[q] = cap + 1;  // nothing stored yet: second pass collects
            next_chunks[q] = 0u;
        } else {
            hist_done[q] = t;
            if (bound[q] < 0 && first_reach >= 0) {
                bound[q] = first_reach;
                t_lo[q] = 0;                // revisit steps 0..t to store under the new bound
            } else {
                if (first_reach >= 0 && (bound[q] < 0 || first_reach < bound[q])) bound[q] = first_reach;
                t_lo[q] = t + 1;
            }
            // one Alg. 3 step per wave, two from step tail_from on (every code
            // within t bits is known after steps 0..t, so the next stopping
            // test is exact either way)
            const int steps = (tail_from >= 0 && t + 1 >= tail_from) ? 2 : 1;
            t_hi[q] = t + steps;
            // Once the next steps alone would push the lookups past the budget,
            // verifying every remaining code once is cheaper (Sec. 3 cost model:
            // a lookup costs about one candidate test).
            if (scan_budget >= 0 &&
                qstats[4ull * q] + steps_lookups(s_len, m, t + 1, t + steps) > static_cast<unsigned long long>(scan_budget))
                exh[q] = 1;
            // chunks of the next wave's steps, for its planning
            next_chunks[q] = static_cast<uint32_t>(query_chunks(s_len, m, n, t_lo, t_hi, exh, q));
            atomicAdd(active, 1u);
        }
    }
}

// Loop control of the graph executor, after the stopping test of a wave:
// counts the wave and lets the while node run its body again while a query is
// still active, no bounded wait has expired and fewer than max_waves waves ran.
__global__ void loop_control_kernel(cudaGraphConditionalHandle h, const unsigned int* __restrict__ active,
                                    const int* __restrict__ timeout, unsigned int* __restrict__ waves,
                                    unsigned int max_waves) {
    const unsigned int w = *waves + 1;
    *waves = w;
    cudaGraphSetConditional(h, (*active != 0u && *timeout == 0 && w < max_waves) ? 1u : 0u);
}

// ------------------------------------------------------------ selection
struct SelectArgs {
    uint32_t nq;
    uint64_t n;
    int q;
    const uint32_t* kq;
    uint32_t k_uniform;
    const uint64_t* out_off;
    const uint32_t* hist;
    const int32_t* dk;
    const uint64_t* buf1;
    uint32_t cap;
    const uint32_t* cnt1;
    const uint64_t* buf2;
    const uint64_t* base2;
    uint32_t* out_ids;
    int32_t* out_dist;
    int* err;
    const TableDesc* tables;   // lazy ids: an entry tagged t in bits 41..49 holds a position of table t - 1
    uint32_t smem_entries;     // shared-memory slots of the launch (a power of two >= min(kmax, n))
};

// Id of a stored entry (distance << 32 | id, or a tagged table position).
__device__ __forceinline__ uint64_t resolved_entry(uint64_t e, const TableDesc* tables) {
    const uint32_t tag = static_cast<uint32_t>(e >> kQueryShift);
    const uint64_t v = e & kEntryMask;
    if (tag == 0 || tables == nullptr) return v;
    return (v & (0x1FFull << 32)) | __ldg(tables[tag - 1].ids + static_cast<uint32_t>(v));
}

// In-place bitonic sort of res[0, S) ascending (S a power of two), one CTA.
__device__ __forceinline__ void bitonic_sort_smem(uint64_t* res, uint32_t S) {
    for (uint32_t size = 2; size <= S; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < S / 2; i += blockDim.x) {
                const uint32_t lo = 2 * i - (i & (stride - 1));
                const uint32_t hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t x = res[lo], y = res[hi];
                if ((x > y) == up) { res[lo] = y; res[hi] = x; }
            }
            __syncthreads();
        }
    }
}

// Top-min(k, n) of one query.  The histogram gives the number of entries
// within d_k (below + ties).  When they fit in shared memory (the usual case)
// one pass gathers them, with ids resolved, and a bitonic sort by (distance,
// id) orders them.  Otherwise ids are resolved in place, every entry closer
// than d_k is kept and the (k - #closer) smallest ids at d_k are found by a
// radix select on the id, then sorted the same way.
__global__ void __launch_bounds__(256) select_kernel(SelectArgs a) {
    extern __shared__ uint64_t res[];
    __shared__ unsigned int s_n, s_hist[256];
    __shared__ uint32_t s_prefix, s_remaining;
    __shared__ unsigned long long s_below;
    const uint32_t q = blockIdx.x;
    const uint32_t k = a.kq ? a.kq[q] : a.k_uniform;
    const uint64_t ob = a.out_off ? a.out_off[q] : static_cast<uint64_t>(q) * a.k_uniform;
    const uint32_t kk = static_cast<uint32_t>(k < a.n ? k : a.n);
    uint32_t* oid = a.out_ids + ob;
    int32_t* odist = a.out_dist + ob;
    if (kk == 0) {
        for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) { oid[i] = kPadId; odist[i] = -1; }
        return;
    }
    const int dk = a.dk[q];
    const uint32_t* h = a.hist + static_cast<uint64_t>(q) * (a.q + 1);
    if (threadIdx.x < 32) {
        // codes closer than d_k: the histogram below d_k, summed by warp 0
        unsigned long long below = 0;
        for (int d = static_cast<int>(threadIdx.x); d < dk; d += 32) below += h[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) below += __shfl_down_sync(0xFFFFFFFFu, below, o);
        if (threadIdx.x == 0) {
            s_below = below;
            s_n = 0;
        }
    }
    __syncthreads();
    const uint32_t ties = h[dk];
    const uint32_t quota = kk - static_cast<uint32_t>(s_below);
    const uint64_t* src;
    uint64_t nsrc;
    // Tagged table positions exist only in the bounded buffer of the k-NN
    // waves; the second-pass buffer holds ids already (its upper bits carry
    // the query index, not a table).
    const TableDesc* tables = nullptr;
    const uint32_t c1 = a.cnt1 ? a.cnt1[q] : 0xFFFFFFFFu;
    if (a.cnt1 && c1 <= a.cap) {
        src = a.buf1 + static_cast<uint64_t>(q) * a.cap;
        nsrc = c1;
        tables = a.tables;
    } else {
        src = a.buf2 + a.base2[q];
        nsrc = s_below + ties;
    }
    const uint64_t within = s_below + ties;
    if (within <= a.smem_entries) {
        // one pass: the entries within d_k, ids resolved, into shared memory
        // (four loads per thread in flight before any is used)
        for (uint64_t i0 = threadIdx.x; i0 < nsrc; i0 += 4ull * blockDim.x) {
            uint64_t e[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint64_t i = i0 + static_cast<uint64_t>(r) * blockDim.x;
                e[r] = i < nsrc ? src[i] : ~0ull;   // ~0: distance field above any d_k
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (static_cast<int>((e[r] & kEntryMask) >> 32) <= dk) {
                    const unsigned int slot = atomicAdd(&s_n, 1u);
                    if (slot < within) res[slot] = resolved_entry(e[r], tables);
                }
            }
        }
        __syncthreads();
        if (s_n != within) {
            if (threadIdx.x == 0) atomicExch(a.err, 1);
            return;
        }
        uint32_t S = 1;
        while (S < within) S <<= 1;
        for (uint32_t i = static_cast<uint32_t>(within) + threadIdx.x; i < S; i += blockDim.x) res[i] = ~0ull;
        __syncthreads();
        bitonic_sort_smem(res, S);
        for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
            if (i < kk) {
                oid[i] = static_cast<uint32_t>(res[i]);
                odist[i] = static_cast<int32_t>(res[i] >> 32);
            } else {
                oid[i] = kPadId;
                odist[i] = -1;
            }
        }
        return;
    }
    if (tables) {
        // large tie sets: ids of the entries within d_k resolved in place
        uint64_t* w = const_cast<uint64_t*>(src);
        for (uint64_t i = threadIdx.x; i < nsrc; i += blockDim.x) {
            const uint64_t e = w[i];
            if ((e >> kQueryShift) != 0 && static_cast<int>((e & kEntryMask) >> 32) <= dk)
                w[i] = resolved_entry(e, tables);
        }
        __syncthreads();
    }
    const bool take_all_ties = quota >= ties;
    uint32_t P = 1;
    while (P < kk) P <<= 1;
    for (uint64_t i = threadIdx.x; i < nsrc; i += blockDim.x) {
        const uint64_t e = src[i] & kEntryMask;
        const int d = static_cast<int>(e >> 32);
        if (d < dk || (d == dk && take_all_ties)) {
            const unsigned int slot = atomicAdd(&s_n, 1u);
            if (slot < P) res[slot] = e;
        }
    }
    if (!take_all_ties) {
        if (threadIdx.x == 0) { s_prefix = 0; s_remaining = quota; }
        for (int pass = 3; pass >= 0; --pass) {
            s_hist[threadIdx.x] = 0;
            __syncthreads();
            const int hi_shift = 8 * (pass + 1);
            const uint32_t prefix = s_prefix;
            for (uint64_t i = threadIdx.x; i < nsrc; i += blockDim.x) {
                const uint64_t e = src[i] & kEntryMask;
                if (static_cast<int>(e >> 32) != dk) continue;
                const uint32_t id = static_cast<uint32_t>(e);
                if (pass < 3 && (id >> hi_shift) != (prefix >> hi_shift)) continue;
                atomicAdd(&s_hist[(id >> (8 * pass)) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t rem = s_remaining, digit = 0;
                for (; digit < 255; ++digit) {
                    if (s_hist[digit] >= rem) break;
                    rem -= s_hist[digit];
                }
                s_remaining = rem;
                s_prefix = prefix | (digit << (8 * pass));
            }
            __syncthreads();
        }
        const uint32_t xid = s_prefix;  // the quota-th smallest tied id
        for (uint64_t i = threadIdx.x; i < nsrc; i += blockDim.x) {
            const uint64_t e = src[i] & kEntryMask;
            if (static_cast<int>(e >> 32) == dk && static_cast<uint32_t>(e) <= xid) {
                const unsigned int slot = atomicAdd(&s_n, 1u);
                if (slot < P) res[slot] = e;
            }
        }
    }
    __syncthreads();
    if (s_n != kk) {
        if (threadIdx.x == 0) atomicExch(a.err, 1);
        return;
    }
    for (uint32_t i = kk + threadIdx.x; i < P; i += blockDim.x) res[i] = ~0ull;
    __syncthreads();
    bitonic_sort_smem(res, P);
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
        if (i < kk) {
            oid[i] = static_cast<uint32_t>(res[i]);
            odist[i] = static_cast<int32_t>(res[i] >> 32);
        } else {
            oid[i] = kPadId;
            odist[i] = -1;
        }
    }
}

// d_k and the buffer size of each overflowed query (second pass).
__global__ void phase2_plan_kernel(uint32_t nq, int qbits, const uint32_t* __restrict__ hist,
                                   const int32_t* __restrict__ dk, const uint32_t* __restrict__ cnt1, uint32_t cap,
                                   int32_t* __restrict__ t_lo, int32_t* __restrict__ t_hi,
                                   int32_t* __restrict__ bound, uint64_t* __restrict__ need,
                                   unsigned int* __restrict__ n_over, const TableDesc* __restrict__ tables, int m,
                                   uint8_t* __restrict__ exh, long long scan_budget) {
    __shared__ int s_len[kMaxTables];
    for (int j = threadIdx.x; j < m; j += blockDim.x) s_len[j] = tables[j].len;
    __syncthreads();
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x) {
        if (q == nq) { need[q] = 0; continue; }
        const bool over = cnt1[q] > cap;
        uint64_t c = 0;
        if (over) {
            const uint32_t* h = hist + static_cast<uint64_t>(q) * (qbits + 1);
            for (int d = 0; d <= dk[q]; ++d) c += h[d];
            atomicAdd(n_over, 1u);
        }
        need[q] = c;
        t_lo[q] = 0;
        t_hi[q] = over ? dk[q] : -1;
        bound[q] = dk[q];
        exh[q] = (over && scan_budget >= 0 &&
                  steps_lookups(s_len, m, 0, dk[q]) > static_cast<unsigned long long>(scan_budget)) ? 1 : 0;
    }
}

__global__ void init_knn_kernel(uint32_t nq, uint64_t n, int32_t* t_lo, int32_t* t_hi, int32_t* bound,
                                int32_t* dk, int32_t* hist_done, uint32_t* chunks) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        t_lo[q] = 0;
        t_hi[q] = n > 0 ? 0 : -1;
        bound[q] = -1;
        dk[q] = 0;
        hist_done[q] = -1;
        chunks[q] = n > 0 ? 1u : 0u;   // step 0: ring 0 of table 0, one key
    }
}

// A first bound on each query's k-th distance, before any step runs: one warp
// per query measures up to `probe` entries of the query's own bucket in every
// table (the buckets of its first m steps).  Any min(k, n) codes of the
// database bound the k-th distance from above, so the smallest D with at
// least min(k, n) probed codes within D is a valid bound; queries that probe
// fewer codes keep bound = -1 (histogram-only steps until one exists).

#ifndef MIH_PROBE_BATCH
#define MIH_PROBE_BATCH 8
#endif
constexpr int kProbeBatch = MIH_PROBE_BATCH;   // records per lane in flight in the bound probe

template <int W>
__global__ void __launch_bounds__(256) bound_probe_kernel(const TableDesc* __restrict__ tables, int m, int qbits,
                                                          const uint64_t* __restrict__ codes,
                                                          const uint64_t* __restrict__ queries, uint32_t nq,
                                                          uint64_t n, const uint32_t* __restrict__ kq,
                                                          uint32_t k_uniform, uint32_t probe,
                                                          int32_t* __restrict__ bound) {
    __shared__ uint32_t s_hist[8][kHistBins];
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    uint32_t* h = s_hist[warp];
    for (int d = lane; d <= qbits; d += 32) h[d] = 0;
    __syncwarp();
    const uint32_t q = blockIdx.x * 8 + warp;
    if (q >= nq) return;
    const Code<W> g = load_query<W>(queries, q);
    // the query's own bucket in every table: lane l looks up tables
    // j0 + l, all 32 lookups in flight together
    uint32_t lb = 0, le = 0;
    for (int j = 0; j < m; ++j) {
        if ((j & 31) == 0) {
            lb = le = 0;
            const int jl = j + static_cast<int>(lane);
            if (jl < m) lookup_bucket(tables[jl], substring_bits<W>(g, tables[jl].off, tables[jl].len), lb, le);
        }
        const TableDesc& t = tables[j];
        const uint32_t b = __shfl_sync(0xFFFFFFFFu, lb, j & 31);
        const uint32_t e = __shfl_sync(0xFFFFFFFFu, le, j & 31);
        const uint32_t end = min(e, b + probe);
        if (t.codes && t.rec_words != 0) {
            // Inline records (every substring one 32-bit word): the table's own
            // word equals the query's in its own bucket, so the distance is the
            // popcount over the record's words (the code's other words), and a
            // code filed under the query's key in table jj < j has record word
            // jj equal to the query's.
            constexpr int R = 2 * W - 1;
            uint32_t g32[2 * W], gq[R];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                g32[2 * w] = static_cast<uint32_t>(g.w[w]);
                g32[2 * w + 1] = static_cast<uint32_t>(g.w[w] >> 32);
            }
#pragma unroll
            for (int i = 0; i < R; ++i) gq[i] = i < j ? g32[i] : g32[i + 1];
            const uint32_t* rec = reinterpret_cast<const uint32_t*>(t.codes);
            // kProbeBatch records per lane per round, their loads in flight together
            for (uint64_t p0 = b; p0 < end; p0 += 32u * kProbeBatch) {
                uint32_t wv[kProbeBatch][R];
#pragma unroll
                for (int u = 0; u < kProbeBatch; ++u) {
                    const uint64_t p = p0 + 32u * u + lane;
#pragma unroll
                    for (int i = 0; i < R; ++i) wv[u][i] = p < end ? __ldg(rec + p * R + i) : 0u;
                }
#pragma unroll
                for (int u = 0; u < kProbeBatch; ++u) {
                    if (p0 + 32u * u + lane >= end) continue;
                    int d = 0;
                    bool first = true;
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        const uint32_t x = wv[u][i] ^ gq[i];
                        d += __popc(x);
                        if (i < j && x == 0u) first = false;
                    }
                    if (first) atomicAdd(&h[d], 1u);
                }
            }
            continue;
        }
        for (uint32_t p = b + lane; p < end; p += 32) {
            const Code<W> c = t.codes ? load_code<W>(t.codes, p) : load_code<W>(codes, __ldg(t.ids + p));
            // a code also filed under the query's key in an earlier table is
            // counted there or not at all: the count never exceeds the number
            // of distinct codes, so the bound stays valid
            Code<W> x;
#pragma unroll
            for (int w = 0; w < W; ++w) x.w[w] = c.w[w] ^ g.w[w];
            bool first = true;
            for (int jj = 0; jj < j && first; ++jj)
                if (substring_bits<W>(x, tables[jj].off, tables[jj].len) == 0u) first = false;
            if (first) atomicAdd(&h[hamming<W>(c, g)], 1u);
        }
    }
    __syncwarp();
    if (lane == 0) {
        const uint64_t kv = kq ? kq[q] : k_uniform;
        const uint32_t kk = static_cast<uint32_t>(kv < n ? kv : n);
        uint32_t cum = 0;
        int bnd = -1;
        for (int d = 0; d <= qbits; ++d) {
            cum += h[d];
            if (cum >= kk) {
                bnd = d;
                break;
            }
        }
        bound[q] = bnd;
    }
}

__global__ void init_range_kernel(uint32_t nq, int32_t lo, int32_t hi, int32_t bnd, int32_t* t_lo, int32_t* t_hi,
                                  int32_t* bound) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        t_lo[q] = lo;
        t_hi[q] = hi;
        bound[q] = bnd;
    }
}

__global__ void widen_counts_kernel(const uint32_t* __restrict__ cnt, uint32_t nq, uint64_t* __restrict__ out) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x)
        out[q] = q < nq ? cnt[q] : 0ull;
}

__global__ void split_entries_kernel(const uint64_t* __restrict__ e, uint64_t total, uint32_t* __restrict__ ids,
                                     int32_t* __restrict__ dist) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t v = e[i];
        ids[i] = static_cast<uint32_t>(v);
        dist[i] = static_cast<int32_t>((v >> 32) & 0x1FFu);
    }
}

// Validation of per-query k: min, max and CSR consistency.
__global__ void check_k_kernel(uint32_t nq, const uint32_t* __restrict__ kq, const uint64_t* __restrict__ off,
                               unsigned int* __restrict__ out /* [min, max, bad] */) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t k = kq[q];
        atomicMin(&out[0], k);
        atomicMax(&out[1], k);
        if (off && off[q + 1] - off[q] != k) atomicOr(&out[2], 1u);
    }
}

unsigned grid1(uint64_t n) {
    uint64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return static_cast<unsigned>(g ? g : 1);
}

// Persistent grids: as many CTAs as fit on the GPU at once.  The occupancy
// queries and the shared-memory attribute run once per kernel, before any
// launch (and so never while a stream is being captured).
struct GridCfg {
    int bps = 0, bps_big = 0, bps_stream[kStreamVariants] = {};
};

template <int W, int MODE, bool ALIGNED, class Shape>
mih_status init_stream_cfg(int* bps) {
    int x = 0;
    MIH_CUDA(cudaFuncSetAttribute(search_stream_kernel<W, MODE, ALIGNED, Shape>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(Shape::kSmem)));
    MIH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x, search_stream_kernel<W, MODE, ALIGNED, Shape>,
                                                           Shape::kWarps * 32, Shape::kSmem));
    *bps = x > 0 ? x : 1;
    return MIH_OK;
}

template <int W, int MODE, bool ALIGNED>
mih_status init_search_cfg(GridCfg* cfg) {
    int v = 0, w = 0;
    MIH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, search_kernel<W, MODE, ALIGNED>, kSearchThreads, 0));
    MIH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&w, search_big_kernel<W, MODE, ALIGNED>, kSearchThreads,
                                                           0));
    MIH_TRY((init_stream_cfg<W, MODE, ALIGNED, Shape0>(&cfg->bps_stream[0])));
    if constexpr (MODE == kModeKnn) {
        MIH_TRY((init_stream_cfg<W, MODE, ALIGNED, Shape1>(&cfg->bps_stream[1])));
        MIH_TRY((init_stream_cfg<W, MODE, ALIGNED, Shape2>(&cfg->bps_stream[2])));
    }
    cfg->bps_big = w > 0 ? w : 1;
    cfg->bps = v > 0 ? v : 1;
    return MIH_OK;
}

// Once per device and kernel variant (the shared-memory attribute is a
// per-device setting), safe when several host threads search at once.
template <int W, int MODE, bool ALIGNED>
mih_status search_cfg(const GridCfg** out) {
    constexpr int kDevs = 64;
    static GridCfg cfg[kDevs];
    static std::once_flag once[kDevs];
    static mih_status st[kDevs];
    int d = 0;
    MIH_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= kDevs) {
        set_error("device ordinal %d out of range", d);
        return MIH_EINVAL;
    }
    std::call_once(once[d], [d] { st[d] = init_search_cfg<W, MODE, ALIGNED>(&cfg[d]); });
    if (st[d] != MIH_OK) {
        set_error("search kernel launch configuration failed on device %d", d);
        return st[d];
    }
    *out = &cfg[d];
    return MIH_OK;
}

template <int W, int MODE, bool ALIGNED>
mih_status launch_search_wa(const SearchArgs& a0, const DeviceInfo& dev, cudaStream_t s, bool launch, bool spans) {
    const GridCfg* cfg = nullptr;
    MIH_TRY((search_cfg<W, MODE, ALIGNED>(&cfg)));
    if (!launch) return MIH_OK;
    // the slice kernel's shape (k-NN waves only) and the slice size it takes
    SearchArgs a = a0;
    a.variant = (MODE == kModeKnn && a.inline_codes && a0.variant > 0 && a0.variant < kStreamVariants) ? a0.variant : 0;
    a.slice_entries = a.inline_codes ? variant_slice_entries<W, ALIGNED>(a.variant) : kSliceEntries;
    {
        KernelSpan ks(s, MIH_PROF_CHUNK, spans);
        search_kernel<W, MODE, ALIGNED><<<dev.sms * cfg->bps, kSearchThreads, 0, s>>>(a);
        MIH_LAUNCH_CHECK();
    }
    KernelSpan ks(s, MIH_PROF_SLICE, spans);
    if (a.inline_codes) {
        const unsigned grid = dev.sms * cfg->bps_stream[a.variant];
        if constexpr (MODE == kModeKnn) {
            if (a.variant == 1)
                search_stream_kernel<W, MODE, ALIGNED, Shape1><<<grid, Shape1::kWarps * 32, Shape1::kSmem, s>>>(a);
            else if (a.variant == 2)
                search_stream_kernel<W, MODE, ALIGNED, Shape2><<<grid, Shape2::kWarps * 32, Shape2::kSmem, s>>>(a);
            else
                search_stream_kernel<W, MODE, ALIGNED, Shape0><<<grid, Shape0::kWarps * 32, Shape0::kSmem, s>>>(a);
        } else {
            search_stream_kernel<W, MODE, ALIGNED, Shape0><<<grid, Shape0::kWarps * 32, Shape0::kSmem, s>>>(a);
        }
    } else {
        search_big_kernel<W, MODE, ALIGNED><<<dev.sms * cfg->bps_big, kSearchThreads, 0, s>>>(a);
    }
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

template <int W, int MODE>
mih_status launch_search_w(const SearchArgs& a, const DeviceInfo& dev, cudaStream_t s, bool launch, bool spans) {
    // every substring is one whole 32-bit word exactly when m = 2W
    if (a.m == 2 * W) return launch_search_wa<W, MODE, true>(a, dev, s, launch, spans);
    return launch_search_wa<W, MODE, false>(a, dev, s, launch, spans);
}

// Launches the chunk and slice kernels (launch = false: only their one-time
// configuration); spans = per-kernel timing events (never while capturing).
template <int MODE>
mih_status launch_search(const SearchArgs& a, int W, const DeviceInfo& dev, cudaStream_t s, bool launch = true,
                         bool spans = false) {
    if (W == 1) return launch_search_w<1, MODE>(a, dev, s, launch, spans);
    if (W == 2) return launch_search_w<2, MODE>(a, dev, s, launch, spans);
    return launch_search_w<4, MODE>(a, dev, s, launch, spans);
}

#ifndef MIH_BIG_CAP_LOG2
#define MIH_BIG_CAP_LOG2 25
#endif

// Per-launch work state (chunk offsets, counters, big list).
struct Plan {
    uint64_t* chunk_off = nullptr;           // [nq + 1]
    unsigned long long* counters = nullptr;  // [0] chunk_next; [1] big_count|big_next (as uint32 x2)
    BigSlice* big = nullptr;
    uint32_t big_cap = 0;
    int* timeout = nullptr;                  // raised by a bounded wait that gave up
    uint64_t* scan_tmp = nullptr;            // block sums of the chunk-offset scan (graph mode)
};

mih_status plan_alloc(Plan& p, uint32_t nq, Workspace& ws) {
    MIH_TRY(ws.alloc(&p.chunk_off, static_cast<size_t>(nq) + 1));
    MIH_TRY(ws.alloc(&p.counters, 2));
    // Slice descriptors per wave (16 B each).  A wave over many medium buckets
    // (1e9 uniform 64-bit codes, 21-bit substrings: ~500 codes per bucket)
    // makes ten million slices or more; a bucket whose slices do not fit is
    // scanned by the chunk kernel's warp itself, which is far slower.
    p.big_cap = 1u << MIH_BIG_CAP_LOG2;
    MIH_TRY(ws.alloc(&p.big, p.big_cap));
    MIH_TRY(ws.alloc(&p.timeout, 1));
    MIH_CUDA(cudaMemsetAsync(p.timeout, 0, sizeof(int), ws.stream()));
    return MIH_OK;
}

// MIH_ETIMEOUT if a kernel of this call gave up a bounded wait (syncs).
mih_status check_timeout(const Plan& p, cudaStream_t s) {
    int h = 0;
    MIH_CUDA(cudaMemcpyAsync(&h, p.timeout, sizeof(int), cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    if (h) {
        set_error("a bounded wait on a bulk copy expired");
        return MIH_ETIMEOUT;
    }
    return MIH_OK;
}

// Compute chunk offsets for the current step ranges and run one search launch.
// With a capture stream cs the launches are recorded into a graph body on cs
// (nothing is allocated and no event is recorded); else they run on the
// workspace's stream.
template <int MODE>
mih_status run_wave(const mih_index* ix, SearchArgs a, Plan& p, const int32_t* t_lo, const int32_t* t_hi,
                    const DeviceInfo& dev, Workspace& ws, cudaStream_t cs = nullptr, const uint32_t* counts = nullptr) {
    const bool in_graph = cs != nullptr;
    cudaStream_t s = in_graph ? cs : ws.stream();
    {
        KernelSpan plan_span(s, MIH_PROF_PLAN, !in_graph);
        if (counts && static_cast<uint64_t>(a.nq) + 1 <= kPlanOneBlockMax) {
            plan_counts_kernel<<<1, kPlanThreads, 0, s>>>(counts, a.nq, p.chunk_off, p.counters);
            MIH_LAUNCH_CHECK();
        } else if (static_cast<uint64_t>(a.nq) + 1 <= kPlanOneBlockMax) {
            plan_scan_kernel<<<1, kPlanThreads, 0, s>>>(ix->dev_tables, ix->m, a.nq, ix->n, t_lo, t_hi, a.exh,
                                                        p.chunk_off, p.counters);
            MIH_LAUNCH_CHECK();
        } else {
            plan_chunks_kernel<<<grid1(a.nq + 1), 256, 0, s>>>(ix->dev_tables, ix->m, a.nq, ix->n, t_lo, t_hi,
                                                              a.exh, p.chunk_off);
            MIH_LAUNCH_CHECK();
            if (in_graph)
                MIH_TRY(scan_exclusive_u64_pre(p.chunk_off, p.chunk_off, static_cast<size_t>(a.nq) + 1, p.scan_tmp,
                                               s));
            else
                MIH_TRY(scan_exclusive_u64(p.chunk_off, p.chunk_off, static_cast<size_t>(a.nq) + 1, ws));
            MIH_CUDA(cudaMemsetAsync(p.counters, 0, 2 * sizeof(unsigned long long), s));
        }
    }
    a.t_lo = t_lo;
    a.t_hi = t_hi;
    a.chunk_off = p.chunk_off;
    a.chunk_next = p.counters;
    a.big = p.big;
    a.big_cap = p.big_cap;
    a.big_count = reinterpret_cast<unsigned int*>(p.counters + 1);
    a.big_next = a.big_count + 1;
    a.inline_codes = ix->inline_codes ? 1 : 0;
    a.timeout = p.timeout;
    a.wait_ns = wait_limit_ns();
    a.wait_test = wait_test_expire() ? 1 : 0;
    a.variant = ix->slice_shape;
    if (in_graph) return launch_search<MODE>(a, ix->W, dev, s);   // events cannot sit in a loop body
    main_kernel_begin(s);
    const mih_status st = launch_search<MODE>(a, ix->W, dev, s, true, true);
    main_kernel_end(s);
    return st;
}

// Lookups after which a query switches to one verification pass over all
// codes: scan_factor * n (default 4 n); -1 = never.
long long scan_budget(const mih_index* ix) {
    if (ix->scan_factor < 0) return -1;
    const long long f = ix->scan_factor == 0 ? 4 : ix->scan_factor;
    return f * static_cast<long long>(ix->n);
}

unsigned long long host_binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned long long c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

// A non-blocking stream per device and host thread on which graph bodies are
// captured (capture cannot run on the legacy default stream a caller may use).
mih_status capture_stream(cudaStream_t* out) {
    constexpr int kDevs = 64;
    static thread_local cudaStream_t cs[kDevs] = {};
    int d = 0;
    MIH_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= kDevs) {
        set_error("device ordinal %d out of range", d);
        return MIH_EINVAL;
    }
    if (!cs[d]) MIH_CUDA(cudaStreamCreateWithFlags(&cs[d], cudaStreamNonBlocking));
    *out = cs[d];
    return MIH_OK;
}

struct GraphGuard {
    cudaGraph_t g = nullptr;
    ~GraphGuard() {
        if (g) cudaGraphDestroy(g);
    }
};

// One instantiated wave graph per device and host thread, reused across calls:
// each call captures its body anew and updates the cached executable in place
// (cudaGraphExecUpdate keeps the instantiation when the topology matches, and
// a thread's previous launch has finished because every call synchronises its
// stream before returning); when the update is refused the call instantiates
// a new one.
struct ExecCache {
    static constexpr int kDevs = 64;
    cudaGraphExec_t e[kDevs] = {};
    ~ExecCache() {
        for (cudaGraphExec_t x : e)
            if (x) cudaGraphExecDestroy(x);
    }
};
thread_local ExecCache t_exec;

// Runs body(cs) -- launches recorded on the capture stream cs -- as the body of
// a while-loop graph node on stream s, the first iteration unconditionally.
// The body must end with loop_control_kernel on `h`.  Returns the launches
// recorded in one body; the graph launch counts as one main launch.  The
// caller synchronises before destroying `gg`.
template <class Body>
mih_status launch_while_graph(GraphGuard& gg, cudaStream_t s, uint64_t* body_launches, Body&& body) {
    cudaStream_t cs = nullptr;
    MIH_TRY(capture_stream(&cs));
    MIH_CUDA(cudaGraphCreate(&gg.g, 0));
    cudaGraphConditionalHandle h;
    MIH_CUDA(cudaGraphConditionalHandleCreate(&h, gg.g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MIH_CUDA(cudaGraphAddNode(&node, gg.g, nullptr, nullptr, 0, &np));
    cudaGraph_t loop_body = np.conditional.phGraph_out[0];
    const uint64_t l0 = launches_so_far();
    MIH_CUDA(cudaStreamBeginCaptureToGraph(cs, loop_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const mih_status st = body(cs, h);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    if (st != MIH_OK) {
        cudaGetLastError();
        return st;
    }
    MIH_CUDA(ce);
    *body_launches = launches_so_far() - l0;
    int d = 0;
    MIH_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= ExecCache::kDevs) {
        set_error("device ordinal %d out of range", d);
        return MIH_EINVAL;
    }
    cudaGraphExec_t& exec = t_exec.e[d];
    bool updated = false;
    if (exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(exec, gg.g, &info) == cudaSuccess) {
            updated = true;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (!updated) MIH_CUDA(cudaGraphInstantiate(&exec, gg.g, 0));
    main_kernel_begin(s);  // the span covers every wave (with its planning and stopping test)
    const cudaError_t le = cudaGraphLaunch(exec, s);
    main_kernel_end(s);
    MIH_CUDA(le);
    return MIH_OK;
}

mih_status check_flag(const int* err, const char* what, cudaStream_t s) {
    int h = 0;
    MIH_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    if (h) {
        set_error("%s", what);
        return MIH_EINTERNAL;
    }
    return MIH_OK;
}

mih_status validate_common(const mih_index* ix, const uint64_t* queries, uint32_t nq) {
    if (!ix) {
        set_error("index is NULL");
        return MIH_EINVAL;
    }
    if (nq > (1u << 23)) {
        set_error("nq must be at most 2^23");
        return MIH_EINVAL;
    }
    int dev = 0;
    MIH_CUDA(cudaGetDevice(&dev));
    if (dev != ix->device) {
        set_error("index was built on device %d, current device is %d", ix->device, dev);
        return MIH_EINVAL;
    }
    if (nq > 0) MIH_TRY(check_device_ptr(queries, "queries"));
    return MIH_OK;
}

// With optimised substrings the index searches bit-permuted codes: the
// queries get the same permutation, in scratch memory, before any kernel.
mih_status permute_queries(const mih_index* ix, const uint64_t** queries, uint32_t nq, Workspace& ws) {
    if (!ix->bit_order) return MIH_OK;
    uint64_t* qp;
    MIH_TRY(ws.alloc(&qp, static_cast<size_t>(nq) * ix->W));
    MIH_TRY(permute_codes(*queries, qp, nq, ix->q, ix->bit_order, ws.stream()));
    *queries = qp;
    return MIH_OK;
}

}  // namespace

// ---------------------------------------------------------------- exported
// k validation shared with the linear scan: fills *kmax.
mih_status check_k_args(uint32_t nq, const uint32_t* k, uint32_t k_uniform, const uint64_t* out_offsets,
                        const uint32_t* out_ids, const int32_t* out_dist, uint32_t* kmax, Workspace& ws) {
    if (nq == 0) {
        *kmax = k ? 0 : k_uniform;
        return MIH_OK;
    }
    MIH_TRY(check_device_ptr(out_ids, "out_ids"));
    MIH_TRY(check_device_ptr(out_dist, "out_dist"));
    if (!k) {
        if (k_uniform < 1 || k_uniform > MIH_MAX_K) {
            set_error("k must be in [1, %u] (got %u)", MIH_MAX_K, k_uniform);
            return MIH_EINVAL;
        }
        if (out_offsets) {
            set_error("out_offsets must be NULL when k is uniform");
            return MIH_EINVAL;
        }
        *kmax = k_uniform;
        return MIH_OK;
    }
    MIH_TRY(check_device_ptr(k, "k"));
    MIH_TRY(check_device_ptr(out_offsets, "out_offsets"));
    unsigned int* d;
    MIH_TRY(ws.alloc(&d, 3));
    unsigned int init[3] = {0xFFFFFFFFu, 0u, 0u};
    MIH_CUDA(cudaMemcpyAsync(d, init, sizeof(init), cudaMemcpyHostToDevice, ws.stream()));
    check_k_kernel<<<grid1(nq), 256, 0, ws.stream()>>>(nq, k, out_offsets, d);
    MIH_LAUNCH_CHECK();
    unsigned int h[3];
    MIH_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, ws.stream()));
    MIH_CUDA(cudaStreamSynchronize(ws.stream()));
    if (h[0] < 1 || h[1] > MIH_MAX_K) {
        set_error("every k must be in [1, %u] (min %u, max %u)", MIH_MAX_K, h[0], h[1]);
        return MIH_EINVAL;
    }
    if (h[2]) {
        set_error("out_offsets[i+1] - out_offsets[i] must equal k[i]");
        return MIH_EINVAL;
    }
    *kmax = h[1];
    return MIH_OK;
}

// Shared-memory slots of a selection launch: room for min(kmax, n) results
// and for the usual number of entries within d_k (one-pass selection).
constexpr uint32_t kSelectSmemEntries = 4096;

uint32_t select_slots(const SelectInputs& in) {
    uint32_t P = 1;
    const uint64_t kk_max = std::min<uint64_t>(in.kmax, in.n);
    while (P < kk_max) P <<= 1;
    return P > kSelectSmemEntries ? P : kSelectSmemEntries;
}

SelectArgs select_args(const SelectInputs& in, int* err, uint32_t slots) {
    SelectArgs a;
    a.nq = in.nq;
    a.n = in.n;
    a.q = in.q;
    a.kq = in.kq;
    a.k_uniform = in.k_uniform;
    a.out_off = in.out_off;
    a.hist = in.hist;
    a.dk = in.dk;
    a.buf1 = in.buf1;
    a.cap = in.cap;
    a.cnt1 = in.cnt1;
    a.buf2 = in.buf2;
    a.base2 = in.base2;
    a.out_ids = in.out_ids;
    a.out_dist = in.out_dist;
    a.err = err;
    a.tables = in.tables;
    a.smem_entries = slots;
    return a;
}

mih_status launch_select(const SelectInputs& in, Workspace& ws) {
    if (in.nq == 0) return MIH_OK;
    const uint32_t slots = select_slots(in);
    const size_t smem = static_cast<size_t>(slots) * sizeof(uint64_t);
    if (smem > 48 * 1024) MIH_CUDA(cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        static_cast<int>(smem)));
    int* err;
    MIH_TRY(ws.alloc(&err, 1));
    MIH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ws.stream()));
    const SelectArgs a = select_args(in, err, slots);
    {
        KernelSpan ks(ws.stream(), MIH_PROF_SELECT);
        select_kernel<<<in.nq, 256, smem, ws.stream()>>>(a);
        MIH_LAUNCH_CHECK();
    }
    int herr = 0;
    MIH_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ws.stream()));
    MIH_CUDA(cudaStreamSynchronize(ws.stream()));
    if (herr) {
        set_error("select: collected entry count differs from min(k, n)");
        return MIH_EINTERNAL;
    }
    return MIH_OK;
}

// Selection with a caller-provided error flag (zeroed by the caller); no
// allocation.  Only while the launch needs at most 48 KB of shared memory.
mih_status launch_select_noalloc(const SelectInputs& in, int* err, cudaStream_t s) {
    if (in.nq == 0) return MIH_OK;
    const uint32_t slots = select_slots(in);
    const size_t smem = static_cast<size_t>(slots) * sizeof(uint64_t);
    if (smem > 48 * 1024) {
        set_error("select: k too large for the fixed-scratch path");
        return MIH_EINVAL;
    }
    const SelectArgs a = select_args(in, err, slots);
    select_kernel<<<in.nq, 256, smem, s>>>(a);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

uint32_t knn_buffer_cap(uint32_t kmax, uint32_t nq) {
    uint64_t c = 16ull * kmax;
    if (c < 16384) c = 16384;
    // at most 2 GiB of buffers per call, but never below 4096 slots
    const uint64_t mem_cap = (1ull << 31) / (8ull * (nq > 0 ? nq : 1));
    if (c > mem_cap) c = mem_cap < 4096 ? 4096 : mem_cap;
    if (c > 65536) c = 65536;
    return static_cast<uint32_t>(c);
}

}  // namespace mih

using namespace mih;

extern "C" {

mih_status mih_knn(const mih_index* ix, const uint64_t* queries, uint32_t nq, const uint32_t* k, uint32_t k_uniform,
                   const uint64_t* out_offsets, uint32_t* out_ids, int32_t* out_dist, uint64_t* query_stats,
                   mih_stats* stats, void* stream) {
    clear_error();
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallScope scope(s);
    MIH_TRY(validate_common(ix, queries, nq));
    Workspace ws(s);
    uint32_t kmax = 0;
    MIH_TRY(check_k_args(nq, k, k_uniform, out_offsets, out_ids, out_dist, &kmax, ws));
    if (query_stats) MIH_TRY(check_device_ptr(query_stats, "query_stats"));
    if (nq == 0) return MIH_OK;
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    const int qb = ix->q;
    const uint32_t cap = knn_buffer_cap(kmax, nq);
    MIH_TRY(permute_queries(ix, &queries, nq, ws));

    int32_t *t_lo, *t_hi, *bound, *dk;
    uint32_t *hist, *cnt1;
    uint64_t* buf1;
    unsigned long long* qstats;
    unsigned int* active;
    MIH_TRY(ws.alloc(&t_lo, nq));
    MIH_TRY(ws.alloc(&t_hi, nq));
    MIH_TRY(ws.alloc(&bound, nq));
    MIH_TRY(ws.alloc(&dk, nq));
    MIH_TRY(ws.alloc(&hist, static_cast<size_t>(nq) * (qb + 1)));
    MIH_TRY(ws.alloc(&cnt1, nq));
    MIH_TRY(ws.alloc(&buf1, static_cast<size_t>(nq) * cap));
    MIH_TRY(ws.alloc(&qstats, 4ull * nq));
    MIH_TRY(ws.alloc(&active, 1));
    unsigned long long* sliced;
    MIH_TRY(ws.alloc(&sliced, 1));
    MIH_CUDA(cudaMemsetAsync(sliced, 0, sizeof(unsigned long long), s));
    uint8_t* exh;
    MIH_TRY(ws.alloc(&exh, nq));
    MIH_CUDA(cudaMemsetAsync(exh, 0, nq, s));
    const long long budget = scan_budget(ix);
    MIH_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nq * (qb + 1), s));
    MIH_CUDA(cudaMemsetAsync(cnt1, 0, sizeof(uint32_t) * nq, s));
    MIH_CUDA(cudaMemsetAsync(qstats, 0, sizeof(unsigned long long) * 4 * nq, s));
    int32_t* hist_done;
    MIH_TRY(ws.alloc(&hist_done, nq));
    uint32_t* wave_chunks;   // chunks of each query's steps in the next wave (written by the stopping test)
    MIH_TRY(ws.alloc(&wave_chunks, nq));
    init_knn_kernel<<<grid1(nq), 256, 0, s>>>(nq, ix->n, t_lo, t_hi, bound, dk, hist_done, wave_chunks);
    MIH_LAUNCH_CHECK();
    if (ix->n > 0 && query_stats == nullptr && ix->probe > 0) {
        // (with per-query counters requested the steps run exactly as Alg. 3
        // counts them, from a histogram-only start)
        KernelSpan ks(s, MIH_PROF_PROBE);
        const unsigned blocks = (nq + 7) / 8;
        if (ix->W == 1)
            bound_probe_kernel<1><<<blocks, 256, 0, s>>>(ix->dev_tables, ix->m, qb, ix->codes, queries, nq, ix->n, k,
                                                         k_uniform, static_cast<uint32_t>(ix->probe), bound);
        else if (ix->W == 2)
            bound_probe_kernel<2><<<blocks, 256, 0, s>>>(ix->dev_tables, ix->m, qb, ix->codes, queries, nq, ix->n, k,
                                                         k_uniform, static_cast<uint32_t>(ix->probe), bound);
        else
            bound_probe_kernel<4><<<blocks, 256, 0, s>>>(ix->dev_tables, ix->m, qb, ix->codes, queries, nq, ix->n, k,
                                                         k_uniform, static_cast<uint32_t>(ix->probe), bound);
        MIH_LAUNCH_CHECK();
    }
    Plan plan;
    MIH_TRY(plan_alloc(plan, nq, ws));

    SearchArgs a;
    memset(&a, 0, sizeof(a));
    a.tables = ix->dev_tables;
    a.m = ix->m;
    a.q = qb;
    a.codes = ix->codes;
    a.queries = queries;
    a.nq = nq;
    a.hist = hist;
    a.bound = bound;
    a.buf = buf1;
    a.cap = cap;
    a.cnt = cnt1;
    a.qstats = qstats;
    a.exh = exh;
    a.hist_done = hist_done;
    a.n = ix->n;
    a.exact_stats = query_stats != nullptr ? 1 : 0;
    a.sliced = sliced;

    // One wave: every active query runs its current Alg. 3 step(s), then the
    // stopping test advances or retires it.  cs = capture stream (graph) or 0.
    auto wave = [&](cudaStream_t cs) -> mih_status {
        cudaStream_t ws_s = cs ? cs : s;
        MIH_TRY(run_wave<kModeKnn>(ix, a, plan, t_lo, t_hi, dev, ws, cs, wave_chunks));
        MIH_CUDA(cudaMemsetAsync(active, 0, sizeof(unsigned int), ws_s));
        KernelSpan ks(ws_s, MIH_PROF_STOP, cs == nullptr);
        knn_stop_kernel<<<grid1(32ull * nq), 256, 0, ws_s>>>(nq, qb, ix->n, k, k_uniform, hist, t_lo, t_hi, bound, dk,
                                                    hist_done, cnt1, cap, qstats, active, ix->dev_tables, ix->m,
                                                    exh, budget, wave_chunks, query_stats ? -1 : ix->tail_from);
        MIH_LAUNCH_CHECK();
        return MIH_OK;
    };
    // At most q + 1 waves: step t <= q reaches every code (Prop. 1 with r = q).
    const unsigned int max_waves = static_cast<unsigned int>(qb) + 1;
    uint64_t waves = 0;
    // per-kernel timing runs the waves from the host so that each launch can be
    // bracketed by events (same kernels, same results)
    if (ix->n > 0 && (ix->executor == MIH_EXEC_HOST || timing_level() >= 2)) {
        for (unsigned int w = 0; w < max_waves; ++w) {
            MIH_TRY(wave(nullptr));
            ++waves;
            unsigned int hact = 0;
            MIH_CUDA(cudaMemcpyAsync(&hact, active, sizeof(hact), cudaMemcpyDeviceToHost, s));
            MIH_TRY(check_timeout(plan, s));
            if (hact == 0) break;
            if (w + 1 == max_waves) {
                set_error("mih_knn: queries still active after q steps");
                return MIH_EINTERNAL;
            }
        }
    } else if (ix->n > 0) {
        // The whole loop as one graph launch: a while node repeats the wave
        // and the loop control on the device, with no host round trip.
        unsigned int* wave_count;
        MIH_TRY(ws.alloc(&wave_count, 1));
        MIH_CUDA(cudaMemsetAsync(wave_count, 0, sizeof(unsigned int), s));
        MIH_TRY(ws.alloc(&plan.scan_tmp, scan_temp_u64(static_cast<size_t>(nq) + 1)));
        MIH_TRY(launch_search<kModeKnn>(a, ix->W, dev, s, false));   // kernel attributes, before capture
        GraphGuard gg;
        uint64_t body_launches = 0;
        MIH_TRY(launch_while_graph(gg, s, &body_launches, [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
            MIH_TRY(wave(cs));
            loop_control_kernel<<<1, 1, 0, cs>>>(h, active, plan.timeout, wave_count, max_waves);
            MIH_LAUNCH_CHECK();
            return MIH_OK;
        }));
        unsigned int hw = 0, hact = 0;
        MIH_CUDA(cudaMemcpyAsync(&hw, wave_count, sizeof(hw), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaMemcpyAsync(&hact, active, sizeof(hact), cudaMemcpyDeviceToHost, s));
        MIH_TRY(check_timeout(plan, s));
        waves = hw;
        if (hw > 1) add_launches((hw - 1) * body_launches, hw - 1);
        if (hact != 0) {
            set_error("mih_knn: queries still active after q steps");
            return MIH_EINTERNAL;
        }
    }

    // Second pass for queries whose bounded buffer overflowed.
    uint64_t* need;
    unsigned int* n_over;
    MIH_TRY(ws.alloc(&need, static_cast<size_t>(nq) + 1));
    MIH_TRY(ws.alloc(&n_over, 1));
    MIH_CUDA(cudaMemsetAsync(n_over, 0, sizeof(unsigned int), s));
    phase2_plan_kernel<<<grid1(nq + 1), 256, 0, s>>>(nq, qb, hist, dk, cnt1, cap, t_lo, t_hi, bound, need, n_over,
                                                    ix->dev_tables, ix->m, exh, budget);
    MIH_LAUNCH_CHECK();
    unsigned int hover = 0;
    MIH_CUDA(cudaMemcpyAsync(&hover, n_over, sizeof(hover), cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    uint64_t* buf2 = nullptr;
    if (hover > 0 && ix->n > 0) {
        MIH_TRY(scan_exclusive_u64(need, need, static_cast<size_t>(nq) + 1, ws));
        uint64_t total = 0;
        MIH_CUDA(cudaMemcpyAsync(&total, need + nq, sizeof(total), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        MIH_TRY(ws.alloc(&buf2, total));
        uint32_t* cursor;
        MIH_TRY(ws.alloc(&cursor, nq));
        MIH_CUDA(cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * nq, s));
        int* err;
        MIH_TRY(ws.alloc(&err, 1));
        MIH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        SearchArgs b = a;
        b.buf = buf2;
        b.cnt = cursor;
        b.out_base = need;
        b.qstats = nullptr;
        b.hist_done = nullptr;
        b.err = err;
        b.sliced = nullptr;
        MIH_TRY(run_wave<kModeCollect>(ix, b, plan, t_lo, t_hi, dev, ws));
        ++waves;
        MIH_TRY(check_timeout(plan, s));
        MIH_TRY(check_flag(err, "mih_knn: second pass found more codes within d_k than counted", s));
    }
    SelectInputs si;
    si.nq = nq;
    si.n = ix->n;
    si.q = qb;
    si.kq = k;
    si.k_uniform = k_uniform;
    si.kmax = kmax;
    si.out_off = out_offsets;
    si.hist = hist;
    si.dk = dk;
    si.buf1 = buf1;
    si.cap = cap;
    si.cnt1 = cnt1;
    si.buf2 = buf2;
    si.base2 = need;
    si.out_ids = out_ids;
    si.out_dist = out_dist;
    si.tables = ix->inline_codes ? ix->dev_tables : nullptr;   // entries hold table positions
    MIH_TRY(launch_select(si, ws));

    if (query_stats)
        MIH_CUDA(cudaMemcpyAsync(query_stats, qstats, sizeof(uint64_t) * 4 * nq, cudaMemcpyDeviceToDevice, s));
    if (stats) {
        std::vector<unsigned long long> h(4ull * nq);
        MIH_CUDA(cudaMemcpyAsync(h.data(), qstats, sizeof(unsigned long long) * 4 * nq, cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        for (uint32_t i = 0; i < nq; ++i) {
            stats->lookups += h[4ull * i];
            stats->candidates_raw += h[4ull * i + 1];
            stats->candidates_unique += query_stats ? h[4ull * i + 2] : 0;
            stats->steps += ix->n > 0 ? h[4ull * i + 3] + 1 : 0;
        }
        stats->phase2_queries = hover;
        stats->waves = waves;
        unsigned long long hs = 0;
        MIH_CUDA(cudaMemcpyAsync(&hs, sliced, sizeof(hs), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        stats->candidates_sliced = hs;
    }
    MIH_CUDA(cudaStreamSynchronize(s));
    return MIH_OK;
}

// CSR offsets of per-query k: out[i] = k[0] + ... + k[i-1], out[nq] = total.
mih_status mih_k_offsets(const uint32_t* k, uint32_t nq, uint64_t* out_offsets, void* stream) {
    clear_error();
    if (nq > (1u << 23)) {
        set_error("mih_k_offsets: nq must be at most 2^23");
        return MIH_EINVAL;
    }
    MIH_TRY(check_device_ptr(out_offsets, "out_offsets"));
    if (nq > 0) MIH_TRY(check_device_ptr(k, "k"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    widen_counts_kernel<<<grid1(static_cast<uint64_t>(nq) + 1), 256, 0, s>>>(k, nq, out_offsets);
    MIH_LAUNCH_CHECK();
    MIH_TRY(scan_exclusive_u64(out_offsets, out_offsets, static_cast<size_t>(nq) + 1, ws));
    return MIH_OK;
}

mih_status mih_rnear(const mih_index* ix, const uint64_t* queries, uint32_t nq, int r, uint64_t capacity,
                     uint64_t* out_offsets, uint32_t* out_ids, int32_t* out_dist, uint64_t* total_out,
                     uint64_t* query_stats, mih_stats* stats, void* stream) {
    clear_error();
    if (stats) memset(stats, 0, sizeof(*stats));
    if (total_out) *total_out = 0;
    CallScope scope(static_cast<cudaStream_t>(stream));
    MIH_TRY(validate_common(ix, queries, nq));
    if (r < 0) {
        set_error("mih_rnear: r must be >= 0");
        return MIH_EINVAL;
    }
    MIH_TRY(check_device_ptr(out_offsets, "out_offsets"));
    if (capacity > 0) {
        MIH_TRY(check_device_ptr(out_ids, "out_ids"));
        MIH_TRY(check_device_ptr(out_dist, "out_dist"));
    }
    if (query_stats) MIH_TRY(check_device_ptr(query_stats, "query_stats"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    const int qb = ix->q;
    const int reff = r < qb ? r : qb;  // every code lies within q bits
    if (nq > 0) MIH_TRY(permute_queries(ix, &queries, nq, ws));
    int32_t *t_lo, *t_hi, *bound;
    uint32_t* cnt;
    unsigned long long* qstats;
    const uint32_t nqa = nq > 0 ? nq : 1;
    MIH_TRY(ws.alloc(&t_lo, nqa));
    MIH_TRY(ws.alloc(&t_hi, nqa));
    MIH_TRY(ws.alloc(&bound, nqa));
    MIH_TRY(ws.alloc(&cnt, nqa));
    MIH_TRY(ws.alloc(&qstats, 4ull * nqa));
    MIH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nqa, s));
    MIH_CUDA(cudaMemsetAsync(qstats, 0, sizeof(unsigned long long) * 4 * nqa, s));
    Plan plan;
    MIH_TRY(plan_alloc(plan, nqa, ws));
    SearchArgs a;
    memset(&a, 0, sizeof(a));
    a.tables = ix->dev_tables;
    a.m = ix->m;
    a.q = qb;
    a.codes = ix->codes;
    a.queries = queries;
    a.nq = nq;
    a.bound = bound;
    a.cnt = cnt;
    a.qstats = qstats;
    a.n = ix->n;
    a.exact_stats = query_stats != nullptr ? 1 : 0;
    unsigned long long* sliced;
    MIH_TRY(ws.alloc(&sliced, 1));
    MIH_CUDA(cudaMemsetAsync(sliced, 0, sizeof(unsigned long long), s));
    a.sliced = sliced;
    uint8_t* exh;
    MIH_TRY(ws.alloc(&exh, nqa));
    {
        // Alg. 2 is steps 0..r; past the lookup budget one verification pass
        // over all codes replaces them.
        const long long budget = scan_budget(ix);
        unsigned long long lk = 0;
        for (int t = 0; t <= reff; ++t) {
            const int s_j = ix->tables[t % ix->m].len, rho = t / ix->m;
            lk += rho <= s_j ? host_binom(s_j, rho) : 0ull;
        }
        MIH_CUDA(cudaMemsetAsync(exh, (budget >= 0 && lk > static_cast<unsigned long long>(budget)) ? 1 : 0, nqa, s));
    }
    a.exh = exh;
    if (nq > 0 && ix->n > 0) {
        init_range_kernel<<<grid1(nq), 256, 0, s>>>(nq, 0, reff, reff, t_lo, t_hi, bound);
        MIH_LAUNCH_CHECK();
        MIH_TRY(run_wave<kModeCount>(ix, a, plan, t_lo, t_hi, dev, ws));
        MIH_TRY(check_timeout(plan, s));
    }
    // CSR offsets of the results: exclusive scan of the counts, last = total
    uint64_t* off64;
    MIH_TRY(ws.alloc(&off64, static_cast<size_t>(nq) + 1));
    widen_counts_kernel<<<grid1(nq + 1), 256, 0, s>>>(cnt, nq, off64);
    MIH_LAUNCH_CHECK();
    MIH_TRY(scan_exclusive_u64(off64, off64, static_cast<size_t>(nq) + 1, ws));
    MIH_CUDA(cudaMemcpyAsync(out_offsets, off64, sizeof(uint64_t) * (nq + 1), cudaMemcpyDeviceToDevice, s));
    uint64_t total = 0;
    MIH_CUDA(cudaMemcpyAsync(&total, off64 + nq, sizeof(total), cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    if (total_out) *total_out = total;
    auto finish_stats = [&]() -> mih_status {
        if (nq == 0) return MIH_OK;
        std::vector<unsigned long long> h(4ull * nq);
        MIH_CUDA(cudaMemcpyAsync(h.data(), qstats, sizeof(unsigned long long) * 4 * nq, cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        for (uint32_t i = 0; i < nq; ++i) h[4ull * i + 3] = static_cast<unsigned long long>(reff);
        if (query_stats)
            MIH_CUDA(cudaMemcpyAsync(query_stats, h.data(), sizeof(uint64_t) * 4 * nq, cudaMemcpyHostToDevice, s));
        if (stats) {
            for (uint32_t i = 0; i < nq; ++i) {
                stats->lookups += h[4ull * i];
                stats->candidates_raw += h[4ull * i + 1];
                stats->candidates_unique += query_stats ? h[4ull * i + 2] : 0;
                stats->steps += ix->n > 0 ? static_cast<uint64_t>(reff) + 1 : 0;
            }
            stats->waves = ix->n > 0 ? 1 : 0;
            unsigned long long hs = 0;
            MIH_CUDA(cudaMemcpyAsync(&hs, sliced, sizeof(hs), cudaMemcpyDeviceToHost, s));
            MIH_CUDA(cudaStreamSynchronize(s));
            stats->candidates_sliced = hs;
        }
        MIH_CUDA(cudaStreamSynchronize(s));
        return MIH_OK;
    };
    if (total > capacity) {
        MIH_TRY(finish_stats());
        set_error("mih_rnear: %llu results exceed capacity %llu", static_cast<unsigned long long>(total),
                  static_cast<unsigned long long>(capacity));
        return MIH_EOVERFLOW;
    }
    if (total >= 0xFFFFFFFFull) {
        set_error("mih_rnear: more than 2^32 - 2 results in one call");
        return MIH_EINVAL;
    }
    if (total > 0) {
        uint64_t *ent, *ent_alt, *sorted;
        MIH_TRY(ws.alloc(&ent, total));
        MIH_TRY(ws.alloc(&ent_alt, total));
        MIH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nq, s));
        int* err;
        MIH_TRY(ws.alloc(&err, 1));
        MIH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        SearchArgs b = a;
        b.buf = ent;
        b.out_base = off64;
        b.qstats = nullptr;
        b.err = err;
        b.sliced = nullptr;
        MIH_TRY(run_wave<kModeCollect>(ix, b, plan, t_lo, t_hi, dev, ws));
        MIH_TRY(check_timeout(plan, s));
        MIH_TRY(check_flag(err, "mih_rnear: fill pass found more results than the count pass", s));
        int qbits = 1;
        while ((1u << qbits) < nq) ++qbits;
        MIH_TRY(radix_sort_keys_u64(ent, ent_alt, total, kQueryShift + qbits, ws, &sorted));
        split_entries_kernel<<<grid1(total), 256, 0, s>>>(sorted, total, out_ids, out_dist);
        MIH_LAUNCH_CHECK();
    }
    MIH_TRY(finish_stats());
    MIH_CUDA(cudaStreamSynchronize(s));
    return MIH_OK;
}

}  // extern "C"
