// mih_internal.cuh -- device-side building blocks shared by the kernels of
// the multi-index hashing library (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mih.h"

namespace mih {

constexpr int kMaxTables = 256;
constexpr uint32_t kPadId = 0xFFFFFFFFu;
constexpr uint32_t kEmptySlot = 0xFFFFFFFFu;
constexpr int kChunkKeys = 256;          // ring keys per work chunk (one warp)
constexpr int kKeysPerLane = kChunkKeys / 32;
#ifndef MIH_BIG_BUCKET
#define MIH_BIG_BUCKET 64
#endif
constexpr uint32_t kBigBucket = MIH_BIG_BUCKET;   // buckets above this go to the slice list

// ---------------------------------------------------------------- tables
// One substring hash table (Sec. 6): either direct-addressed CSR offsets over
// all 2^s buckets, or a sparse form: the distinct keys in an open-addressing
// index (4 slots of {key, rank} per 32-byte bucket) plus CSR begins by rank.
struct TableDesc {
    int32_t off;        // first code bit of the substring
    int32_t len;        // s_j (1..32)
    int32_t kind;       // MIH_TABLE_DIRECT / MIH_TABLE_SPARSE
    int32_t rec_words;  // inline records of this many 32-bit words: the code without the
                        // table's own word (every substring one 32-bit word); 0 = full codes
    const uint32_t* ids;       // n ids ordered by (key, id)
    const uint32_t* offsets;   // direct: offsets[2^s + 1]; sparse: begins[U + 1]
    const uint2* slots;        // sparse: 4 * nbuckets slots {key, rank}
    uint64_t bucket_mask;      // sparse: nbuckets - 1 (power of two)
    uint32_t max_probe;        // sparse: longest probe sequence at build
    uint32_t pad2_;
    const uint64_t* codes;     // optional: codes in the order of `ids`: W uint64 words each, or
                               // (rec_words > 0) records of rec_words uint32 words
};

// ---------------------------------------------------------------- binomials
// C(n, k) for 0 <= k <= n <= 32 (substrings hold at most 32 bits), built at
// compile time (Pascal's rule) and read through the L1 cache: lanes of a warp
// index it divergently, which a __constant__ bank would serialise.
struct BinomTable {
    uint64_t v[33][33];
    constexpr BinomTable() : v() {
        for (int a = 0; a <= 32; ++a) {
            v[a][0] = 1;
            for (int b = 1; b <= a; ++b) v[a][b] = v[a - 1][b - 1] + (b <= a - 1 ? v[a - 1][b] : 0);
        }
    }
};

static __device__ const BinomTable g_binom = BinomTable();

__device__ __forceinline__ uint64_t binom(int n, int k) {
    return (k < 0 || n < 0 || k > n) ? 0ull : __ldg(&g_binom.v[n][k]);
}

// ---------------------------------------------------------------- codes
template <int W>
struct Code {
    uint64_t w[W];
};

template <int W>
__device__ __forceinline__ Code<W> load_code(const uint64_t* __restrict__ codes, uint64_t i) {
    Code<W> c;
    const uint64_t* p = codes + i * W;
    if constexpr (W == 1) {
        c.w[0] = __ldg(p);
    } else if constexpr (W == 2) {
        ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
        c.w[0] = v.x;
        c.w[1] = v.y;
    } else {
        ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(p));
        ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2*>(p) + 1);
        c.w[0] = a.x; c.w[1] = a.y; c.w[2] = b.x; c.w[3] = b.y;
    }
    return c;
}

template <int W>
__device__ __forceinline__ int hamming(const Code<W>& a, const Code<W>& b) {
    int d = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) d += __popcll(a.w[w] ^ b.w[w]);
    return d;
}

// Bits [off, off + len) of a W-word code (len <= 32), bit 0 = code bit off.
template <int W>
__device__ __forceinline__ uint32_t substring_bits(const Code<W>& c, int off, int len) {
    const int w0 = off >> 6, sh = off & 63;
    uint64_t lo = 0, hi = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        if (w == w0) lo = c.w[w];
        if (w == w0 + 1) hi = c.w[w];
    }
    uint64_t v = lo >> sh;
    if (sh != 0 && sh + len > 64) v |= hi << (64 - sh);
    const uint64_t mask = (len >= 64) ? ~0ull : ((1ull << len) - 1ull);
    return static_cast<uint32_t>(v & mask);
}

// ---------------------------------------------------------------- rings
// Keys at exactly rho bits from a query key are key ^ x with popcount(x) = rho
// and x < 2^s (the bucket ring of one Alg. 3 step).  x runs through the
// rho-subsets of {0..s-1} in increasing numeric order (colex order), so a
// rank maps to a subset by the combinatorial number system and consecutive
// ranks are one Gosper step apart.
// The element c_i of each position is the largest c below the previous one
// with C(c, i) <= rank: found by binary search (C(c, i) grows with c), and
// for i = 1 it is the rank itself.
__device__ __forceinline__ uint64_t unrank_subset(uint64_t rank, int s, int rho) {
    uint64_t x = 0;
    int hi = s;   // c < hi
    for (int i = rho; i >= 1; --i) {
        int c;
        if (i == 1) {
            c = static_cast<int>(rank);
        } else {
            int lo = i - 1, h = hi - 1;
            while (lo < h) {
                const int mid = (lo + h + 1) >> 1;
                if (binom(mid, i) <= rank) lo = mid;
                else h = mid - 1;
            }
            c = lo;
        }
        rank -= binom(c, i);
        x |= 1ull << c;
        hi = c;
    }
    return x;
}

// Next larger integer with the same popcount (Gosper); x != 0.
__device__ __forceinline__ uint64_t next_subset(uint64_t x) {
    const uint64_t c = x & (0ull - x);
    const uint64_t r = x + c;
    return (((r ^ x) >> 2) >> (__ffsll(static_cast<long long>(c)) - 1)) | r;
}

// ---------------------------------------------------------------- lookup
__device__ __forceinline__ uint32_t hash_key(uint32_t k) {
    // 32-bit finaliser (xorshift-multiply), spreads clustered keys over buckets.
    k ^= k >> 16;
    k *= 0x7feb352dU;
    k ^= k >> 15;
    k *= 0x846ca68bU;
    k ^= k >> 16;
    return k;
}

// Bucket [begin, end) of `key` in table t (empty when absent).
__device__ __forceinline__ void lookup_bucket(const TableDesc& t, uint32_t key, uint32_t& begin,
                                              uint32_t& end) {
    if (t.kind == MIH_TABLE_DIRECT) {
        begin = __ldg(t.offsets + key);
        end = __ldg(t.offsets + key + 1);
        return;
    }
    uint64_t b = hash_key(key) & t.bucket_mask;
    begin = end = 0;
    for (uint32_t p = 0; p <= t.max_probe; ++p) {
        const uint4* s4 = reinterpret_cast<const uint4*>(t.slots + 4 * b);
        const uint4 s01 = __ldg(s4);
        const uint4 s23 = __ldg(s4 + 1);
        uint32_t rank = kEmptySlot;
        bool open = false;
        if (s01.y != kEmptySlot) { if (s01.x == key) rank = s01.y; } else open = true;
        if (rank == kEmptySlot && !open) {
            if (s01.w != kEmptySlot) { if (s01.z == key) rank = s01.w; } else open = true;
        }
        if (rank == kEmptySlot && !open) {
            if (s23.y != kEmptySlot) { if (s23.x == key) rank = s23.y; } else open = true;
        }
        if (rank == kEmptySlot && !open) {
            if (s23.w != kEmptySlot) { if (s23.z == key) rank = s23.w; } else open = true;
        }
        if (rank != kEmptySlot) {
            begin = __ldg(t.offsets + rank);
            end = __ldg(t.offsets + rank + 1);
            return;
        }
        if (open) return;
        b = (b + 1) & t.bucket_mask;
    }
}

// ------------------------------------------------------- bulk async copies
// Global -> shared copies by the bulk-copy engine (cp.async.bulk), completion
// counted in bytes on an mbarrier, and bounded waits on that barrier.
constexpr uint32_t kWaitHintNs = 20000;          // longest suspension of one try_wait
constexpr uint64_t kWaitNs = 1000000000ull;      // a bulk copy not done after 1 s is an error

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bulk_copy_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `bar` with the given parity.  Each try_wait may
// suspend the warp (up to kWaitHintNs, woken early when the phase completes)
// instead of spinning, so waiting warps leave the issue slots to the warps
// that verify codes.  Gives up after limit_ns of global time, and in any case
// after a bounded number of polls (each takes at least a few nanoseconds).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    const uint32_t hint = limit_ns < kWaitHintNs ? static_cast<uint32_t>(limit_ns) : kWaitHintNs;
    const uint64_t max_polls = limit_ns / 4u + 4096u;
    uint64_t t0 = 0;
    for (uint64_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint)
            : "memory");
        if (ok) return true;
        if ((it & 7u) == 0) {
            const uint64_t now = global_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
        if (it >= max_polls) return false;
    }
}

// ---------------------------------------------------------------- warp utils
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane_id() >= static_cast<uint32_t>(o)) v += u;
    }
    return v;
}

// Packed result entry: distance in the high word so that uint64 order is
// (distance, id) order.
__device__ __forceinline__ uint64_t pack_entry(int d, uint32_t id) {
    return (static_cast<uint64_t>(static_cast<uint32_t>(d)) << 32) | id;
}

}  // namespace mih
