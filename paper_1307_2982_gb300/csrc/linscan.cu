// linscan.cu -- the linear-scan baseline (Sec. 5.2): exact k-NN by computing
// the Hamming distance from each query to every code (Sec. 6 "Hamming
// Distance": xor and population count per 64 bits).
//
// Batched design.  A CTA holds a tile of queries in shared memory and streams
// a contiguous range of codes; each thread keeps a few codes in registers and
// runs them against every query of the tile.  A pair is kept only if its
// distance is at most the query's running bound thr_q on the k-th smallest
// distance; kept pairs go to a bounded per-query buffer and a per-query
// distance histogram in global memory, from which every CTA periodically
// tightens thr_q (thr_q = the smallest D with at least min(k, n) kept codes
// within D bits, always >= the true k-th distance).  The initial bound comes
// from an exact histogram over a prefix sample of the database.
//
// Most pairs are far from the bound, so the kernel first tests a cheaper
// lower bound: the popcount of the OR of G consecutive 32-bit words of
// (code xor query) never exceeds their total popcount.  Only pairs that pass
// it pay for the exact distance.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "launch.h"
#include "mih_internal.cuh"
#include "search.h"

namespace mih {
namespace {

constexpr int kLsThreads = 256;
constexpr int kLsTile = kLsThreads * 8;                    // codes per tile (split granularity)
constexpr int kLsQueries = 64;                             // queries per CTA
constexpr int kLsRefresh = 8;                              // tiles between bound refreshes
constexpr uint32_t kSampleMax = 1u << 18;                  // prefix sample for the first bound

struct ScanArgs {
    const uint64_t* codes;
    uint64_t n;
    const uint64_t* queries;
    uint32_t nq;
    int qbits;
    const uint32_t* kq;
    uint32_t k_uniform;
    uint64_t split_len;        // codes per CTA column (multiple of kLsTile)
    int32_t* thr;              // [nq] running bound (read at start, written by refresh)
    uint32_t* hist;            // [nq][q+1] kept distances (first pass)
    uint64_t* buf;             // first pass: [nq][cap]; second pass: entries at base[q]
    uint32_t cap;
    uint32_t* cnt;             // first pass: kept count; second pass: cursor
    const uint64_t* base;      // second pass only: [nq + 1]
    int second_pass;
    int* err;                  // set when a second-pass write would leave its query's range
    int* timeout;              // tensor-core form: set when a bounded wait on a stage copy gave up
};

__device__ __forceinline__ uint32_t kk_of(const uint32_t* kq, uint32_t k_uniform, uint32_t q, uint64_t n) {
    const uint64_t k = kq ? kq[q] : k_uniform;
    return static_cast<uint32_t>(k < n ? k : n);
}

// (a ^ b) | c in one LOP3 (truth table 0xBE over inputs 0xF0, 0xCC, 0xAA).
__device__ __forceinline__ uint32_t xor_or(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm("lop3.b32 %0, %1, %2, %3, 0xBE;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Lower bound on the distance from ORs of G consecutive 32-bit words of
// code ^ query (G = 1: the exact distance).  Words are 32-bit halves,
// little-endian, so the chain folds the xor into each OR step.
template <int NW, int G>
__device__ __forceinline__ int or_bound32(const uint32_t (&c)[NW], const uint32_t (&g)[NW]) {
    int d = 0;
    if constexpr (G == 1) {
#pragma unroll
        for (int i = 0; i < NW; ++i) d += __popc(c[i] ^ g[i]);
    } else {
#pragma unroll
        for (int grp = 0; grp < NW / G; ++grp) {
            uint32_t t = c[grp * G + G - 1] ^ g[grp * G + G - 1];
#pragma unroll
            for (int i = G - 2; i >= 0; --i) t = xor_or(c[grp * G + i], g[grp * G + i], t);
            d += __popc(t);
        }
    }
    return d;
}

template <int W>
struct ScanShape {
    static constexpr int J = W <= 2 ? 8 : 4;   // codes per thread per tile
};

template <int W, int G>
__global__ void __launch_bounds__(kLsThreads) linscan_kernel(ScanArgs a) {
    constexpr int NW = 2 * W;
    constexpr int J = ScanShape<W>::J;
    constexpr int kTile = kLsThreads * J;
    __shared__ uint32_t s_q[kLsQueries][NW];
    __shared__ int s_thr[kLsQueries];
    const uint32_t q0 = blockIdx.x * kLsQueries;
    const uint32_t nql = min(static_cast<uint32_t>(kLsQueries), a.nq - q0);
    for (int i = threadIdx.x; i < kLsQueries * NW; i += blockDim.x) {
        const int qi = i / NW, w = i % NW;
        uint32_t v = 0;
        if (static_cast<uint32_t>(qi) < nql) {
            const uint64_t word = a.queries[static_cast<uint64_t>(q0 + qi) * W + w / 2];
            v = static_cast<uint32_t>(w & 1 ? word >> 32 : word);
        }
        s_q[qi][w] = v;
    }
    for (int i = threadIdx.x; i < kLsQueries; i += blockDim.x)
        s_thr[i] = (static_cast<uint32_t>(i) < nql) ? a.thr[q0 + i] : -1;
    __syncthreads();
    const uint64_t begin = static_cast<uint64_t>(blockIdx.y) * a.split_len;
    const uint64_t end = min(a.n, begin + a.split_len);
    int tile_no = 0;
    for (uint64_t t0 = begin; t0 < end; t0 += kTile, ++tile_no) {
        const bool full = t0 + kTile <= end;   // only the last tile checks its codes
        uint32_t c[J][NW];
        bool ok[J];
#pragma unroll
        for (int jj = 0; jj < J; ++jj) {
            const uint64_t i = t0 + static_cast<uint64_t>(jj) * kLsThreads + threadIdx.x;
            ok[jj] = full || i < end;
            const Code<W> v = ok[jj] ? load_code<W>(a.codes, i) : Code<W>{};
#pragma unroll
            for (int w = 0; w < W; ++w) {
                c[jj][2 * w] = static_cast<uint32_t>(v.w[w]);
                c[jj][2 * w + 1] = static_cast<uint32_t>(v.w[w] >> 32);
            }
        }
        for (uint32_t qi = 0; qi < nql; ++qi) {
            uint32_t g[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) g[w] = s_q[qi][w];
            const int th = s_thr[qi];
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
                const int lb = or_bound32<NW, G>(c[jj], g);
                if (lb <= th && (full || ok[jj])) {
                    const int d = (G == 1) ? lb : or_bound32<NW, 1>(c[jj], g);
                    if (d <= th) {
                        const uint32_t q = q0 + qi;
                        const uint32_t id = static_cast<uint32_t>(t0 + static_cast<uint64_t>(jj) * kLsThreads + threadIdx.x);
                        const uint32_t p = atomicAdd(&a.cnt[q], 1u);
                        if (!a.second_pass) {
                            if (p < a.cap) a.buf[static_cast<uint64_t>(q) * a.cap + p] = pack_entry(d, id);
                            atomicAdd(&a.hist[static_cast<uint64_t>(q) * (a.qbits + 1) + d], 1u);
                        } else {
                            const uint64_t slot = a.base[q] + p;
                            if (slot < a.base[q + 1]) a.buf[slot] = pack_entry(d, id);
                            else atomicExch(a.err, 1);
                        }
                    }
                }
            }
        }
        if (!a.second_pass && (tile_no % kLsRefresh) == kLsRefresh - 1) {
            __syncthreads();
            if (threadIdx.x < nql) {
                const uint32_t q = q0 + threadIdx.x;
                const uint32_t kk = kk_of(a.kq, a.k_uniform, q, a.n);
                const uint32_t* h = a.hist + static_cast<uint64_t>(q) * (a.qbits + 1);
                const int old = s_thr[threadIdx.x];
                uint32_t cum = 0;
                for (int d = 0; d < old; ++d) {
                    cum += __ldcg(h + d);  // written by other CTAs' atomics: bypass L1
                    if (cum >= kk) {
                        s_thr[threadIdx.x] = d;
                        break;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ tensor-core form
// The same scan with the distances from fp8 tensor-core products.  A code bit
// b becomes the e4m3 value (-1)^b (0x38 = +1.0, 0xB8 = -1.0), so the dot
// product of two q-bit codes is (#equal bits - #differing bits) = q - 2 d and
// d = (q - <g, c>) / 2 (Sec. 6's distance, on the tensor pipe); every partial
// sum is an integer of magnitude <= 256, exact in the f32 accumulators.  One
// 32-bit code word is one K-step of mma.m16n8k32.
//
// A warp holds the A fragments of its 16 MT queries in registers for the whole
// scan and takes 8 NT codes per step, building their B fragments from code
// words that the CTA stages in shared memory; the CTA's warps scan the same
// codes for different queries.  A pair is kept when dot >= q - 2 thr_q, i.e. d <= thr_q; the warp
// only looks at single pairs when one of its lanes has such a pair.
constexpr int kMmaWarps = 4;
constexpr int kMmaStageCodes = 256;   // codes per shared-memory stage
constexpr int kMmaSlots = 3;          // stages in flight per CTA (a ring of slots)

template <int W>
struct MmaShape {
    static constexpr int MT = W == 4 ? 2 : 4;   // 16-query tiles per warp (A fragments in registers)
    static constexpr int NT = 2;                // 8-code tiles per step
};

// Four code bits (bit i of `nibble`) -> four e4m3 bytes 0x38 | (bit_i << 7):
// the multiplier puts bit i at bit 8 i + 7 (the copies of the nibble do not overlap).
__device__ __forceinline__ uint32_t pm1_e4m3x4(uint32_t nibble) {
    return ((nibble * 0x10204080u) & 0x80808080u) | 0x38383838u;
}

__device__ __forceinline__ void mma_e4m3(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A W-word code from shared memory (16-byte loads for W >= 2).
template <int W>
__device__ __forceinline__ Code<W> smem_code(const uint64_t* sc, uint32_t i) {
    Code<W> c;
    if constexpr (W == 1) {
        c.w[0] = sc[i];
    } else {
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(sc + static_cast<uint64_t>(i) * W);
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
            const ulonglong2 v = p[h];
            c.w[2 * h] = v.x;
            c.w[2 * h + 1] = v.y;
        }
    }
    return c;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The CTA's codes arrive in stages of kMmaStageCodes, copied into a ring of
// kMmaSlots shared-memory slots by the bulk-copy engine (thread 0 issues,
// completion counted on a per-slot mbarrier), so the warps read code words
// from shared memory.  Every wait is bounded and the decision to go on is
// taken by the whole CTA; on expiry the CTA raises a.timeout, waits (bounded)
// for its copies in flight and leaves.
template <int W>
__global__ void __launch_bounds__(kMmaWarps * 32) linscan_mma_kernel(ScanArgs a) {
    constexpr int KS = 2 * W;                       // K-steps: 32-bit words per code
    constexpr int MT = MmaShape<W>::MT, NT = MmaShape<W>::NT;
    constexpr int QW = 16 * MT, QC = QW * kMmaWarps, CT = 8 * NT;
    constexpr int kRefreshStages = kLsRefresh * kLsTile / kMmaStageCodes;
    __shared__ __align__(16) uint64_t s_codes[kMmaSlots][kMmaStageCodes * W];
    __shared__ __align__(8) uint64_t s_bar[kMmaSlots];
    __shared__ int s_thr[QC];
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id(), g = lane >> 2, t = lane & 3;
    const uint32_t q0 = blockIdx.x * QC;
    const uint32_t nql = min(static_cast<uint32_t>(QC), a.nq - q0);
    for (int i = threadIdx.x; i < QC; i += blockDim.x) s_thr[i] = static_cast<uint32_t>(i) < nql ? a.thr[q0 + i] : -1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kMmaSlots; ++i) mbar_init(&s_bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // A fragments: rows g and g + 8 of each query tile; bits 4t..4t+3 of a
    // word in registers 0/1, bits 16+4t..16+4t+3 in registers 2/3
    uint32_t A[MT][KS][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t r = warp * QW + mt * 16 + g + 8 * h;
            Code<W> v{};
            if (r < nql) v = load_code<W>(a.queries, q0 + r);
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const uint32_t wd = static_cast<uint32_t>(v.w[ks >> 1] >> (32 * (ks & 1)));
                A[mt][ks][h] = pm1_e4m3x4((wd >> (4 * t)) & 0xFu);
                A[mt][ks][2 + h] = pm1_e4m3x4((wd >> (16 + 4 * t)) & 0xFu);
            }
        }
    }
    // Kept when dot >= cut = q - 2 thr (thr = -1: cut = q + 2, never).  The
    // accumulators start at 0.5 - cut, so they end at dot - cut + 0.5: at
    // least +0.5 for a kept pair, at most -0.5 otherwise (exact in f32, never
    // zero), and the sign bit alone decides.
    float cut[MT][2];
    auto load_cuts = [&]() {
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                cut[mt][h] = static_cast<float>(a.qbits - 2 * s_thr[warp * QW + mt * 16 + g + 8 * h]);
    };
    load_cuts();
    const uint64_t begin = static_cast<uint64_t>(blockIdx.y) * a.split_len;
    const uint64_t end = min(a.n, begin + a.split_len);
    const uint64_t nstages = (end - begin + kMmaStageCodes - 1) / kMmaStageCodes;
    // thread 0: copy stage st into its slot.  Whole 16-byte multiples go by
    // bulk copy; with 8-byte codes an odd last code is stored by a plain load,
    // before the arrival that publishes the stage.
    auto issue = [&](uint64_t st) {
        const uint64_t c0 = begin + st * kMmaStageCodes;
        const uint32_t cnt = static_cast<uint32_t>(min(static_cast<uint64_t>(kMmaStageCodes), end - c0));
        const int slot = static_cast<int>(st % kMmaSlots);
        uint64_t* dst = s_codes[slot];
        uint32_t bulk = cnt;
        if constexpr (W == 1) {
            bulk = cnt & ~1u;
            if (bulk < cnt) dst[cnt - 1] = __ldg(a.codes + c0 + cnt - 1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the slot are done
        if (bulk > 0) bulk_copy_to_smem(dst, a.codes + c0 * W, bulk * 8u * W, &s_bar[slot]);
        else mbar_arrive(&s_bar[slot]);
    };
    if (threadIdx.x == 0)
        for (uint64_t st = 0; st < kMmaSlots && st < nstages; ++st) issue(st);
    uint32_t parities = 0u;
    for (uint64_t st = 0; st < nstages; ++st) {
        const int slot = static_cast<int>(st % kMmaSlots);
        const bool ok = mbar_wait_bounded(&s_bar[slot], (parities >> slot) & 1u, kWaitNs);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                if (a.timeout) atomicExch(a.timeout, 1);
                // the copies still in flight land before the CTA leaves
                for (uint64_t s2 = st; s2 < st + kMmaSlots && s2 < nstages; ++s2) {
                    const int sl = static_cast<int>(s2 % kMmaSlots);
                    mbar_wait_bounded(&s_bar[sl], (parities >> sl) & 1u, kWaitNs);
                }
            }
            __syncthreads();
            return;
        }
        parities ^= 1u << slot;
        const uint64_t c0 = begin + st * kMmaStageCodes;
        const uint32_t cnt = static_cast<uint32_t>(min(static_cast<uint64_t>(kMmaStageCodes), end - c0));
        const uint64_t* sc = s_codes[slot];
        for (uint32_t lb = 0; lb < cnt; lb += CT) {
            uint32_t cw[NT][KS];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const uint32_t idx = lb + nt * 8 + g;
                Code<W> v{};
                if (idx < cnt) v = smem_code<W>(sc, idx);
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) cw[nt][ks] = static_cast<uint32_t>(v.w[ks >> 1] >> (32 * (ks & 1)));
            }
            float D[MT][NT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) D[mt][nt][e] = 0.5f - cut[mt][e >> 1];
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                uint32_t b0[NT], b1[NT];
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    b0[nt] = pm1_e4m3x4((cw[nt][ks] >> (4 * t)) & 0xFu);
                    b1[nt] = pm1_e4m3x4((cw[nt][ks] >> (16 + 4 * t)) & 0xFu);
                }
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_e4m3(D[mt][nt], A[mt][ks], b0[nt], b1[nt]);
            }
            // accumulator e: row g + 8 (e >> 1) of the query tile, code 2t + (e & 1)
            // of the code tile; a clear sign bit in the AND of all of them means
            // some pair of this lane is kept
            uint32_t signs = 0xFFFFFFFFu;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) signs &= __float_as_uint(D[mt][nt][e]);
            if (__any_sync(0xFFFFFFFFu, (signs >> 31) == 0u)) {
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int h = e >> 1;
                            const uint32_t idx = lb + nt * 8 + 2 * t + (e & 1);
                            if (idx >= cnt || (__float_as_uint(D[mt][nt][e]) >> 31) != 0u) continue;
                            const int dot = __float2int_rn(D[mt][nt][e] - 0.5f + cut[mt][h]);
                            const int d = (a.qbits - dot) >> 1;
                            const uint32_t q = q0 + warp * QW + mt * 16 + g + 8 * h;
                            const uint32_t id = static_cast<uint32_t>(c0 + idx);
                            const uint32_t p = atomicAdd(&a.cnt[q], 1u);
                            if (!a.second_pass) {
                                if (p < a.cap) a.buf[static_cast<uint64_t>(q) * a.cap + p] = pack_entry(d, id);
                                atomicAdd(&a.hist[static_cast<uint64_t>(q) * (a.qbits + 1) + d], 1u);
                            } else {
                                const uint64_t slot2 = a.base[q] + p;
                                if (slot2 < a.base[q + 1]) a.buf[slot2] = pack_entry(d, id);
                                else atomicExch(a.err, 1);
                            }
                        }
            }
        }
        __syncthreads();   // every warp is done with this slot
        if (threadIdx.x == 0 && st + kMmaSlots < nstages) issue(st + kMmaSlots);
        if (!a.second_pass && (st % kRefreshStages) == kRefreshStages - 1) {
            for (uint32_t r = threadIdx.x; r < nql; r += blockDim.x) {
                const uint32_t q = q0 + r;
                const uint32_t kk = kk_of(a.kq, a.k_uniform, q, a.n);
                const uint32_t* h = a.hist + static_cast<uint64_t>(q) * (a.qbits + 1);
                const int old = s_thr[r];
                uint32_t cum = 0;
                for (int d = 0; d < old; ++d) {
                    cum += __ldcg(h + d);  // written by other CTAs' atomics: bypass L1
                    if (cum >= kk) {
                        s_thr[r] = d;
                        break;
                    }
                }
            }
            __syncthreads();
            load_cuts();
        }
    }
}

// Exact distance histogram of the first S codes per query (one warp per
// query, lane-private columns in shared memory), then the bound: the smallest
// D with at least min(k, n) sample codes within D bits (q if S < min(k, n)).
template <int W>
__global__ void __launch_bounds__(128) sample_bound_kernel(const uint64_t* __restrict__ codes, uint64_t S,
                                                           const uint64_t* __restrict__ queries, uint32_t nq,
                                                           int qbits, const uint32_t* kq, uint32_t k_uniform,
                                                           uint64_t n, int32_t* __restrict__ thr) {
    extern __shared__ uint16_t s_h[];  // [warps][qbits+1][32]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q = blockIdx.x * (blockDim.x >> 5) + warp;
    uint16_t* h = s_h + static_cast<size_t>(warp) * (qbits + 1) * 32;
    for (int d = 0; d <= qbits; ++d) h[d * 32 + lane] = 0;
    __syncwarp();
    if (q >= nq) return;
    Code<W> g;
#pragma unroll
    for (int w = 0; w < W; ++w) g.w[w] = queries[static_cast<uint64_t>(q) * W + w];
    for (uint64_t i = lane; i < S; i += 32) {
        const Code<W> c = load_code<W>(codes, i);
        const int d = hamming<W>(c, g);
        h[d * 32 + lane] += 1;
    }
    __syncwarp();
    const uint32_t kk = kk_of(kq, k_uniform, q, n);
    uint32_t cum = 0;
    int bound = qbits;
    for (int d0 = 0; d0 <= qbits; d0 += 32) {
        const int d = d0 + lane;
        uint32_t v = 0;
        if (d <= qbits)
            for (int l = 0; l < 32; ++l) v += h[d * 32 + l];
        const uint32_t incl = warp_inclusive_scan(v);
        const uint32_t reach = __ballot_sync(0xFFFFFFFFu, d <= qbits && cum + incl >= kk);
        if (reach) {
            bound = d0 + __ffs(reach) - 1;
            break;
        }
        cum += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) thr[q] = bound;
}

// d_k from the kept-distance histogram (exact up to d_k); overflowed queries
// get their exact buffer size and thr = d_k for the second pass, the others
// thr = -1 (skipped).
__global__ void finish_first_pass_kernel(uint32_t nq, int qbits, uint64_t n, const uint32_t* kq, uint32_t k_uniform,
                                         const uint32_t* __restrict__ hist, const uint32_t* __restrict__ cnt,
                                         uint32_t cap, int32_t* __restrict__ dk, int32_t* __restrict__ thr,
                                         uint64_t* __restrict__ need, unsigned int* __restrict__ n_over) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q <= nq; q += gridDim.x * blockDim.x) {
        if (q == nq) { need[q] = 0; continue; }
        const uint32_t kk = kk_of(kq, k_uniform, q, n);
        const uint32_t* h = hist + static_cast<uint64_t>(q) * (qbits + 1);
        uint64_t cum = 0;
        int d = 0;
        for (; d <= qbits; ++d) {
            cum += h[d];
            if (cum >= kk) break;
        }
        if (d > qbits) d = qbits;
        dk[q] = d;
        const bool over = cnt[q] > cap;
        need[q] = over ? cum : 0;
        thr[q] = over ? d : -1;
        if (over) atomicAdd(n_over, 1u);
    }
}

unsigned grid1(uint64_t n) {
    uint64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return static_cast<unsigned>(g ? g : 1);
}

template <int W>
mih_status launch_sample(const uint64_t* codes, uint64_t S, const uint64_t* queries, uint32_t nq, int qbits,
                         const uint32_t* kq, uint32_t k_uniform, uint64_t n, int32_t* thr, cudaStream_t s) {
    const int warps = 4;
    const size_t smem = static_cast<size_t>(warps) * (qbits + 1) * 32 * sizeof(uint16_t);
    if (smem > 48 * 1024)
        MIH_CUDA(cudaFuncSetAttribute(sample_bound_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    sample_bound_kernel<W><<<(nq + warps - 1) / warps, warps * 32, smem, s>>>(codes, S, queries, nq, qbits, kq,
                                                                              k_uniform, n, thr);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

template <int W, int G>
mih_status launch_scan_wg(const ScanArgs& a, dim3 grid, cudaStream_t s) {
    linscan_kernel<W, G><<<grid, kLsThreads, 0, s>>>(a);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

template <int W>
mih_status launch_scan_w(const ScanArgs& a, int G, dim3 grid, cudaStream_t s) {
    if (G >= 4 && W >= 2) return launch_scan_wg<W, (W >= 2 ? 4 : 2)>(a, grid, s);
    if (G >= 2) return launch_scan_wg<W, 2>(a, grid, s);
    return launch_scan_wg<W, 1>(a, grid, s);
}
// (split lengths are multiples of kLsTile = 2048 codes, a multiple of every
// per-W tile, so only each CTA's last tile can be partial)

mih_status launch_scan(const ScanArgs& a, int W, int G, dim3 grid, cudaStream_t s) {
    if (W == 1) return launch_scan_w<1>(a, G, grid, s);
    if (W == 2) return launch_scan_w<2>(a, G, grid, s);
    return launch_scan_w<4>(a, G, grid, s);
}

// Grid of a scan: query tiles x CTA columns over the codes, enough columns to
// fill the GPU about 4 times over; columns are whole multiples of kLsTile.
struct ScanGrid {
    dim3 grid;
    uint64_t split_len;
};

ScanGrid scan_grid(uint64_t n, uint32_t nq, uint32_t queries_per_cta, int sms) {
    const uint32_t qtiles = (nq + queries_per_cta - 1) / queries_per_cta;
    const uint64_t target = static_cast<uint64_t>(sms) * 4;
    uint64_t splits = (target + qtiles - 1) / qtiles;
    const uint64_t max_splits = (n + kLsTile - 1) / kLsTile;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    if (splits > 65535) splits = 65535;
    uint64_t split_len = (n + splits - 1) / splits;
    split_len = (split_len + kLsTile - 1) / kLsTile * kLsTile;
    splits = (n + split_len - 1) / split_len;
    return {dim3(qtiles, static_cast<unsigned>(splits)), split_len};
}

uint32_t mma_queries_per_cta(int W) { return (W == 4 ? 2u : 4u) * 16u * kMmaWarps; }

mih_status launch_scan_mma(const ScanArgs& a, int W, dim3 grid, cudaStream_t s) {
    if (W == 1) linscan_mma_kernel<1><<<grid, kMmaWarps * 32, 0, s>>>(a);
    else if (W == 2) linscan_mma_kernel<2><<<grid, kMmaWarps * 32, 0, s>>>(a);
    else linscan_mma_kernel<4><<<grid, kMmaWarps * 32, 0, s>>>(a);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

// OR-group width: the widest G whose expected lower bound on a random pair,
// (2W/G) * 32 * (1 - 2^-G), stays clear of the typical first bound.
int choose_group(int W, int typical_thr) {
    int best = 1;
    for (int G = 2; G <= 4 && G <= 2 * W; G *= 2) {
        const double e = (2.0 * W / G) * 32.0 * (1.0 - 1.0 / (1 << G));
        if (e > typical_thr + 6) best = G;
    }
    return best;
}

}  // namespace
}  // namespace mih

using namespace mih;

extern "C" mih_status linscan_knn(const uint64_t* codes, uint64_t n, int q, const uint64_t* queries, uint32_t nq,
                                  const uint32_t* k, uint32_t k_uniform, const uint64_t* out_offsets,
                                  uint32_t* out_ids, int32_t* out_dist, void* stream) {
    clear_error();
    if (q != 64 && q != 128 && q != 256) {
        set_error("linscan_knn: q must be 64, 128 or 256 (got %d)", q);
        return MIH_EINVAL;
    }
    if (n >= 0xFFFFFFFFull) {
        set_error("linscan_knn: n must be below 2^32 - 1");
        return MIH_EINVAL;
    }
    if (nq > (1u << 23)) {
        set_error("linscan_knn: nq must be at most 2^23");
        return MIH_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallScope scope(s);
    Workspace ws(s);
    uint32_t kmax = 0;
    MIH_TRY(check_k_args(nq, k, k_uniform, out_offsets, out_ids, out_dist, &kmax, ws));
    if (nq == 0) return MIH_OK;
    MIH_TRY(check_device_ptr(queries, "queries"));
    if (n > 0) {
        MIH_TRY(check_device_ptr(codes, "codes"));
        MIH_TRY(check_code_alignment(codes, q / 64, "codes"));
    }
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    const int W = q / 64;
    const uint32_t cap = std::max<uint32_t>(16384u, std::min<uint32_t>(16u * kmax, 65536u));

    int32_t *thr, *dk;
    uint32_t *hist, *cnt;
    uint64_t *buf, *need;
    unsigned int* n_over;
    MIH_TRY(ws.alloc(&thr, nq));
    MIH_TRY(ws.alloc(&dk, nq));
    MIH_TRY(ws.alloc(&hist, static_cast<size_t>(nq) * (q + 1)));
    MIH_TRY(ws.alloc(&cnt, nq));
    MIH_TRY(ws.alloc(&buf, static_cast<size_t>(nq) * cap));
    MIH_TRY(ws.alloc(&need, static_cast<size_t>(nq) + 1));
    MIH_TRY(ws.alloc(&n_over, 1));
    MIH_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nq * (q + 1), s));
    MIH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nq, s));
    MIH_CUDA(cudaMemsetAsync(n_over, 0, sizeof(unsigned int), s));

    uint64_t* buf2 = nullptr;
    unsigned int hover = 0;
    if (n > 0) {
        const uint64_t S = std::min<uint64_t>(n, kSampleMax);
        if (W == 1) MIH_TRY(launch_sample<1>(codes, S, queries, nq, q, k, k_uniform, n, thr, s));
        else if (W == 2) MIH_TRY(launch_sample<2>(codes, S, queries, nq, q, k, k_uniform, n, thr, s));
        else MIH_TRY(launch_sample<4>(codes, S, queries, nq, q, k, k_uniform, n, thr, s));
        // typical first bound -> OR-group width
        std::vector<int32_t> hthr(nq);
        MIH_CUDA(cudaMemcpyAsync(hthr.data(), thr, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        std::nth_element(hthr.begin(), hthr.begin() + nq / 2, hthr.end());
#ifdef MIH_LINSCAN_G
        const int G = MIH_LINSCAN_G;   // build-time override for tuning
#else
        const int G = choose_group(W, hthr[nq / 2]);
#endif

        // the popcount form unless the tensor-core form (fp8 products) is asked for
        // (its stage copies start on 16-byte boundaries: 8-byte codes must be
        // 16-byte aligned for it)
        const bool tensor = scan_kernel_choice() == MIH_SCAN_TENSOR &&
                            (W >= 2 || reinterpret_cast<uintptr_t>(codes) % 16 == 0);
        const ScanGrid sg = scan_grid(n, nq, tensor ? mma_queries_per_cta(W) : kLsQueries, dev.sms);
        const uint64_t split_len = sg.split_len;

        ScanArgs a;
        memset(&a, 0, sizeof(a));
        a.codes = codes;
        a.n = n;
        a.queries = queries;
        a.nq = nq;
        a.qbits = q;
        a.kq = k;
        a.k_uniform = k_uniform;
        a.split_len = split_len;
        a.thr = thr;
        a.hist = hist;
        a.buf = buf;
        a.cap = cap;
        a.cnt = cnt;
        int* timeout = nullptr;
        if (tensor) {
            MIH_TRY(ws.alloc(&timeout, 1));
            MIH_CUDA(cudaMemsetAsync(timeout, 0, sizeof(int), s));
            a.timeout = timeout;
        }
        const dim3 grid = sg.grid;
        main_kernel_begin(s);
        {
            KernelSpan ks(s, MIH_PROF_SCAN);
            if (tensor) MIH_TRY(launch_scan_mma(a, W, grid, s));
            else MIH_TRY(launch_scan(a, W, G, grid, s));
        }
        main_kernel_end(s);

        finish_first_pass_kernel<<<grid1(nq + 1), 256, 0, s>>>(nq, q, n, k, k_uniform, hist, cnt, cap, dk, thr, need,
                                                              n_over);
        MIH_LAUNCH_CHECK();
        MIH_CUDA(cudaMemcpyAsync(&hover, n_over, sizeof(hover), cudaMemcpyDeviceToHost, s));
        int htimeout = 0;
        if (timeout) MIH_CUDA(cudaMemcpyAsync(&htimeout, timeout, sizeof(int), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        if (htimeout) {
            set_error("linscan_knn: a bounded wait on a bulk copy expired");
            return MIH_ETIMEOUT;
        }
        if (hover > 0) {
            // Second pass over the database for queries whose buffer overflowed:
            // collect exactly the codes within d_k bits.
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
            ScanArgs b = a;
            b.buf = buf2;
            b.cnt = cursor;
            b.base = need;
            b.second_pass = 1;
            b.err = err;
            if (tensor) MIH_TRY(launch_scan_mma(b, W, grid, s));
            else MIH_TRY(launch_scan(b, W, 1, grid, s));
            int herr = 0;
            MIH_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            if (timeout) MIH_CUDA(cudaMemcpyAsync(&htimeout, timeout, sizeof(int), cudaMemcpyDeviceToHost, s));
            MIH_CUDA(cudaStreamSynchronize(s));
            if (htimeout) {
                set_error("linscan_knn: a bounded wait on a bulk copy expired");
                return MIH_ETIMEOUT;
            }
            if (herr) {
                set_error("linscan_knn: second pass found more codes within d_k than counted");
                return MIH_EINTERNAL;
            }
        }
    } else {
        MIH_CUDA(cudaMemsetAsync(dk, 0, sizeof(int32_t) * nq, s));
    }

    SelectInputs si;
    si.nq = nq;
    si.n = n;
    si.q = q;
    si.kq = k;
    si.k_uniform = k_uniform;
    si.kmax = kmax;
    si.out_off = out_offsets;
    si.hist = hist;
    si.dk = dk;
    si.buf1 = buf;
    si.cap = cap;
    si.cnt1 = cnt;
    si.buf2 = buf2;
    si.base2 = need;
    si.out_ids = out_ids;
    si.out_dist = out_dist;
    MIH_TRY(launch_select(si, ws));
    MIH_CUDA(cudaStreamSynchronize(s));
    return MIH_OK;
}

// ---------------------------------------------------------------------------
// linscan_knn_noalloc: the same linear scan with all scratch memory in one
// fixed array inside the library, for callers that must not allocate device
// memory during a search (see include/mih.h).  The array lives in device
// memory of every GPU that loads the library until the process exits.
namespace mih {
namespace {

constexpr uint32_t kNaMaxQueries = 256;        // queries per call
constexpr uint32_t kNaMaxK = 256;              // k per call
constexpr uint32_t kNaCap = 16 * kNaMaxK;      // first-pass slots per query (4096); a query that
                                               // keeps more is collected by a second scan
constexpr uint64_t kNaSecond = 1ull << 20;     // second-pass slots per call

constexpr size_t na_align(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr size_t kNaThr = 0;
constexpr size_t kNaDk = na_align(kNaThr + 4 * kNaMaxQueries);
constexpr size_t kNaCnt = na_align(kNaDk + 4 * kNaMaxQueries);
constexpr size_t kNaCursor = na_align(kNaCnt + 4 * kNaMaxQueries);
constexpr size_t kNaFlags = na_align(kNaCursor + 4 * kNaMaxQueries);   // n_over, scan error, select error
constexpr size_t kNaNeed = na_align(kNaFlags + 16);
constexpr size_t kNaHist = na_align(kNaNeed + 8 * (kNaMaxQueries + 1));
constexpr size_t kNaBuf = na_align(kNaHist + 4ull * kNaMaxQueries * 257);
constexpr size_t kNaBuf2 = na_align(kNaBuf + 8ull * kNaMaxQueries * kNaCap);
constexpr size_t kNaBytes = na_align(kNaBuf2 + 8ull * kNaSecond);   // about 16.3 MiB

static __device__ __align__(256) unsigned char g_linscan_scratch[kNaBytes];

std::mutex g_na_mu;
void* g_na_addr[64] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not its address).
mih_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    MIH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d out of range", dev);
        return MIH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_linscan_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            set_error("linscan_knn_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return MIH_ECUDA;
        }
        g_na_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_na_addr[dev]);
    return MIH_OK;
}

}  // namespace
}  // namespace mih

extern "C" mih_status linscan_knn_noalloc(const uint64_t* codes, uint64_t n, int q, const uint64_t* queries,
                                          uint32_t nq, uint32_t k, uint32_t* out_ids, int32_t* out_dist,
                                          void* stream) {
    using namespace mih;
    clear_error();
    if (q != 64 && q != 128 && q != 256) {
        set_error("linscan_knn_noalloc: q must be 64, 128 or 256 (got %d)", q);
        return MIH_EINVAL;
    }
    if (n >= 0xFFFFFFFFull) {
        set_error("linscan_knn_noalloc: n must be below 2^32 - 1");
        return MIH_EINVAL;
    }
    if (nq > kNaMaxQueries) {
        set_error("linscan_knn_noalloc: at most %u queries per call (got %u)", kNaMaxQueries, nq);
        return MIH_EINVAL;
    }
    if (k < 1 || k > kNaMaxK) {
        set_error("linscan_knn_noalloc: k must be in [1, %u] (got %u)", kNaMaxK, k);
        return MIH_EINVAL;
    }
    if (nq == 0) return MIH_OK;
    MIH_TRY(check_device_ptr(queries, "queries"));
    MIH_TRY(check_device_ptr(out_ids, "out_ids"));
    MIH_TRY(check_device_ptr(out_dist, "out_dist"));
    if (n > 0) {
        MIH_TRY(check_device_ptr(codes, "codes"));
        MIH_TRY(check_code_alignment(codes, q / 64, "codes"));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = nullptr;
    MIH_TRY(noalloc_scratch(&base));
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    const int W = q / 64;
    int32_t* thr = reinterpret_cast<int32_t*>(base + kNaThr);
    int32_t* dk = reinterpret_cast<int32_t*>(base + kNaDk);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(base + kNaCnt);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(base + kNaCursor);
    unsigned int* n_over = reinterpret_cast<unsigned int*>(base + kNaFlags);
    int* scan_err = reinterpret_cast<int*>(base + kNaFlags + 4);
    int* select_err = reinterpret_cast<int*>(base + kNaFlags + 8);
    uint64_t* need = reinterpret_cast<uint64_t*>(base + kNaNeed);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kNaHist);
    uint64_t* buf = reinterpret_cast<uint64_t*>(base + kNaBuf);
    uint64_t* buf2 = reinterpret_cast<uint64_t*>(base + kNaBuf2);

    // The array keeps the previous call's contents: clear what must start at zero.
    MIH_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nq * (q + 1), s));
    MIH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nq, s));
    MIH_CUDA(cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * nq, s));
    MIH_CUDA(cudaMemsetAsync(base + kNaFlags, 0, 16, s));
    MIH_CUDA(cudaMemsetAsync(need, 0, sizeof(uint64_t) * (nq + 1), s));

    bool second = false;
    if (n > 0) {
        const uint64_t S = std::min<uint64_t>(n, kSampleMax);
        if (W == 1) MIH_TRY(launch_sample<1>(codes, S, queries, nq, q, nullptr, k, n, thr, s));
        else if (W == 2) MIH_TRY(launch_sample<2>(codes, S, queries, nq, q, nullptr, k, n, thr, s));
        else MIH_TRY(launch_sample<4>(codes, S, queries, nq, q, nullptr, k, n, thr, s));
        int32_t hthr[kNaMaxQueries];
        MIH_CUDA(cudaMemcpyAsync(hthr, thr, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        std::nth_element(hthr, hthr + nq / 2, hthr + nq);
        const int G = choose_group(W, hthr[nq / 2]);

        const uint32_t qtiles = (nq + kLsQueries - 1) / kLsQueries;
        uint64_t splits = (static_cast<uint64_t>(dev.sms) * 4 + qtiles - 1) / qtiles;
        const uint64_t max_splits = (n + kLsTile - 1) / kLsTile;
        if (splits > max_splits) splits = max_splits;
        if (splits < 1) splits = 1;
        if (splits > 65535) splits = 65535;
        uint64_t split_len = (n + splits - 1) / splits;
        split_len = (split_len + kLsTile - 1) / kLsTile * kLsTile;
        splits = (n + split_len - 1) / split_len;

        ScanArgs a;
        memset(&a, 0, sizeof(a));
        a.codes = codes;
        a.n = n;
        a.queries = queries;
        a.nq = nq;
        a.qbits = q;
        a.kq = nullptr;
        a.k_uniform = k;
        a.split_len = split_len;
        a.thr = thr;
        a.hist = hist;
        a.buf = buf;
        a.cap = kNaCap;
        a.cnt = cnt;
        const dim3 grid(qtiles, static_cast<unsigned>(splits));
        MIH_TRY(launch_scan(a, W, G, grid, s));
        finish_first_pass_kernel<<<grid1(nq + 1), 256, 0, s>>>(nq, q, n, nullptr, k, hist, cnt, kNaCap, dk, thr,
                                                              need, n_over);
        MIH_LAUNCH_CHECK();
        unsigned int hover = 0;
        MIH_CUDA(cudaMemcpyAsync(&hover, n_over, sizeof(hover), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        if (hover > 0) {
            // Offsets of the second pass (exact counts within d_k), on the host.
            uint64_t h[kNaMaxQueries + 1];
            MIH_CUDA(cudaMemcpyAsync(h, need, sizeof(uint64_t) * (nq + 1), cudaMemcpyDeviceToHost, s));
            MIH_CUDA(cudaStreamSynchronize(s));
            uint64_t run = 0;
            for (uint32_t i = 0; i <= nq; ++i) {
                const uint64_t c = i < nq ? h[i] : 0;
                h[i] = run;
                run += c;
            }
            if (run > kNaSecond) {
                set_error("linscan_knn_noalloc: %llu codes tie within the k-th distance; the fixed scratch holds "
                          "%llu (use linscan_knn)",
                          static_cast<unsigned long long>(run), static_cast<unsigned long long>(kNaSecond));
                return MIH_ENOMEM;
            }
            MIH_CUDA(cudaMemcpyAsync(need, h, sizeof(uint64_t) * (nq + 1), cudaMemcpyHostToDevice, s));
            ScanArgs b = a;
            b.buf = buf2;
            b.cnt = cursor;
            b.base = need;
            b.second_pass = 1;
            b.err = scan_err;
            MIH_TRY(launch_scan(b, W, 1, grid, s));
            second = true;
        }
    } else {
        MIH_CUDA(cudaMemsetAsync(dk, 0, sizeof(int32_t) * nq, s));
    }

    SelectInputs si;
    si.nq = nq;
    si.n = n;
    si.q = q;
    si.kq = nullptr;
    si.k_uniform = k;
    si.kmax = k;
    si.out_off = nullptr;
    si.hist = hist;
    si.dk = dk;
    si.buf1 = buf;
    si.cap = kNaCap;
    si.cnt1 = cnt;
    si.buf2 = second ? buf2 : nullptr;
    si.base2 = need;
    si.out_ids = out_ids;
    si.out_dist = out_dist;
    MIH_TRY(launch_select_noalloc(si, select_err, s));
    int herr[2] = {0, 0};
    MIH_CUDA(cudaMemcpyAsync(herr, scan_err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    if (herr[0] || herr[1]) {
        set_error("linscan_knn_noalloc: internal count mismatch (scan %d, select %d)", herr[0], herr[1]);
        return MIH_EINTERNAL;
    }
    return MIH_OK;
}
