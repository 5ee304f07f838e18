// rerank.cu -- re-ranking of candidate lists by an asymmetric Hamming
// distance.  Sec. 5.1 notes that Hamming distance leaves equidistant codes
// unordered and that a re-ranking phase with an asymmetric Hamming distance
// helps; the Conclusion describes it: the query stays real-valued, multi-index
// hashing supplies the candidates and the asymmetric distance culls them.
// The distance (the paper gives no formula) is
//     a(y, h) = sum of |y_b| over the bits b where h_b != [y_b > 0],
// with y the query's q real projections (their signs are its code), summed
// exactly on a fixed-point grid: with 2^E <= max |y_b| < 2^(E+1) the weights
// are w_b = floor(|y_b| 2^(53-E)) (below 2^54), their sum is an exact
// integer (below 2^62) in any order, and a is that sum rounded to double,
// times 2^-(53-E).
//
// Rows of up to 256 candidates take one warp each (the row sorted in
// registers and by shuffles); longer rows one CTA each: the row's weights and
// sign code go to shared memory, every thread scores candidates (a 16- or
// 32-byte code gathered by id, then one 64-bit integer add per disagreeing
// bit), and a bitonic network over the row sorts the (sum, id) pairs in
// shared memory.
#include <cuda_runtime.h>

#include <algorithm>

#include "launch.h"
#include "mih_internal.cuh"

namespace mih {
namespace {

struct RerankArgs {
    const uint64_t* codes;
    uint64_t n;
    const float* proj;    // [nq][64 W]
    const uint32_t* ids;  // [nq][k_in]
    uint32_t k_in, k, P;  // P: power of two >= k_in, the sort width
    uint32_t* out_ids;    // [nq][k]
    double* out_a;
    unsigned int* bad;    // bit 0: a candidate id >= n; bit 1: a row longer than k_in;
                          // bit 2: a result row longer than MIH_MAX_K
    const uint64_t* in_off;    // CSR rows (nullable: uniform rows of k_in)
    const uint64_t* out_off;   // CSR results (nullable: uniform rows of k)
};

// Row `row`'s candidates ids[ib, ib + len) and result slots [ob, ob + kr).
struct RowSpan {
    uint64_t ib, ob;
    uint32_t len, kr;
};

__device__ __forceinline__ RowSpan row_span(const RerankArgs& a, uint64_t row, bool report) {
    RowSpan r;
    if (a.in_off) {
        r.ib = a.in_off[row];
        const uint64_t e = a.in_off[row + 1];
        const bool over = e < r.ib || e - r.ib > a.k_in;
        if (over && report) atomicOr(a.bad, 2u);
        r.len = over ? 0u : static_cast<uint32_t>(e - r.ib);
    } else {
        r.ib = row * a.k_in;
        r.len = a.k_in;
    }
    if (a.out_off) {
        r.ob = a.out_off[row];
        const uint64_t e = a.out_off[row + 1];
        const bool over = e < r.ob || e - r.ob > MIH_MAX_K;
        if (over && report) atomicOr(a.bad, 4u);
        r.kr = over ? 0u : static_cast<uint32_t>(e - r.ob);
    } else {
        r.ob = row * a.k;
        r.kr = a.k;
    }
    return r;
}

// Shared memory of a row: sort keys (the integer sums), the weights, the
// sign code, ids, and the row's largest |y_b| (as its fp32 bit pattern).
template <int W>
constexpr size_t rerank_smem_bytes(uint32_t P) {
    return static_cast<size_t>(P) * 12 + W * 64 * 8 + W * 8 + 8;
}

// 2^e as a double, for -1022 <= e <= 1023 (built from its bits: exact).
__device__ __forceinline__ double pow2(int e) {
    return __longlong_as_double(static_cast<long long>(1023 + e) << 52);
}

template <int W>
__global__ void __launch_bounds__(512) rerank_asym_kernel(RerankArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* key = reinterpret_cast<uint64_t*>(smem);
    uint64_t* wt = key + a.P;          // [64 W] grid weights
    uint64_t* qcode = wt + 64 * W;     // [W] sign code
    uint32_t* cid = reinterpret_cast<uint32_t*>(qcode + W);
    uint32_t* ymax = cid + a.P;        // largest |y_b|, fp32 bits (nonnegative: they order as integers)

    const uint64_t row = blockIdx.x;
    const RowSpan rs = row_span(a, row, threadIdx.x == 0);
    const float* y = a.proj + row * (64 * W);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    if (threadIdx.x == 0) *ymax = 0u;
    __syncthreads();
    for (int w32 = warp; w32 < 2 * W; w32 += warps) {
        const float v = __ldg(y + w32 * 32 + lane);
        const unsigned bits = __ballot_sync(0xffffffffu, v > 0.f);
        const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(v)));
        if (lane == 0) {
            reinterpret_cast<uint32_t*>(qcode)[w32] = bits;   // little-endian words
            atomicMax(ymax, m);
        }
    }
    __syncthreads();
    // the grid: s = 53 - E, E the binary exponent of the largest |y_b|
    const double M = static_cast<double>(__uint_as_float(*ymax));
    const int s = M > 0.0 ? 53 - (static_cast<int>((__double_as_longlong(M) >> 52) & 0x7FF) - 1023) : 0;
    const double scale = pow2(s);
    for (int b = threadIdx.x; b < 64 * W; b += blockDim.x)
        wt[b] = __double2ull_rz(static_cast<double>(fabsf(__ldg(y + b))) * scale);   // exact product, floor
    __syncthreads();

    uint32_t g[2 * W];
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) g[w] = reinterpret_cast<const uint32_t*>(qcode)[w];
    for (uint32_t i = threadIdx.x; i < a.P; i += blockDim.x) {
        uint64_t kk = ~0ull;
        uint32_t id = kPadId;
        if (i < rs.len) {
            id = __ldg(a.ids + rs.ib + i);
            if (id != kPadId && id >= a.n) {
                atomicOr(a.bad, 1u);
                id = kPadId;
            }
            if (id != kPadId) {
                const Code<W> h = load_code<W>(a.codes, id);
                uint64_t acc = 0;
#pragma unroll
                for (int w = 0; w < 2 * W; ++w) {
                    const uint64_t hw = h.w[w >> 1];
                    uint32_t x = static_cast<uint32_t>((w & 1) ? (hw >> 32) : hw) ^ g[w];
                    while (x) {
                        acc += wt[32 * w + __ffs(x) - 1];
                        x &= x - 1;
                    }
                }
                kk = acc;
            }
        }
        key[i] = kk;
        cid[i] = id;
    }

    // bitonic sort of (sum, id), ascending; padding (key ~0, id ~0) goes last
    for (uint32_t size = 2; size <= a.P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < a.P / 2; t += blockDim.x) {
                const uint32_t lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
                const uint64_t kl = key[lo], kh = key[hi];
                const uint32_t il = cid[lo], ih = cid[hi];
                const bool greater = kl > kh || (kl == kh && il > ih);
                if (greater == ((lo & size) == 0)) {
                    key[lo] = kh;
                    key[hi] = kl;
                    cid[lo] = ih;
                    cid[hi] = il;
                }
            }
        }
    }
    __syncthreads();

    for (uint32_t p = threadIdx.x; p < rs.kr; p += blockDim.x) {
        const bool real = p < a.P && key[p] != ~0ull;
        a.out_ids[rs.ob + p] = real ? cid[p] : kPadId;
        a.out_a[rs.ob + p] = real ? __ull2double_rn(key[p]) * pow2(-s) : -1.0;
    }
}

// Rows of up to 256 candidates: one warp per row, no block barriers.  The
// row's P = 32 E slots are held E per lane (slot x = 32 e + lane): the lane
// scores its E candidates with their gathers in flight together, then a
// bitonic network sorts the slots, exchanging across lanes by shuffles
// (strides below 32) and within a lane in registers (strides 32 and up).
constexpr int kRowWarps = 8;

// Keep the smaller (ascending) or larger of (k, i) and its partner (pk, pi).
__device__ __forceinline__ void keep_side(uint64_t& k, uint32_t& i, uint64_t pk, uint32_t pi, bool smaller) {
    const bool mine_less = k < pk || (k == pk && i < pi);
    if (mine_less != smaller) {
        k = pk;
        i = pi;
    }
}

template <int W, int E>
__global__ void __launch_bounds__(kRowWarps * 32) rerank_warp_kernel(RerankArgs a, uint32_t nq) {
    __shared__ uint64_t s_wt[kRowWarps][64 * W];
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t row = static_cast<uint64_t>(blockIdx.x) * kRowWarps + warp;
    if (row >= nq) return;   // warp-uniform; the kernel has no block barrier
    const RowSpan rs = row_span(a, row, threadIdx.x % 32 == 0);
    uint64_t* wt = s_wt[warp];
    const float* y = a.proj + row * (64 * W);

    // sign code (ballots) and the grid of the largest |y_b|
    uint32_t g[2 * W];
    float v[2 * W];
    uint32_t mx = 0u;
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) {
        v[w] = __ldg(y + 32 * w + lane);
        g[w] = __ballot_sync(0xffffffffu, v[w] > 0.f);
        mx = max(mx, __float_as_uint(fabsf(v[w])));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    const double M = static_cast<double>(__uint_as_float(mx));
    const int s = M > 0.0 ? 53 - (static_cast<int>((__double_as_longlong(M) >> 52) & 0x7FF) - 1023) : 0;
    const double scale = pow2(s);
#pragma unroll
    for (int w = 0; w < 2 * W; ++w)
        wt[32 * w + lane] = __double2ull_rz(static_cast<double>(fabsf(v[w])) * scale);   // exact product, floor
    __syncwarp();

    uint64_t key[E];
    uint32_t cid[E];
    Code<W> h[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t x = 32u * e + lane;
        cid[e] = x < rs.len ? __ldg(a.ids + rs.ib + x) : kPadId;
        if (cid[e] != kPadId && cid[e] >= a.n) {
            atomicOr(a.bad, 1u);
            cid[e] = kPadId;
        }
        if (cid[e] != kPadId) h[e] = load_code<W>(a.codes, cid[e]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        key[e] = ~0ull;
        if (cid[e] != kPadId) {
            uint64_t acc = 0;
#pragma unroll
            for (int w = 0; w < 2 * W; ++w) {
                const uint64_t hw = h[e].w[w >> 1];
                uint32_t x = static_cast<uint32_t>((w & 1) ? (hw >> 32) : hw) ^ g[w];
                while (x) {
                    acc += wt[32 * w + __ffs(x) - 1];
                    x &= x - 1;
                }
            }
            key[e] = acc;
        }
    }

    // bitonic sort of the 32 E slots by (sum, id), ascending
#pragma unroll
    for (uint32_t size = 2; size <= 32u * E; size <<= 1) {
#pragma unroll
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int se = static_cast<int>(stride >> 5);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int f = e ^ se;
                    if (f > e) {
                        const bool asc = ((32u * e + lane) & size) == 0;
                        const bool greater = key[e] > key[f] || (key[e] == key[f] && cid[e] > cid[f]);
                        if (greater == asc) {
                            const uint64_t tk = key[e];
                            const uint32_t ti = cid[e];
                            key[e] = key[f];
                            cid[e] = cid[f];
                            key[f] = tk;
                            cid[f] = ti;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t pk = __shfl_xor_sync(0xffffffffu, key[e], stride);
                    const uint32_t pi = __shfl_xor_sync(0xffffffffu, cid[e], stride);
                    const bool asc = ((32u * e + lane) & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    keep_side(key[e], cid[e], pk, pi, lower == asc);
                }
            }
        }
    }

    const double unscale = pow2(-s);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t x = 32u * e + lane;
        if (x < rs.kr) {
            const bool real = key[e] != ~0ull;
            a.out_ids[rs.ob + x] = real ? cid[e] : kPadId;
            a.out_a[rs.ob + x] = real ? __ull2double_rn(key[e]) * unscale : -1.0;
        }
    }
    for (uint32_t x = 32u * E + lane; x < rs.kr; x += 32) {
        a.out_ids[rs.ob + x] = kPadId;
        a.out_a[rs.ob + x] = -1.0;
    }
}

template <int W, int E>
mih_status launch_rerank_rows(const RerankArgs& a, uint32_t nq, cudaStream_t s) {
    const unsigned blocks = (nq + kRowWarps - 1) / kRowWarps;
    main_kernel_begin(s);
    {
        KernelSpan span(s, MIH_PROF_RERANK);
        rerank_warp_kernel<W, E><<<blocks, kRowWarps * 32, 0, s>>>(a, nq);
    }
    main_kernel_end(s);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

template <int W>
mih_status launch_rerank(const RerankArgs& a, uint32_t nq, cudaStream_t s) {
    // rows of up to 256 candidates: a warp per row
    if (a.P <= 32) return launch_rerank_rows<W, 1>(a, nq, s);
    if (a.P == 64) return launch_rerank_rows<W, 2>(a, nq, s);
    if (a.P == 128) return launch_rerank_rows<W, 4>(a, nq, s);
    if (a.P == 256) return launch_rerank_rows<W, 8>(a, nq, s);

    const size_t smem = rerank_smem_bytes<W>(a.P);
    if (smem > 48 * 1024)
        MIH_CUDA(cudaFuncSetAttribute(rerank_asym_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
    const unsigned threads = std::min<unsigned>(512u, std::max<unsigned>(64u, a.P));
    main_kernel_begin(s);
    {
        KernelSpan span(s, MIH_PROF_RERANK);
        rerank_asym_kernel<W><<<nq, threads, smem, s>>>(a);
    }
    main_kernel_end(s);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

}  // namespace
}  // namespace mih

namespace mih {
namespace {

// The checks and the launch shared by both entry points (`name` prefixes
// error messages).  in_off / out_off null: uniform rows of k_in / k.
mih_status rerank_call(const char* name, const uint64_t* codes, uint64_t n, int q, const float* proj, uint32_t nq,
                       const uint32_t* ids, const uint64_t* in_off, uint32_t k_in, const uint64_t* out_off,
                       uint32_t k, uint32_t* out_ids, double* out_a, void* stream) {
    clear_error();
    if (q != 64 && q != 128 && q != 256) {
        set_error("%s: q must be 64, 128 or 256 (got %d)", name, q);
        return MIH_EINVAL;
    }
    if (n >= 0xFFFFFFFFull) {
        set_error("%s: n must be below 2^32 - 1", name);
        return MIH_EINVAL;
    }
    if (k_in < 1 || k_in > MIH_MAX_K || (out_off == nullptr && (k < 1 || k > MIH_MAX_K))) {
        set_error("%s: k_in and k must be in [1, %u]", name, MIH_MAX_K);
        return MIH_EINVAL;
    }
    if (nq > (1u << 23)) {
        set_error("%s: nq must be at most 2^23", name);
        return MIH_EINVAL;
    }
    if (nq == 0) return MIH_OK;
    const int W = q / 64;
    if (n > 0) {
        MIH_TRY(check_device_ptr(codes, "rerank: codes"));
        MIH_TRY(check_code_alignment(codes, W, "rerank: codes"));
    }
    MIH_TRY(check_device_ptr(proj, "rerank: proj"));
    MIH_TRY(check_device_ptr(ids, "rerank: ids"));
    MIH_TRY(check_device_ptr(out_ids, "rerank: out_ids"));
    MIH_TRY(check_device_ptr(out_a, "rerank: out_a"));
    if (in_off) MIH_TRY(check_device_ptr(in_off, "rerank: in_offsets"));
    if (out_off) MIH_TRY(check_device_ptr(out_off, "rerank: out_offsets"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallScope scope(s);
    Workspace ws(s);
    unsigned int* bad;
    MIH_TRY(ws.alloc(&bad, 1));
    MIH_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));

    RerankArgs a;
    a.codes = codes;
    a.n = n;
    a.proj = proj;
    a.ids = ids;
    a.k_in = k_in;
    a.k = k;
    a.P = 2;
    while (a.P < k_in) a.P <<= 1;
    a.out_ids = out_ids;
    a.out_a = out_a;
    a.bad = bad;
    a.in_off = in_off;
    a.out_off = out_off;
    if (W == 1) MIH_TRY(launch_rerank<1>(a, nq, s));
    else if (W == 2) MIH_TRY(launch_rerank<2>(a, nq, s));
    else MIH_TRY(launch_rerank<4>(a, nq, s));
    unsigned int hbad = 0;
    MIH_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    if (hbad & 1u) {
        set_error("%s: a candidate id is >= n (0xFFFFFFFF is the only padding id)", name);
        return MIH_EINVAL;
    }
    if (hbad & 2u) {
        set_error("%s: a candidate row is longer than k_in (or its offsets decrease)", name);
        return MIH_EINVAL;
    }
    if (hbad & 4u) {
        set_error("%s: a result row is longer than MIH_MAX_K (or its offsets decrease)", name);
        return MIH_EINVAL;
    }
    return MIH_OK;
}

}  // namespace
}  // namespace mih

extern "C" mih_status mih_rerank_asym(const uint64_t* codes, uint64_t n, int q, const float* proj, uint32_t nq,
                                      const uint32_t* ids, uint32_t k_in, uint32_t k, uint32_t* out_ids,
                                      double* out_a, void* stream) {
    return mih::rerank_call("mih_rerank_asym", codes, n, q, proj, nq, ids, nullptr, k_in, nullptr, k, out_ids,
                            out_a, stream);
}

extern "C" mih_status mih_rerank_asym_csr(const uint64_t* codes, uint64_t n, int q, const float* proj,
                                          uint32_t nq, const uint32_t* ids, const uint64_t* in_offsets,
                                          uint32_t k_in_max, const uint64_t* out_offsets, uint32_t* out_ids,
                                          double* out_a, void* stream) {
    if (in_offsets == nullptr || out_offsets == nullptr) {
        mih::clear_error();
        mih::set_error("mih_rerank_asym_csr: in_offsets and out_offsets are required");
        return MIH_EINVAL;
    }
    return mih::rerank_call("mih_rerank_asym_csr", codes, n, q, proj, nq, ids, in_offsets, k_in_max, out_offsets,
                            0u, out_ids, out_a, stream);
}
