// util_kernels.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// The table build of Algorithm 1 is written as a stable radix sort of
// (substring key, id) pairs; the r-neighbour output is ordered with the same
// sort.  Both are bandwidth-bound streaming passes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "mih_internal.cuh"

namespace mih {
namespace {

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem_warp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_inclusive_scan(v);
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < kScanThreads / 32) ? smem_warp[lane] : T(0);
        T wi = warp_inclusive_scan(w);
        if (lane < kScanThreads / 32) smem_warp[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) smem_warp[kScanThreads / 32] = wi;
    }
    __syncthreads();
    T out = smem_warp[warp] + incl - v;
    *total = smem_warp[kScanThreads / 32];
    return out;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const T* __restrict__ in, size_t n,
                                                                   T* __restrict__ block_sums) {
    __shared__ T sw[kScanThreads / 32 + 1];
    const size_t base = static_cast<size_t>(blockIdx.x) * kScanTile;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        size_t idx = base + static_cast<size_t>(i) * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    T total;
    block_exclusive_scan(s, sw, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const T* in, T* out, size_t n,
                                                                 const T* __restrict__ block_prefix) {
    __shared__ T sw[kScanThreads / 32 + 1];
    const size_t base = static_cast<size_t>(blockIdx.x) * kScanTile +
                        static_cast<size_t>(threadIdx.x) * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        s += v[i];
    }
    T total;
    T run = block_exclusive_scan(s, sw, &total);
    if (block_prefix) run += block_prefix[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

template <typename T>
mih_status scan_exclusive(const T* in, T* out, size_t n, Workspace& ws) {
    if (n == 0) return MIH_OK;
    const size_t blocks = (n + kScanTile - 1) / kScanTile;
    if (blocks > 0x7FFFFFFFull) {
        set_error("scan: too many elements");
        return MIH_EINVAL;
    }
    T* sums = nullptr;
    if (blocks > 1) {
        MIH_TRY(ws.alloc(&sums, blocks));
        scan_reduce_kernel<T><<<static_cast<unsigned>(blocks), kScanThreads, 0, ws.stream()>>>(in, n, sums);
        MIH_LAUNCH_CHECK();
        MIH_TRY(scan_exclusive<T>(sums, sums, blocks, ws));
    }
    scan_down_kernel<T><<<static_cast<unsigned>(blocks), kScanThreads, 0, ws.stream()>>>(in, out, n, sums);
    MIH_LAUNCH_CHECK();
    if (sums) ws.release(sums);
    return MIH_OK;
}

// ------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRadix = 256;

// Per-tile digit counts, digit-major: counts[d * tiles + t].
template <typename K>
__global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const K* __restrict__ keys, size_t n, int shift,
                                                             uint32_t dmask, uint32_t* __restrict__ counts,
                                                             uint32_t tiles) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = static_cast<size_t>(blockIdx.x) * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsRounds; ++r) {
        size_t i = base + static_cast<size_t>(r) * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[static_cast<uint32_t>(keys[i] >> shift) & dmask], 1u);
    }
    __syncthreads();
    counts[static_cast<size_t>(threadIdx.x) * tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items are ranked in (round, thread) order, which is input
// order, so equal digits keep their relative order.
template <typename K, bool HAS_VAL, bool VAL_IOTA>
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(
    const K* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, size_t n, int shift,
    uint32_t dmask, const uint32_t* __restrict__ offsets, uint32_t tiles, K* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t base[kRadix];
    __shared__ uint32_t wcnt[kRsWarps][kRadix];
    __shared__ uint32_t wpos[kRsWarps][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offsets[static_cast<size_t>(threadIdx.x) * tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const size_t tile0 = static_cast<size_t>(blockIdx.x) * kRsTile;
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kRsRounds; ++r) {
        const size_t i = tile0 + static_cast<size_t>(r) * kRsThreads + threadIdx.x;
        const bool valid = i < n;
        K key = valid ? keys_in[i] : K(0);
        uint32_t val = 0;
        if constexpr (HAS_VAL) val = VAL_IOTA ? static_cast<uint32_t>(i) : (valid ? vals_in[i] : 0u);
        const uint32_t digit = valid ? (static_cast<uint32_t>(key >> shift) & dmask) : kRadix;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, digit);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t run = base[d];
#pragma unroll
            for (int w = 0; w < kRsWarps; ++w) {
                wpos[w][d] = run;
                run += wcnt[w][d];
                wcnt[w][d] = 0;
            }
            base[d] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wpos[warp][digit] + rank;
            keys_out[pos] = key;
            if constexpr (HAS_VAL) vals_out[pos] = val;
        }
    }
}

template <typename K, bool HAS_VAL>
mih_status radix_sort(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, bool vals_iota,
                      size_t n, int bits, Workspace& ws, K** keys_out, uint32_t** vals_out) {
    *keys_out = keys;
    if (vals_out) *vals_out = vals;
    if (n == 0) return MIH_OK;
    if (bits <= 0) {
        if (HAS_VAL && vals_iota) {
            set_error("radix sort: identity values need at least one pass");
            return MIH_EINTERNAL;
        }
        return MIH_OK;
    }
    if (n >= 0xFFFFFFFFull) {
        set_error("radix sort: n must be below 2^32 - 1");
        return MIH_EINVAL;
    }
    const uint32_t tiles = static_cast<uint32_t>((n + kRsTile - 1) / kRsTile);
    uint32_t* counts = nullptr;
    MIH_TRY(ws.alloc(&counts, static_cast<size_t>(tiles) * kRadix));
    K* kin = keys;
    K* kout = keys_alt;
    uint32_t* vin = vals;
    uint32_t* vout = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        const int width = (bits - shift) < 8 ? (bits - shift) : 8;
        const uint32_t dmask = (1u << width) - 1u;
        rs_hist_kernel<K><<<tiles, kRsThreads, 0, ws.stream()>>>(kin, n, shift, dmask, counts, tiles);
        MIH_LAUNCH_CHECK();
        MIH_TRY(scan_exclusive<uint32_t>(counts, counts, static_cast<size_t>(tiles) * kRadix, ws));
        if (HAS_VAL && vals_iota && shift == 0) {
            rs_scatter_kernel<K, HAS_VAL, true><<<tiles, kRsThreads, 0, ws.stream()>>>(
                kin, nullptr, n, shift, dmask, counts, tiles, kout, vout);
        } else {
            rs_scatter_kernel<K, HAS_VAL, false><<<tiles, kRsThreads, 0, ws.stream()>>>(
                kin, vin, n, shift, dmask, counts, tiles, kout, vout);
        }
        MIH_LAUNCH_CHECK();
        K* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    ws.release(counts);
    *keys_out = kin;
    if (vals_out) *vals_out = vin;
    return MIH_OK;
}

__global__ void fill_u32_kernel(uint32_t* p, uint32_t v, size_t n) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        p[i] = v;
}

}  // namespace

mih_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, size_t n, Workspace& ws) {
    return scan_exclusive<uint32_t>(in, out, n, ws);
}

// Scan with caller-provided block sums (no allocation; usable while a stream
// is being captured into a graph): tmp must hold scan_temp_u64(n) elements.
size_t scan_temp_u64(size_t n) {
    size_t total = 0;
    while (n > static_cast<size_t>(kScanTile)) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n;
    }
    return total > 0 ? total : 1;
}

mih_status scan_exclusive_u64_pre(const uint64_t* in, uint64_t* out, size_t n, uint64_t* tmp, cudaStream_t s) {
    if (n == 0) return MIH_OK;
    const size_t blocks = (n + kScanTile - 1) / kScanTile;
    uint64_t* sums = nullptr;
    if (blocks > 1) {
        sums = tmp;
        scan_reduce_kernel<uint64_t><<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(in, n, sums);
        MIH_LAUNCH_CHECK();
        MIH_TRY(scan_exclusive_u64_pre(sums, sums, blocks, tmp + blocks, s));
    }
    scan_down_kernel<uint64_t><<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(in, out, n, sums);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

mih_status scan_exclusive_u64(const uint64_t* in, uint64_t* out, size_t n, Workspace& ws) {
    return scan_exclusive<uint64_t>(in, out, n, ws);
}

mih_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                                bool vals_iota, size_t n, int bits, Workspace& ws,
                                uint32_t** keys_out, uint32_t** vals_out) {
    if (vals == nullptr || vals_alt == nullptr) {
        set_error("radix sort: both value buffers are required");
        return MIH_EINTERNAL;
    }
    return radix_sort<uint32_t, true>(keys, vals, keys_alt, vals_alt, vals_iota, n, bits, ws, keys_out,
                                      vals_out);
}

mih_status radix_sort_keys_u64(uint64_t* keys, uint64_t* keys_alt, size_t n, int bits, Workspace& ws,
                               uint64_t** keys_out) {
    return radix_sort<uint64_t, false>(keys, nullptr, keys_alt, nullptr, false, n, bits, ws, keys_out,
                                       nullptr);
}

mih_status fill_u32(uint32_t* p, uint32_t v, size_t n, cudaStream_t s) {
    if (n == 0) return MIH_OK;
    size_t blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    fill_u32_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p, v, n);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

}  // namespace mih
