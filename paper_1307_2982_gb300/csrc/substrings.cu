// substrings.cu -- substring optimisation (Sec. 5.5 "Substring Optimization"):
// the correlation between code bits measured on the GPU, the paper's greedy
// assignment of bits to substrings, and the bit permutation applied to codes.
//
// The permutation changes no result: the same permutation of the bits of two
// codes keeps their Hamming distance, and ids are row positions, which the
// permuted copy keeps.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "launch.h"
#include "substrings.h"

namespace mih {
namespace {

constexpr int kTile = 8;   // bits per side of a pair-count tile

// planes[a][w] bit i = bit a of code 32 w + i (0 past n).  One warp per 32
// codes: lane i holds code 32 w + i, and a ballot per bit builds the plane
// word; lane (a mod 32) keeps the words of bits a = lane, lane + 32, ...
template <int W>
__global__ void bitplanes_kernel(const uint64_t* __restrict__ codes, uint64_t n, uint64_t nw,
                                 uint32_t* __restrict__ planes) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t w = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; w < nw; w += warps) {
        const uint64_t i = 32 * w + lane;
        uint64_t c[W];
#pragma unroll
        for (int k = 0; k < W; ++k) c[k] = i < n ? codes[i * W + k] : 0ull;
        uint32_t mine[2 * W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t half = static_cast<uint32_t>(c[k] >> (32 * h));
                // bits 64 k + 32 h + b, b = 0..31: bit b of `half`
                uint32_t keep = 0;
                for (int b = 0; b < 32; ++b) {
                    const uint32_t word = __ballot_sync(0xFFFFFFFFu, (half >> b) & 1u);
                    if (static_cast<uint32_t>(b) == lane) keep = word;
                }
                mine[2 * k + h] = keep;
            }
        }
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) planes[static_cast<uint64_t>(32 * k + lane) * nw + w] = mine[k];
    }
}

// counts[a][b] += sum_w popc(planes[a][w] & planes[b][w]) for the 8 x 8 tile
// (blockIdx.x, blockIdx.y); blockIdx.z strides the words.
__global__ void __launch_bounds__(256) pair_counts_kernel(const uint32_t* __restrict__ planes, uint64_t nw, int q,
                                                          unsigned long long* __restrict__ counts) {
    __shared__ unsigned int s_cnt[kTile * kTile];
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) s_cnt[i] = 0;
    __syncthreads();
    const int a0 = blockIdx.x * kTile, b0 = blockIdx.y * kTile;
    unsigned int acc[kTile * kTile];
#pragma unroll
    for (int i = 0; i < kTile * kTile; ++i) acc[i] = 0;
    const uint64_t stride = static_cast<uint64_t>(gridDim.z) * blockDim.x;
    for (uint64_t w = blockIdx.z * static_cast<uint64_t>(blockDim.x) + threadIdx.x; w < nw; w += stride) {
        uint32_t pa[kTile], pb[kTile];
#pragma unroll
        for (int i = 0; i < kTile; ++i) {
            pa[i] = __ldg(planes + static_cast<uint64_t>(a0 + i) * nw + w);
            pb[i] = __ldg(planes + static_cast<uint64_t>(b0 + i) * nw + w);
        }
#pragma unroll
        for (int i = 0; i < kTile; ++i)
#pragma unroll
            for (int j = 0; j < kTile; ++j) acc[i * kTile + j] += __popc(pa[i] & pb[j]);
    }
#pragma unroll
    for (int i = 0; i < kTile * kTile; ++i)
        if (acc[i]) atomicAdd(&s_cnt[i], acc[i]);
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
        const int a = a0 + i / kTile, b = b0 + i % kTile;
        if (s_cnt[i] && a < q && b < q) atomicAdd(&counts[a * q + b], static_cast<unsigned long long>(s_cnt[i]));
    }
}

// out bit p of each code = in bit order[p].
template <int W>
__global__ void permute_bits_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n,
                                    const int32_t* __restrict__ order) {
    __shared__ int32_t s_order[64 * W];
    for (int p = threadIdx.x; p < 64 * W; p += blockDim.x) s_order[p] = order[p];
    __syncthreads();
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t c[W], r[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            c[k] = in[i * W + k];
            r[k] = 0ull;
        }
#pragma unroll
        for (int k = 0; k < W; ++k) {
            for (int b = 0; b < 64; ++b) {
                const int src = s_order[64 * k + b];
                uint64_t word = c[0];
#pragma unroll
                for (int u = 1; u < W; ++u)
                    if ((src >> 6) == u) word = c[u];
                r[k] |= ((word >> (src & 63)) & 1ull) << b;
            }
        }
#pragma unroll
        for (int k = 0; k < W; ++k) out[i * W + k] = r[k];
    }
}

unsigned grid_for_codes(uint64_t n, int sms) {
    const uint64_t want = (n + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(sms) * 32;
    return static_cast<unsigned>(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

mih_status check_bit_order(const int32_t* order, int q) {
    std::vector<char> seen(q, 0);
    for (int p = 0; p < q; ++p) {
        const int32_t b = order[p];
        if (b < 0 || b >= q || seen[b]) {
            set_error("bit_order must list each of the q = %d bit indices once (entry %d is %d)", q, p, b);
            return MIH_EINVAL;
        }
        seen[b] = 1;
    }
    return MIH_OK;
}

mih_status permute_codes(const uint64_t* in, uint64_t* out, uint64_t n, int q, const int32_t* order_dev,
                         cudaStream_t s) {
    if (n == 0) return MIH_OK;
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    const unsigned grid = grid_for_codes(n, dev.sms);
    if (q == 64) permute_bits_kernel<1><<<grid, 256, 0, s>>>(in, out, n, order_dev);
    else if (q == 128) permute_bits_kernel<2><<<grid, 256, 0, s>>>(in, out, n, order_dev);
    else permute_bits_kernel<4><<<grid, 256, 0, s>>>(in, out, n, order_dev);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

}  // namespace mih

using namespace mih;

extern "C" {

mih_status mih_bit_correlation(const uint64_t* codes, uint64_t n, int q, double* corr, void* stream) {
    clear_error();
    if (q != 64 && q != 128 && q != 256) {
        set_error("mih_bit_correlation: q must be 64, 128 or 256 (got %d)", q);
        return MIH_EINVAL;
    }
    if (n == 0 || n >= 0xFFFFFFFFull) {
        set_error("mih_bit_correlation: need 1 <= n < 2^32 - 1");
        return MIH_EINVAL;
    }
    if (!corr) {
        set_error("mih_bit_correlation: corr is NULL");
        return MIH_EINVAL;
    }
    MIH_TRY(check_device_ptr(codes, "mih_bit_correlation: codes"));
    MIH_TRY(check_code_alignment(codes, q / 64, "mih_bit_correlation: codes"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallScope scope(s);
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    Workspace ws(s);
    const uint64_t nw = (n + 31) / 32;
    uint32_t* planes;
    unsigned long long* counts;
    MIH_TRY(ws.alloc(&planes, static_cast<size_t>(q) * nw));
    MIH_TRY(ws.alloc(&counts, static_cast<size_t>(q) * q));
    MIH_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * q * q, s));
    const unsigned warps_grid = grid_for_codes(nw * 32, dev.sms);
    if (q == 64) bitplanes_kernel<1><<<warps_grid, 256, 0, s>>>(codes, n, nw, planes);
    else if (q == 128) bitplanes_kernel<2><<<warps_grid, 256, 0, s>>>(codes, n, nw, planes);
    else bitplanes_kernel<4><<<warps_grid, 256, 0, s>>>(codes, n, nw, planes);
    MIH_LAUNCH_CHECK();
    const int tiles = q / kTile;
    uint64_t zs = (nw + 255) / 256;
    const uint64_t zmax = (static_cast<uint64_t>(dev.sms) * 8 + tiles * tiles - 1) / (tiles * tiles);
    if (zs > zmax) zs = zmax;
    if (zs < 1) zs = 1;
    pair_counts_kernel<<<dim3(tiles, tiles, static_cast<unsigned>(zs)), 256, 0, s>>>(planes, nw, q, counts);
    MIH_LAUNCH_CHECK();
    std::vector<unsigned long long> h(static_cast<size_t>(q) * q);
    MIH_CUDA(cudaMemcpyAsync(h.data(), counts, sizeof(unsigned long long) * q * q, cudaMemcpyDeviceToHost, s));
    MIH_CUDA(cudaStreamSynchronize(s));
    const double nn = static_cast<double>(n);
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            const double ca = static_cast<double>(h[a * q + a]), cb = static_cast<double>(h[b * q + b]);
            const double den = ca * (nn - ca) * cb * (nn - cb);
            corr[a * q + b] = den > 0.0 ? (nn * static_cast<double>(h[a * q + b]) - ca * cb) / sqrt(den) : 0.0;
        }
    return MIH_OK;
}

mih_status mih_greedy_substrings(const double* corr, int q, int m, uint64_t seed, int32_t* bit_order) {
    clear_error();
    if (q != 64 && q != 128 && q != 256) {
        set_error("mih_greedy_substrings: q must be 64, 128 or 256 (got %d)", q);
        return MIH_EINVAL;
    }
    if (m < 1 || m > q) {
        set_error("mih_greedy_substrings: need 1 <= m <= q (m = %d)", m);
        return MIH_EINVAL;
    }
    if (!corr || !bit_order) {
        set_error("mih_greedy_substrings: NULL pointer");
        return MIH_EINVAL;
    }
    std::vector<int32_t> off(m), len(m);
    MIH_TRY(static_cast<mih_status>(mih_substring_layout(q, m, off.data(), len.data())));
    std::vector<std::vector<int>> sub(m);
    std::vector<char> used(q, 0);
    auto c = [&](int a, int b) { return fabs(corr[a * q + b]); };
    auto take = [&](int j, int b) {
        sub[j].push_back(b);
        used[b] = 1;
    };
    // first bit of every substring: a seeded bit for substring 0, then the
    // unused bit most correlated with the previous substring's first bit
    take(0, static_cast<int>(seed % static_cast<uint64_t>(q)));
    for (int j = 1; j < m; ++j) {
        const int prev = sub[j - 1][0];
        int best = -1;
        double bv = -1.0;
        for (int b = 0; b < q; ++b)
            if (!used[b] && c(prev, b) > bv) {
                bv = c(prev, b);
                best = b;
            }
        take(j, best);
    }
    // then one bit at a time, substrings in turn: the unused bit whose largest
    // correlation with the substring's bits is smallest
    int placed = m;
    for (int j = 0; placed < q; j = (j + 1) % m) {
        if (static_cast<int>(sub[j].size()) >= len[j]) continue;
        int best = -1;
        double bv = 0.0;
        for (int b = 0; b < q; ++b) {
            if (used[b]) continue;
            double worst = 0.0;
            for (int a : sub[j]) worst = fmax(worst, c(a, b));
            if (best < 0 || worst < bv) {
                bv = worst;
                best = b;
            }
        }
        take(j, best);
        ++placed;
    }
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < len[j]; ++i) bit_order[off[j] + i] = sub[j][i];
    return MIH_OK;
}

}  // extern "C"
