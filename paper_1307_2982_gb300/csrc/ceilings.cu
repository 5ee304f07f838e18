// ceilings.cu -- throughput ceilings of the current GPU that the kernels'
// rooflines are quoted against (not part of the paper): the integer
// population count the linear scan is bound by, the tensor-core forms of the
// Hamming distance (Sec. 6 "Hamming Distance" computes it with xor and
// popcount; on tensor cores popc(a xor b) = popc a + popc b - 2 popc(a and b)
// over b1 operands, or (q - <a, b>) / 2 over +-1 operands), and the bandwidth
// of random 32-byte reads, which bounds gathering codes by id.
//
// Each measurement is one timed launch (after an untimed one) of a kernel that
// keeps independent chains of the operation in flight on every SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace mih {
namespace {

constexpr int kCeilThreads = 256;

// POPC: every thread keeps 8 independent chains (x -> popc(x) + x + c).
__global__ void __launch_bounds__(kCeilThreads) popc_rate_kernel(uint32_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = seed * (threadIdx.x + 1u) + i * 0x9E3779B9u + blockIdx.x;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = static_cast<uint32_t>(__popc(v[i])) + v[i] + 0x3Bu;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= v[i];
    if (acc == 0x12345678u) sink[0] = acc;   // keeps the chains alive
}

// b1 tensor op: m16n8k128, AND then popcount, s32 accumulators; 4
// independent accumulator tiles per warp.
__global__ void __launch_bounds__(kCeilThreads) b1_mma_rate_kernel(uint32_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[2], b[1];
    a[0] = seed ^ threadIdx.x;
    a[1] = seed * 3u + threadIdx.x;
    b[0] = seed * 7u ^ blockIdx.x;
    int32_t c[4][4] = {};
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
            asm volatile(
                "mma.sync.aligned.m16n8k128.row.col.s32.b1.b1.s32.and.popc "
                "{%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};"
                : "+r"(c[t][0]), "+r"(c[t][1]), "+r"(c[t][2]), "+r"(c[t][3])
                : "r"(a[0]), "r"(a[1]), "r"(b[0]));
    }
    int32_t acc = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) acc ^= c[t][0] ^ c[t][1] ^ c[t][2] ^ c[t][3];
    if (acc == 0x12345678) sink[0] = static_cast<uint32_t>(acc);
}

// fp8 tensor op: m16n8k32 e4m3 x e4m3 -> f32; 4 independent accumulator tiles.
__global__ void __launch_bounds__(kCeilThreads) fp8_mma_rate_kernel(uint32_t iters, uint32_t seed, uint32_t* sink) {
    // +-1.0 in e4m3 (0x38 / 0xB8) in every byte
    const uint32_t a0 = 0x38B838B8u ^ ((seed & 1u) << 7), a1 = 0xB838B838u, a2 = 0x3838B8B8u, a3 = 0xB8B83838u;
    const uint32_t b0 = 0x38383838u, b1 = 0xB838B838u ^ ((seed & 2u) << 6);
    float c[4][4] = {};
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 "
                "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                : "+f"(c[t][0]), "+f"(c[t][1]), "+f"(c[t][2]), "+f"(c[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) acc += c[t][0] + c[t][1] + c[t][2] + c[t][3];
    if (acc == 1234.5f) sink[0] = 1u;
}

// Random 32-byte reads: every thread reads `per` sectors at hashed positions
// of a buffer of nsec 32-byte sectors, 8 in flight.
__global__ void __launch_bounds__(kCeilThreads) gather_rate_kernel(const uint4* __restrict__ buf, uint64_t nsec,
                                                                   uint32_t per, uint32_t seed, uint32_t* sink) {
    uint64_t x = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 0x9E3779B97F4A7C15ull + seed;
    uint32_t acc = 0;
    for (uint32_t i = 0; i < per; i += 8) {
        uint4 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            x ^= x >> 31;
            x *= 0xBF58476D1CE4E5B9ull;
            x ^= x >> 29;
            const uint64_t s = x % nsec;
            const uint4 lo = __ldg(buf + 2 * s);
            const uint4 hi = __ldg(buf + 2 * s + 1);
            v[r] = make_uint4(lo.x ^ hi.x, lo.y ^ hi.y, lo.z ^ hi.z, lo.w ^ hi.w);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) acc ^= v[r].x ^ v[r].y ^ v[r].z ^ v[r].w;
    }
    if (acc == 0x12345678u) sink[0] = acc;
}

template <class Launch>
mih_status time_launch(cudaStream_t s, Launch&& launch, double* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MIH_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0);
        set_error("ceilings: event creation failed");
        return MIH_ECUDA;
    }
    launch();   // untimed
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    const cudaError_t e = cudaEventSynchronize(e1);
    float f = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&f, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MIH_CUDA(e);
    MIH_CUDA(cudaGetLastError());
    *ms = f;
    return MIH_OK;
}

}  // namespace
}  // namespace mih

extern "C" mih_status mih_measure_ceilings(mih_ceilings* out, uint64_t gather_bytes, void* stream) {
    using namespace mih;
    clear_error();
    if (!out) {
        set_error("mih_measure_ceilings: out is NULL");
        return MIH_EINVAL;
    }
    *out = mih_ceilings{};
    if (gather_bytes < (64ull << 20)) gather_bytes = 64ull << 20;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));
    Workspace ws(s);
    uint32_t* sink;
    MIH_TRY(ws.alloc(&sink, 1));
    const unsigned blocks = static_cast<unsigned>(dev.sms) * 8u;   // 8 x 256 threads per SM
    const double threads = static_cast<double>(blocks) * kCeilThreads;

    double ms = 0.0;
    const uint32_t it_popc = 4096;
    MIH_TRY(time_launch(s, [&] { popc_rate_kernel<<<blocks, kCeilThreads, 0, s>>>(it_popc, 7u, sink); }, &ms));
    out->popc_per_s = threads * it_popc * 8.0 / (ms * 1e-3);

    const uint32_t it_mma = 2048;
    const double warps = threads / 32.0;
    MIH_TRY(time_launch(s, [&] { b1_mma_rate_kernel<<<blocks, kCeilThreads, 0, s>>>(it_mma, 5u, sink); }, &ms));
    // one m16n8k128 = 16 x 8 (row, column) pairs of 128-bit operands
    out->b1_mma_pairs128_per_s = warps * it_mma * 4.0 * 128.0 / (ms * 1e-3);
    MIH_TRY(time_launch(s, [&] { fp8_mma_rate_kernel<<<blocks, kCeilThreads, 0, s>>>(it_mma, 3u, sink); }, &ms));
    // one m16n8k32 = 16 x 8 x 32 multiply-adds; a 128-bit pair needs 128
    out->fp8_mma_tflops = warps * it_mma * 4.0 * 16.0 * 8.0 * 32.0 * 2.0 / (ms * 1e-3) / 1e12;
    out->fp8_mma_pairs128_per_s = out->fp8_mma_tflops * 1e12 / 256.0;

    // random sectors of a buffer far larger than L2
    uint4* buf = nullptr;
    MIH_TRY(ws.alloc(&buf, gather_bytes / 16));
    MIH_CUDA(cudaMemsetAsync(buf, 0x5A, gather_bytes, s));
    const uint64_t nsec = gather_bytes / 32;
    const uint32_t per = 256;
    MIH_TRY(time_launch(s, [&] { gather_rate_kernel<<<blocks, kCeilThreads, 0, s>>>(buf, nsec, per, 11u, sink); },
                        &ms));
    out->gather32_gbs = threads * per * 32.0 / (ms * 1e-3) / 1e9;
    out->sms = dev.sms;
    int clk = 0;
    if (cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev.device) == cudaSuccess) out->sm_clock_mhz = clk / 1000.0;
    cudaGetLastError();
    MIH_CUDA(cudaStreamSynchronize(s));
    return MIH_OK;
}
