// build.cu -- Algorithm 1: one hash table per substring (mih_build).
//
// Per table j: extract the s_j-bit substring keys of all codes, stable radix
// sort (key, id), then write the buckets as CSR.  Short substrings get a
// direct-addressed offsets array over all 2^s buckets; long ones (s > 24,
// where 2^s offsets would dominate memory) keep only the distinct keys, in an
// open-addressing index of 32-byte buckets, each holding four {key, rank}
// slots, next to begins[rank].  This stands in for the paper's sparse
// direct-address tables of Sec. 6: the occupancy words and group pointers
// become a hash probe that usually touches one 32-byte sector.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "index.h"
#include "launch.h"
#include "substrings.h"

namespace mih {
namespace {

constexpr int kDirectMaxAuto = 24;   // s above this uses the sparse form by default
constexpr int kDirectMaxForced = 28; // 2^28 + 1 offsets = 1 GiB

template <int W>
__global__ void extract_keys_kernel(const uint64_t* __restrict__ codes, uint64_t n, int off, int len,
                                    uint32_t* __restrict__ keys) {
    const int w0 = off >> 6;
    const int w1 = (off + len - 1) >> 6;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t* c = codes + i * W;
        const uint64_t lo = __ldg(c + w0);
        const uint64_t hi = (w1 != w0) ? __ldg(c + w1) : 0ull;
        const int sh = off & 63;
        uint64_t v = lo >> sh;
        if (w1 != w0) v |= hi << (64 - sh);
        keys[i] = static_cast<uint32_t>(v & ((len >= 64) ? ~0ull : ((1ull << len) - 1ull)));
    }
}

// codes_out[p] = codes[ids[p]]: the table's codes in bucket order.
template <int W>
__global__ void gather_codes_kernel(const uint64_t* __restrict__ codes, const uint32_t* __restrict__ ids, uint64_t n,
                                    uint64_t* __restrict__ out) {
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const Code<W> c = load_code<W>(codes, __ldg(ids + p));
#pragma unroll
        for (int w = 0; w < W; ++w) out[p * W + w] = c.w[w];
    }
}

// Inline records of table j when every substring is one 32-bit word: the
// code's 2W words except word j, in order (the table's key fixes word j up to
// the ring: its distance to the query's word is the ring radius).
template <int W>
__global__ void gather_records_kernel(const uint64_t* __restrict__ codes, const uint32_t* __restrict__ ids,
                                      uint64_t n, int j, uint32_t* __restrict__ out) {
    constexpr int R = 2 * W - 1;
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const Code<W> c = load_code<W>(codes, __ldg(ids + p));
        uint32_t w32[2 * W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            w32[2 * w] = static_cast<uint32_t>(c.w[w]);
            w32[2 * w + 1] = static_cast<uint32_t>(c.w[w] >> 32);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) out[p * R + i] = w32[i < j ? i : i + 1];
    }
}

__global__ void count_keys_kernel(const uint32_t* __restrict__ keys, uint64_t n, uint32_t* __restrict__ counts) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&counts[keys[i]], 1u);
}

// Non-empty buckets and the largest bucket over a counts array.
__global__ void bucket_stats_kernel(const uint32_t* __restrict__ counts, uint64_t nb,
                                    unsigned long long* __restrict__ out /* [distinct, max] */) {
    unsigned long long distinct = 0, mx = 0;
    for (uint64_t b = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; b < nb;
         b += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t c = counts[b];
        distinct += (c != 0);
        mx = c > mx ? c : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        distinct += __shfl_down_sync(0xFFFFFFFFu, distinct, o);
        unsigned long long m2 = __shfl_down_sync(0xFFFFFFFFu, mx, o);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], distinct);
        atomicMax(&out[1], mx);
    }
}

// heads[i] = 1 where a run of equal sorted keys starts.
__global__ void mark_heads_kernel(const uint32_t* __restrict__ sorted, uint64_t n, uint32_t* __restrict__ heads) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        heads[i] = (i == 0 || sorted[i] != sorted[i - 1]) ? 1u : 0u;
}

// For each run head: uniq[rank] = key, begins[rank] = position; begins[U] = n.
__global__ void write_runs_kernel(const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ rank, uint64_t n,
                                  uint32_t U, uint32_t* __restrict__ uniq, uint32_t* __restrict__ begins) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        if (i == 0 || sorted[i] != sorted[i - 1]) {
            const uint32_t r = rank[i];
            uniq[r] = sorted[i];
            begins[r] = static_cast<uint32_t>(i);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) begins[U] = static_cast<uint32_t>(n);
}

// Largest bucket of a sparse table: max over ranks of begins[u+1] - begins[u].
__global__ void max_run_kernel(const uint32_t* __restrict__ begins, uint32_t U,
                               unsigned long long* __restrict__ max_bucket) {
    unsigned long long mx = 0;
    for (uint64_t u = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; u < U;
         u += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const unsigned long long sz = begins[u + 1] - begins[u];
        mx = sz > mx ? sz : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long m2 = __shfl_down_sync(0xFFFFFFFFu, mx, o);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(max_bucket, mx);
}

__global__ void hash_insert_kernel(const uint32_t* __restrict__ uniq, uint32_t U, uint2* __restrict__ slots,
                                   uint64_t bucket_mask, unsigned int* __restrict__ max_probe) {
    for (uint64_t u = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; u < U;
         u += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t key = uniq[u];
        uint64_t b = hash_key(key) & bucket_mask;
        for (uint64_t p = 0; p <= bucket_mask; ++p) {
            bool done = false;
            for (int s = 0; s < 4 && !done; ++s) {
                unsigned int* rank_slot = &slots[4 * b + s].y;
                if (atomicCAS(rank_slot, kEmptySlot, static_cast<unsigned int>(u)) == kEmptySlot) {
                    slots[4 * b + s].x = key;
                    atomicMax(max_probe, static_cast<unsigned int>(p));
                    done = true;
                }
            }
            if (done) break;
            b = (b + 1) & bucket_mask;
        }
    }
}

unsigned grid_for(uint64_t n, int sms) {
    uint64_t g = (n + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(sms) * 16;
    if (g > cap) g = cap;
    if (g == 0) g = 1;
    return static_cast<unsigned>(g);
}

mih_status index_alloc(mih_index* ix, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("index allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? MIH_ENOMEM : MIH_ECUDA;
    }
    ix->allocs.push_back(*p);
    ix->bytes += bytes;
    return MIH_OK;
}

template <int W>
mih_status launch_extract(const uint64_t* codes, uint64_t n, int off, int len, uint32_t* keys, int sms,
                          cudaStream_t s) {
    extract_keys_kernel<W><<<grid_for(n, sms), 256, 0, s>>>(codes, n, off, len, keys);
    MIH_LAUNCH_CHECK();
    return MIH_OK;
}

mih_status build_table(mih_index* ix, int j, int kind, const DeviceInfo& dev, cudaStream_t s) {
    TableDesc& t = ix->tables[j];
    const uint64_t n = ix->n;
    const int len = t.len;
    Workspace ws(s);
    uint32_t *keys, *keys_alt, *vals_alt, *ids;
    MIH_TRY(ws.alloc(&keys, n));
    MIH_TRY(ws.alloc(&keys_alt, n));
    MIH_TRY(ws.alloc(&vals_alt, n));
    MIH_TRY(index_alloc(ix, reinterpret_cast<void**>(&ids), n * sizeof(uint32_t)));
    if (n > 0) {
        if (ix->W == 1) MIH_TRY(launch_extract<1>(ix->codes, n, t.off, len, keys, dev.sms, s));
        else if (ix->W == 2) MIH_TRY(launch_extract<2>(ix->codes, n, t.off, len, keys, dev.sms, s));
        else MIH_TRY(launch_extract<4>(ix->codes, n, t.off, len, keys, dev.sms, s));
    }
    uint32_t *skeys = keys, *sids = ids;
    MIH_TRY(radix_sort_pairs_u32(keys, ids, keys_alt, vals_alt, true, n, len, ws, &skeys, &sids));
    if (sids != ids && n > 0) MIH_CUDA(cudaMemcpyAsync(ids, sids, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    t.ids = ids;
    t.kind = kind;
    t.codes = nullptr;
    t.rec_words = 0;
    if (ix->inline_codes && n > 0 && ix->m == 2 * ix->W) {
        // every substring is one 32-bit word: records without the table's own word
        const int R = 2 * ix->W - 1;
        uint32_t* rec;
        // 16 bytes of padding: streamed copies are widened to 16-byte boundaries
        MIH_TRY(index_alloc(ix, reinterpret_cast<void**>(&rec), n * R * sizeof(uint32_t) + 16));
        if (ix->W == 1) gather_records_kernel<1><<<grid_for(n, dev.sms), 256, 0, s>>>(ix->codes, ids, n, j, rec);
        else if (ix->W == 2) gather_records_kernel<2><<<grid_for(n, dev.sms), 256, 0, s>>>(ix->codes, ids, n, j, rec);
        else gather_records_kernel<4><<<grid_for(n, dev.sms), 256, 0, s>>>(ix->codes, ids, n, j, rec);
        MIH_LAUNCH_CHECK();
        t.codes = reinterpret_cast<const uint64_t*>(rec);
        t.rec_words = R;
    } else if (ix->inline_codes && n > 0) {
        uint64_t* inl;
        // 16 bytes of padding: streamed copies of 8-byte codes are widened to
        // 16-byte boundaries and may read one code past the end
        MIH_TRY(index_alloc(ix, reinterpret_cast<void**>(&inl), n * ix->W * sizeof(uint64_t) + 16));
        if (ix->W == 1) gather_codes_kernel<1><<<grid_for(n, dev.sms), 256, 0, s>>>(ix->codes, ids, n, inl);
        else if (ix->W == 2) gather_codes_kernel<2><<<grid_for(n, dev.sms), 256, 0, s>>>(ix->codes, ids, n, inl);
        else gather_codes_kernel<4><<<grid_for(n, dev.sms), 256, 0, s>>>(ix->codes, ids, n, inl);
        MIH_LAUNCH_CHECK();
        t.codes = inl;
    }

    unsigned long long* stats;  // [distinct, max bucket]
    MIH_TRY(ws.alloc(&stats, 2));
    MIH_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), s));
    unsigned long long hstats[2] = {0, 0};

    if (kind == MIH_TABLE_DIRECT) {
        const uint64_t nb = 1ull << len;
        uint32_t* offsets;
        MIH_TRY(index_alloc(ix, reinterpret_cast<void**>(&offsets), (nb + 1) * sizeof(uint32_t)));
        MIH_CUDA(cudaMemsetAsync(offsets, 0, (nb + 1) * sizeof(uint32_t), s));
        if (n > 0) {
            count_keys_kernel<<<grid_for(n, dev.sms), 256, 0, s>>>(skeys, n, offsets);
            MIH_LAUNCH_CHECK();
        }
        bucket_stats_kernel<<<grid_for(nb, dev.sms), 256, 0, s>>>(offsets, nb, stats);
        MIH_LAUNCH_CHECK();
        MIH_TRY(scan_exclusive_u32(offsets, offsets, nb + 1, ws));
        MIH_CUDA(cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        t.offsets = offsets;
        t.slots = nullptr;
        t.bucket_mask = 0;
        t.max_probe = 0;
    } else {
        uint32_t* rank;
        MIH_TRY(ws.alloc(&rank, n + 1));
        uint32_t U = 0;
        if (n > 0) {
            mark_heads_kernel<<<grid_for(n, dev.sms), 256, 0, s>>>(skeys, n, rank);
            MIH_LAUNCH_CHECK();
            uint32_t last_head = 0;
            MIH_CUDA(cudaMemcpyAsync(&last_head, rank + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            MIH_TRY(scan_exclusive_u32(rank, rank, n, ws));
            uint32_t last_rank = 0;
            MIH_CUDA(cudaMemcpyAsync(&last_rank, rank + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            MIH_CUDA(cudaStreamSynchronize(s));
            U = last_rank + last_head;
        }
        uint32_t *uniq, *begins;
        MIH_TRY(ws.alloc(&uniq, static_cast<size_t>(U) + 1));
        MIH_TRY(index_alloc(ix, reinterpret_cast<void**>(&begins), (static_cast<size_t>(U) + 1) * sizeof(uint32_t)));
        if (n > 0) {
            write_runs_kernel<<<grid_for(n, dev.sms), 256, 0, s>>>(skeys, rank, n, U, uniq, begins);
            MIH_LAUNCH_CHECK();
            max_run_kernel<<<grid_for(U, dev.sms), 256, 0, s>>>(begins, U, &stats[1]);
            MIH_LAUNCH_CHECK();
        } else {
            MIH_CUDA(cudaMemsetAsync(begins, 0, sizeof(uint32_t), s));
        }
        uint64_t nbk = 1;
        while (nbk * 2 < static_cast<uint64_t>(U)) nbk <<= 1;  // load factor U / (4 nbk) <= 1/2
        uint2* slots;
        MIH_TRY(index_alloc(ix, reinterpret_cast<void**>(&slots), 4 * nbk * sizeof(uint2)));
        MIH_CUDA(cudaMemsetAsync(slots, 0xFF, 4 * nbk * sizeof(uint2), s));
        unsigned int* probe;
        MIH_TRY(ws.alloc(&probe, 1));
        MIH_CUDA(cudaMemsetAsync(probe, 0, sizeof(unsigned int), s));
        if (U > 0) {
            hash_insert_kernel<<<grid_for(U, dev.sms), 256, 0, s>>>(uniq, U, slots, nbk - 1, probe);
            MIH_LAUNCH_CHECK();
        }
        unsigned int hprobe = 0;
        MIH_CUDA(cudaMemcpyAsync(&hprobe, probe, sizeof(hprobe), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
        MIH_CUDA(cudaStreamSynchronize(s));
        hstats[0] = U;
        t.offsets = begins;
        t.slots = slots;
        t.bucket_mask = nbk - 1;
        t.max_probe = hprobe;
    }
    ix->distinct_keys[j] = hstats[0];
    ix->max_bucket[j] = hstats[1];
    return MIH_OK;
}

}  // namespace
}  // namespace mih

extern "C" {

mih_status mih_build(const uint64_t* codes, uint64_t n, int q, int m, const mih_params* params, void* stream,
                     mih_index** out) {
    using namespace mih;
    clear_error();
    if (!out) {
        set_error("mih_build: out is NULL");
        return MIH_EINVAL;
    }
    *out = nullptr;
    if (q != 64 && q != 128 && q != 256) {
        set_error("mih_build: q must be 64, 128 or 256 (got %d)", q);
        return MIH_EINVAL;
    }
    const int32_t* lengths = params ? params->substring_length : nullptr;
    if (m < 1 || m > q || m > kMaxTables || (!lengths && (q + m - 1) / m > 32)) {
        set_error("mih_build: need 1 <= m <= min(q, %d) and substrings of at most 32 bits (q=%d m=%d)", kMaxTables,
                  q, m);
        return MIH_EINVAL;
    }
    if (lengths) {
        int sum = 0;
        for (int j = 0; j < m; ++j) {
            if (lengths[j] < 1 || lengths[j] > 32) {
                set_error("mih_build: substring_length[%d] = %d is outside 1..32", j, lengths[j]);
                return MIH_EINVAL;
            }
            sum += lengths[j];
        }
        if (sum != q) {
            set_error("mih_build: substring lengths sum to %d, not q = %d", sum, q);
            return MIH_EINVAL;
        }
    }
    if (n >= 0xFFFFFFFFull) {
        set_error("mih_build: n must be below 2^32 - 1 (ids are uint32)");
        return MIH_EINVAL;
    }
    int kind_req = MIH_TABLE_AUTO;
    if (params) {
        if (params->slice_shape < MIH_SLICE_SHAPE_3K_8W || params->slice_shape > MIH_SLICE_SHAPE_4K_8W) {
            set_error("mih_build: unknown slice_shape %d", params->slice_shape);
            return MIH_EINVAL;
        }
        for (int i = 0; i < 5; ++i)
            if (params->reserved[i] != 0) {
                set_error("mih_build: params.reserved must be zero");
                return MIH_EINVAL;
            }
        if (params->bit_order) MIH_TRY(check_bit_order(params->bit_order, q));
        if (params->executor < MIH_EXEC_AUTO || params->executor > MIH_EXEC_GRAPH) {
            set_error("mih_build: unknown executor %d", params->executor);
            return MIH_EINVAL;
        }
        kind_req = params->table_kind;
        if (kind_req < MIH_TABLE_AUTO || kind_req > MIH_TABLE_SPARSE) {
            set_error("mih_build: unknown table_kind %d", kind_req);
            return MIH_EINVAL;
        }
    }
    if (n > 0) {
        MIH_TRY(check_device_ptr(codes, "mih_build: codes"));
        MIH_TRY(check_code_alignment(codes, q / 64, "mih_build: codes"));
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceInfo dev;
    MIH_TRY(device_info(&dev));

    mih_index* ix = new (std::nothrow) mih_index();
    if (!ix) {
        set_error("mih_build: host allocation failed");
        return MIH_ENOMEM;
    }
    ix->device = dev.device;
    ix->q = q;
    ix->m = m;
    ix->W = q / 64;
    ix->n = n;
    ix->codes = codes;
    ix->scan_factor = params ? params->scan_factor : 0;
    ix->probe = (!params || params->probe == 0) ? 4096 : (params->probe < 0 ? 0 : params->probe);
    ix->executor = params ? params->executor : MIH_EXEC_AUTO;
    ix->tail_from = (!params || params->tail_from <= 0) ? -1 : params->tail_from;
    ix->slice_shape = params ? params->slice_shape : MIH_SLICE_SHAPE_3K_8W;
    if (params && params->bit_order) {
        // Optimised substrings (Sec. 5.5): the tables see codes whose bits are
        // permuted; the index keeps that copy and the order for the queries.
        mih_status pst = index_alloc(ix, reinterpret_cast<void**>(&ix->bit_order), q * sizeof(int32_t));
        uint64_t* perm = nullptr;
        if (pst == MIH_OK)
            pst = index_alloc(ix, reinterpret_cast<void**>(&perm), static_cast<size_t>(n) * (q / 64) * 8 + 16);
        if (pst == MIH_OK) {
            const cudaError_t e = cudaMemcpyAsync(ix->bit_order, params->bit_order, q * sizeof(int32_t),
                                                  cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                set_error("mih_build: bit order upload failed: %s", cudaGetErrorString(e));
                pst = MIH_ECUDA;
            }
        }
        if (pst == MIH_OK) pst = permute_codes(codes, perm, n, q, ix->bit_order, s);
        if (pst == MIH_OK) pst = cudaStreamSynchronize(s) == cudaSuccess ? MIH_OK : MIH_ECUDA;
        if (pst != MIH_OK) {
            mih_free(ix);
            return pst;
        }
        ix->codes = perm;
    }
    {
        // Inline codes: m * n * q/8 bytes on top of ids (4 m n) and tables;
        // automatic when the whole index fits in half the free memory.
        const int req = params ? params->inline_codes : 0;
        if (req > 0) {
            ix->inline_codes = true;
        } else if (req == 0 && n > 0) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
                cudaGetLastError();
                free_b = 0;
            }
            // ids (4 B) + inline codes (q/8 B, 4 B less when every substring
            // is one 32-bit word) per entry and table, plus the build's
            // transient key/id buffers (12 B per code)
            const int rec_b = (m == 2 * (q / 64)) ? q / 8 - 4 : q / 8;
            const double est = static_cast<double>(m) * n * (rec_b + 4) + 12.0 * n;
            ix->inline_codes = est < 0.6 * static_cast<double>(free_b);
        }
    }
    ix->tables.resize(m);
    ix->distinct_keys.assign(m, 0);
    ix->max_bucket.assign(m, 0);
    int32_t off[kMaxTables], len[kMaxTables];
    if (lengths) {
        for (int j = 0, o = 0; j < m; o += lengths[j], ++j) {
            off[j] = o;
            len[j] = lengths[j];
        }
    } else {
        mih_substring_layout(q, m, off, len);
    }
    mih_status st = MIH_OK;
    for (int j = 0; j < m && st == MIH_OK; ++j) {
        memset(&ix->tables[j], 0, sizeof(TableDesc));
        ix->tables[j].off = off[j];
        ix->tables[j].len = len[j];
        int kind = kind_req;
        if (kind == MIH_TABLE_AUTO) kind = len[j] <= kDirectMaxAuto ? MIH_TABLE_DIRECT : MIH_TABLE_SPARSE;
        if (kind == MIH_TABLE_DIRECT && len[j] > kDirectMaxForced) {
            set_error("mih_build: direct tables need substrings of at most %d bits", kDirectMaxForced);
            st = MIH_EINVAL;
            break;
        }
        st = build_table(ix, j, kind, dev, s);
    }
    if (st == MIH_OK) {
        st = index_alloc(ix, reinterpret_cast<void**>(&ix->dev_tables), m * sizeof(TableDesc));
        if (st == MIH_OK) {
            cudaError_t e = cudaMemcpyAsync(ix->dev_tables, ix->tables.data(), m * sizeof(TableDesc),
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                set_error("mih_build: descriptor upload failed: %s", cudaGetErrorString(e));
                st = MIH_ECUDA;
            }
        }
    }
    if (st == MIH_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("mih_build: %s", cudaGetErrorString(e));
            st = MIH_ECUDA;
        }
    }
    trim_pool();
    if (st != MIH_OK) {
        mih_free(ix);
        return st;
    }
    *out = ix;
    return MIH_OK;
}

void mih_free(mih_index* ix) {
    if (!ix) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != ix->device) cudaSetDevice(ix->device);
    for (void* p : ix->allocs) cudaFree(p);
    if (cur != ix->device) cudaSetDevice(cur);
    delete ix;
}

mih_status mih_index_get_info(const mih_index* ix, mih_index_info* info) {
    if (!ix || !info) {
        mih::set_error("mih_index_get_info: NULL argument");
        return MIH_EINVAL;
    }
    memset(info, 0, sizeof(*info));
    info->q = ix->q;
    info->m = ix->m;
    info->W = ix->W;
    info->n = ix->n;
    info->index_bytes = ix->bytes;
    info->inline_codes = ix->inline_codes ? 1 : 0;
    for (int j = 0; j < ix->m; ++j) {
        info->substring_offset[j] = ix->tables[j].off;
        info->substring_length[j] = ix->tables[j].len;
        info->table_kind[j] = ix->tables[j].kind;
        info->distinct_keys[j] = ix->distinct_keys[j];
        info->max_bucket[j] = ix->max_bucket[j];
    }
    return MIH_OK;
}

}  // extern "C"
