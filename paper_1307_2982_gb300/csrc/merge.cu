// merge.cu -- exact merge of k-NN lists answered over disjoint id ranges of
// one database (a database split across GPUs).  Each list holds one shard's
// min(k, n_shard) nearest codes in (distance, id) order, ids relative to the
// shard; the merged list is the k smallest (distance, global id) pairs over
// all shards, which by the k-NN definition (Sec. 1.1) is the k-NN of the
// whole database because the shards partition it and (distance, id) is a
// total order.
#include <cuda_runtime.h>

#include "launch.h"
#include "mih_internal.cuh"

namespace mih {
namespace {

constexpr int kMergeMaxParts = 64;

struct MergeArgs {
    const uint32_t* ids;      // [parts][nq][k_in]
    const int32_t* dist;
    uint32_t parts, nq, k_in, k;
    uint32_t* out_ids;        // [nq][k]
    int32_t* out_dist;
    uint32_t base[kMergeMaxParts];
};

// Sort key of entry i of a list: (distance, global id); padding (distance
// -1) sorts after every code.
__device__ __forceinline__ uint64_t merge_key(const MergeArgs& a, uint32_t part, uint64_t row, uint32_t i) {
    const uint64_t at = (static_cast<uint64_t>(part) * a.nq + row) * a.k_in + i;
    const int32_t d = __ldg(a.dist + at);
    if (d < 0) return ~0ull;
    return (static_cast<uint64_t>(static_cast<uint32_t>(d)) << 32) | (__ldg(a.ids + at) + a.base[part]);
}

// Entries of list `part` (sorted) whose key is below `key`, or at most `key`
// when `or_equal`: a binary search.
__device__ __forceinline__ uint32_t count_below(const MergeArgs& a, uint32_t part, uint64_t row, uint64_t key,
                                                bool or_equal) {
    uint32_t lo = 0, hi = a.k_in;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint64_t v = merge_key(a, part, row, mid);
        if (v < key || (or_equal && v == key)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One CTA per query row.  The merged position of entry i of list p is i plus,
// for every other list p', its entries below the key (at or below it when
// p' < p, so that equal keys -- only padding -- keep list order): a stable
// merge, computed independently for every entry.
__global__ void __launch_bounds__(256) merge_topk_kernel(MergeArgs a) {
    const uint64_t row = blockIdx.x;
    for (uint32_t t = threadIdx.x; t < a.parts * a.k_in; t += blockDim.x) {
        const uint32_t p = t / a.k_in, i = t % a.k_in;
        const uint64_t key = merge_key(a, p, row, i);
        uint64_t rank = i;
        for (uint32_t pp = 0; pp < a.parts && rank < a.k; ++pp)
            if (pp != p) rank += count_below(a, pp, row, key, pp < p);
        if (rank < a.k) {
            const uint64_t o = row * a.k + rank;
            a.out_ids[o] = key == ~0ull ? kPadId : static_cast<uint32_t>(key);
            a.out_dist[o] = key == ~0ull ? -1 : static_cast<int32_t>(key >> 32);
        }
    }
    // positions no entry reached (k above the lists' total): padding
    for (uint32_t i = a.parts * a.k_in + threadIdx.x; i < a.k; i += blockDim.x) {
        a.out_ids[row * a.k + i] = kPadId;
        a.out_dist[row * a.k + i] = -1;
    }
}

}  // namespace
}  // namespace mih

extern "C" mih_status mih_merge_topk(const uint32_t* ids, const int32_t* dist, uint32_t parts, uint32_t nq,
                                     uint32_t k_in, const uint32_t* id_base, uint32_t k, uint32_t* out_ids,
                                     int32_t* out_dist, void* stream) {
    using namespace mih;
    clear_error();
    if (parts < 1 || parts > static_cast<uint32_t>(kMergeMaxParts)) {
        set_error("mih_merge_topk: parts must be in [1, %d] (got %u)", kMergeMaxParts, parts);
        return MIH_EINVAL;
    }
    if (k < 1 || k > MIH_MAX_K || k_in < 1 || k_in > MIH_MAX_K) {
        set_error("mih_merge_topk: k and k_in must be in [1, %u]", MIH_MAX_K);
        return MIH_EINVAL;
    }
    if (!id_base) {
        set_error("mih_merge_topk: id_base is NULL");
        return MIH_EINVAL;
    }
    for (uint32_t p = 1; p < parts; ++p)
        if (id_base[p] < id_base[p - 1]) {
            set_error("mih_merge_topk: id_base must be non-decreasing (shards in id order)");
            return MIH_EINVAL;
        }
    if (nq == 0) return MIH_OK;
    MIH_TRY(check_device_ptr(ids, "mih_merge_topk: ids"));
    MIH_TRY(check_device_ptr(dist, "mih_merge_topk: dist"));
    MIH_TRY(check_device_ptr(out_ids, "mih_merge_topk: out_ids"));
    MIH_TRY(check_device_ptr(out_dist, "mih_merge_topk: out_dist"));
    MergeArgs a;
    a.ids = ids;
    a.dist = dist;
    a.parts = parts;
    a.nq = nq;
    a.k_in = k_in;
    a.k = k;
    a.out_ids = out_ids;
    a.out_dist = out_dist;
    for (uint32_t p = 0; p < static_cast<uint32_t>(kMergeMaxParts); ++p) a.base[p] = p < parts ? id_base[p] : 0u;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    merge_topk_kernel<<<nq, 256, 0, s>>>(a);
    MIH_LAUNCH_CHECK();
    MIH_CUDA(cudaStreamSynchronize(s));
    return MIH_OK;
}
