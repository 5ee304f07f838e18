// autotune.cu -- choose m by timing the search on hold-out queries (Sec. 6
// "Number of Substrings").  Host code over the library's own entry points.
#include <cuda_runtime.h>

#include <vector>

#include "launch.h"

extern "C" mih_status mih_autotune(const uint64_t* codes, uint64_t n, int q, const uint64_t* queries, uint32_t nq,
                                   uint32_t k, const int* candidates, int n_candidates, const mih_params* params,
                                   void* stream, int* best_m, double* ms_per_query) {
    using namespace mih;
    clear_error();
    if (!best_m) {
        set_error("mih_autotune: best_m is NULL");
        return MIH_EINVAL;
    }
    *best_m = 0;
    if (nq == 0 || k == 0 || k > MIH_MAX_K) {
        set_error("mih_autotune: need at least one hold-out query and 1 <= k <= %u", MIH_MAX_K);
        return MIH_EINVAL;
    }
    std::vector<int> cand;
    if (candidates) {
        if (n_candidates < 1) {
            set_error("mih_autotune: n_candidates must be positive");
            return MIH_EINVAL;
        }
        cand.assign(candidates, candidates + n_candidates);
    } else {
        const int m0 = mih_suggest_m(q, n);
        cand = {m0 - 1, m0, m0 + 1};
    }
    for (size_t i = 0; i < cand.size(); ++i)
        if (ms_per_query) ms_per_query[i] = -1.0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *ids = nullptr;
    int32_t *dist = nullptr;
    MIH_CUDA(cudaMalloc(&ids, sizeof(uint32_t) * nq * static_cast<size_t>(k)));
    if (cudaMalloc(&dist, sizeof(int32_t) * nq * static_cast<size_t>(k)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ids);
        set_error("mih_autotune: output allocation failed");
        return MIH_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    mih_status st = MIH_OK;
    double best = -1.0;
    for (size_t i = 0; i < cand.size() && st == MIH_OK; ++i) {
        const int m = cand[i];
        if (m < 1 || m > q || (q + m - 1) / m > 32) continue;
        mih_index* ix = nullptr;
        st = mih_build(codes, n, q, m, params, stream, &ix);
        if (st != MIH_OK) break;
        st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, nullptr, nullptr, stream);   // warm
        if (st == MIH_OK) {
            cudaEventRecord(e0, s);
            st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, nullptr, nullptr, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
        }
        mih_free(ix);
        if (st != MIH_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per_q = ms / nq;
        if (ms_per_query) ms_per_query[i] = per_q;
        if (best < 0 || per_q < best) {
            best = per_q;
            *best_m = m;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ids);
    cudaFree(dist);
    if (st == MIH_OK && *best_m == 0) {
        set_error("mih_autotune: no valid candidate m for q=%d", q);
        return MIH_EINVAL;
    }
    return st;
}
