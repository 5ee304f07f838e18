// autotune.cu -- choose m by timing the search on hold-out queries (Sec. 6
// "Number of Substrings"), and per-table substring lengths for a given m the
// same way.  Host code over the library's own entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "index.h"
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
    if (params && params->substring_length) {
        set_error("mih_autotune: params.substring_length must be NULL (lengths depend on m)");
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

// Per-table lengths for a given m: the stop steps of the hold-out queries on
// the Sec. 2.1 layout (per-query counters), mih_cost_layout's lengths for
// their histogram, then one timed mih_knn of each layout.
extern "C" mih_status mih_autotune_layout(const uint64_t* codes, uint64_t n, int q, const uint64_t* queries,
                                          uint32_t nq, uint32_t k, int m, const mih_params* params, void* stream,
                                          int32_t* best_length, double* ms_per_query) {
    using namespace mih;
    clear_error();
    if (!best_length) {
        set_error("mih_autotune_layout: best_length is NULL");
        return MIH_EINVAL;
    }
    if (nq == 0 || k == 0 || k > MIH_MAX_K) {
        set_error("mih_autotune_layout: need at least one hold-out query and 1 <= k <= %u", MIH_MAX_K);
        return MIH_EINVAL;
    }
    if (m < 1 || m > q || (q + m - 1) / m > 32) {
        set_error("mih_autotune_layout: need 1 <= m <= q and substrings of at most 32 bits (q=%d m=%d)", q, m);
        return MIH_EINVAL;
    }
    if (params && params->substring_length) {
        set_error("mih_autotune_layout: params.substring_length must be NULL (the call chooses it)");
        return MIH_EINVAL;
    }
    if (ms_per_query) ms_per_query[0] = ms_per_query[1] = -1.0;
    mih_params base = {};
    if (params) base = *params;
    std::vector<int32_t> uni_off(m), uni_len(m);
    MIH_TRY(mih_substring_layout(q, m, uni_off.data(), uni_len.data()));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* ids = nullptr;
    int32_t* dist = nullptr;
    uint64_t* qstats = nullptr;
    MIH_CUDA(cudaMalloc(&ids, sizeof(uint32_t) * nq * static_cast<size_t>(k)));
    if (cudaMalloc(&dist, sizeof(int32_t) * nq * static_cast<size_t>(k)) != cudaSuccess ||
        cudaMalloc(&qstats, sizeof(uint64_t) * 4 * static_cast<size_t>(nq)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ids);
        cudaFree(dist);
        set_error("mih_autotune_layout: output allocation failed");
        return MIH_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // time one layout: untimed call, timed call; ms per query
    auto time_layout = [&](const int32_t* len, double* per_q, bool stop_steps, std::vector<double>* hist) {
        mih_params p = base;
        p.substring_length = len;
        mih_index* ix = nullptr;
        mih_status st = mih_build(codes, n, q, m, &p, stream, &ix);
        if (st != MIH_OK) return st;
        if (stop_steps) {
            st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, qstats, nullptr, stream);
            if (st == MIH_OK) {
                std::vector<uint64_t> h(4ull * nq);
                if (cudaMemcpy(h.data(), qstats, sizeof(uint64_t) * 4 * nq, cudaMemcpyDeviceToHost) != cudaSuccess) {
                    cudaGetLastError();
                    set_error("mih_autotune_layout: counter copy failed");
                    st = MIH_ECUDA;
                } else {
                    hist->assign(static_cast<size_t>(q) + 1, 0.0);
                    for (uint32_t i = 0; i < nq; ++i) (*hist)[std::min<uint64_t>(h[4ull * i + 3], q)] += 1.0;
                }
            }
        }
        if (st == MIH_OK) st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, nullptr, nullptr, stream);
        if (st == MIH_OK) {
            cudaEventRecord(e0, s);
            st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, nullptr, nullptr, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            *per_q = ms / nq;
        }
        mih_free(ix);
        return st;
    };
    double t_uni = -1.0, t_cost = -1.0;
    std::vector<double> hist;
    std::vector<int32_t> cost_len(m);
    mih_status st = time_layout(uni_len.data(), &t_uni, n > 0, &hist);
    bool same = true;
    if (st == MIH_OK && n > 0) {
        if (mih_cost_layout(q, n, m, hist.data(), static_cast<int>(hist.size()), cost_len.data()) < 0) {
            set_error("mih_autotune_layout: cost model failed");
            st = MIH_EINTERNAL;
        } else {
            for (int j = 0; j < m; ++j) same = same && cost_len[j] == uni_len[j];
            if (!same) st = time_layout(cost_len.data(), &t_cost, false, nullptr);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ids);
    cudaFree(dist);
    cudaFree(qstats);
    if (st != MIH_OK) return st;
    if (same) t_cost = t_uni;
    if (ms_per_query) {
        ms_per_query[0] = t_uni;
        ms_per_query[1] = t_cost;
    }
    const int32_t* best = (!same && t_cost < t_uni) ? cost_len.data() : uni_len.data();
    for (int j = 0; j < m; ++j) best_length[j] = best[j];
    return MIH_OK;
}

// Launch choices of an index's k-NN waves by timing on hold-out queries: the
// slice kernel's shape x the step from which queries run two steps per wave.
extern "C" mih_status mih_tune_search(mih_index* ix, const uint64_t* queries, uint32_t nq, uint32_t k, void* stream,
                                      mih_search_tuning* best, double* ms_per_query) {
    using namespace mih;
    clear_error();
    if (!ix) {
        set_error("mih_tune_search: index is NULL");
        return MIH_EINVAL;
    }
    if (nq == 0 || k == 0 || k > MIH_MAX_K) {
        set_error("mih_tune_search: need at least one hold-out query and 1 <= k <= %u", MIH_MAX_K);
        return MIH_EINVAL;
    }
    constexpr int kShapes = 3, kTails = 3;
    if (ms_per_query)
        for (int i = 0; i < kShapes * kTails; ++i) ms_per_query[i] = -1.0;
    const int tails[kTails] = {2 * ix->m, ix->m, -1};
    const int old_shape = ix->slice_shape, old_tail = ix->tail_from;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* ids = nullptr;
    int32_t* dist = nullptr;
    MIH_CUDA(cudaMalloc(&ids, sizeof(uint32_t) * nq * static_cast<size_t>(k)));
    if (cudaMalloc(&dist, sizeof(int32_t) * nq * static_cast<size_t>(k)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ids);
        set_error("mih_tune_search: output allocation failed");
        return MIH_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    mih_status st = MIH_OK;
    double best_ms = -1.0;
    int best_shape = old_shape, best_tail = old_tail;
    // without inline codes big buckets go through the by-id kernel: the shape
    // does not apply
    const int shapes = ix->inline_codes ? kShapes : 1;
    for (int sh = 0; sh < shapes && st == MIH_OK; ++sh) {
        for (int ti = 0; ti < kTails && st == MIH_OK; ++ti) {
            ix->slice_shape = sh;
            ix->tail_from = tails[ti];
            st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, nullptr, nullptr, stream);   // warm
            if (st != MIH_OK) break;
            cudaEventRecord(e0, s);
            st = mih_knn(ix, queries, nq, nullptr, k, nullptr, ids, dist, nullptr, nullptr, stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            if (st != MIH_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per_q = ms / nq;
            if (ms_per_query) ms_per_query[sh * kTails + ti] = per_q;
            if (best_ms < 0 || per_q < best_ms) {
                best_ms = per_q;
                best_shape = sh;
                best_tail = tails[ti];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ids);
    cudaFree(dist);
    ix->slice_shape = st == MIH_OK ? best_shape : old_shape;
    ix->tail_from = st == MIH_OK ? best_tail : old_tail;
    if (best) {
        best->slice_shape = ix->slice_shape;
        best->tail_from = ix->tail_from;
    }
    return st;
}
