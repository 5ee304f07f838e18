// search.h -- pieces of the k-NN path shared by the MIH search and the
// linear scan: argument checks, the bounded per-query buffer size and the
// final k-selection.
#pragma once

#include <stdint.h>

#include "launch.h"

namespace mih {

struct TableDesc;

// Per-query inputs of the selection kernel.  For query q the candidate
// entries (distance << 32 | id) are buf1[q*cap, q*cap + cnt1[q]) when
// cnt1[q] <= cap, else buf2[base2[q], ...) holding exactly the codes within
// dk[q] bits.  hist[q][d] must be exact for every d <= dk[q].
struct SelectInputs {
    uint32_t nq;
    uint64_t n;
    int q;
    const uint32_t* kq;        // per-query k or null
    uint32_t k_uniform;
    uint32_t kmax;
    const uint64_t* out_off;   // CSR output offsets or null (uniform k)
    const uint32_t* hist;      // [nq][q+1]
    const int32_t* dk;         // k-th smallest distance per query
    const uint64_t* buf1;
    uint32_t cap;
    const uint32_t* cnt1;
    const uint64_t* buf2;
    const uint64_t* base2;
    uint32_t* out_ids;
    int32_t* out_dist;
    const TableDesc* tables = nullptr;   // device; set when entries may hold tagged table positions
};

mih_status launch_select(const SelectInputs& in, Workspace& ws);

// The same selection writing a failure into `err` (device int, zeroed by the
// caller) instead of allocating a flag; for min(kmax, n) <= 4096 (32 KB of
// shared memory).
mih_status launch_select_noalloc(const SelectInputs& in, int* err, cudaStream_t s);

// Validate k (uniform or per query, device) and the output pointers; *kmax
// receives the largest k.
mih_status check_k_args(uint32_t nq, const uint32_t* k, uint32_t k_uniform, const uint64_t* out_offsets,
                        const uint32_t* out_ids, const int32_t* out_dist, uint32_t* kmax, Workspace& ws);

// Slots of the bounded per-query candidate buffer for a given largest k and
// batch size.
uint32_t knn_buffer_cap(uint32_t kmax, uint32_t nq);

}  // namespace mih
