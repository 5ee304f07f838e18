// index.h -- host-side layout of a multi-index hashing index (one hash table
// per substring, Algorithm 1).  Shared by the build and search units.
#pragma once

#include <stdint.h>

#include <vector>

#include "mih_internal.cuh"

struct mih_index {
    int device = 0;
    int q = 0, m = 0, W = 0;
    uint64_t n = 0;
    const uint64_t* codes = nullptr;            // borrowed, device
    std::vector<mih::TableDesc> tables;         // host copy of the descriptors
    mih::TableDesc* dev_tables = nullptr;       // device copy (m entries)
    std::vector<void*> allocs;                  // device memory owned by the index
    std::vector<uint64_t> distinct_keys;        // non-empty buckets per table
    std::vector<uint64_t> max_bucket;           // largest bucket per table
    uint64_t bytes = 0;                         // device bytes owned
    int scan_factor = 0;                        // lookup budget factor (see mih_params)
    bool inline_codes = false;                  // tables hold codes in bucket order
    int probe = 1024;                           // bound-probe entries per bucket (0 = off)
    int executor = 0;                           // MIH_EXEC_* for the k-NN wave loop
    int tail_from = 0;                          // step from which queries run two steps per wave (-1: never)
    int slice_shape = 0;                        // slice-kernel shape of the k-NN waves (MIH_SLICE_SHAPE_*)
    int32_t* bit_order = nullptr;               // device, q entries: optimised substrings (Sec. 5.5), or null
};
