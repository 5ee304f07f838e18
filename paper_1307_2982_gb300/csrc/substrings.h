// substrings.h -- bit permutation of codes for optimised substrings (Sec. 5.5).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mih.h"

namespace mih {

// MIH_EINVAL unless order (host, q entries) lists each bit index 0..q-1 once.
mih_status check_bit_order(const int32_t* order, int q);

// out[i] = in[i] with bit p taken from bit order_dev[p] (device order, q entries).
mih_status permute_codes(const uint64_t* in, uint64_t* out, uint64_t n, int q, const int32_t* order_dev,
                         cudaStream_t s);

}  // namespace mih
