// launch.h -- host-side helpers shared by the library's translation units:
// error reporting, the stream-ordered scratch pool and utility launches.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/mih.h"

namespace mih {

// Thread-local error detail (returned by mih_last_error).
void set_error(const char* fmt, ...);
void clear_error();

// Per-call profile (mih_last_profile): launch counts and, with timing on,
// CUDA-event times of the main kernels.  A CallScope brackets one C-ABI call.
void note_launch();
uint64_t launches_so_far();                                  // launches counted in this call
void add_launches(uint64_t launches, uint64_t main_launches);  // work a graph repeated on the device
void main_kernel_begin(cudaStream_t s);
void main_kernel_end(cudaStream_t s);
// Bounded device waits of the calling host thread (mih_set_wait_limit): the
// limit in ns (default one second) and the timeout test switch.
uint64_t wait_limit_ns();
bool wait_test_expire();
// Timing level of the calling thread (mih_set_timing).
int timing_level();

// Linear-scan kernel form chosen by the calling thread (MIH_SCAN_*).
int scan_kernel_choice();

// An event pair around one kernel launch of the given MIH_PROF_* kind, on
// stream s, recorded only with per-kernel timing (level 2) inside a C-ABI
// call and when `active` (false while the stream is being captured).
class KernelSpan {
   public:
    KernelSpan(cudaStream_t s, int kind, bool active = true);
    ~KernelSpan();
    KernelSpan(const KernelSpan&) = delete;
    KernelSpan& operator=(const KernelSpan&) = delete;

   private:
    cudaStream_t s_;
    bool on_;
};

class CallScope {
   public:
    explicit CallScope(cudaStream_t s);
    ~CallScope();

   private:
    cudaStream_t s_;
};

#define MIH_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::mih::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                             __FILE__, __LINE__);                                         \
            return MIH_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

#define MIH_LAUNCH_CHECK()                                                                \
    do {                                                                                  \
        ::mih::note_launch();                                                             \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            ::mih::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),  \
                             __FILE__, __LINE__);                                         \
            return MIH_ECUDA;                                                             \
        }                                                                                 \
    } while (0)

#define MIH_TRY(expr)                                                                     \
    do {                                                                                  \
        mih_status s_ = (expr);                                                           \
        if (s_ != MIH_OK) return s_;                                                      \
    } while (0)

// Scratch memory: stream-ordered allocations from a private pool of the
// current device (kept warm between calls: its release threshold is raised).
// A Workspace frees everything it allocated, in stream order, on destruction.
class Workspace {
   public:
    explicit Workspace(cudaStream_t s) : stream_(s) {}
    ~Workspace();
    Workspace(const Workspace&) = delete;
    Workspace& operator=(const Workspace&) = delete;

    template <typename T>
    mih_status alloc(T** p, size_t count) {
        void* v = nullptr;
        mih_status st = raw_alloc(&v, count * sizeof(T));
        *p = static_cast<T*>(v);
        return st;
    }
    mih_status raw_alloc(void** p, size_t bytes);
    void release(void* p);  // free one allocation early
    cudaStream_t stream() const { return stream_; }

   private:
    cudaStream_t stream_;
    std::vector<void*> ptrs_;
};

// Return the pool's unused memory to the device (after a large build).
mih_status trim_pool();

// Reject pointers that are not device (or managed) memory of this process.
mih_status check_device_ptr(const void* p, const char* what);

// Code arrays are read with 16-byte vector loads when W >= 2.
mih_status check_code_alignment(const void* p, int W, const char* what);

// Device properties of the current device (cached per device).
struct DeviceInfo {
    int device;
    int sms;
    int max_smem_optin;
};
mih_status device_info(DeviceInfo* out);

// ---------------------------------------------------------------- utilities
// Exclusive prefix sum over n elements; out may alias in.  Uses `ws`.
mih_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, size_t n, Workspace& ws);
mih_status scan_exclusive_u64(const uint64_t* in, uint64_t* out, size_t n, Workspace& ws);
size_t scan_temp_u64(size_t n);
mih_status scan_exclusive_u64_pre(const uint64_t* in, uint64_t* out, size_t n, uint64_t* tmp, cudaStream_t s);

// Stable LSD radix sort of (uint32 key, uint32 value) pairs on key bits
// [0, bits), ping-ponging between the buffers and their alternates.  With
// `vals_iota` the input values are the positions 0..n-1 and `vals` is not
// read.  Results land in (*keys_out, *vals_out), which point at either the
// input buffers or the alternate buffers.
mih_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                                uint32_t* vals_alt, bool vals_iota, size_t n, int bits,
                                Workspace& ws, uint32_t** keys_out, uint32_t** vals_out);

// Stable LSD radix sort of uint64 keys on bits [0, bits); result pointer as above.
mih_status radix_sort_keys_u64(uint64_t* keys, uint64_t* keys_alt, size_t n, int bits,
                               Workspace& ws, uint64_t** keys_out);

// Fill helpers.
mih_status fill_u32(uint32_t* p, uint32_t v, size_t n, cudaStream_t s);

}  // namespace mih
