// api.cu -- host-side entry points that need no kernels: status text, error
// detail, the scratch pool, substring layout and the cost-model helpers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "launch.h"

namespace mih {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

// ---------------------------------------------------------------- profile
namespace {
struct Profiler {
    int timing = 0;                   // 0 off, 1 main spans, 2 also per-kernel spans
    int depth = 0;
    mih_profile last = {};
    mih_profile cur = {};
    std::vector<cudaEvent_t> events;  // pool; pairs [2i, 2i+1] are main-kernel spans
    size_t used = 0;
    std::vector<cudaEvent_t> kevents; // pool; pairs [2i, 2i+1] are kernel spans of kind kkind[i]
    size_t kused = 0;
    std::vector<int> kkind;
    cudaEvent_t call_start = nullptr, call_stop = nullptr;
};
thread_local Profiler g_prof;

cudaEvent_t pooled_event(std::vector<cudaEvent_t>& pool, size_t& used) {
    if (used == pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        pool.push_back(e);
    }
    return pool[used++];
}

cudaEvent_t next_event() { return pooled_event(g_prof.events, g_prof.used); }
}  // namespace

int timing_level() { return g_prof.timing; }

KernelSpan::KernelSpan(cudaStream_t s, int kind, bool active) : s_(s), on_(false) {
    Profiler& p = g_prof;
    if (!active || p.timing < 2 || p.depth == 0 || kind < 0 || kind >= MIH_PROF_KINDS) return;
    cudaEvent_t e = pooled_event(p.kevents, p.kused);
    if (!e) return;
    if (cudaEventRecord(e, s) != cudaSuccess) {
        cudaGetLastError();
        --p.kused;
        return;
    }
    p.kkind.push_back(kind);
    on_ = true;
}

KernelSpan::~KernelSpan() {
    if (!on_) return;
    Profiler& p = g_prof;
    cudaEvent_t e = pooled_event(p.kevents, p.kused);
    if (e && cudaEventRecord(e, s_) == cudaSuccess) return;
    cudaGetLastError();
    // drop this span: its end event (if taken) and its begin event
    if (e) --p.kused;
    --p.kused;
    p.kkind.pop_back();
}

// Limit of the bounded waits on bulk copies, and the timeout test switch
// (mih_set_wait_limit), per host thread.
// Linear-scan kernel form (mih_set_scan_kernel), per host thread.
thread_local int g_scan_kernel = MIH_SCAN_AUTO;
int scan_kernel_choice() { return g_scan_kernel; }

thread_local uint64_t g_wait_ns = 1000000000ull;
thread_local bool g_wait_test = false;
uint64_t wait_limit_ns() { return g_wait_ns; }
bool wait_test_expire() { return g_wait_test; }

void note_launch() { g_prof.cur.launches++; }
uint64_t launches_so_far() { return g_prof.cur.launches; }
void add_launches(uint64_t launches, uint64_t main_launches) {
    g_prof.cur.launches += launches;
    g_prof.cur.main_launches += main_launches;
}

void main_kernel_begin(cudaStream_t s) {
    g_prof.cur.main_launches++;
    if (!g_prof.timing) return;
    if (g_prof.used % 2 == 1) return;  // unbalanced: ignore
    cudaEvent_t e = next_event();
    if (e) cudaEventRecord(e, s);
}

void main_kernel_end(cudaStream_t s) {
    if (!g_prof.timing) return;
    if (g_prof.used % 2 == 0) return;
    cudaEvent_t e = next_event();
    if (e) cudaEventRecord(e, s);
}

CallScope::CallScope(cudaStream_t s) : s_(s) {
    Profiler& p = g_prof;
    if (p.depth++ > 0) return;
    p.cur = mih_profile{};
    p.used = 0;
    p.kused = 0;
    p.kkind.clear();
    if (p.timing) {
        if (!p.call_start) cudaEventCreate(&p.call_start);
        if (!p.call_stop) cudaEventCreate(&p.call_stop);
        cudaEventRecord(p.call_start, s_);
    }
}

CallScope::~CallScope() {
    Profiler& p = g_prof;
    if (--p.depth > 0) return;
    if (p.timing && p.call_stop) {
        cudaEventRecord(p.call_stop, s_);
        if (cudaEventSynchronize(p.call_stop) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.call_start, p.call_stop) == cudaSuccess) p.cur.call_ms = ms;
            double main_ms = 0.0;
            for (size_t i = 0; i + 1 < p.used; i += 2) {
                float m = 0.f;
                if (cudaEventElapsedTime(&m, p.events[i], p.events[i + 1]) == cudaSuccess) main_ms += m;
            }
            p.cur.main_ms = main_ms;
            for (size_t i = 0; i + 1 < p.kused && i / 2 < p.kkind.size(); i += 2) {
                const int kind = p.kkind[i / 2];
                float m = 0.f;
                if (kind >= 0 && cudaEventElapsedTime(&m, p.kevents[i], p.kevents[i + 1]) == cudaSuccess) {
                    p.cur.kernel_ms[kind] += m;
                    p.cur.kernel_launches[kind] += 1;
                }
            }
        }
        cudaGetLastError();
    }
    p.last = p.cur;
}

// ------------------------------------------------------------ scratch pool
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
DeviceInfo g_dev[kMaxDevices] = {};
bool g_dev_ok[kMaxDevices] = {};

mih_status pool_for_current(cudaMemPool_t* out) {
    int dev = 0;
    MIH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return MIH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        MIH_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t thr = UINT64_MAX;
        MIH_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return MIH_OK;
}
}  // namespace

mih_status Workspace::raw_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool;
    MIH_TRY(pool_for_current(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, stream_);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? MIH_ENOMEM : MIH_ECUDA;
    }
    ptrs_.push_back(*p);
    return MIH_OK;
}

void Workspace::release(void* p) {
    for (size_t i = 0; i < ptrs_.size(); ++i) {
        if (ptrs_[i] == p) {
            cudaFreeAsync(p, stream_);
            ptrs_[i] = ptrs_.back();
            ptrs_.pop_back();
            return;
        }
    }
}

Workspace::~Workspace() {
    for (void* p : ptrs_) cudaFreeAsync(p, stream_);
}

mih_status trim_pool() {
    cudaMemPool_t pool;
    MIH_TRY(pool_for_current(&pool));
    MIH_CUDA(cudaMemPoolTrimTo(pool, 0));
    return MIH_OK;
}

mih_status check_device_ptr(const void* p, const char* what) {
    if (!p) {
        set_error("%s is NULL", what);
        return MIH_EINVAL;
    }
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("%s: cudaPointerGetAttributes failed: %s", what, cudaGetErrorString(e));
        return MIH_EINVAL;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) {
        set_error("%s must be CUDA device memory", what);
        return MIH_EINVAL;
    }
    int dev = 0;
    MIH_CUDA(cudaGetDevice(&dev));
    if (a.type == cudaMemoryTypeDevice && a.device != dev) {
        set_error("%s lives on device %d, current device is %d", what, a.device, dev);
        return MIH_EINVAL;
    }
    return MIH_OK;
}

mih_status check_code_alignment(const void* p, int W, const char* what) {
    const uintptr_t need = W >= 2 ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(p) % need != 0) {
        set_error("%s must be %u-byte aligned", what, static_cast<unsigned>(need));
        return MIH_EINVAL;
    }
    return MIH_OK;
}

mih_status device_info(DeviceInfo* out) {
    int dev = 0;
    MIH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return MIH_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (g_dev_ok[dev]) {
            *out = g_dev[dev];
            return MIH_OK;
        }
    }
    DeviceInfo d;
    d.device = dev;
    MIH_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    MIH_CUDA(cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_dev[dev] = d;
    g_dev_ok[dev] = true;
    *out = d;
    return MIH_OK;
}

}  // namespace mih

// ------------------------------------------------------------------ C-ABI
extern "C" {

const char* mih_status_str(mih_status s) {
    switch (s) {
        case MIH_OK: return "MIH_OK";
        case MIH_EINVAL: return "MIH_EINVAL: invalid argument";
        case MIH_ENOMEM: return "MIH_ENOMEM: device memory allocation failed";
        case MIH_ECUDA: return "MIH_ECUDA: CUDA runtime error";
        case MIH_EOVERFLOW: return "MIH_EOVERFLOW: result capacity exceeded";
        case MIH_ETIMEOUT: return "MIH_ETIMEOUT: bounded device wait expired";
        case MIH_EINTERNAL: return "MIH_EINTERNAL: internal consistency check failed";
    }
    return "unknown mih_status";
}

const char* mih_last_error(void) { return mih::g_err; }

void mih_set_timing(int level) { mih::g_prof.timing = level < 0 ? 0 : (level > 2 ? 2 : level); }

mih_status mih_set_scan_kernel(int kind) {
    if (kind < MIH_SCAN_AUTO || kind > MIH_SCAN_TENSOR) {
        mih::set_error("mih_set_scan_kernel: unknown kind %d", kind);
        return MIH_EINVAL;
    }
    mih::g_scan_kernel = kind;
    return MIH_OK;
}

mih_status mih_set_wait_limit(uint32_t limit_us, int expire_first_wait) {
    if (limit_us > 60u * 1000u * 1000u) {
        mih::set_error("mih_set_wait_limit: limit above one minute (%u us)", limit_us);
        return MIH_EINVAL;
    }
    mih::g_wait_ns = limit_us == 0 ? 1000000000ull : 1000ull * limit_us;
    mih::g_wait_test = expire_first_wait != 0;
    return MIH_OK;
}

mih_status mih_last_profile(mih_profile* out) {
    if (!out) {
        mih::set_error("mih_last_profile: out is NULL");
        return MIH_EINVAL;
    }
    *out = mih::g_prof.last;
    return MIH_OK;
}

const char* mih_version(void) { return "mih-gb300 0.1 (sm_103a)"; }

// Sec. 2.1 footnote: substrings of floor(q/m) or ceil(q/m) bits; the first
// m - (q mod m) are the short ones.
mih_status mih_substring_layout(int q, int m, int32_t* offset, int32_t* length) {
    if (q < 1 || m < 1 || m > q || !offset || !length) {
        mih::set_error("substring layout: need 1 <= m <= q and non-null outputs (q=%d m=%d)", q, m);
        return MIH_EINVAL;
    }
    const int shortl = q / m, nlong = q % m;
    int o = 0;
    for (int j = 0; j < m; ++j) {
        length[j] = shortl + (j >= m - nlong ? 1 : 0);
        offset[j] = o;
        o += length[j];
    }
    return MIH_OK;
}

// Eq. 7: cost(s) = (1 + n / 2^s) (q / s) sum_{z=0}^{floor(s r / q)} C(s, z).
double mih_cost_model(int q, uint64_t n, int s, int r) {
    if (q < 1 || s < 1 || s > q || r < 0) return -1.0;
    const int zmax = static_cast<int>((static_cast<int64_t>(s) * r) / q);
    double ball = 0.0, c = 1.0;
    for (int z = 0; z <= zmax && z <= s; ++z) {
        ball += c;
        c = c * (s - z) / (z + 1);
    }
    return (1.0 + static_cast<double>(n) / ldexp(1.0, s)) * (static_cast<double>(q) / s) * ball;
}

// Eq. 7 table by table over Algorithm 3's schedule (see include/mih.h): the
// cost of table j with s bits, weighted over the stop steps, is
// (1 + n / 2^s) sum_t w[t] sum_{rho <= floor((t - j)/m)} C(s, rho); the layout
// is the exact minimum of the sum over tables with sum_j s_j = q, by dynamic
// programming over (tables done, bits used).
double mih_cost_layout(int q, uint64_t n, int m, const double* w, int n_steps, int32_t* length) {
    if (q < 1 || m < 1 || m > q || q > 32 * m || n_steps < 1 || !w || !length) return -1.0;
    for (int t = 0; t < n_steps; ++t)
        if (!(w[t] >= 0.0)) return -1.0;
    // C(s, rho) for s <= 32
    double C[33][33] = {};
    for (int a = 0; a <= 32; ++a) {
        C[a][0] = 1.0;
        for (int b = 1; b <= a; ++b) C[a][b] = C[a - 1][b - 1] + (b <= a - 1 ? C[a - 1][b] : 0.0);
    }
    // table cost cost[j][s]
    std::vector<double> cost(static_cast<size_t>(m) * 33, 0.0);
    for (int j = 0; j < m; ++j)
        for (int sb = 1; sb <= 32; ++sb) {
            double rings = 0.0;
            for (int t = j; t < n_steps; ++t) {
                if (w[t] == 0.0) continue;
                const int rmax = (t - j) / m;
                double ball = 0.0;
                for (int r = 0; r <= rmax && r <= sb; ++r) ball += C[sb][r];
                rings += w[t] * ball;
            }
            cost[static_cast<size_t>(j) * 33 + sb] = (1.0 + static_cast<double>(n) / ldexp(1.0, sb)) * rings;
        }
    // best[j][b]: (cost, squared deviation from q/m) of tables 0..j-1 on b bits
    const double inf = HUGE_VAL, mean = static_cast<double>(q) / m;
    std::vector<double> bc(static_cast<size_t>(m + 1) * (q + 1), inf), bd = bc;
    std::vector<int> pick(static_cast<size_t>(m + 1) * (q + 1), 0);
    auto at = [q](int j, int b) { return static_cast<size_t>(j) * (q + 1) + b; };
    bc[at(0, 0)] = 0.0;
    bd[at(0, 0)] = 0.0;
    for (int j = 0; j < m; ++j)
        for (int b = 0; b <= q; ++b) {
            if (bc[at(j, b)] == inf) continue;
            for (int sb = 1; sb <= 32 && b + sb <= q; ++sb) {
                const double c = bc[at(j, b)] + cost[static_cast<size_t>(j) * 33 + sb];
                const double d = bd[at(j, b)] + (sb - mean) * (sb - mean);
                double& oc = bc[at(j + 1, b + sb)];
                double& od = bd[at(j + 1, b + sb)];
                const double tol = 1e-12 * (c > oc ? c : oc);
                const bool better = oc == inf || c < oc - tol || (c <= oc + tol && d < od);
                if (better) {
                    oc = c;
                    od = d;
                    pick[at(j + 1, b + sb)] = sb;
                }
            }
        }
    if (bc[at(m, q)] == inf) return -1.0;
    for (int j = m, b = q; j > 0; --j) {
        length[j - 1] = pick[at(j, b)];
        b -= length[j - 1];
    }
    return bc[at(m, q)];
}

// Sec. 3.1 / Table 4: m close to q / log2(n); no substring above 32 bits.
int mih_suggest_m(int q, uint64_t n) {
    if (q < 1) return 0;
    int m = (n > 1) ? static_cast<int>(lround(q / log2(static_cast<double>(n)))) : q;
    const int mmin = (q + 31) / 32;
    if (m < mmin) m = mmin;
    if (m > q) m = q;
    if (m < 1) m = 1;
    return m;
}

}  // extern "C"
