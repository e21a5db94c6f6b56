// Error reporting and small C-ABI helpers of the PSL library.
#include <cuda_runtime.h>

#include <string>

#include "psl_internal.cuh"

#include <atomic>

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void psl_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int64_t psl_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void psl_set_error(const std::string &msg) { g_last_error = msg; }

int psl_fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

extern "C" const char *psl_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------------
// Failure-detection hooks (psl_debug_waits): the polls a bounded device
// wait makes before it gives up, and the stalls and queue cap that let a
// test make a wait run out or a queue overflow without faulting the GPU.
namespace {
std::atomic<long long> g_dbg_polls{0};
std::atomic<unsigned> g_dbg_flags{0};
std::atomic<long long> g_dbg_queue_cap{0};
}  // namespace

long long psl_wait_polls(long long dflt) {
    const long long v = g_dbg_polls.load(std::memory_order_relaxed);
    return v > 0 ? v : dflt;
}
unsigned psl_debug_flags() { return g_dbg_flags.load(std::memory_order_relaxed); }
long long psl_debug_queue_cap() { return g_dbg_queue_cap.load(std::memory_order_relaxed); }

extern "C" int psl_debug_waits(int64_t polls, uint32_t flags, int64_t queue_cap) {
    if (polls < 0 || queue_cap < 0 || (flags & ~(uint32_t)(PSL_DEBUG_LOOKBACK_STALL | PSL_DEBUG_FEED_STALL)))
        return psl_fail(PSL_EINVAL, "psl_debug_waits: bad argument");
    g_dbg_polls.store(polls, std::memory_order_relaxed);
    g_dbg_flags.store(flags, std::memory_order_relaxed);
    g_dbg_queue_cap.store(queue_cap, std::memory_order_relaxed);
    return PSL_OK;
}

// ------------------------------------------------------------------------
// Device memory pool of the library: one per device, created on first use,
// keeping freed blocks (release threshold = unlimited) so that the large
// stream-ordered scratch of psl_build, psl_plan_create and psl_stream_bin is
// mapped once, not at every call.  psl_memory_trim hands memory back.
#include <mutex>

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[256] = {};

cudaError_t pool_of_current(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if ((e = cudaMemPoolCreate(&p, &props)) != cudaSuccess) return e;
        uint64_t keep = ~0ull;
        if ((e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t psl_malloc_async(void **ptr, size_t bytes, cudaStream_t st) {
    cudaMemPool_t p = nullptr;
    cudaError_t e = pool_of_current(&p);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(ptr, bytes, p, st);
}

void workspace_cache_trim();

extern "C" int psl_memory_trim(uint64_t keep_bytes, uint64_t *held_bytes) {
    workspace_cache_trim();
    cudaMemPool_t p = nullptr;
    cudaError_t e = pool_of_current(&p);
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, std::string("psl_memory_trim: ") + cudaGetErrorString(e));
    if ((e = cudaDeviceSynchronize()) != cudaSuccess)
        return psl_fail(PSL_ECUDA, std::string("psl_memory_trim: ") + cudaGetErrorString(e));
    if ((e = cudaMemPoolTrimTo(p, (size_t)keep_bytes)) != cudaSuccess)
        return psl_fail(PSL_ECUDA, std::string("psl_memory_trim: ") + cudaGetErrorString(e));
    if (held_bytes) {
        uint64_t v = 0;
        if ((e = cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &v)) != cudaSuccess)
            return psl_fail(PSL_ECUDA, std::string("psl_memory_trim: ") + cudaGetErrorString(e));
        *held_bytes = v;
    }
    return PSL_OK;
}

extern "C" void psl_physics_default(psl_physics_t *out) {
    if (!out) return;
    out->photon_cut = 0.010f;                        // Sec. 2.6
    out->electron_cut = (float)(0.700 - 0.51099895);  // 0.700 MeV total energy, Sec. 2.6
    out->wcc = 0.200f;
    out->wcb = 0.200f;
    out->flags = 0u;
}

// ------------------------------------------------------------------------
// Opt-in per-kernel timing: CUDA events recorded on the launching stream
// around the launches of the main kernels, resolved when read.
#include <mutex>
#include <vector>

namespace {
const char *K_NAMES[PSL_NK] = {"key", "onesweep", "gather", "source", "photon", "electron", "band_sort", "readout",
                               "conv3d"};
struct TimerState {
    std::mutex mu;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[PSL_NK];
    std::vector<cudaEvent_t> pool;
    double ms[PSL_NK] = {0};
    long long n[PSL_NK] = {0};
};
TimerState &timers() {
    static TimerState t;
    return t;
}
cudaEvent_t take_event(TimerState &t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
void resolve(TimerState &t) {
    for (int k = 0; k < PSL_NK; ++k) {
        for (auto &pr : t.pending[k]) {
            cudaEventSynchronize(pr.second);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            t.ms[k] += ms;
            t.n[k] += 1;
            t.pool.push_back(pr.first);
            t.pool.push_back(pr.second);
        }
        t.pending[k].clear();
    }
}
}  // namespace

bool psl_timer_on() { return timers().on; }

void psl_timer_begin(int k, cudaStream_t st, void **tok) {
    TimerState &t = timers();
    std::lock_guard<std::mutex> lk(t.mu);
    cudaEvent_t a = take_event(t);
    cudaEventRecord(a, st);
    *tok = a;
}

void psl_timer_end(int k, cudaStream_t st, void *tok) {
    TimerState &t = timers();
    std::lock_guard<std::mutex> lk(t.mu);
    cudaEvent_t b = take_event(t);
    cudaEventRecord(b, st);
    t.pending[k].push_back({(cudaEvent_t)tok, b});
}

extern "C" int psl_profile(int enable) {
    TimerState &t = timers();
    std::lock_guard<std::mutex> lk(t.mu);
    resolve(t);
    for (int k = 0; k < PSL_NK; ++k) { t.ms[k] = 0; t.n[k] = 0; }
    t.on = enable != 0;
    return PSL_OK;
}

extern "C" int psl_profile_read(int32_t kernel, double *total_ms, int64_t *launches, const char **name) {
    if (kernel < 0 || kernel >= PSL_NK) return psl_fail(PSL_EINVAL, "psl_profile_read: kernel index out of range");
    TimerState &t = timers();
    std::lock_guard<std::mutex> lk(t.mu);
    resolve(t);
    if (total_ms) *total_ms = t.ms[kernel];
    if (launches) *launches = t.n[kernel];
    if (name) *name = K_NAMES[kernel];
    return PSL_OK;
}
