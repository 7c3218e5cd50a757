// Library-wide C ABI helpers: status strings and the launch counter.
#include <atomic>

#include "common.cuh"

namespace fastcq {
static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Optional CUDA events around the main kernel of the latest fp2s_solve /
// tensor-core cq_history_direct call, recorded on the caller's stream.
static bool g_timing = false, g_timed = false;
static cudaEvent_t g_ev0 = nullptr, g_ev1 = nullptr;

// Event pairs around the sub-launches of one part (the tensor-core contractions of
// the mixed-precision direct solve) inside the timed region; reset by timing_begin.
static cudaEvent_t g_part_ev[2 * kMaxTimedParts];
static int g_part_created = 0, g_part_used = 0;
static bool g_part_open = false;          // a begin event of the current sub-launch was recorded

int timing_begin(cudaStream_t s) {
    if (!g_timing) return CQ_OK;
    g_part_used = 0;
    g_part_open = false;
    return cudaEventRecord(g_ev0, s) == cudaSuccess ? CQ_OK : CQ_ECUDA;
}

int timing_part(cudaStream_t s, bool end) {
    if (!g_timing) return CQ_OK;
    if (!end && g_part_used >= kMaxTimedParts) return CQ_OK;     // beyond the pool: not timed
    if (end && !g_part_open) return CQ_OK;                         // its begin was not recorded
    const int k = 2 * (end ? g_part_used - 1 : g_part_used) + (end ? 1 : 0);
    if (k < 0) return CQ_OK;
    while (g_part_created <= k) {
        if (cudaEventCreate(&g_part_ev[g_part_created]) != cudaSuccess) return CQ_ECUDA;
        ++g_part_created;
    }
    if (cudaEventRecord(g_part_ev[k], s) != cudaSuccess) return CQ_ECUDA;
    if (!end) ++g_part_used;
    g_part_open = !end;
    return CQ_OK;
}

int smem_attr_once(const void *func, int bytes, unsigned long long *done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CQ_ECUDA;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (__atomic_load_n(done, __ATOMIC_ACQUIRE) & bit)) return CQ_OK;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return CQ_ECUDA;
    if (bit) __atomic_fetch_or(done, bit, __ATOMIC_RELEASE);
    return CQ_OK;
}

int device_sms() {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev < 64 && sms[dev] > 0) return sms[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    if (dev < 64) sms[dev] = n;
    return n;
}

int timing_end(cudaStream_t s) {
    if (!g_timing) return CQ_OK;
    if (cudaEventRecord(g_ev1, s) != cudaSuccess) return CQ_ECUDA;
    g_timed = true;
    return CQ_OK;
}
}  // namespace fastcq

extern "C" int cq_timing_enable(int on) {
    using namespace fastcq;
    if (on && !g_ev0) {
        if (cudaEventCreate(&g_ev0) != cudaSuccess || cudaEventCreate(&g_ev1) != cudaSuccess) return CQ_ECUDA;
    }
    g_timing = on != 0;
    return CQ_OK;
}

extern "C" int cq_timing_last(double *ms) {
    using namespace fastcq;
    if (!ms || !g_timed) return CQ_EINVAL;
    float f = 0.0f;
    if (cudaEventSynchronize(g_ev1) != cudaSuccess) return CQ_ECUDA;
    if (cudaEventElapsedTime(&f, g_ev0, g_ev1) != cudaSuccess) return CQ_ECUDA;
    *ms = f;
    return CQ_OK;
}

extern "C" int cq_timing_part(int part, double *ms) {
    using namespace fastcq;
    if (!ms || !g_timed || part < 0 || part > 1) return CQ_EINVAL;
    if (part == 0) return cq_timing_last(ms);
    double tot = 0.0;
    for (int i = 0; i < g_part_used; ++i) {
        float f = 0.0f;
        if (cudaEventSynchronize(g_part_ev[2 * i + 1]) != cudaSuccess) return CQ_ECUDA;
        if (cudaEventElapsedTime(&f, g_part_ev[2 * i], g_part_ev[2 * i + 1]) != cudaSuccess) return CQ_ECUDA;
        tot += f;
    }
    *ms = tot;
    return CQ_OK;
}

extern "C" const char *cq_strerror(int status) {
    switch (status) {
        case CQ_OK: return "ok";
        case CQ_EINVAL: return "invalid argument";
        case CQ_ENOMEM: return "workspace too small";
        case CQ_ECUDA: return "CUDA runtime error";
        case CQ_ESINGULAR: return "singular 2x2 step matrix";
        case CQ_ENONFINITE: return "result contains Inf or NaN";
        case CQ_ETIMEOUT: return "bounded device wait expired";
        case CQ_EUNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

extern "C" int64_t cq_launch_count(void) { return fastcq::g_launches.load(std::memory_order_relaxed); }
