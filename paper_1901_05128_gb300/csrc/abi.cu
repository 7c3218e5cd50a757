// Library-wide C ABI helpers: status strings and the launch counter.
#include <atomic>

#include "common.cuh"

namespace fastcq {
static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace fastcq

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
