// profile.cu -- launch counting and opt-in per-kernel-class timing.
//
// Every kernel launch of the library passes through NLH_CHECK_LAUNCH(),
// which bumps a process-wide counter.  When profiling is enabled, the hot
// kernels are bracketed by CUDA events recorded on their own stream, so the
// measured duration is the device time of that launch.
#include "common.cuh"

#include <atomic>
#include <mutex>

namespace nlh {

static std::atomic<long long> g_launches{0};
static std::mutex g_mu;
static bool g_enabled = false;
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfRange::ProfRange(int cls, cudaStream_t s) : idx_(-1), s_(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_enabled) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return;  // event records are not allowed inside a solve graph
    ProfRec r{cls, take_event(), take_event()};
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    idx_ = (int)g_recs.size() - 1;
}

ProfRange::~ProfRange() {
    if (idx_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (idx_ < (int)g_recs.size()) cudaEventRecord(g_recs[idx_].b, s_);
}

}  // namespace nlh

using namespace nlh;

extern "C" {

int64_t nlh_kernel_launches(void) { return (int64_t)g_launches.load(); }

nlh_status nlh_profile_enable(int enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_enabled = enable != 0;
    return NLH_OK;
}

nlh_status nlh_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    return NLH_OK;
}

nlh_status nlh_profile_read(int kernel_class, int64_t *launches, double *total_ms) {
    clear_error();
    if (!launches || !total_ms || kernel_class < 0 || kernel_class >= NLH_K_NCLASSES) {
        set_error("nlh_profile_read: bad arguments");
        return NLH_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t cnt = 0;
    double ms = 0.0;
    for (auto &r : g_recs) {
        if (r.cls != kernel_class) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            set_error("nlh_profile_read: event synchronisation failed");
            return NLH_ERR_CUDA;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        ms += t;
        ++cnt;
    }
    *launches = cnt;
    *total_ms = ms;
    return NLH_OK;
}

}  // extern "C"
