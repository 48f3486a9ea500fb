// Kernel tracing: a process-wide launch counter (always on) and, when enabled, a CUDA
// event pair around every launch with the launch's algorithmic bytes and flops, summed
// per kernel name when read. Used by the benchmark to time kernels inside a registration.
#include "common.cuh"
#include "lddmm.h"

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace lddmm {

namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
    double bytes, flops;
};
std::atomic<long> g_launches{0};
thread_local bool t_capturing = false;   // this thread is capturing a CUDA graph
thread_local long t_captured = 0;        // launches recorded into the graph so far
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
struct Sum {
    long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
};
std::map<std::string, Sum> g_sums;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_locked() {
    for (auto& r : g_recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            Sum& s = g_sums[r.name];
            s.launches++;
            s.ms += ms;
            s.bytes += r.bytes;
            s.flops += r.flops;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}
}  // namespace

KTrace::KTrace(const char* name, cudaStream_t st, double bytes, double flops)
    : name_(name), st_(st), bytes_(bytes), flops_(flops), a_(nullptr) {
    if (t_capturing) {  // counted when the graph is launched; no events inside a graph
        ++t_captured;
        return;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_enabled.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_mu);
        a_ = get_event();
        cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
    }
}

KTrace::~KTrace() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    cudaEventRecord(b, st_);
    g_recs.push_back(Rec{name_, static_cast<cudaEvent_t>(a_), b, bytes_, flops_});
    if (g_recs.size() > 4096) drain_locked();
}

void capture_begin() {
    t_capturing = true;
    t_captured = 0;
}
long capture_end() {
    t_capturing = false;
    return t_captured;
}
void count_launches(long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool tracing() { return g_enabled.load(std::memory_order_relaxed); }

}  // namespace lddmm

using namespace lddmm;

extern "C" {

long lddmm_launch_count(void) { return g_launches.load(); }

int lddmm_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    g_enabled.store(on != 0);
    return LDDMM_OK;
}

int lddmm_trace_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    g_sums.clear();
    return LDDMM_OK;
}

int lddmm_trace_read(char* buf, int len) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    std::string s = "{";
    bool first = true;
    for (auto& kv : g_sums) {
        char tmp[512];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %ld, \"ms\": %.6f, \"bytes\": %.6e, \"flops\": %.6e}",
                 first ? "" : ", ", kv.first.c_str(), kv.second.launches, kv.second.ms,
                 kv.second.bytes, kv.second.flops);
        s += tmp;
        first = false;
    }
    s += "}";
    if (!buf || len <= 0) return (int)s.size() + 1;
    if ((int)s.size() + 1 > len) {
        set_error("lddmm_trace_read: buffer too small");
        return LDDMM_EINVAL;
    }
    memcpy(buf, s.c_str(), s.size() + 1);
    return LDDMM_OK;
}

}  // extern "C"
