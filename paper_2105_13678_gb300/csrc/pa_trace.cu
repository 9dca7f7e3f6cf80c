// pa_trace.cu -- per-kernel device timing (pa_trace_enable / pa_trace_collect).
//
// While tracing is on, each kernel launch of the library is bracketed by two
// CUDA events recorded on the stream it is launched on.  pa_trace_collect
// waits for the recorded events and returns launches and total milliseconds
// per (kernel, stage).  Launches made while a stream is being captured into a
// graph are not traced.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pa_gb300.h"
#include "pa_internal.h"

namespace {

struct Rec {
    std::string name;
    cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::string g_only;  // non-empty: record only launches with this name
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

namespace pa {

void *trace_begin(const char *name, u32 stage, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return nullptr;
    Rec r;
    // stage 2: Eq. 4's seed operand transformed beside the Eq. 2 stage
    r.name = std::string(stage == 0 ? "mmh." : stage == 1 ? "mh." : "mh_b.") + name;
    if (!g_only.empty() && r.name != g_only) return nullptr;
    r.a = take_event();
    r.b = take_event();
    cudaEventRecord(r.a, (cudaStream_t)stream);
    g_recs.push_back(r);
    return (void *)(uintptr_t)g_recs.size();  // 1-based index
}

void trace_end(void *token, void *stream) {
    if (!token) return;
    std::lock_guard<std::mutex> lk(g_mu);
    const size_t i = (size_t)(uintptr_t)token - 1;
    if (i < g_recs.size()) cudaEventRecord(g_recs[i].b, (cudaStream_t)stream);
}

}  // namespace pa

extern "C" {

int pa_trace_select(const char *name) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_only = name ? std::string(name) : std::string();
    return PA_OK;
}

int pa_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_on = on != 0;
    return PA_OK;
}

int pa_trace_collect(pa_trace_entry *out, int max_entries, int *count) {
    if (!count) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    std::map<std::string, std::pair<uint64_t, double>> agg;
    for (auto &r : g_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return PA_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return PA_ERR_CUDA;
        auto &e = agg[r.name];
        e.first += 1;
        e.second += ms;
    }
    int n = 0;
    for (auto &kv : agg) {
        if (out && n < max_entries) {
            memset(&out[n], 0, sizeof(out[n]));
            strncpy(out[n].name, kv.first.c_str(), sizeof(out[n].name) - 1);
            out[n].launches = kv.second.first;
            out[n].total_ms = kv.second.second;
        }
        n++;
    }
    *count = n;
    return PA_OK;
}

}  // extern "C"
