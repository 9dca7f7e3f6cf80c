// pa_batch.cu -- many independent privacy-amplification blocks in one CUDA
// graph launch (pa_hash_batch).
//
// Each block is Algorithm 1 on its own plan.  The blocks are spread over up to
// kBranches concurrent graph branches, heaviest first onto the least loaded
// branch (longest-processing-time list scheduling, cost ~ sum of N log N of
// the block's transforms), so that the small blocks fill the SMs left idle by
// the large ones.  The captured graph is cached per argument list and
// replayed by later calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/pa_gb300.h"

namespace {

constexpr int kBranches = 16;

struct CachedGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<pa_plan_t *> plans;
};

std::mutex g_mu;
std::map<std::vector<uintptr_t>, CachedGraph> g_cache;

double block_cost(pa_plan_t *pl) {
    pa_plan_info info;
    pa_plan_info_get(pl, &info);
    auto nlogn = [](double n) { return n * std::max(1.0, std::log2(n)); };
    return (2.0 * (double)info.k + 1.0) * nlogn((double)info.mmh_len) + 3.0 * nlogn((double)info.mh_len);
}

int capture(pa_plan_t *const *plans, const uint64_t *const *keys, const uint64_t *const *seeds,
            uint64_t *const *outs, int *statuses, int count, cudaGraphExec_t *exec) {
    const int nb = std::min(count, kBranches);
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> br(nb, nullptr);
    std::vector<cudaEvent_t> ev(nb + 1, nullptr);
    cudaGraph_t graph = nullptr;
    int rc = PA_OK;
    auto fail = [&](int code) {
        if (rc == PA_OK) rc = code;
    };
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) fail(PA_ERR_CUDA);
    for (int b = 0; b < nb && rc == PA_OK; b++)
        if (cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking)) fail(PA_ERR_CUDA);
    for (int b = 0; b <= nb && rc == PA_OK; b++)
        if (cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming)) fail(PA_ERR_CUDA);
    if (rc == PA_OK) {
        // list scheduling: heaviest block first onto the least loaded branch
        std::vector<int> order(count);
        std::iota(order.begin(), order.end(), 0);
        std::vector<double> cost(count);
        for (int i = 0; i < count; i++) cost[i] = block_cost(plans[i]);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        std::vector<double> load(nb, 0.0);
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) fail(PA_ERR_CUDA);
        if (rc == PA_OK && cudaEventRecord(ev[nb], cs)) fail(PA_ERR_CUDA);
        for (int b = 0; b < nb && rc == PA_OK; b++)
            if (cudaStreamWaitEvent(br[b], ev[nb], 0)) fail(PA_ERR_CUDA);
        for (int i : order) {
            if (rc != PA_OK) break;
            const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            load[b] += cost[i];
            int e = pa_hash(plans[i], keys[i], seeds[i], outs[i], statuses ? statuses + i : nullptr, br[b]);
            if (e) fail(e);
        }
        for (int b = 0; b < nb && rc == PA_OK; b++) {
            if (cudaEventRecord(ev[b], br[b])) fail(PA_ERR_CUDA);
            if (rc == PA_OK && cudaStreamWaitEvent(cs, ev[b], 0)) fail(PA_ERR_CUDA);
        }
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (ce) fail(PA_ERR_CUDA);
        if (rc == PA_OK && cudaGraphInstantiate(exec, graph, 0)) fail(PA_ERR_CUDA);
    }
    if (graph) cudaGraphDestroy(graph);
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    for (auto s : br)
        if (s) cudaStreamDestroy(s);
    if (cs) cudaStreamDestroy(cs);
    cudaGetLastError();
    return rc;
}

}  // namespace

extern "C" {

int pa_hash_batch(pa_plan_t *const *plans, const uint64_t *const *keys, const uint64_t *const *seeds,
                  uint64_t *const *outs, int *statuses, int count, void *stream) {
    if (count <= 0 || !plans || !keys || !seeds || !outs) return PA_ERR_INVALID;
    std::vector<uintptr_t> key;
    key.reserve(4 * count + 2);
    key.push_back((uintptr_t)count);
    key.push_back((uintptr_t)statuses);
    for (int i = 0; i < count; i++) {
        if (!plans[i] || !keys[i] || !seeds[i] || !outs[i]) return PA_ERR_INVALID;
        key.push_back((uintptr_t)plans[i]);
        key.push_back((uintptr_t)keys[i]);
        key.push_back((uintptr_t)seeds[i]);
        key.push_back((uintptr_t)outs[i]);
    }
    {
        std::vector<pa_plan_t *> sorted(plans, plans + count);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return PA_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end()) {
        CachedGraph cg;
        int rc = capture(plans, keys, seeds, outs, statuses, count, &cg.exec);
        if (rc) return rc;
        cg.plans.assign(plans, plans + count);
        it = g_cache.emplace(key, cg).first;
    }
    if (cudaGraphLaunch(it->second.exec, (cudaStream_t)stream)) return PA_ERR_CUDA;
    return PA_OK;
}

int pa_batch_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &kv : g_cache) cudaGraphExecDestroy(kv.second.exec);
    g_cache.clear();
    return PA_OK;
}

// Called by pa_plan_destroy: graphs that reference the plan's workspace die with it.
int pa_batch_drop_plan(pa_plan_t *pl) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        if (std::find(it->second.plans.begin(), it->second.plans.end(), pl) != it->second.plans.end()) {
            cudaGraphExecDestroy(it->second.exec);
            it = g_cache.erase(it);
        } else {
            ++it;
        }
    }
    return PA_OK;
}

}  // extern "C"
