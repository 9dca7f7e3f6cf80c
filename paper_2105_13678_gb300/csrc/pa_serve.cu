// pa_serve.cu -- continuous-batching request loop for privacy-amplification
// jobs on one GPU (pa_serve_*).
//
// A worker thread owns `slots` CUDA streams.  Jobs wait in a FIFO and are
// admitted, in order, when a stream is free and the workspace of a plan for
// the job's (n, r) fits in the HBM budget next to everything the server
// already holds (busy plans plus idle cached plans; idle plans of other sizes
// are released first when memory is short).  Admitted jobs run concurrently,
// one per stream, so a request that arrives while others are on the GPU starts
// as soon as a slot and memory free up.  Completion is detected with events;
// latency is measured from submit to the host observing completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pa_gb300.h"

extern "C" int pa_plan_estimate_bytes(uint64_t n_bits, uint64_t r_bits, const pa_params *params, uint64_t *bytes);

namespace {

using Clock = std::chrono::steady_clock;

enum JobState { kQueued, kRunning, kDone };

struct Job {
    uint64_t ticket, n, r;
    const uint64_t *key, *seed;
    uint64_t *out;
    Clock::time_point t_submit, t_done;
    JobState state = kQueued;
    int status = PA_OK;
    int slot = -1;
    pa_plan_t *plan = nullptr;
    uint64_t bytes = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int *dstatus = nullptr;
    int *hstatus = nullptr;  // pinned
    uint64_t ticket = 0;
    bool busy = false;
};

struct PlanEntry {
    pa_plan_t *plan;
    uint64_t bytes;
};

}  // namespace

struct pa_server_s {
    pa_serve_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> fifo;
    std::unordered_map<uint64_t, Job> jobs;
    std::vector<Slot> slots;
    std::map<std::pair<uint64_t, uint64_t>, std::vector<PlanEntry>> idle;  // (n, r) -> idle plans
    uint64_t held_bytes = 0, peak_bytes = 0;
    uint64_t next_ticket = 1;
    std::vector<double> latencies_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, bits_completed = 0;
    Clock::time_point t_first_submit, t_last_done;
    bool have_first = false;
    std::atomic<bool> stop{false};
    std::thread worker;

    // ---- worker-side helpers (called with mu held) ----
    void release_idle_for(uint64_t need) {
        for (auto it = idle.begin(); it != idle.end() && held_bytes + need > cfg.hbm_budget_bytes;) {
            auto &vec = it->second;
            while (!vec.empty() && held_bytes + need > cfg.hbm_budget_bytes) {
                pa_plan_destroy(vec.back().plan);
                held_bytes -= vec.back().bytes;
                vec.pop_back();
            }
            it = vec.empty() ? idle.erase(it) : std::next(it);
        }
    }

    bool try_admit(Job &j, int slot_idx) {
        auto key = std::make_pair(j.n, j.r);
        auto it = idle.find(key);
        if (it != idle.end() && !it->second.empty()) {
            j.plan = it->second.back().plan;
            j.bytes = it->second.back().bytes;
            it->second.pop_back();
        } else {
            uint64_t need = 0;
            if (pa_plan_estimate_bytes(j.n, j.r, &cfg.params, &need)) {
                j.status = PA_ERR_INVALID;
                return true;  // consumed: fails immediately
            }
            if (held_bytes + need > cfg.hbm_budget_bytes) release_idle_for(need);
            if (held_bytes + need > cfg.hbm_budget_bytes) return false;  // wait for memory
            int rc = pa_plan(j.n, j.r, &cfg.params, &j.plan);
            if (rc) {
                j.status = rc;
                j.plan = nullptr;
                return true;
            }
            pa_plan_info info;
            pa_plan_info_get(j.plan, &info);
            j.bytes = info.workspace_bytes;
            held_bytes += j.bytes;
            peak_bytes = std::max(peak_bytes, held_bytes);
        }
        Slot &s = slots[slot_idx];
        int rc = pa_hash(j.plan, j.key, j.seed, j.out, s.dstatus, s.stream);
        if (!rc && cudaMemcpyAsync(s.hstatus, s.dstatus, sizeof(int), cudaMemcpyDeviceToHost, s.stream)) rc = PA_ERR_CUDA;
        if (!rc && cudaEventRecord(s.done, s.stream)) rc = PA_ERR_CUDA;
        if (rc) {
            j.status = rc;
            return true;
        }
        s.busy = true;
        s.ticket = j.ticket;
        j.slot = slot_idx;
        j.state = kRunning;
        return true;
    }

    void finish(Job &j, int status) {
        j.state = kDone;
        j.status = status;
        j.t_done = Clock::now();
        if (j.plan) {
            idle[std::make_pair(j.n, j.r)].push_back(PlanEntry{j.plan, j.bytes});
            j.plan = nullptr;
        }
        if (status == PA_OK || status == PA_RELOAD) {
            completed++;
            bits_completed += j.n;
            latencies_ms.push_back(std::chrono::duration<double, std::milli>(j.t_done - j.t_submit).count());
            t_last_done = j.t_done;
        } else if (status == PA_ERR_CANCELLED) {
            cancelled++;
        } else {
            failed++;
        }
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progressed = false;
            // completions
            for (size_t i = 0; i < slots.size(); i++) {
                Slot &s = slots[i];
                if (!s.busy) continue;
                cudaError_t q = cudaEventQuery(s.done);
                if (q == cudaErrorNotReady) continue;
                Job &j = jobs[s.ticket];
                finish(j, q == cudaSuccess ? (*s.hstatus ? PA_RELOAD : PA_OK) : PA_ERR_CUDA);
                s.busy = false;
                progressed = true;
            }
            if (progressed) cv_done.notify_all();
            // admissions, FIFO order
            while (!fifo.empty()) {
                int free_slot = -1;
                for (size_t i = 0; i < slots.size(); i++)
                    if (!slots[i].busy) {
                        free_slot = (int)i;
                        break;
                    }
                if (free_slot < 0) break;
                Job &j = jobs[fifo.front()];
                if (!try_admit(j, free_slot)) break;
                fifo.pop_front();
                if (j.state != kRunning) {
                    finish(j, j.status);
                    cv_done.notify_all();
                }
                progressed = true;
            }
            bool any_busy = false;
            for (auto &s : slots) any_busy = any_busy || s.busy;
            if (stop && !any_busy) break;
            if (!progressed) {
                if (any_busy)
                    cv_work.wait_for(lk, std::chrono::microseconds(20));
                else
                    cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
};

extern "C" {

int pa_serve_create(const pa_serve_config *cfg, pa_server_t **out) {
    if (!cfg || !out || cfg->slots == 0 || cfg->hbm_budget_bytes == 0) return PA_ERR_INVALID;
    *out = nullptr;
    pa_server_t *srv = new (std::nothrow) pa_server_s();
    if (!srv) return PA_ERR_NOMEM;
    srv->cfg = *cfg;
    if (srv->cfg.max_queue == 0) srv->cfg.max_queue = 1u << 20;
    cudaGetDevice(&srv->device);
    srv->slots.resize(cfg->slots);
    int rc = PA_OK;
    for (auto &s : srv->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) || cudaMalloc(&s.dstatus, sizeof(int)) ||
            cudaMallocHost(&s.hstatus, sizeof(int))) {
            rc = PA_ERR_CUDA;
            break;
        }
    }
    if (rc) {
        pa_serve_destroy(srv);
        return rc;
    }
    srv->worker = std::thread([srv] { srv->loop(); });
    *out = srv;
    return PA_OK;
}

int pa_serve_submit(pa_server_t *srv, uint64_t n_bits, uint64_t r_bits, const uint64_t *key, const uint64_t *seed,
                    uint64_t *out, uint64_t *ticket) {
    if (!srv || !key || !seed || !out || !ticket || n_bits == 0 || r_bits == 0) return PA_ERR_INVALID;
    uint64_t need = 0;
    int rc = pa_plan_estimate_bytes(n_bits, r_bits, &srv->cfg.params, &need);
    if (rc) return rc;
    if (need > srv->cfg.hbm_budget_bytes) return PA_ERR_BUDGET;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return PA_ERR_CANCELLED;
    if (srv->fifo.size() >= srv->cfg.max_queue) return PA_ERR_BUSY;
    Job j;
    j.ticket = srv->next_ticket++;
    j.n = n_bits;
    j.r = r_bits;
    j.key = key;
    j.seed = seed;
    j.out = out;
    j.t_submit = Clock::now();
    if (!srv->have_first) {
        srv->t_first_submit = j.t_submit;
        srv->have_first = true;
    }
    srv->jobs.emplace(j.ticket, j);
    srv->fifo.push_back(j.ticket);
    srv->submitted++;
    *ticket = j.ticket;
    srv->cv_work.notify_one();
    return PA_OK;
}

int pa_serve_poll(pa_server_t *srv, uint64_t ticket, int *status) {
    if (!srv || !status) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return PA_ERR_INVALID;
    if (it->second.state != kDone) return PA_ERR_BUSY;
    *status = it->second.status;
    return PA_OK;
}

int pa_serve_wait(pa_server_t *srv, uint64_t ticket, uint64_t timeout_ns, int *status) {
    if (!srv || !status) return PA_ERR_INVALID;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return PA_ERR_INVALID;
    const auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns);
    while (it->second.state != kDone) {
        if (srv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state != kDone)
            return PA_ERR_TIMEOUT;
    }
    *status = it->second.status;
    return PA_OK;
}

int pa_serve_stats_get(pa_server_t *srv, pa_serve_stats *st) {
    if (!srv || !st) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    *st = pa_serve_stats{};
    st->submitted = srv->submitted;
    st->completed = srv->completed;
    st->failed = srv->failed;
    st->cancelled = srv->cancelled;
    st->queued = srv->fifo.size();
    for (auto &s : srv->slots) st->running += s.busy ? 1 : 0;
    st->bits_completed = srv->bits_completed;
    st->peak_budget_bytes = srv->peak_bytes;
    std::vector<double> lat = srv->latencies_ms;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto q = [&](double p) { return lat[std::min(lat.size() - 1, (size_t)(p * (double)(lat.size() - 1) + 0.5))]; };
        st->p50_latency_ms = q(0.50);
        st->p99_latency_ms = q(0.99);
        st->max_latency_ms = lat.back();
        st->busy_seconds = std::chrono::duration<double>(srv->t_last_done - srv->t_first_submit).count();
    }
    return PA_OK;
}

int pa_serve_destroy(pa_server_t *srv) {
    if (!srv) return PA_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (uint64_t t : srv->fifo) srv->finish(srv->jobs[t], PA_ERR_CANCELLED);
        srv->fifo.clear();
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    for (auto &kv : srv->idle)
        for (auto &pe : kv.second) pa_plan_destroy(pe.plan);
    for (auto &s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.dstatus) cudaFree(s.dstatus);
        if (s.hstatus) cudaFreeHost(s.hstatus);
    }
    delete srv;
    return PA_OK;
}

}  // extern "C"
