// pa_serve.cu -- continuous-batching request loop for privacy-amplification
// jobs on one GPU (pa_serve_*).
//
// A worker thread owns `slots` CUDA streams.  Jobs wait in a FIFO and are
// admitted, in order, when a stream is free and the workspace of a plan for
// the job's (n, r) fits in the HBM budget next to everything the server
// already holds (busy plans plus idle cached plans; idle plans of other sizes
// are released first when memory is short).  Admitted jobs run concurrently,
// one per stream, so a request that arrives while others are on the GPU starts
// as soon as a slot and memory free up.
//
// Nothing the worker does waits for the device as a whole: server plans keep
// their memory stream-ordered on a private stream (cudaMallocAsync /
// cudaFreeAsync), a new plan is built with the server lock released (its table
// fills are waited for on its own stream), and an idle plan -- all of whose
// work has completed -- is dropped without a device synchronisation.
// Completion is signalled by a host function enqueued behind each job on its
// stream: it stamps the completion time (latency = submit -> that stamp) and
// wakes the worker, so neither admission nor the latency figures depend on a
// polling interval.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pa_gb300.h"
#include "pa_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum JobState { kQueued, kAdmitting, kRunning, kDone };

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
    // set by the host function behind the job (a CUDA driver thread)
    std::atomic<bool> fired{false};
    Clock::time_point t_fired;
    pa_server_s *srv = nullptr;
};

struct PlanEntry {
    pa_plan_t *plan;
    uint64_t bytes;
};

}  // namespace

struct pa_server_s {
    pa_serve_config cfg;
    int device = 0;
    std::mutex mu;                    // jobs, fifo, slots' busy/ticket, plans, statistics
    std::condition_variable cv_done;  // a job finished (with mu)
    std::mutex wake_mu;               // the worker's wake-up flag (never held across CUDA calls)
    std::condition_variable cv_wake;
    bool wake = false;
    std::deque<uint64_t> fifo;
    std::unordered_map<uint64_t, Job> jobs;
    std::vector<std::unique_ptr<Slot>> slots;
    std::map<std::pair<uint64_t, uint64_t>, std::vector<PlanEntry>> idle;  // (n, r) -> idle plans
    uint64_t held_bytes = 0, peak_bytes = 0;
    uint64_t next_ticket = 1;
    std::vector<double> latencies_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, bits_completed = 0;
    Clock::time_point t_first_submit, t_last_done;
    bool have_first = false;
    bool stop = false;     // shutdown requested: no new admissions
    bool exited = false;   // the worker has left its loop
    std::thread worker;

    void poke() {
        {
            std::lock_guard<std::mutex> lk(wake_mu);
            wake = true;
        }
        cv_wake.notify_one();
    }

    static void CUDART_CB on_job_done(void *arg) {  // no CUDA calls here
        Slot *s = static_cast<Slot *>(arg);
        s->t_fired = Clock::now();
        s->fired.store(true, std::memory_order_release);
        s->srv->poke();
    }

    // ---- worker-side helpers (called with mu held) ----
    void release_idle_for(uint64_t need) {
        for (auto it = idle.begin(); it != idle.end() && held_bytes + need > cfg.hbm_budget_bytes;) {
            auto &vec = it->second;
            while (!vec.empty() && held_bytes + need > cfg.hbm_budget_bytes) {
                pa::plan_destroy_idle(vec.back().plan);  // its work is complete: frees are stream-ordered
                held_bytes -= vec.back().bytes;
                vec.pop_back();
            }
            it = vec.empty() ? idle.erase(it) : std::next(it);
        }
    }

    void launch(Job &j, int slot_idx) {
        Slot &s = *slots[slot_idx];
        s.fired.store(false, std::memory_order_relaxed);
        int rc = pa_hash(j.plan, j.key, j.seed, j.out, s.dstatus, s.stream);
        if (!rc && cudaMemcpyAsync(s.hstatus, s.dstatus, sizeof(int), cudaMemcpyDeviceToHost, s.stream)) rc = PA_ERR_CUDA;
        if (!rc && cudaEventRecord(s.done, s.stream)) rc = PA_ERR_CUDA;
        if (!rc && cudaLaunchHostFunc(s.stream, on_job_done, &s)) rc = PA_ERR_CUDA;
        if (rc) {
            finish(j, rc);
            return;
        }
        s.busy = true;
        s.ticket = j.ticket;
        j.slot = slot_idx;
        j.state = kRunning;
    }

    void finish(Job &j, int status, const Clock::time_point *t = nullptr) {
        j.state = kDone;
        j.status = status;
        j.t_done = t ? *t : Clock::now();
        if (j.plan) {
            idle[std::make_pair(j.n, j.r)].push_back(PlanEntry{j.plan, j.bytes});
            j.plan = nullptr;
        }
        if (status == PA_OK || status == PA_RELOAD) {
            completed++;
            bits_completed += j.n;
            latencies_ms.push_back(std::chrono::duration<double, std::milli>(j.t_done - j.t_submit).count());
            t_last_done = std::max(t_last_done, j.t_done);
        } else if (status == PA_ERR_CANCELLED) {
            cancelled++;
        } else {
            failed++;
        }
    }

    int free_slot() const {
        for (size_t i = 0; i < slots.size(); i++)
            if (!slots[i]->busy) return (int)i;
        return -1;
    }

    // Admissions in FIFO order while a slot is free; a job whose plan does not
    // fit the budget yet waits (and holds back the ones behind it).  A new plan
    // is built with `lk` released.
    void admit(std::unique_lock<std::mutex> &lk) {
        while (!fifo.empty()) {
            const int si = free_slot();
            if (si < 0) return;
            Job &j = jobs[fifo.front()];
            auto key = std::make_pair(j.n, j.r);
            auto it = idle.find(key);
            if (it != idle.end() && !it->second.empty()) {
                j.plan = it->second.back().plan;
                j.bytes = it->second.back().bytes;
                it->second.pop_back();
                fifo.pop_front();
                launch(j, si);
                continue;
            }
            uint64_t need = 0;
            if (pa_plan_estimate_bytes(j.n, j.r, &cfg.params, &need)) {
                fifo.pop_front();
                finish(j, PA_ERR_INVALID);
                cv_done.notify_all();
                continue;
            }
            if (held_bytes + need > cfg.hbm_budget_bytes) release_idle_for(need);
            if (held_bytes + need > cfg.hbm_budget_bytes) return;  // wait for memory
            fifo.pop_front();
            j.state = kAdmitting;
            held_bytes += need;  // reserved while the plan is built
            peak_bytes = std::max(peak_bytes, held_bytes);
            const uint64_t n = j.n, r = j.r;
            pa_plan_t *plan = nullptr;
            lk.unlock();
            const int rc = pa::plan_create(n, r, &cfg.params, true, &plan);
            lk.lock();
            Job &jj = jobs[j.ticket];
            held_bytes -= need;
            if (rc) {
                finish(jj, rc);
                cv_done.notify_all();
                continue;
            }
            pa_plan_info info;
            pa_plan_info_get(plan, &info);
            jj.plan = plan;
            jj.bytes = info.workspace_bytes;
            held_bytes += jj.bytes;
            peak_bytes = std::max(peak_bytes, held_bytes);
            launch(jj, si);  // only this thread admits, so slot si is still free
        }
    }

    bool any_busy() const {
        for (auto &s : slots)
            if (s->busy) return true;
        return false;
    }

    void loop() {
        cudaSetDevice(device);
        while (true) {
            {
                std::unique_lock<std::mutex> lk(mu);
                bool done_any = false;
                for (auto &sp : slots) {
                    Slot &s = *sp;
                    if (!s.busy || !s.fired.load(std::memory_order_acquire)) continue;
                    const cudaError_t q = cudaEventQuery(s.done);  // complete: the host function ran after it
                    Job &j = jobs[s.ticket];
                    finish(j, q == cudaSuccess ? (*s.hstatus ? PA_RELOAD : PA_OK) : PA_ERR_CUDA, &s.t_fired);
                    s.busy = false;
                    done_any = true;
                }
                if (done_any) cv_done.notify_all();
                if (!stop) admit(lk);
                if (stop && !any_busy()) {
                    exited = true;
                    cv_done.notify_all();
                    return;
                }
            }
            std::unique_lock<std::mutex> wl(wake_mu);
            cv_wake.wait_for(wl, std::chrono::milliseconds(2), [&] { return wake; });
            wake = false;
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
    int rc = PA_OK;
    for (uint32_t i = 0; i < cfg->slots && rc == PA_OK; i++) {
        srv->slots.emplace_back(new (std::nothrow) Slot());
        Slot *s = srv->slots.back().get();
        if (!s) {
            srv->slots.pop_back();
            rc = PA_ERR_NOMEM;
            break;
        }
        s->srv = srv;
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) ||
            cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) || cudaMalloc(&s->dstatus, sizeof(int)) ||
            cudaMallocHost(&s->hstatus, sizeof(int)))
            rc = PA_ERR_CUDA;
    }
    if (rc) {
        srv->exited = true;  // no worker was started
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
    {
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
    }
    srv->poke();
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
    for (auto &s : srv->slots) st->running += s->busy ? 1 : 0;
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

int pa_serve_stats_reset(pa_server_t *srv) {
    if (!srv) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->latencies_ms.clear();
    srv->submitted = srv->completed = srv->failed = srv->cancelled = srv->bits_completed = 0;
    srv->have_first = false;
    srv->t_last_done = Clock::time_point{};
    srv->peak_bytes = srv->held_bytes;
    return PA_OK;
}

int pa_serve_shutdown(pa_server_t *srv) {
    if (!srv) return PA_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (uint64_t t : srv->fifo) srv->finish(srv->jobs[t], PA_ERR_CANCELLED);
        srv->fifo.clear();
        srv->cv_done.notify_all();
    }
    srv->poke();
    if (srv->worker.joinable()) srv->worker.join();  // returns once no job is running
    return PA_OK;
}

int pa_serve_destroy(pa_server_t *srv) {
    if (!srv) return PA_ERR_INVALID;
    pa_serve_shutdown(srv);
    for (auto &kv : srv->idle)
        for (auto &pe : kv.second) pa::plan_destroy_idle(pe.plan);
    srv->idle.clear();
    for (auto &sp : srv->slots) {
        Slot &s = *sp;
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
