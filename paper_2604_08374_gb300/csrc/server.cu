// server.cu -- a request loop that serves HyperBall analyses of device-resident
// graphs, with continuous batching.
//
// Requests (graph, p, d, seed, convergence rule, host outputs) arrive from any
// thread.  Their device state (counters, estimates, sums, outputs) is charged
// to an HBM budget; a request is admitted when its bytes fit.  Two lanes share
// the budget and run on their own streams, so their work overlaps on the GPU:
//
//   batched lane  graphs up to `solo_nodes` nodes.  Between any two passes it
//                 admits waiting requests that fit (up to `max_batch` at once),
//                 starts their counters, then advances every admitted request
//                 by one pass with the batched engine (engine.cu: one union,
//                 estimate, step and finalize launch for all of them), and
//                 retires the ones that stopped.  Requests join and leave
//                 between passes: continuous batching at pass granularity.
//   solo lane     larger graphs, one at a time, through hyperball_run_dev
//                 (run-aware union) on its own stream.
//
// Each request's results are bit-identical to running it alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.cuh"

namespace vga {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    const vga_graph *g = nullptr;
    int p = 10, d = 0, conv = 0;
    uint64_t seed = 0;
    double *md_host = nullptr, *ball_host = nullptr;
    Clock::time_point t_submit, t_admit, t_done;
    int lane = 0;          // 0 batched, 1 solo
    uint64_t bytes = 0;    // budget charge
    JobLayout L;
    bool done = false;
    int status = VGA_OK;
    int iterations = 0;
    std::string error;
    uint8_t *ws = nullptr;  // device block: layout, then md, ball
};

}  // namespace
}  // namespace vga

struct vga_server {
    vga_server_config cfg{};
    int device = 0;
    uint64_t l2_budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<vga::Request>> pending_batched, pending_solo;
    std::unordered_map<uint64_t, std::shared_ptr<vga::Request>> requests;
    uint64_t next_id = 1;
    uint64_t budget_used = 0, budget_peak = 0;
    uint64_t submitted = 0, completed = 0, passes = 0, batched_peak = 0;
    bool stopping = false;
    std::thread lane_batched, lane_solo;
    // batched-lane device state
    cudaStream_t stream_batched = nullptr, stream_solo = nullptr;
    // requests' workspaces come from the server's own stream-ordered pool, which
    // keeps freed memory (up to the HBM budget) for the next request instead of
    // returning it to the driver at every synchronisation
    cudaMemPool_t pool = nullptr;
    std::atomic<int> solo_active{0};  // a solo-lane analysis is on the GPU
    uint8_t *arrays = nullptr;  // active and start arrays, LC tables
};

namespace vga {
namespace {

uint64_t request_bytes_batched(const JobLayout &L, uint32_t n) { return L.bytes + align256(16ull * n); }

// Copy a finished request's outputs to the caller's host buffers, release its
// device block and budget, and wake its waiters.
void retire(vga_server *S, const std::shared_ptr<Request> &r, double *md_dev, double *ball_dev, cudaStream_t stream) {
    int rc = VGA_OK;
    std::string msg;
    const size_t n = r->g->n;
    if (r->status == VGA_OK && n) {
        cudaError_t e = cudaSuccess;
        if (r->md_host) e = cudaMemcpyAsync(r->md_host, md_dev, 8 * n, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess && r->ball_host)
            e = cudaMemcpyAsync(r->ball_host, ball_dev, 8 * n, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            rc = VGA_ECUDA;
            msg = cudaGetErrorString(e);
        }
    }
    if (r->ws) cudaFreeAsync(r->ws, stream);
    r->ws = nullptr;
    std::lock_guard<std::mutex> lock(S->mu);
    if (rc != VGA_OK) {
        r->status = rc;
        r->error = msg;
    }
    S->budget_used -= r->bytes;
    r->done = true;
    r->t_done = Clock::now();
    S->completed++;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

void fail(vga_server *S, const std::shared_ptr<Request> &r, int status, const char *what, cudaStream_t stream) {
    r->status = status;
    r->error = what;
    retire(S, r, nullptr, nullptr, stream);
}

void batched_lane(vga_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t stream = S->stream_batched;
    const int cap = S->cfg.max_batch;
    const EngineArrays A_run = engine_arrays_at(S->arrays, cap);
    const EngineArrays A_new = engine_arrays_at(S->arrays + align256(engine_arrays_bytes(cap)), cap);
    const double *lc_base = reinterpret_cast<const double *>(S->arrays + 2 * align256(engine_arrays_bytes(cap)));
    std::vector<std::shared_ptr<Request>> active;
    std::vector<JobDev> host;  // device state of `active`, refreshed after every pass
    EngineForks forks;         // the pass's union kernels of different slice widths run side by side
    for (;;) {
        std::vector<std::shared_ptr<Request>> fresh;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            while (!S->stopping && active.empty() && S->pending_batched.empty()) S->cv_work.wait(lock);
            if (S->stopping && active.empty() && S->pending_batched.empty()) break;
            // admit every waiting request that fits, in arrival order
            for (auto it = S->pending_batched.begin(); it != S->pending_batched.end();) {
                const auto &r = *it;
                if ((int)(active.size() + fresh.size()) >= cap) break;
                if (S->budget_used + r->bytes > S->cfg.hbm_budget_bytes) {
                    ++it;
                    continue;
                }
                S->budget_used += r->bytes;
                S->budget_peak = std::max(S->budget_peak, S->budget_used);
                r->t_admit = Clock::now();
                fresh.push_back(r);
                it = S->pending_batched.erase(it);
            }
            S->batched_peak = std::max<uint64_t>(S->batched_peak, active.size() + fresh.size());
        }
        // start the admitted requests' counters
        std::vector<JobDev> start;
        std::vector<std::shared_ptr<Request>> started;
        for (const auto &r : fresh) {
            void *mem = nullptr;
            if (cudaMallocFromPoolAsync(&mem, r->bytes, S->pool, stream) != cudaSuccess) {
                cudaGetLastError();
                fail(S, r, VGA_ENOMEM, "device allocation for the request failed", stream);
                continue;
            }
            r->ws = static_cast<uint8_t *>(mem);
            double *md = reinterpret_cast<double *>(r->ws + r->L.bytes);
            JobDev J{};
            vga_tune_entry te{};
            const bool tabled = tune_table_lookup(r->g, &te);
            const uint32_t hub = tabled ? (uint32_t)te.hub_lookups : 0u;
            const int rc = make_jobdev(r->g, r->p, r->d, r->seed, r->conv, r->L, r->ws, lc_base + lc_offset(r->p) / 8,
                                       md, md + r->g->n, hub, stream, &J, tabled ? te.group_nodes : 0);
            if (rc != VGA_OK) {
                fail(S, r, rc, vga_last_error(), stream);
                continue;
            }
            start.push_back(J);
            started.push_back(r);
        }
        if (!start.empty()) {
            EngineSet E;
            int rc = engine_upload(A_new, start, &E, stream);
            if (rc == VGA_OK) rc = engine_start(A_new, start, E, stream);
            if (rc == VGA_OK) {  // the scattered pass 1 left its change flags in the descriptors
                cudaError_t e = cudaMemcpyAsync(start.data(), A_new.jobs, sizeof(JobDev) * start.size(),
                                                cudaMemcpyDeviceToHost, stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
                if (e != cudaSuccess) {
                    set_error("reading the started requests' state failed: %s", cudaGetErrorString(e));
                    rc = VGA_ECUDA;
                }
            }
            if (rc != VGA_OK) {
                for (const auto &r : started) fail(S, r, rc, vga_last_error(), stream);
                started.clear();
                start.clear();
            }
            for (size_t k = 0; k < started.size(); k++) {
                active.push_back(started[k]);
                host.push_back(start[k]);
            }
        }
        if (active.empty()) continue;
        // one pass for every admitted request
        EngineSet E;
        int rc = engine_upload(A_run, host, &E, stream);
        const int share = S->solo_active.load() ? S->cfg.batched_share : 100;
        if (rc == VGA_OK) rc = engine_pass(A_run, E, stream, 0, 0, share, &forks);
        cudaError_t e = cudaSuccess;
        int err = 0;
        if (rc == VGA_OK) {
            e = cudaMemcpyAsync(host.data(), A_run.jobs, sizeof(JobDev) * host.size(), cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&err, A_run.error, sizeof(int), cudaMemcpyDeviceToHost, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) rc = VGA_ECUDA;
            if (err) rc = VGA_ETIMEOUT;
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->passes++;
        }
        if (rc != VGA_OK) {
            for (const auto &r : active) fail(S, r, rc, "batched pass failed", stream);
            active.clear();
            host.clear();
            continue;
        }
        // retire the requests that stopped (their epilogue ran in this pass)
        std::vector<std::shared_ptr<Request>> keep_r;
        std::vector<JobDev> keep_h;
        for (size_t k = 0; k < active.size(); k++) {
            if (host[k].state != 0) {
                active[k]->iterations = host[k].t;
                retire(S, active[k], host[k].md, host[k].ball, stream);
            } else {
                keep_r.push_back(active[k]);
                keep_h.push_back(host[k]);
            }
        }
        active.swap(keep_r);
        host.swap(keep_h);
    }
}

void solo_lane(vga_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t stream = S->stream_solo;
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            for (;;) {
                if (!S->pending_solo.empty()) {
                    auto &front = S->pending_solo.front();
                    if (S->budget_used + front->bytes <= S->cfg.hbm_budget_bytes) break;
                } else if (S->stopping) {
                    return;
                }
                S->cv_work.wait(lock);
            }
            r = S->pending_solo.front();
            S->pending_solo.pop_front();
            S->budget_used += r->bytes;
            S->budget_peak = std::max(S->budget_peak, S->budget_used);
            r->t_admit = Clock::now();
        }
        void *mem = nullptr;
        if (cudaMallocFromPoolAsync(&mem, r->bytes, S->pool, stream) != cudaSuccess) {
            cudaGetLastError();
            fail(S, r, VGA_ENOMEM, "device allocation for the request failed", stream);
            continue;
        }
        r->ws = static_cast<uint8_t *>(mem);
        const uint64_t ws_bytes = r->bytes - align256(16ull * r->g->n);
        double *md = reinterpret_cast<double *>(r->ws + ws_bytes);
        int it = 0;
        S->solo_active.store(1);
        const int rc = hyperball_run_dev(r->g, r->p, r->d, r->seed, r->conv, md, md + r->g->n, &it, r->ws, ws_bytes,
                                         stream, nullptr);
        S->solo_active.store(0);
        if (rc != VGA_OK) {
            fail(S, r, rc, vga_last_error(), stream);
            continue;
        }
        r->iterations = it;
        retire(S, r, md, md + r->g->n, stream);
    }
}

}  // namespace
}  // namespace vga

using namespace vga;

extern "C" {

int vga_server_create(const vga_server_config *cfg, vga_server **out) {
    clear_error();
    if (!out) {
        set_error("vga_server_create: null argument");
        return VGA_EINVAL;
    }
    auto S = std::make_unique<vga_server>();
    if (cfg) S->cfg = *cfg;
    if (S->cfg.hbm_budget_bytes == 0) S->cfg.hbm_budget_bytes = 150ull << 30;
    if (S->cfg.max_batch <= 0) S->cfg.max_batch = 256;
    if (S->cfg.solo_nodes == 0) S->cfg.solo_nodes = 32768;
    if (S->cfg.lane_priority < -1 || S->cfg.lane_priority > 1) {
        set_error("vga_server_create: lane_priority = %d is outside -1..1", S->cfg.lane_priority);
        return VGA_EINVAL;
    }
    if (S->cfg.batched_share < 0 || S->cfg.batched_share > 100) {
        set_error("vga_server_create: batched_share = %d is outside 0..100", S->cfg.batched_share);
        return VGA_EINVAL;
    }
    VGA_CHECK_CUDA(cudaGetDevice(&S->device));
    S->l2_budget = l2_budget_bytes(S->device);
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        VGA_CHECK_CUDA(cudaMemPoolCreate(&S->pool, &props));
        uint64_t keep = S->cfg.hbm_budget_bytes;
        VGA_CHECK_CUDA(cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    const uint64_t arrays = 2 * align256(engine_arrays_bytes(S->cfg.max_batch)) + lc_all_bytes();
    void *mem = nullptr;
    VGA_CHECK_CUDA(cudaMalloc(&mem, arrays));
    S->arrays = static_cast<uint8_t *>(mem);
    int prio_low = 0, prio_high = 0;
    VGA_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    const int prio_batched = S->cfg.lane_priority < 0 ? prio_high : prio_low;
    const int prio_solo = S->cfg.lane_priority > 0 ? prio_high : prio_low;
    VGA_CHECK_CUDA(cudaStreamCreateWithPriority(&S->stream_batched, cudaStreamNonBlocking, prio_batched));
    VGA_CHECK_CUDA(cudaStreamCreateWithPriority(&S->stream_solo, cudaStreamNonBlocking, prio_solo));
    VGA_TRY(upload_lc_tables(S->arrays + 2 * align256(engine_arrays_bytes(S->cfg.max_batch)), nullptr,
                             S->stream_batched));
    VGA_CHECK_CUDA(cudaStreamSynchronize(S->stream_batched));
    vga_server *raw = S.release();
    raw->lane_batched = std::thread(batched_lane, raw);
    raw->lane_solo = std::thread(solo_lane, raw);
    *out = raw;
    return VGA_OK;
}

int vga_server_submit(vga_server *S, const vga_graph *g, int p, int d, uint64_t seed, int conv_mode,
                      double *mean_depth_host, double *ball_size_host, uint64_t *request_id) {
    clear_error();
    if (!S || !g || !request_id || p < 4 || p > 16 || (conv_mode != 0 && conv_mode != 1)) {
        set_error("vga_server_submit: null argument, p outside 4..16 or bad conv_mode");
        return VGA_EINVAL;
    }
    if (g->device != S->device) {
        set_error("vga_server_submit: graph on device %d, server on device %d", g->device, S->device);
        return VGA_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->g = g;
    r->p = p;
    r->d = d;
    r->seed = seed;
    r->conv = conv_mode;
    r->md_host = mean_depth_host;
    r->ball_host = ball_size_host;
    r->t_submit = Clock::now();
    r->lane = g->n > (uint32_t)S->cfg.solo_nodes ? 1 : 0;
    if (r->lane == 0) {
        r->L = job_layout(g->n, p, 0, S->l2_budget, 0, g->lk_scheme);
        r->bytes = request_bytes_batched(r->L, g->n);
    } else {
        uint64_t ws = 0;
        VGA_TRY(hyperball_workspace_bytes(g, p, &ws));
        r->bytes = align256(ws) + align256(16ull * g->n);
    }
    if (r->bytes > S->cfg.hbm_budget_bytes) {
        set_error("vga_server_submit: the request needs %llu bytes, more than the whole budget (%llu)",
                  (unsigned long long)r->bytes, (unsigned long long)S->cfg.hbm_budget_bytes);
        return VGA_EBUSY;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) {
        set_error("vga_server_submit: server is shutting down");
        return VGA_EBUSY;
    }
    r->id = S->next_id++;
    S->requests[r->id] = r;
    S->submitted++;
    if (g->n == 0) {  // nothing to compute
        r->done = true;
        r->t_admit = r->t_done = Clock::now();
        S->completed++;
        S->cv_done.notify_all();
    } else {
        (r->lane ? S->pending_solo : S->pending_batched).push_back(r);
        S->cv_work.notify_all();
    }
    *request_id = r->id;
    return VGA_OK;
}

int vga_server_wait(vga_server *S, uint64_t request_id, double timeout_s, int *iterations, double *latency_s,
                    double *queued_s) {
    clear_error();
    if (!S) {
        set_error("vga_server_wait: null server");
        return VGA_EINVAL;
    }
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->requests.find(request_id);
    if (it == S->requests.end()) {
        set_error("vga_server_wait: unknown request %llu", (unsigned long long)request_id);
        return VGA_EINVAL;
    }
    std::shared_ptr<Request> r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    while (!r->done) {
        if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && !r->done) {
            set_error("vga_server_wait: request %llu not done after %.3f s", (unsigned long long)request_id,
                      timeout_s);
            return VGA_ETIMEOUT;
        }
    }
    if (iterations) *iterations = r->iterations;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (queued_s) *queued_s = std::chrono::duration<double>(r->t_admit - r->t_submit).count();
    const int status = r->status;
    if (status != VGA_OK) set_error("request %llu failed: %s", (unsigned long long)request_id, r->error.c_str());
    S->requests.erase(it);
    return status;
}

int vga_server_stats(vga_server *S, vga_server_stats_t *out) {
    clear_error();
    if (!S || !out) {
        set_error("vga_server_stats: null argument");
        return VGA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->batched_passes = S->passes;
    out->budget_used = S->budget_used;
    out->budget_peak = S->budget_peak;
    out->batched_peak = S->batched_peak;
    out->queued = S->pending_batched.size() + S->pending_solo.size();
    return VGA_OK;
}

void vga_server_destroy(vga_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->lane_batched.joinable()) S->lane_batched.join();
    if (S->lane_solo.joinable()) S->lane_solo.join();
    cudaSetDevice(S->device);
    if (S->stream_batched) cudaStreamSynchronize(S->stream_batched);
    if (S->stream_solo) cudaStreamSynchronize(S->stream_solo);
    if (S->arrays) cudaFree(S->arrays);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->stream_batched) cudaStreamDestroy(S->stream_batched);
    if (S->stream_solo) cudaStreamDestroy(S->stream_solo);
    delete S;
}

}  // extern "C"
