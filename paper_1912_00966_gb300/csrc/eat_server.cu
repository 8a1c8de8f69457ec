// Serving loop of libeat (eat_server_* in eat.h): continuous batching of
// earliest-arrival queries over resident networks.
//
// Requests go into a host queue.  A dispatcher thread owns a fixed pool of
// slots, each a CUDA stream with pre-allocated device buffers (query arrays,
// arrival rows, workspace) and pinned host staging.  The number of slots is set
// by a device-memory budget: a request is admitted to the GPU only when a slot,
// i.e. its memory, is free.  A free slot takes up to max_batch pending requests
// (any mix of networks) and runs them as one multi-network batch on its stream,
// so batches launched while others are still running overlap on the device.
// When a slot's completion event fires its rows are copied to the callers'
// buffers and the results (tag, status, latency) are queued for eat_server_poll.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <new>
#include <thread>

#include "eat_launch.h"

namespace eat {

using Clock = std::chrono::steady_clock;

struct ServerReq {
    int32_t net, s, ts;
    int32_t *out;
    uint64_t tag;
    Clock::time_point t_submit;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int32_t *d_idx = nullptr, *d_src = nullptr, *d_ts = nullptr, *d_out = nullptr,
            *d_status = nullptr;
    int64_t *d_off = nullptr;
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    int32_t *h_idx = nullptr, *h_src = nullptr, *h_ts = nullptr, *h_out = nullptr,
            *h_status = nullptr;
    int64_t *h_off = nullptr;
    std::vector<ServerReq> reqs;
    Clock::time_point t_launch;
    bool busy = false;
};

}  // namespace eat

struct eat_server {
    std::vector<const eat_net *> nets;
    int device = 0;
    eat_server_opts opts{};
    int32_t vmax = 0;
    std::vector<eat::Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<eat::ServerReq> pending;
    std::deque<eat_server_result> done;
    std::thread dispatcher;
    bool stop = false;
    int last_error = EAT_OK;
    eat_server_stats stats{};
};

namespace eat {

int fail(int code, const std::string &msg);
void clear_error();

static int server_cuda_fail(cudaError_t e, const char *what) {
    return fail(EAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static void free_slot(Slot &s) {
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    for (void *p : {(void *)s.d_idx, (void *)s.d_src, (void *)s.d_ts, (void *)s.d_out,
                    (void *)s.d_status, (void *)s.d_off, s.d_ws})
        if (p) cudaFree(p);
    for (void *p : {(void *)s.h_idx, (void *)s.h_src, (void *)s.h_ts, (void *)s.h_out,
                    (void *)s.h_status, (void *)s.h_off})
        if (p) cudaFreeHost(p);
    s = Slot();
}

// Launch the slot's batch: stage queries, run them, copy rows and statuses back.
static int launch_slot(eat_server *sv, Slot &sl) {
    const int32_t n = (int32_t)sl.reqs.size();
    int64_t off = 0;
    for (int32_t i = 0; i < n; ++i) {
        const ServerReq &r = sl.reqs[i];
        sl.h_idx[i] = r.net;
        sl.h_src[i] = r.s;
        sl.h_ts[i] = r.ts;
        sl.h_off[i] = off;
        off += sv->nets[r.net]->host.n_stops;
    }
    cudaStream_t st = sl.stream;
    cudaError_t e = cudaMemcpyAsync(sl.d_idx, sl.h_idx, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_src, sl.h_src, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_ts, sl.h_ts, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_off, sl.h_off, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return server_cuda_fail(e, "server staging copy");
    eat_query_opts qo{};
    qo.status = sl.d_status;
    int rc = eat_query_batch_multi(sv->nets.data(), (int32_t)sv->nets.size(), sl.d_idx, sl.d_src,
                                   sl.d_ts, n, sl.d_out, sl.d_off, sl.d_ws, sl.ws_bytes, &qo, st);
    if (rc) return rc;
    e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)off * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_status, sl.d_status, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
    if (e != cudaSuccess) return server_cuda_fail(e, "server result copy");
    sl.busy = true;
    sl.t_launch = Clock::now();
    return EAT_OK;
}

// Deliver a finished slot's rows to the callers (called without the lock held).
static void finish_slot(eat_server *sv, Slot &sl, std::vector<eat_server_result> &out) {
    const auto now = Clock::now();
    int64_t off = 0;
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const ServerReq &r = sl.reqs[i];
        const int32_t V = sv->nets[r.net]->host.n_stops;
        std::memcpy(r.out, sl.h_out + off, (size_t)V * 4);
        off += V;
        eat_server_result res;
        res.tag = r.tag;
        res.status = sl.h_status[i];
        res.net = r.net;
        res.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - r.t_submit).count();
        out.push_back(res);
    }
    sl.reqs.clear();
    sl.busy = false;
}

static void dispatcher_main(eat_server *sv) {
    cudaSetDevice(sv->device);
    const auto wait = std::chrono::microseconds(std::max(1, sv->opts.batch_wait_us));
    std::vector<eat_server_result> results;
    for (;;) {
        // 1. Retire finished batches.
        results.clear();
        for (Slot &sl : sv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                std::lock_guard<std::mutex> g(sv->mu);
                sv->last_error = EAT_ERR_CUDA;
                for (ServerReq &r : sl.reqs) {
                    eat_server_result res{r.tag, EAT_ERR_CUDA, r.net, 0};
                    sv->done.push_back(res);
                }
                sl.reqs.clear();
                sl.busy = false;
                sv->cv_done.notify_all();
                continue;
            }
            finish_slot(sv, sl, results);
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        if (!results.empty()) {
            for (const eat_server_result &r : results) sv->done.push_back(r);
            sv->stats.completed += (int64_t)results.size();
            sv->cv_done.notify_all();
        }
        int busy = 0;
        for (const Slot &sl : sv->slots) busy += sl.busy;
        if (sv->stop && sv->pending.empty() && busy == 0) break;
        // 2. Admit pending requests into free slots (continuous batching).
        for (Slot &sl : sv->slots) {
            if (sl.busy || sv->pending.empty()) continue;
            const auto age = Clock::now() - sv->pending.front().t_submit;
            const bool full = (int32_t)sv->pending.size() >= sv->opts.max_batch;
            if (!full && busy > 0 && age < wait && !sv->stop) break;   // let the batch fill
            const int32_t n = std::min<int32_t>((int32_t)sv->pending.size(), sv->opts.max_batch);
            sl.reqs.assign(sv->pending.begin(), sv->pending.begin() + n);
            sv->pending.erase(sv->pending.begin(), sv->pending.begin() + n);
            lk.unlock();
            const int rc = launch_slot(sv, sl);
            lk.lock();
            if (rc) {
                sv->last_error = rc;
                for (ServerReq &r : sl.reqs) sv->done.push_back({r.tag, rc, r.net, 0});
                sl.reqs.clear();
                sv->cv_done.notify_all();
                continue;
            }
            ++busy;
            ++sv->stats.batches;
            sv->stats.batched_queries += n;
            sv->stats.max_batch_seen = std::max<int64_t>(sv->stats.max_batch_seen, n);
            sv->stats.max_inflight_seen = std::max<int64_t>(sv->stats.max_inflight_seen, busy);
        }
        // 3. Sleep until new work arrives or a running batch may have finished.
        sv->cv_work.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::microseconds(500));
    }
}

}  // namespace eat

using namespace eat;

extern "C" {

int eat_server_create(const eat_net *const *nets, int32_t n_nets, const eat_server_opts *opts,
                      eat_server **out) {
    clear_error();
    if (!out) return fail(EAT_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (!nets || n_nets < 1 || n_nets > EAT_MAX_NETS) return fail(EAT_ERR_INVALID, "bad nets");
    for (int i = 0; i < n_nets; ++i) {
        if (!nets[i]) return fail(EAT_ERR_INVALID, "NULL network");
        if (nets[i]->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
        if (nets[i]->device != nets[0]->device) return fail(EAT_ERR_INVALID, "networks on different devices");
    }
    eat_server_opts o{};
    if (opts) o = *opts;
    if (o.max_batch <= 0) o.max_batch = 256;
    if (o.max_inflight <= 0) o.max_inflight = 4;
    if (o.batch_wait_us <= 0) o.batch_wait_us = 200;
    if (o.mem_budget <= 0) o.mem_budget = (int64_t)1 << 30;
    if (o.max_batch > (1 << 20) || o.max_inflight > 64)
        return fail(EAT_ERR_INVALID, "max_batch or max_inflight too large");
    eat_server *sv = new (std::nothrow) eat_server();
    if (!sv) return fail(EAT_ERR_OOM, "host allocation failed");
    sv->nets.assign(nets, nets + n_nets);
    sv->device = nets[0]->device;
    sv->opts = o;
    for (const eat_net *n : sv->nets) sv->vmax = std::max(sv->vmax, n->host.n_stops);
    const size_t ws = eat_workspace_bytes(nets, n_nets, o.max_batch, nullptr);
    if (!ws) {
        delete sv;
        return EAT_ERR_INVALID;
    }
    const size_t rows = (size_t)o.max_batch * (size_t)sv->vmax * 4;
    const size_t per_slot = rows + ws + (size_t)o.max_batch * 24 + 4096;
    const int64_t fit = o.mem_budget / (int64_t)per_slot;
    if (fit < 1) {
        delete sv;
        return fail(EAT_ERR_OOM, "mem_budget of " + std::to_string(o.mem_budget) +
                                     " bytes holds no slot of " + std::to_string(per_slot) + " bytes");
    }
    const int n_slots = (int)std::min<int64_t>(fit, o.max_inflight);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    sv->slots.resize(n_slots);
    int rc = EAT_OK;
    for (Slot &sl : sv->slots) {
        const size_t n = (size_t)o.max_batch;
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_idx, n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_src, n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_ts, n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_status, n * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_off, n * 8);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.d_out, rows);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_ws, ws);
        sl.ws_bytes = ws;
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_idx, n * 4);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_src, n * 4);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_ts, n * 4);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_status, n * 4);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_off, n * 8);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_out, rows);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(EAT_ERR_OOM, std::string("server slot allocation: ") + cudaGetErrorString(e));
            break;
        }
    }
    if (rc) {
        for (Slot &sl : sv->slots) free_slot(sl);
        cudaSetDevice(prev);
        delete sv;
        return rc;
    }
    sv->stats.slots = n_slots;
    sv->stats.slot_bytes = (int64_t)per_slot;
    cudaSetDevice(prev);
    sv->dispatcher = std::thread(dispatcher_main, sv);
    *out = sv;
    return EAT_OK;
}

int eat_server_submit(eat_server *sv, int32_t net, int32_t s, int32_t t_s, int32_t *arr_out,
                      uint64_t tag) {
    clear_error();
    if (!sv || !arr_out) return fail(EAT_ERR_INVALID, "NULL argument");
    if (net < 0 || net >= (int32_t)sv->nets.size()) return fail(EAT_ERR_INVALID, "net out of range");
    if (s < 0 || s >= sv->nets[net]->host.n_stops) return fail(EAT_ERR_INVALID, "source out of range");
    {
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->stop) return fail(EAT_ERR_INVALID, "server is shutting down");
        sv->pending.push_back({net, s, t_s, arr_out, tag, Clock::now()});
        ++sv->stats.submitted;
        sv->stats.max_pending_seen = std::max<int64_t>(sv->stats.max_pending_seen, (int64_t)sv->pending.size());
    }
    sv->cv_work.notify_one();
    return EAT_OK;
}

int32_t eat_server_poll(eat_server *sv, eat_server_result *results, int32_t max, int32_t timeout_us) {
    clear_error();
    if (!sv || !results || max <= 0) return 0;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done.empty() && timeout_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !sv->done.empty(); });
    int32_t k = 0;
    while (k < max && !sv->done.empty()) {
        results[k++] = sv->done.front();
        sv->done.pop_front();
    }
    return k;
}

int eat_server_get_stats(eat_server *sv, eat_server_stats *out) {
    clear_error();
    if (!sv || !out) return fail(EAT_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> g(sv->mu);
    *out = sv->stats;
    out->pending = (int64_t)sv->pending.size();
    out->last_error = sv->last_error;
    return EAT_OK;
}

void eat_server_destroy(eat_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->dispatcher.joinable()) sv->dispatcher.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    for (Slot &sl : sv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        free_slot(sl);
    }
    cudaSetDevice(prev);
    delete sv;
}

}  // extern "C"
