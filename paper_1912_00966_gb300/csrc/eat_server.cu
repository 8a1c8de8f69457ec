// Serving loop of libeat (eat_server_* in eat.h): continuous batching of
// earliest-arrival queries over resident networks.
//
// Requests go into a host queue; a dispatcher thread admits them to the GPU.
//
// Ring admission (default): one persistent launch of the per-query kernel serves a
// ring of request entries in page-locked host memory.  The dispatcher writes an
// admitted request into the next ring entry once that entry (and its row of the
// page-locked result pool) is free, then publishes the ring's tail with a release
// store; a block that has finished its query claims the next published entry (a CAS
// on a device-side head), runs it, writes the row into the pool in place and sets
// the entry's done flag with a system-scope release.  The dispatcher sees the flag,
// copies the row to the caller and frees the entry.  When nothing has been in
// flight for a while it sets the stop flag and the launch ends (idle blocks leave);
// the next request starts a new launch.  Ring capacity = admission by memory.
//
// Batch admission: a fixed pool of slots, each a CUDA stream with pre-allocated
// device buffers (query arrays, arrival rows, workspace) and pinned host staging,
// the number of slots set by the memory budget.  A free slot takes up to max_batch
// pending requests (any mix of networks) and runs them as one multi-network batch
// on its stream, so batches launched while others are still running overlap on
// the device; a slot's completion event hands its rows back.
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

struct RingState {
    RingLaunch rl;
    int32_t cap = 0;                     // entries (a power of two)
    RingEntry *h_ring = nullptr, *d_ring = nullptr;
    int64_t *h_tail = nullptr, *d_tail = nullptr;
    int32_t *h_stop = nullptr, *d_stop = nullptr;
    unsigned long long *d_head = nullptr;
    int32_t *h_pool = nullptr, *d_pool = nullptr;   // [cap][row_stride] result rows
    int64_t row_stride = 0;
    void *d_ws = nullptr;
    int32_t *d_rows = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ended = nullptr;
    std::vector<ServerReq> req;          // request held by each entry
    std::vector<char> busy;              // entry published and not yet delivered
    int64_t tail = 0;                    // requests published so far
    int64_t inflight = 0;
    bool running = false, stopping = false;
    Clock::time_point last_busy;
};

constexpr int32_t kRingIdleIters = 5000;     // polls before an idle block leaves (~100 ms)
constexpr auto kRingIdleStop = std::chrono::microseconds(2000);

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
    int admission = EAT_ADMIT_RING;
    eat::RingState ring;
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

static void free_ring(RingState &R) {
    if (R.stream) {
        cudaStreamSynchronize(R.stream);
        cudaStreamDestroy(R.stream);
    }
    if (R.ended) cudaEventDestroy(R.ended);
    for (void *p : {(void *)R.d_head, R.d_ws, (void *)R.d_rows})
        if (p) cudaFree(p);
    for (void *p : {(void *)R.h_ring, (void *)R.h_tail, (void *)R.h_stop, (void *)R.h_pool})
        if (p) cudaFreeHost(p);
    R = RingState();
}

// Fails every request in the ring (the launch could not run or ended in an error).
static void fail_ring(eat_server *sv, int rc) {
    RingState &R = sv->ring;
    sv->last_error = rc;
    for (int32_t i = 0; i < R.cap; ++i) {
        if (!R.busy[i]) continue;
        const ServerReq &r = R.req[i];
        sv->done.push_back({r.tag, rc, r.net, 0});
        R.busy[i] = 0;
    }
    R.inflight = 0;
    sv->cv_done.notify_all();
}

static void dispatcher_ring(eat_server *sv) {
    cudaSetDevice(sv->device);
    RingState &R = sv->ring;
    std::vector<eat_server_result> results;
    R.last_busy = Clock::now();
    for (;;) {
        // 1. Deliver finished requests (any order: blocks finish out of order).
        results.clear();
        const auto now = Clock::now();
        for (int32_t i = 0; i < R.cap && R.inflight > 0; ++i) {
            if (!R.busy[i] || __atomic_load_n(&R.h_ring[i].done, __ATOMIC_ACQUIRE) == 0) continue;
            const ServerReq &r = R.req[i];
            const int32_t V = sv->nets[r.net]->host.n_stops;
            std::memcpy(r.out, R.h_pool + (int64_t)i * R.row_stride, (size_t)V * 4);
            eat_server_result res;
            res.tag = r.tag;
            res.status = R.h_ring[i].status;
            res.net = r.net;
            res.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - r.t_submit).count();
            results.push_back(res);
            R.busy[i] = 0;
            --R.inflight;
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        if (!results.empty()) {
            for (const eat_server_result &r : results) sv->done.push_back(r);
            sv->stats.completed += (int64_t)results.size();
            sv->cv_done.notify_all();
        }
        // 2. Has the launch ended?  Its blocks finish every request they claimed, so
        // requests still in the ring afterwards were never claimed.
        if (R.running) {
            const cudaError_t q = cudaEventQuery(R.ended);
            if (q != cudaErrorNotReady) {
                R.running = false;
                R.stopping = false;
                if (q != cudaSuccess) fail_ring(sv, EAT_ERR_CUDA);
            }
        }
        if (sv->stop && sv->pending.empty() && R.inflight == 0 && !R.running) break;
        // 3. Admit pending requests into free entries, in ring order.
        int64_t admitted = 0;
        while (!sv->pending.empty()) {
            const int32_t slot = (int32_t)(R.tail & (int64_t)(R.cap - 1));
            if (R.busy[slot]) break;                       // that entry is still in flight
            const ServerReq r = sv->pending.front();
            sv->pending.pop_front();
            RingEntry &e = R.h_ring[slot];
            e.net = r.net;
            e.src = r.s;
            e.ts = r.ts;
            e.row = slot;
            e.status = EAT_OK;
            e.seq = R.tail;
            __atomic_store_n(&e.done, 0, __ATOMIC_RELAXED);
            R.req[slot] = r;
            R.busy[slot] = 1;
            ++R.inflight;
            ++R.tail;
            ++admitted;
        }
        if (admitted) {
            __atomic_store_n(R.h_tail, R.tail, __ATOMIC_RELEASE);   // publish the entries
            sv->stats.batched_queries += admitted;
            if (R.running && !R.stopping) sv->stats.admitted_running += admitted;
            sv->stats.max_batch_seen = std::max<int64_t>(sv->stats.max_batch_seen, R.inflight);
            sv->stats.max_inflight_seen = std::max<int64_t>(sv->stats.max_inflight_seen, R.inflight);
        }
        if (R.inflight > 0) R.last_busy = Clock::now();
        // 4. Start a launch when requests wait in the ring and none runs.
        if (!R.running && R.inflight > 0) {
            __atomic_store_n(R.h_stop, 0, __ATOMIC_RELEASE);
            RingArgs rg;
            rg.ring = R.d_ring;
            rg.tail = R.d_tail;
            rg.stop = R.d_stop;
            rg.head = R.d_head;
            rg.row_stride = R.row_stride;
            rg.mask = R.cap - 1;
            rg.idle_iters = kRingIdleIters;
            lk.unlock();
            int rc = ring_launch(sv->nets.data(), (int)sv->nets.size(), R.rl, R.d_ws, R.d_rows,
                                 R.d_pool, rg, R.stream);
            if (rc == EAT_OK) {
                const cudaError_t e = cudaEventRecord(R.ended, R.stream);
                if (e != cudaSuccess) rc = server_cuda_fail(e, "server ring event");
            }
            lk.lock();
            if (rc) {
                fail_ring(sv, rc);
            } else {
                R.running = true;
                ++sv->stats.batches;
            }
        }
        // 5. Let a launch with nothing to do end (idle blocks read the stop flag).
        if (R.running && !R.stopping && R.inflight == 0 &&
            (sv->stop || Clock::now() - R.last_busy > kRingIdleStop)) {
            __atomic_store_n(R.h_stop, 1, __ATOMIC_RELEASE);
            R.stopping = true;
        }
        // 6. Sleep until new work arrives or a request may have finished.
        sv->cv_work.wait_for(lk, R.inflight ? std::chrono::microseconds(10)
                                 : R.running ? std::chrono::microseconds(200)
                                             : std::chrono::microseconds(500));
    }
}

// Ring admission: plan, ring and pool in page-locked host memory, device workspace.
static int create_ring(eat_server *sv, const eat_server_opts &o) {
    RingState &R = sv->ring;
    int rc = ring_setup(sv->nets.data(), (int)sv->nets.size(), R.rl);
    if (rc) return rc;
    R.row_stride = (int64_t)((sv->vmax + 63) / 64 * 64);
    const int64_t per_entry = R.row_stride * 4 + (int64_t)sizeof(RingEntry);
    const int64_t base = (int64_t)R.rl.ws_bytes + (int64_t)R.rl.rows_bytes + 4096;
    const int64_t fit = (o.mem_budget - base) / per_entry;
    const int64_t want = std::min<int64_t>(fit, (int64_t)o.max_batch * o.max_inflight);
    if (want < 1)
        return fail(EAT_ERR_OOM, "mem_budget of " + std::to_string(o.mem_budget) +
                                     " bytes holds no ring entry (" + std::to_string(base) +
                                     " bytes of workspace + " + std::to_string(per_entry) +
                                     " per entry)");
    int32_t cap = 1;
    while ((int64_t)cap * 2 <= want && cap < (1 << 20)) cap *= 2;
    R.cap = cap;
    cudaError_t e = cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.ended, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&R.h_ring, (size_t)cap * sizeof(RingEntry), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&R.h_tail, 64, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&R.h_stop, 64, cudaHostAllocMapped);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&R.h_pool, (size_t)cap * (size_t)R.row_stride * 4, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc((void **)&R.d_head, 64);
    if (e == cudaSuccess) e = cudaMalloc(&R.d_ws, R.rl.ws_bytes);
    if (e == cudaSuccess && R.rl.rows_bytes) e = cudaMalloc((void **)&R.d_rows, R.rl.rows_bytes);
    if (e == cudaSuccess) e = cudaMemset(R.d_head, 0, 64);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&R.d_ring, R.h_ring, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&R.d_tail, R.h_tail, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&R.d_stop, R.h_stop, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&R.d_pool, R.h_pool, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EAT_ERR_OOM, std::string("server ring allocation: ") + cudaGetErrorString(e));
    }
    std::memset(R.h_ring, 0, (size_t)cap * sizeof(RingEntry));
    *R.h_tail = 0;
    *R.h_stop = 0;
    R.req.assign((size_t)cap, ServerReq{});
    R.busy.assign((size_t)cap, 0);
    sv->stats.slots = cap;
    sv->stats.slot_bytes = per_entry;
    sv->stats.base_bytes = base;
    return EAT_OK;
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
    if (o.admission != EAT_ADMIT_RING && o.admission != EAT_ADMIT_BATCH)
        return fail(EAT_ERR_INVALID, "admission must be EAT_ADMIT_RING or EAT_ADMIT_BATCH");
    eat_server *sv = new (std::nothrow) eat_server();
    if (!sv) return fail(EAT_ERR_OOM, "host allocation failed");
    sv->nets.assign(nets, nets + n_nets);
    sv->device = nets[0]->device;
    sv->opts = o;
    sv->admission = o.admission;
    for (const eat_net *n : sv->nets) sv->vmax = std::max(sv->vmax, n->host.n_stops);
    if (o.admission == EAT_ADMIT_RING) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(sv->device);
        const int rc = create_ring(sv, o);
        if (rc) {
            free_ring(sv->ring);
            cudaSetDevice(prev);
            delete sv;
            return rc;
        }
        cudaSetDevice(prev);
        sv->dispatcher = std::thread(dispatcher_ring, sv);
        *out = sv;
        return EAT_OK;
    }
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
    sv->stats.base_bytes = 0;
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
    free_ring(sv->ring);
    cudaSetDevice(prev);
    delete sv;
}

}  // extern "C"
