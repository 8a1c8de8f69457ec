// Topology-driven variants of Section II (A to F), the paper's own execution
// model: one query at a time, every round one kernel over all connections, types
// or edges, host-driven rounds with a flag read every `flag_every` rounds
// (Section IV-C).  Kept as a baseline for the frontier-driven kernels of
// eat_kernels.cu and to show what each pruning step buys.
//
// Active stops (Section III-B's active / nextactive pair) are two arrays of round
// stamps: stop u is active in round i if stamp[i & 1][u] == i, and a stop lowered
// in round i gets stamp[(i + 1) & 1][v] = i + 1, so neither array is ever
// cleared.  `last` holds the latest round that lowered some arrival: after round
// i the query has converged iff last < i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "eat_device.cuh"
#include "eat_internal.h"

namespace eat {

struct LadderDev {
    const int32_t *cu, *cv, *cdep, *cdur;   // connections [C]
    const int4 *ty;                         // {tail, head, duration, 0} [T]
    const int32_t *dep_ptr, *dep;           // sorted unique departures per type
    const int32_t *ap_ptr;                  // whole-day APs per type
    const int4 *ap;                         // {first, difference, terms, last term}
    const int32_t *edge_ptr, *edge_u;       // edge e = types [edge_ptr[e], edge_ptr[e+1])
    int32_t *e;                             // [V] arrivals
    int32_t *stamp;                         // [2 V] round stamps
    int32_t *last;                          // latest round that lowered an arrival
    int32_t *round;                         // round index for launches that read it here
    int32_t V, T, E;
    int64_t C;
};

namespace {

// Round index of a launch: the argument, or (when it is negative: graph replay, where
// every launch of the graph is the same) the device counter that ladder_advance_kernel
// moves on after each round.
__device__ __forceinline__ int32_t round_of(const LadderDev &L, int32_t it) {
    return it >= 0 ? it : __ldcg(L.round);
}

__device__ __forceinline__ bool ladder_active(const LadderDev &L, int32_t u, int32_t it) {
    return __ldcg(L.stamp + (int64_t)(it & 1) * L.V + u) == it;
}

// Relax (Algorithm 3): lower e[v] to cand if that is earlier; the winner marks v
// active for the next round and records that round `it` changed something.
__device__ __forceinline__ void ladder_relax(const LadderDev &L, int32_t v, int32_t cand,
                                             int32_t it) {
    if (cand >= __ldcg(L.e + v)) return;
    if (atomicMin(L.e + v, cand) <= cand) return;
    L.stamp[(int64_t)((it + 1) & 1) * L.V + v] = it + 1;
    if (__ldcg(L.last) < it) atomicMax(L.last, it);
}

__global__ void ladder_init_kernel(LadderDev L, int32_t s, int32_t t_s) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.V; i += stride) {
        L.e[i] = i == s ? t_s : kInf;
        L.stamp[i] = i == s ? 0 : -1;
        L.stamp[L.V + i] = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *L.last = -1;
        *L.round = 0;
    }
}

__global__ void ladder_advance_kernel(LadderDev L) { *L.round += 1; }

// Algorithm 4: one thread per connection.
__global__ void ladder_connection_kernel(LadderDev L, int32_t it_arg) {
    const int32_t it = round_of(L, it_arg);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < L.C; c += stride) {
        const int32_t u = __ldg(L.cu + c);
        if (!ladder_active(L, u, it)) continue;
        const int32_t t = __ldg(L.cdep + c);
        if (__ldcg(L.e + u) > t) continue;
        ladder_relax(L, __ldg(L.cv + c), t + __ldg(L.cdur + c), it);
    }
}

// Algorithm 5: one thread per type, getConnection by linear search.
__global__ void ladder_type_kernel(LadderDev L, int32_t it_arg) {
    const int32_t it = round_of(L, it_arg);
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < L.T; t += stride) {
        const int4 r = __ldg(L.ty + t);
        if (!ladder_active(L, r.x, it)) continue;
        const int32_t eu = __ldcg(L.e + r.x);
        const int32_t end = __ldg(L.dep_ptr + t + 1);
        for (int32_t j = __ldg(L.dep_ptr + t); j < end; ++j) {
            const int32_t d = __ldg(L.dep + j);
            if (d >= eu) {
                ladder_relax(L, r.y, d + r.z, it);
                break;
            }
        }
    }
}

// Section II-C: one thread per type, getConnectionFromAPs (Algorithm 6) over the
// type's whole-day AP tuples.
__global__ void ladder_type_ap_kernel(LadderDev L, int32_t it_arg) {
    const int32_t it = round_of(L, it_arg);
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < L.T; t += stride) {
        const int4 r = __ldg(L.ty + t);
        if (!ladder_active(L, r.x, it)) continue;
        const int32_t eu = __ldcg(L.e + r.x);
        int32_t tc = kInf;
        const int32_t end = __ldg(L.ap_ptr + t + 1);
        for (int32_t a = __ldg(L.ap_ptr + t); a < end; ++a) {
            const int4 q = __ldg(L.ap + a);                 // {start, difference, terms, end}
            if (q.x < eu && eu <= q.w) {
                const int64_t i = ((int64_t)eu - q.x + q.y - 1) / q.y;
                tc = min(tc, (int32_t)(q.x + i * q.y));
            }
            if (eu <= q.x) tc = min(tc, q.x);
        }
        if (tc != kInf) ladder_relax(L, r.y, tc + r.z, it);
    }
}

// Cluster-AP lookup of type t at e[u] and its relaxation.
__device__ __forceinline__ void cluster_ap_relax(const LadderDev &L, const NetDev &N, int32_t t,
                                                 int32_t eu, int32_t k, int32_t it) {
    const int4 tr = __ldg(N.tr + t);                     // {v, lambda|d, row of v, last}
    if (eu > tr.w) return;                               // no departure left
    int4 a, b;
    load_entry(entry_at(N, k, t), a, b);
    int32_t n, x, aps = 0;
    entry_aps(b, n, x);
    const int32_t tc = cluster_lookup(a, b, n, x, cluster_base(N, k), eu, N.apx, aps);
    ladder_relax(L, tr.x, tc + (tr.y & 0xffffff), it);
}

// Section II-D: one thread per type, Cluster-AP lookup.
__global__ void ladder_cluster_ap_kernel(LadderDev L, NetDev N, int32_t it_arg) {
    const int32_t it = round_of(L, it_arg);
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < L.T; t += stride) {
        const int32_t u = __ldg(L.ty + t).x;
        if (!ladder_active(L, u, it)) continue;
        const int32_t eu = __ldcg(L.e + u);
        const int32_t k = cluster_slot(N, eu);
        if (k < N.y) cluster_ap_relax(L, N, t, eu, k, it);
    }
}

// Section II-E: one thread per edge, all its types by Cluster-AP.
__global__ void ladder_edge_kernel(LadderDev L, NetDev N, int32_t it_arg) {
    const int32_t it = round_of(L, it_arg);
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < L.E; e += stride) {
        const int32_t u = __ldg(L.edge_u + e);
        if (!ladder_active(L, u, it)) continue;
        const int32_t eu = __ldcg(L.e + u);
        const int32_t k = cluster_slot(N, eu);
        if (k >= N.y) continue;
        const int32_t end = __ldg(L.edge_ptr + e + 1);
        for (int32_t t = __ldg(L.edge_ptr + e); t < end; ++t) cluster_ap_relax(L, N, t, eu, k, it);
    }
}

// Section II-F: one warp per edge, the edge's types over the lanes.
__global__ void ladder_warp_kernel(LadderDev L, NetDev N, int32_t it_arg) {
    const int32_t it = round_of(L, it_arg);
    const int32_t lane = threadIdx.x & 31;
    const int32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (int32_t e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < L.E; e += nw) {
        const int32_t u = __ldg(L.edge_u + e);
        if (!ladder_active(L, u, it)) continue;             // the same for the whole warp
        const int32_t eu = __ldcg(L.e + u);
        const int32_t k = cluster_slot(N, eu);
        if (k >= N.y) continue;
        const int32_t end = __ldg(L.edge_ptr + e + 1);
        for (int32_t t = __ldg(L.edge_ptr + e) + lane; t < end; t += 32)
            cluster_ap_relax(L, N, t, eu, k, it);
    }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace eat

using namespace eat;

struct eat_ladder {
    eat_net *net = nullptr;                  // the Cluster-AP network (eat_build)
    int32_t device = -1;
    int32_t n_stops = 0;
    std::vector<int32_t> u, v, dep, dur;     // connections, as given
    std::vector<int32_t> type_uvl, dep_ptr, deps, ap_ptr, ap, edge_ptr, edge_u;
    void *blob = nullptr;
    int32_t *pinned = nullptr;               // host copy of `last`
    cudaStream_t stream = nullptr;
    LadderDev dev{};
    int sms = 0;
    struct Graph {
        int variant, rounds;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;               // instantiated round groups, by (variant, rounds)
    std::mutex lock;
};

namespace {

// Per-type departures (expanded from the type's cluster APs) and whole-day AP
// cover, for types [t0, t1).
void type_tables(const HostNet &h, int32_t t0, int32_t t1, std::vector<int32_t> &dep_cnt,
                 std::vector<int32_t> &deps, std::vector<int32_t> &ap_cnt, std::vector<int32_t> &ap) {
    std::vector<int32_t> d;
    std::vector<int32_t> cover;
    for (int32_t t = t0; t < t1; ++t) {
        d.clear();
        const int32_t first = h.type_rec[4 * (size_t)t + 2], last = h.type_rec[4 * (size_t)t + 3];
        const int32_t kf = (first - h.t0) / h.width, kl = (last - h.t0) / h.width;
        for (int32_t k = kf; k <= kl; ++k) {
            const int32_t c = h.type_cl[t] + k;
            for (int32_t a = h.cl[c]; a < h.cl[c + 1]; ++a) {
                const int32_t start = (int32_t)h.ap[2 * (size_t)a];
                const uint32_t sc = h.ap[2 * (size_t)a + 1];
                const int32_t step = (int32_t)(sc >> 16), terms = (int32_t)(sc & 0xffffu);
                for (int32_t m = 0; m < terms; ++m) d.push_back(start + m * step);
            }
        }
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
        dep_cnt.push_back((int32_t)d.size());
        deps.insert(deps.end(), d.begin(), d.end());
        cover.clear();
        if (!d.empty()) ap_cover_wide(d.data(), (int32_t)d.size(), cover);
        ap_cnt.push_back((int32_t)(cover.size() / 3));
        ap.insert(ap.end(), cover.begin(), cover.end());
    }
}

int ladder_upload(eat_ladder *l) {
    const int64_t C = (int64_t)l->u.size();
    const int32_t T = (int32_t)(l->type_uvl.size() / 3), E = (int32_t)l->edge_u.size();
    const int32_t V = l->n_stops;
    const int64_t A = (int64_t)l->ap.size() / 3;
    std::vector<int4> ty((size_t)T), apq((size_t)A);
    for (int32_t t = 0; t < T; ++t)
        ty[t] = make_int4(l->type_uvl[3 * (size_t)t], l->type_uvl[3 * (size_t)t + 1],
                          l->type_uvl[3 * (size_t)t + 2], 0);
    for (int64_t a = 0; a < A; ++a) {
        const int32_t f = l->ap[3 * a], d = l->ap[3 * a + 1], n = l->ap[3 * a + 2];
        apq[a] = make_int4(f, d, n, f + (n - 1) * d);
    }
    struct Piece { const void *src; size_t bytes; size_t off; };
    std::vector<Piece> p = {
        {l->u.data(), (size_t)C * 4, 0}, {l->v.data(), (size_t)C * 4, 0},
        {l->dep.data(), (size_t)C * 4, 0}, {l->dur.data(), (size_t)C * 4, 0},
        {ty.data(), (size_t)T * 16, 0}, {l->dep_ptr.data(), l->dep_ptr.size() * 4, 0},
        {l->deps.data(), l->deps.size() * 4, 0}, {l->ap_ptr.data(), l->ap_ptr.size() * 4, 0},
        {apq.data(), (size_t)A * 16, 0}, {l->edge_ptr.data(), l->edge_ptr.size() * 4, 0},
        {l->edge_u.data(), (size_t)E * 4, 0},
        {nullptr, (size_t)V * 4, 0}, {nullptr, (size_t)V * 8, 0}, {nullptr, 4, 0}, {nullptr, 4, 0}};
    size_t total = 0;
    for (Piece &q : p) {
        q.off = total;
        total += align256(std::max<size_t>(q.bytes, 4));
    }
    cudaError_t e = cudaMalloc(&l->blob, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        l->blob = nullptr;
        return fail(EAT_ERR_OOM, "cudaMalloc of the ladder arrays failed");
    }
    char *b = (char *)l->blob;
    for (const Piece &q : p)
        if (q.src && q.bytes) {
            e = cudaMemcpy(b + q.off, q.src, q.bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(EAT_ERR_CUDA, std::string("ladder upload: ") + cudaGetErrorString(e));
        }
    LadderDev &L = l->dev;
    L.cu = (const int32_t *)(b + p[0].off);
    L.cv = (const int32_t *)(b + p[1].off);
    L.cdep = (const int32_t *)(b + p[2].off);
    L.cdur = (const int32_t *)(b + p[3].off);
    L.ty = (const int4 *)(b + p[4].off);
    L.dep_ptr = (const int32_t *)(b + p[5].off);
    L.dep = (const int32_t *)(b + p[6].off);
    L.ap_ptr = (const int32_t *)(b + p[7].off);
    L.ap = (const int4 *)(b + p[8].off);
    L.edge_ptr = (const int32_t *)(b + p[9].off);
    L.edge_u = (const int32_t *)(b + p[10].off);
    L.e = (int32_t *)(b + p[11].off);
    L.stamp = (int32_t *)(b + p[12].off);
    L.last = (int32_t *)(b + p[13].off);
    L.round = (int32_t *)(b + p[14].off);
    L.V = V;
    L.T = T;
    L.E = E;
    L.C = C;
    e = cudaMallocHost(&l->pinned, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l->sms, cudaDevAttrMultiProcessorCount, l->device);
    if (e != cudaSuccess) return fail(EAT_ERR_CUDA, std::string("ladder setup: ") + cudaGetErrorString(e));
    return EAT_OK;
}

}  // namespace

// One round of `variant`; it < 0: the kernels read the round from the device.
static cudaError_t launch_round(eat_ladder *l, int32_t variant, int32_t it, int grid, int block,
                                cudaStream_t st) {
    const LadderDev &L = l->dev;
    const NetDev &N = l->net->dev;
    switch (variant) {
        case EAT_VAR_CONNECTION: ladder_connection_kernel<<<grid, block, 0, st>>>(L, it); break;
        case EAT_VAR_TYPE: ladder_type_kernel<<<grid, block, 0, st>>>(L, it); break;
        case EAT_VAR_TYPE_AP: ladder_type_ap_kernel<<<grid, block, 0, st>>>(L, it); break;
        case EAT_VAR_CLUSTER_AP: ladder_cluster_ap_kernel<<<grid, block, 0, st>>>(L, N, it); break;
        case EAT_VAR_EDGE: ladder_edge_kernel<<<grid, block, 0, st>>>(L, N, it); break;
        default: ladder_warp_kernel<<<grid, block, 0, st>>>(L, N, it); break;
    }
    return cudaGetLastError();
}

extern "C" {

int eat_ladder_build(const eat_connections *conn, const eat_build_opts *opts, eat_ladder **out) {
    if (!out) return fail(EAT_ERR_INVALID, "NULL out");
    *out = nullptr;
    if (opts && opts->subtrips != EAT_SUBTRIPS_NONE)
        return fail(EAT_ERR_INVALID, "the topology-driven variants take the timetable without sub-trips");
    eat_ladder *l = new (std::nothrow) eat_ladder;
    if (!l) return fail(EAT_ERR_OOM, "host allocation failed");
    int rc = eat_build(conn, opts, &l->net);
    if (rc) {
        delete l;
        return rc;
    }
    clear_error();
    const HostNet &h = l->net->host;
    l->device = l->net->device;
    l->n_stops = h.n_stops;
    const int64_t C = conn->n_conn;
    l->u.assign(conn->u, conn->u + C);
    l->v.assign(conn->v, conn->v + C);
    l->dep.assign(conn->dep, conn->dep + C);
    l->dur.assign(conn->dur, conn->dur + C);
    const int32_t T = h.n_types;
    l->type_uvl.resize(3 * (size_t)T);
    for (int32_t u = 0; u < h.n_stops; ++u)
        for (int32_t t = h.row_ptr[u]; t < h.row_ptr[u + 1]; ++t) {
            l->type_uvl[3 * (size_t)t] = u;
            l->type_uvl[3 * (size_t)t + 1] = h.type_rec[4 * (size_t)t];
            l->type_uvl[3 * (size_t)t + 2] = h.type_rec[4 * (size_t)t + 1];
            if (t == h.row_ptr[u] || h.type_rec[4 * (size_t)t] != h.type_rec[4 * (size_t)(t - 1)]) {
                l->edge_ptr.push_back(t);
                l->edge_u.push_back(u);
            }
        }
    l->edge_ptr.push_back(T);
    // Departures and whole-day covers, types split over the host threads.
    const int nth = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    struct Part { std::vector<int32_t> dc, d, ac, a; };
    std::vector<Part> parts((size_t)nth);
    std::vector<std::thread> th;
    for (int k = 0; k < nth; ++k)
        th.emplace_back([&, k] {
            const int32_t a = (int32_t)((int64_t)T * k / nth), b = (int32_t)((int64_t)T * (k + 1) / nth);
            type_tables(h, a, b, parts[k].dc, parts[k].d, parts[k].ac, parts[k].a);
        });
    for (std::thread &x : th) x.join();
    l->dep_ptr.assign(1, 0);
    l->ap_ptr.assign(1, 0);
    for (const Part &q : parts) {
        for (int32_t c : q.dc) l->dep_ptr.push_back(l->dep_ptr.back() + c);
        for (int32_t c : q.ac) l->ap_ptr.push_back(l->ap_ptr.back() + c);
        l->deps.insert(l->deps.end(), q.d.begin(), q.d.end());
        l->ap.insert(l->ap.end(), q.a.begin(), q.a.end());
    }
    if (l->device >= 0) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(l->device);
        rc = ladder_upload(l);
        if (prev >= 0) cudaSetDevice(prev);
        if (rc) {
            eat_ladder_free(l);
            return rc;
        }
    }
    *out = l;
    return EAT_OK;
}

void eat_ladder_free(eat_ladder *l) {
    if (!l) return;
    if (l->blob || l->stream || l->pinned) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(l->device);
        for (const eat_ladder::Graph &g : l->graphs) cudaGraphExecDestroy(g.exec);
        if (l->stream) cudaStreamDestroy(l->stream);
        if (l->pinned) cudaFreeHost(l->pinned);
        if (l->blob) cudaFree(l->blob);
        if (prev >= 0) cudaSetDevice(prev);
    }
    eat_free(l->net);
    delete l;
}

int eat_ladder_host_view(const eat_ladder *l, eat_ladder_view *view) {
    if (!l || !view) return fail(EAT_ERR_INVALID, "NULL argument");
    view->n_types = (int32_t)(l->type_uvl.size() / 3);
    view->n_edges = (int32_t)l->edge_u.size();
    view->n_dep = (int64_t)l->deps.size();
    view->n_ap = (int64_t)l->ap.size() / 3;
    view->type_uvl = l->type_uvl.data();
    view->dep_ptr = l->dep_ptr.data();
    view->dep = l->deps.data();
    view->ap_ptr = l->ap_ptr.data();
    view->ap = l->ap.data();
    view->edge_ptr = l->edge_ptr.data();
    return EAT_OK;
}

int eat_ladder_query(eat_ladder *l, int32_t variant, int32_t s, int32_t t_s, int32_t flag_every,
                     int32_t graph, int32_t *arr_out, eat_ladder_stats *stats) {
    clear_error();
    if (!l || !arr_out) return fail(EAT_ERR_INVALID, "NULL argument");
    if (l->device < 0) return fail(EAT_ERR_NO_DEVICE, "ladder was built host-only");
    if (variant < EAT_VAR_CONNECTION || variant > EAT_VAR_WARP)
        return fail(EAT_ERR_INVALID, "variant must be one of EAT_VAR_*");
    if (s < 0 || s >= l->n_stops) return fail(EAT_ERR_INVALID, "source out of range");
    if (flag_every < 1) return fail(EAT_ERR_INVALID, "flag_every must be >= 1");
    std::lock_guard<std::mutex> g(l->lock);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(l->device);
    cudaStream_t st = l->stream;
    const int block = 256, grid = l->sms * 8;
    const int32_t cap = l->n_stops + flag_every;
    int32_t it = 0, reads = 0;
    int rc = EAT_OK;
    cudaError_t e = cudaSuccess;
    cudaGraphExec_t exec = nullptr;
    if (graph) {
        for (const eat_ladder::Graph &gr : l->graphs)
            if (gr.variant == variant && gr.rounds == flag_every) exec = gr.exec;
        if (!exec) {   // capture flag_every (round, advance) pairs once per (variant, cadence)
            cudaGraph_t gph = nullptr;
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            for (int32_t r = 0; r < flag_every && e == cudaSuccess; ++r) {
                e = launch_round(l, variant, -1, grid, block, st);
                if (e == cudaSuccess) {
                    ladder_advance_kernel<<<1, 1, 0, st>>>(l->dev);
                    e = cudaGetLastError();
                }
            }
            const cudaError_t e2 = cudaStreamEndCapture(st, &gph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, gph, 0);
            if (gph) cudaGraphDestroy(gph);
            if (e == cudaSuccess) l->graphs.push_back({variant, flag_every, exec});
        }
    }
    if (e == cudaSuccess) {
        ladder_init_kernel<<<grid, block, 0, st>>>(l->dev, s, t_s);
        e = cudaGetLastError();
    }
    while (e == cudaSuccess) {
        if (graph) {
            e = cudaGraphLaunch(exec, st);
            it += flag_every;
        } else {
            e = launch_round(l, variant, it, grid, block, st);
            ++it;
            if (e != cudaSuccess || it % flag_every) {
                if (e == cudaSuccess && it > cap) rc = fail(EAT_ERR_NO_CONVERGENCE, "round cap reached");
                if (rc) break;
                continue;
            }
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(l->pinned, l->dev.last, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        ++reads;
        if (*l->pinned < it - 1) break;          // the last round lowered nothing
        if (it > cap) {
            rc = fail(EAT_ERR_NO_CONVERGENCE, "round cap reached");
            break;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(arr_out, l->dev.e, (size_t)l->n_stops * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EAT_ERR_CUDA, std::string("eat_ladder_query: ") + cudaGetErrorString(e));
    }
    if (stats) {
        stats->rounds = it;
        stats->flag_reads = reads;
    }
    return rc;
}

}  // extern "C"
