// sm_103a kernels for earliest-arrival-time queries (Cluster-AP fixpoint).
//
// Per query (Algorithms 2-5 with the Cluster-AP lookup of Section II-D):
//   init     e[] = INF, e[s] = t_s, frontier = {s}                 (Algorithm 2)
//   round    for every stop u of the frontier and every connection type
//            (u, v, lambda) leaving u: find the first departure t_c >= e[u]
//            (the APs of e[u]'s cluster, else the next non-empty cluster;
//            Algorithm 6), and if t_c + lambda < e[v] lower e[v] with atomicMin
//            and put v on the next frontier                        (Algorithm 3)
//   stop     when a round puts nobody on the next frontier.
// The frontier replaces the paper's active[]/nextactive[] flags (Section III-B):
// a stop joins the next frontier only after its e[] was lowered, through a
// test-and-set on a per-round bitmap, so each stop appears at most once per
// round; atomicMin resolves concurrent lowerings (Section III-C).
//
// CTA mode: one thread block owns one query at a time (persistent blocks take
// queries from an atomic counter), so rounds are separated by one block barrier
// and there is no grid-wide synchronisation and no spin-wait.  The round-free
// mode (eat_async_kernel) and the cluster mode (eat_cluster_kernel) are
// described at their kernels below.
//
// Work items: when a stop v joins the next frontier, the thread that lowered e[v]
// writes one (v, type) item per connection type leaving v into shared memory (one
// 32- or 64-bit store each), so the next round hands every thread one (stop, type)
// pair: the paper's one thread per connection type (Algorithm 5), restricted to the
// active tails.  Per item, the type's 16-byte record (head, duration, head row, last
// departure) and e[u] are loaded together, then the 32-byte cluster entry of e[u]'s
// cluster, then e[v] beside any further APs.  Stops whose items do not fit spill to a
// global queue and are expanded by `vwarp`-lane sub-warps (Section II-F's virtual
// warps).
//
// Horizon (qa.horizon > 0, an option; not in the paper): Algorithms 4-5 expand every
// improved stop in the next round, so a stop first reached late by a path of few
// connections is expanded, and its successors with it, again each time a later round
// improves it.  With a horizon H a stop lowered to an arrival >= H is not queued but
// waits (once, in a per-block list with a bitmap); when no stop below H is left to
// expand, waiting stops whose arrival has since dropped below H are dropped (they
// were queued by that lowering), H moves to the earliest remaining arrival + horizon,
// and the stops below the new H become the next round's spilled stops.  Every
// lowered stop is still expanded with its arrival at some round after the lowering,
// so the fixpoint is the same; only the order of relaxations changes (as
// delta-stepping orders Bellman-Ford's).
//
// Buffers per query: arrivals in shared memory (ARR = kArrShared), in global
// memory (kArrGlobal: the output row, or the block's scratch row when the output
// is host memory), or per query whichever the query's network allows
// (kArrPerQuery: shared when n_stops <= smem_arr_cap, for batches over networks
// of uneven size); two frontier bitmaps (this round's pushes, last round's) in
// shared memory when they fit (SMEM_MASK).  Arrivals not kept in the output row
// are copied there when the query converges.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "eat_device.cuh"
#include "eat_launch.h"

namespace eat {

enum { kArrGlobal = 0, kArrShared = 1, kArrPerQuery = 2 };

// Arrival load that sees the block's own atomics: shared memory through a
// volatile read, global memory from L2 (not a possibly stale L1 line).
__device__ __forceinline__ int32_t load_arr(const int32_t *arr, int32_t i, bool shared) {
    if (shared) return *((const volatile int32_t *)arr + i);
    return __ldcg(arr + i);
}

// A converged query's row from its arrivals (shared memory, or a global row) to `out`
// (device or page-locked host memory) by the block's threads: 16-byte loads and stores
// when both start on a 16-byte boundary (a quarter of the transactions, which matters
// most for rows written to host memory), else 4-byte ones.  The caller has passed a
// barrier since the last write to `arr`.
__device__ __forceinline__ void copy_row(int32_t *out, const int32_t *arr, int32_t V, bool shared,
                                         int tid, int nthr) {
    int32_t done = 0;
    if (((reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(arr)) & 15) == 0) {
        const int32_t n4 = V >> 2;
        int4 *const o4 = reinterpret_cast<int4 *>(out);
        const int4 *const a4 = reinterpret_cast<const int4 *>(arr);
        for (int32_t i = tid; i < n4; i += nthr) o4[i] = shared ? a4[i] : __ldcg(a4 + i);
        done = n4 << 2;
    }
    for (int32_t i = done + tid; i < V; i += nthr) out[i] = shared ? arr[i] : __ldcg(arr + i);
}

// Index of the next query a persistent block takes: the work counter's next value,
// through the start order when there is one (values >= n end the block's loop).
__device__ __forceinline__ int32_t next_query(const QueryArgs &qa) {
    const int32_t w = atomicAdd(qa.work, 1);
    return (qa.order && w < qa.n) ? __ldg(qa.order + w) : w;
}

// Ring mode: thread 0 of a block claims the next published request (a CAS on the
// device-side head below the host's tail, read with acquire semantics so that the
// entry written before it is visible), copies its fields to s_ring and returns its
// ring slot; it returns -1 when the host's stop flag is set and nothing is left, or
// after rg.idle_iters polls without a request (every wait bounded: polls 2 us apart
// for the first 512, then 20 us apart).
__device__ __forceinline__ int64_t ld_acquire_sys(const int64_t *p) {
    int64_t v;
    asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ int32_t ring_next(const RingArgs &R, int32_t *s_ring) {
    for (int32_t it = 0; it < R.idle_iters; ++it) {
        const int64_t tail = ld_acquire_sys(R.tail);
        unsigned long long h = *(volatile unsigned long long *)R.head;
        while ((int64_t)h < tail) {
            const unsigned long long was = atomicCAS(R.head, h, h + 1);
            if (was == h) {
                const int32_t slot = (int32_t)(h & (unsigned long long)R.mask);
                const volatile RingEntry *e = R.ring + slot;
                s_ring[0] = e->net;
                s_ring[1] = e->src;
                s_ring[2] = e->ts;
                s_ring[3] = e->row;
                return slot;
            }
            h = was;
        }
        if (*(const volatile int32_t *)R.stop) return -1;
        __nanosleep(it < 512 ? 2000 : 20000);       // back off after about 1 ms idle
    }
    return -1;
}

// Ring mode: publish request `slot` as finished (its row is already written by the
// block, ordered before this by the block barrier and the release).
__device__ __forceinline__ void ring_done(const RingArgs &R, int32_t slot, int32_t status) {
    RingEntry *e = R.ring + slot;
    *(volatile int32_t *)&e->status = status;
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(&e->done), "r"(1) : "memory");
}

constexpr int32_t kNullItem = -1;           // hole left by a stop that spilled
constexpr int32_t kFirstItem = INT32_MIN;    // flag on the first item of a stop

// Items are (stop, type) pairs in two int32 arrays per buffer, or, with PACK (networks
// of at most 32,767 stops and 65,535 types), one word per item: first-item flag << 31 |
// stop << 16 | type, which doubles the items a buffer holds in the same shared memory
// (kNullItem is then no valid item: it would be stop 32,767, type 65,535).
// COUNT: the build that fills qa.counters; without it the per-thread work counters are
// dead code and compiled away (the timed launches pass no counters).  HZ: the build that
// honours qa.horizon (the packed build also comes without, for launches with none).
template <int NETS, int ARR, bool SMEM_MASK, bool PACK = false, bool RING = false, bool COUNT = false,
          bool HZ = true>
__global__ void __launch_bounds__(1024, 1)
eat_cta_kernel(const __grid_constant__ NetTable<NETS> nets, const QueryArgs qa) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ int32_t s_q;
    __shared__ int32_t s_ring[4];     // ring mode: net, source, t_s, row of the request
    __shared__ int32_t s_items[3];    // items reserved per round (rotating)
    __shared__ int32_t s_spill[3];    // stops spilled per round (rotating)
    __shared__ unsigned long long s_cnt[6];
    __shared__ int32_t s_def[4];      // waiting stops: count, kept, released, least arrival

    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int vw = 1 << qa.vw_log2;
    const int lane = tid & (vw - 1);
    const int sub = tid >> qa.vw_log2;
    const int nsub = nthr >> qa.vw_log2;
    const int32_t icap = qa.qcap;

    // Item buffers (stop, type) and spill queues; round r writes buffer r & 1.
    int32_t *const item_base = smem + qa.smem_q_off;
    int32_t *const spill_base = qa.spill + (int64_t)blockIdx.x * qa.spill_stride;
    uint32_t *const mask_base = SMEM_MASK ? (uint32_t *)(smem + qa.smem_mask_off)
                                          : qa.gmask + (int64_t)blockIdx.x * qa.mask_stride;
    // Stops waiting beyond the horizon: two lists of vmax stops and their bitmap.
    int32_t *const def_base = spill_base + 2 * (int64_t)qa.vmax;
    uint32_t *const dmask = (uint32_t *)(spill_base + 4 * (int64_t)qa.vmax);

    for (;;) {
        if (tid == 0) s_q = RING ? ring_next(qa.rg, s_ring) : next_query(qa);
        if (tid < 6) s_cnt[tid] = 0;
        __syncthreads();
        const int q = s_q;
        if (RING ? q < 0 : q >= qa.n) break;

        const int ni = RING ? s_ring[0] : qa.net_idx == nullptr ? 0 : __ldg(qa.net_idx + q);
        const bool net_ok = (unsigned)ni < (unsigned)qa.n_nets;
        const NetDev &N = nets.net[net_ok ? ni : 0];
        const int32_t V = N.n_stops;
        const int64_t off = RING         ? (int64_t)s_ring[3] * qa.rg.row_stride
                            : qa.arr_off ? __ldg(qa.arr_off + q)
                                         : (int64_t)q * V;
        int32_t *const out = qa.arr_out + off;
        const bool arr_shared = ARR == kArrShared || (ARR == kArrPerQuery && V <= qa.smem_arr_cap);
        // Arrivals: shared memory, else the block's scratch row (when the output is
        // host memory), else the output row itself.
        int32_t *const arr = arr_shared ? smem
                             : qa.arr_rows ? qa.arr_rows + (int64_t)blockIdx.x * qa.arr_rows_stride
                                           : out;
        const int32_t nwords = (V + 31) >> 5;
        uint32_t *const mask0 = mask_base;
        uint32_t *const mask1 = mask_base + qa.mask_words;

        // Algorithm 2: every stop passive at infinity.
        for (int32_t i = tid; i < V; i += nthr) arr[i] = kInf;
        for (int32_t i = tid; i < nwords; i += nthr) {
            mask0[i] = 0u;
            mask1[i] = 0u;
        }
        const bool hz_on = HZ && qa.horizon > 0;
        if (hz_on)
            for (int32_t i = tid; i < nwords; i += nthr) dmask[i] = 0u;
        if (tid < 3) {
            s_items[tid] = 0;
            s_spill[tid] = 0;
        }
        if (tid == 0) s_def[0] = 0;
        const int32_t s = RING ? s_ring[1] : __ldg(qa.src + q);
        const int32_t t_s = RING ? s_ring[2] : __ldg(qa.ts + q);
        const bool valid = net_ok && (unsigned)s < (unsigned)V;
        __syncthreads();
        // The source is the frontier of "round -1": spill queue of buffer 1, counter slot 2.
        if (tid == 0 && valid) {
            arr[s] = t_s;
            spill_base[qa.vmax] = s;
            s_spill[2] = 1;
        }
        __syncthreads();

        int32_t n_items = 0, n_spill = valid ? 1 : 0;
        int32_t rounds = 0;
        // Horizon H (kInf when there is none): a stop lowered to an arrival at or after
        // H waits until no stop below H is left to expand.
        int32_t H = hz_on && t_s < kInf - qa.horizon ? t_s + qa.horizon : kInf;
        int dl = 0;                                       // list that new waiting stops join
        int cs = 0;                                       // counter slot written this round
        int32_t c_vert = 0, c_types = 0, c_evals = 0, c_lookups = 0, c_aps = 0, c_relax = 0;
        while (n_items + n_spill > 0 && rounds < qa.max_rounds) {
            const int wr = rounds & 1, rd = wr ^ 1;
            // One-word items (PACK) or two-word items {stop | first flag, type}.
            int32_t *const iu_rd = item_base + (PACK ? rd : 2 * rd) * icap;
            int32_t *const iu_wr = item_base + (PACK ? wr : 2 * wr) * icap;
            const int2 *const i2_rd = reinterpret_cast<const int2 *>(iu_rd);
            int2 *const i2_wr = reinterpret_cast<int2 *>(iu_wr);
            const int32_t *const sp_rd = spill_base + (int64_t)rd * qa.vmax;
            int32_t *const sp_wr = spill_base + (int64_t)wr * qa.vmax;
            uint32_t *const pmask = wr ? mask1 : mask0;    // stops pushed this round
            uint32_t *const cmask = wr ? mask0 : mask1;    // stops pushed last round
            // The slot used next round was last read two barriers ago.
            if (tid == 0) {
                const int nx = cs == 2 ? 0 : cs + 1;
                s_items[nx] = 0;
                s_spill[nx] = 0;
            }

            // Relaxation (Algorithm 3 with getConnection, Algorithm 6) in two steps.
            // lookup: t_c + lambda of one type of tail u from its cluster entry and type
            // record, for e[u] at or before the type's last departure (so that some
            // departure is at or after e[u]).  lower: when that candidate is below the
            // e[v] read beside the lookup, e[v] is lowered with an atomic min whose result
            // is not waited for and v goes on the next frontier as items or as a spilled
            // stop: every lowering is made by a thread whose candidate was below its read,
            // so every lowering pushes v (at most once a round: the bitmap); a push whose
            // min lost to a lower one made meanwhile only repeats work.  In EAT_MODE_EDGE
            // a stop with at least vwarp types is queued whole for a vwarp-lane sub-warp
            // (the mapping chosen by degree).
            auto lookup = [&](int32_t e_u, int32_t k, const int4 ca, const int4 cb,
                              const int4 tr) -> int32_t {  // tr = {v, lambda|d, row of v, last}
                ++c_lookups;
                ++c_evals;
                int32_t n, x;
                entry_aps(cb, n, x);
                return cluster_lookup(ca, cb, n, x, cluster_base(N, k), e_u, N.apx, c_aps) +
                       (tr.y & 0xffffff);
            };
            auto lower = [&](const int4 tr, int32_t cand, int32_t ev) {
                if (cand >= ev) return;
                const int32_t v = tr.x;
                atomicMin(arr + v, cand);
                ++c_relax;
                int32_t d = (int32_t)((uint32_t)tr.y >> 24);  // types leaving v
                if (d == kCountOverflow) d = __ldg(N.row_ptr + v + 1) - tr.z;
                if (d <= 0) return;
                const uint32_t bit = 1u << (v & 31);
                if (HZ && cand >= H) {                      // beyond the horizon: wait
                    if (!(atomicOr(dmask + (v >> 5), bit) & bit))
                        def_base[(int64_t)dl * qa.vmax + atomicAdd(&s_def[0], 1)] = v;
                    return;
                }
                if (atomicOr(pmask + (v >> 5), bit) & bit) return;   // already queued
                if (qa.edge && d >= vw) {                   // a sub-warp expands v whole
                    sp_wr[atomicAdd(&s_spill[cs], 1)] = v;
                    return;
                }
                const int32_t base = atomicAdd(&s_items[cs], d);
                if (base + d > icap) {
                    for (int32_t j = base; j < icap; ++j) {
                        if (PACK) iu_wr[j] = kNullItem;
                        else i2_wr[j].x = kNullItem;
                    }
                    sp_wr[atomicAdd(&s_spill[cs], 1)] = v;
                    return;
                }
                if (PACK) {
                    const int32_t hv = (v << 16) | tr.z;
                    iu_wr[base] = hv | kFirstItem;
                    for (int32_t j = 1; j < d; ++j) iu_wr[base + j] = hv + j;
                } else {
                    i2_wr[base] = make_int2(v | kFirstItem, tr.z);
                    for (int32_t j = 1; j < d; ++j) i2_wr[base + j] = make_int2(v, tr.z + j);
                }
            };
            // Item i: its stop u and type t (clearing u's bit in last round's bitmap at
            // u's first item); loads the type record and e[u], then the cluster entry of
            // e[u]'s cluster.  Returns whether the type has a departure at or after e[u]
            // (else it stops here, Section III-D).
            auto load_item = [&](int32_t i, int32_t &e_u, int32_t &k, int4 &ca, int4 &cb,
                                 int4 &tr) -> bool {
                int32_t u, t;
                if (PACK) {
                    const int32_t raw = iu_rd[i];
                    if (raw == kNullItem) return false;
                    u = (raw >> 16) & 0x7fff;
                    t = raw & 0xffff;
                    if (raw < 0) {
                        atomicAnd(cmask + (u >> 5), ~(1u << (u & 31)));
                        ++c_vert;
                    }
                } else {
                    const int2 it = i2_rd[i];
                    if (it.x == kNullItem) return false;
                    u = it.x & 0x7fffffff;
                    t = it.y;
                    if (it.x < 0) {
                        atomicAnd(cmask + (u >> 5), ~(1u << (u & 31)));
                        ++c_vert;
                    }
                }
                ++c_types;
                tr = __ldg(N.tr + t);
                e_u = load_arr(arr, u, arr_shared);
                k = cluster_slot(N, e_u);
                if (k < N.y) load_entry(entry_at(N, k, t), ca, cb);
                return e_u <= tr.w;
            };

            if (!qa.edge) {
                // One thread per (stop, type) item.
                for (int32_t i = tid; i < n_items; i += nthr) {
                    int32_t e_u, k;
                    int4 ca = make_int4(0, 0, 0, 0), cb = ca, tr;
                    if (!load_item(i, e_u, k, ca, cb, tr)) continue;
                    const int32_t ev = load_arr(arr, tr.x, arr_shared);
                    lower(tr, lookup(e_u, k, ca, cb, tr), ev);
                }
            } else {
                // EAT_MODE_EDGE: a warp's lanes take consecutive items and every lane runs
                // every pass (lanes past the end carry none); lanes whose types share a head
                // stop v (the types of one edge, or of edges into one stop) reduce their
                // candidates with a warp min, and one lane per head stop lowers e[v].
                for (int32_t ib = tid & ~31; ib < n_items; ib += nthr) {
                    const int32_t i = ib + (tid & 31);
                    int32_t e_u = 0, k = 0, ev = kInf, cand = kInf;
                    int4 ca = make_int4(0, 0, 0, 0), cb = ca, tr = ca;
                    bool live = i < n_items && load_item(i, e_u, k, ca, cb, tr);
                    if (live) {
                        ev = load_arr(arr, tr.x, arr_shared);
                        cand = lookup(e_u, k, ca, cb, tr);
                    }
                    const unsigned grp = __match_any_sync(0xffffffffu, live ? tr.x : -1 - (tid & 31));
                    const int32_t m = __reduce_min_sync(grp, cand);
                    const unsigned first = __ballot_sync(0xffffffffu, cand == m) & grp;
                    if (live && (tid & 31) == __ffs(first) - 1) lower(tr, cand, ev);
                }
            }
            // Spilled stops: `vw` lanes per stop stride over its types.
            for (int32_t i = sub; i < n_spill; i += nsub) {
                const int32_t u = __ldcg(sp_rd + i);
                const int32_t beg = __ldg(N.row_ptr + u);
                const int32_t end = __ldg(N.row_ptr + u + 1);
                if (lane == 0) {
                    atomicAnd(cmask + (u >> 5), ~(1u << (u & 31)));
                    ++c_vert;
                }
                const int32_t e_u = load_arr(arr, u, arr_shared);
                const int32_t k = cluster_slot(N, e_u);
                if (k >= N.y) {                             // no departure left anywhere
                    if (lane == 0) c_types += end - beg;
                    continue;
                }
                for (int32_t t = beg + lane; t < end; t += vw) {
                    ++c_types;
                    int4 ca, cb;
                    load_entry(entry_at(N, k, t), ca, cb);
                    const int4 tr = __ldg(N.tr + t);
                    if (e_u > tr.w) continue;
                    const int32_t ev = load_arr(arr, tr.x, arr_shared);
                    lower(tr, lookup(e_u, k, ca, cb, tr), ev);
                }
            }
            __syncthreads();
            n_items = min(s_items[cs], icap);
            n_spill = s_spill[cs];
            cs = cs == 2 ? 0 : cs + 1;
            ++rounds;
            if (hz_on && n_items + n_spill == 0) {
                // No stop below H is left: waiting stops since lowered below H were queued
                // by that lowering and drop out; H moves to the earliest remaining arrival
                // + horizon and the stops below it become next round's spilled stops, the
                // others wait on (in the other list).  (Releasing while a few stops below
                // H are still queued moves H every round and loses the horizon.)  The
                // waiting count is read before a barrier that no change to it precedes.
                const int32_t nd = s_def[0];
                if (tid == 0) {
                    s_def[1] = 0;
                    s_def[2] = 0;
                    s_def[3] = kInf;
                }
                __syncthreads();
                if (nd > 0) {
                    const int32_t *const L = def_base + (int64_t)dl * qa.vmax;
                    int32_t *const K = def_base + (int64_t)(dl ^ 1) * qa.vmax;
                    int32_t *const sp_next = spill_base + (int64_t)((rounds & 1) ^ 1) * qa.vmax;
                    int32_t m = kInf;
                    for (int32_t i = tid; i < nd; i += nthr) {
                        const int32_t e = load_arr(arr, __ldcg(L + i), arr_shared);
                        if (e >= H) m = min(m, e);
                    }
                    m = __reduce_min_sync(0xffffffffu, m);
                    if ((tid & 31) == 0 && m < kInf) atomicMin(&s_def[3], m);
                    __syncthreads();
                    const int32_t lo = s_def[3];
                    const int32_t Hn = lo < kInf - qa.horizon ? lo + qa.horizon : kInf;
                    for (int32_t i = tid; i < nd; i += nthr) {
                        const int32_t v = __ldcg(L + i);
                        const int32_t e = load_arr(arr, v, arr_shared);
                        if (e < H) continue;
                        if (e < Hn) sp_next[atomicAdd(&s_def[2], 1)] = v;
                        else K[atomicAdd(&s_def[1], 1)] = v;
                    }
                    __syncthreads();
                    n_spill = s_def[2];
                    H = Hn;
                    dl ^= 1;
                    if (tid == 0) s_def[0] = s_def[1];   // no thread reads [0] or [1] before this
                    __syncthreads();
                }
            }
        }
        const int32_t F = n_items + n_spill;

        if (arr_shared || qa.arr_rows) {
            __syncthreads();
            copy_row(out, arr, V, arr_shared, tid, nthr);
        }
        const int32_t q_status = !valid ? EAT_ERR_INVALID : (F > 0 ? EAT_ERR_NO_CONVERGENCE : EAT_OK);
        if (RING) {
            __syncthreads();                              // the whole row is written
            if (tid == 0) ring_done(qa.rg, q, q_status);
        } else if (tid == 0 && qa.status) {
            qa.status[q] = q_status;
        }
        if (COUNT && !RING && qa.counters) {
            unsigned long long c[6] = {(unsigned long long)c_vert, (unsigned long long)c_types,
                                       (unsigned long long)c_evals, (unsigned long long)c_lookups,
                                       (unsigned long long)c_aps, (unsigned long long)c_relax};
#pragma unroll
            for (int j = 0; j < 6; ++j)
                for (int o = 16; o > 0; o >>= 1) c[j] += __shfl_down_sync(0xffffffffu, c[j], o);
            if ((tid & 31) == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) atomicAdd(&s_cnt[j], c[j]);
            }
            __syncthreads();
            if (tid == 0) {
                eat_counters r;
                r.rounds = rounds;
                r.vertices = (int64_t)s_cnt[0];
                r.types = (int64_t)s_cnt[1];
                r.evals = (int64_t)s_cnt[2];
                r.lookups = (int64_t)s_cnt[3];
                r.aps = (int64_t)s_cnt[4];
                r.relaxed = (int64_t)s_cnt[5];
                qa.counters[q] = r;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ paired mode
//
// Two queries on one small network share a 1,024-thread block and its rounds: both
// arrival rows and their bitmaps sit in shared memory, and every round hands the
// items of both queries to all threads.  When one query converges its threads go
// to the other (and the slot takes the next query), so a block is not left with
// half its threads idle behind its deeper query; batches larger than the SM count
// fill every SM with one block.  Items are packed as in eat_cta_kernel.  Slot 0's
// items fill a buffer from the front, slot 1's from the back; one 32-bit counter
// per round reserves both (slot 0 in the low half, slot 1 in the high half: a slot
// reserves at most one item per connection type in a round, and there are at most
// 65,535 types), so a reservation fits if the two totals before it plus its own
// items stay within the buffer.  Once one does not, none after it does: the
// counter state before that first failure (saved by the failing thread) gives each
// slot's valid items.
constexpr int kSlots = 2;

// Per-thread work counters of both slots (COUNT builds only): vertices, types,
// evaluations, lookups, AP records, relaxations.
struct PairCounters {
    int32_t c[kSlots][6];
    __device__ __forceinline__ void add(int j, int k, int32_t x) {
        if (j) c[1][k] += x;
        else c[0][k] += x;
    }
};

template <bool COUNT>
__global__ void __launch_bounds__(1024, 1)
eat_pair_kernel(const __grid_constant__ NetTable<1> nets, const QueryArgs qa) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ uint32_t s_res[3];               // items reserved per round (rotating)
    __shared__ uint32_t s_cross[3];             // reservations before the first that failed
    __shared__ int32_t s_spill[3][kSlots];      // stops spilled per round and slot
    __shared__ int32_t s_q[kSlots];
    __shared__ unsigned long long s_cnt[kSlots][6];

    const NetDev &N = nets.net[0];
    const int32_t V = N.n_stops;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int vw = 1 << qa.vw_log2;
    const int lane = tid & (vw - 1);
    const int sub = tid >> qa.vw_log2;
    const int nsub = nthr >> qa.vw_log2;
    const int32_t icap = qa.qcap;               // items per buffer, both slots together
    const int32_t vpad = qa.smem_arr_cap;       // ints per arrival row
    const int32_t nwords = (V + 31) >> 5;
    PairCounters pc;
#pragma unroll
    for (int j = 0; j < kSlots; ++j)
#pragma unroll
        for (int k = 0; k < 6; ++k) pc.c[j][k] = 0;
    int32_t *const items = smem + qa.smem_q_off;
    uint32_t *const masks = (uint32_t *)(smem + qa.smem_mask_off);   // [slot][buffer][words]
    int32_t *const spill_base = qa.spill + (int64_t)blockIdx.x * qa.spill_stride;  // [slot][buffer][vmax]

    if (tid < 3) {
        s_res[tid] = 0u;
        s_spill[tid][0] = 0;
        s_spill[tid][1] = 0;
    }
    // Per slot (uniform over the block): query, rounds, items and spilled stops
    // queued for the coming round, and whether the slot must take a new query.
    int32_t qs[kSlots], rr[kSlots], ni[kSlots], ns[kSlots];
    bool vq[kSlots], need[kSlots], fresh[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        qs[j] = -1;
        rr[j] = ni[j] = ns[j] = 0;
        vq[j] = false;
        need[j] = true;
        fresh[j] = true;       // the first query of slot j is j * grid + block
    }
    int32_t R = 0;             // block round: round R writes buffer R & 1
    int cs = 0;                // counter slot written this round

    for (;;) {
        if (need[0] || need[1]) {
            if (COUNT) {   // block totals of the finishing slots' counters
#pragma unroll
                for (int j = 0; j < kSlots; ++j) {
                    if (!need[j] || qs[j] < 0) continue;
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        unsigned long long x = (unsigned long long)pc.c[j][k];
                        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                        if ((tid & 31) == 0) atomicAdd(&s_cnt[j][k], x);
                        pc.c[j][k] = 0;
                    }
                }
                __syncthreads();
            }
            // Finish converged (or capped) queries: result row, status, counters.
#pragma unroll
            for (int j = 0; j < kSlots; ++j) {
                if (!need[j] || qs[j] < 0) continue;
                const int32_t q = qs[j];
                const int64_t off = qa.arr_off ? __ldg(qa.arr_off + q) : (int64_t)q * V;
                int32_t *const out = qa.arr_out + off;
                const int32_t *const a = smem + j * vpad;
                copy_row(out, a, V, true, tid, nthr);
                if (tid == 0) {
                    if (qa.status)
                        qa.status[q] = !vq[j] ? EAT_ERR_INVALID
                                       : (ni[j] + ns[j] > 0 ? EAT_ERR_NO_CONVERGENCE : EAT_OK);
                    if (COUNT) {
                        eat_counters r;
                        r.rounds = rr[j];
                        r.vertices = (int64_t)s_cnt[j][0];
                        r.types = (int64_t)s_cnt[j][1];
                        r.evals = (int64_t)s_cnt[j][2];
                        r.lookups = (int64_t)s_cnt[j][3];
                        r.aps = (int64_t)s_cnt[j][4];
                        r.relaxed = (int64_t)s_cnt[j][5];
                        qa.counters[q] = r;
                    }
                }
            }
            if (tid == 0) {
#pragma unroll
                for (int j = 0; j < kSlots; ++j) {
                    if (!need[j]) continue;
                    const int32_t w = fresh[j] ? j * (int32_t)gridDim.x + (int32_t)blockIdx.x
                                               : kSlots * (int32_t)gridDim.x + atomicAdd(qa.work, 1);
                    s_q[j] = w >= qa.n ? -1 : qa.order ? __ldg(qa.order + w) : w;
                }
            }
            __syncthreads();   // result rows read; new queries visible
            const int rd = (R & 1) ^ 1;                    // buffer the coming round reads
#pragma unroll
            for (int j = 0; j < kSlots; ++j) {
                if (!need[j]) continue;
                need[j] = false;
                fresh[j] = false;
                qs[j] = s_q[j];
                rr[j] = ni[j] = ns[j] = 0;
                vq[j] = false;
                if (qs[j] < 0) continue;                   // no query left for this slot
                // Algorithm 2 for the slot's new query; its source is the one
                // spilled stop of the coming round.
                const int32_t s = __ldg(qa.src + qs[j]);
                const int32_t t_s = __ldg(qa.ts + qs[j]);
                const int32_t ni_q = qa.net_idx ? __ldg(qa.net_idx + qs[j]) : 0;
                vq[j] = ni_q == 0 && (unsigned)s < (unsigned)V;
                int32_t *const a = smem + j * vpad;
                for (int32_t i = tid; i < V; i += nthr) a[i] = (vq[j] && i == s) ? t_s : kInf;
                uint32_t *const m = masks + j * 2 * qa.mask_words;
                for (int32_t i = tid; i < nwords; i += nthr) {
                    m[i] = 0u;
                    m[qa.mask_words + i] = 0u;
                }
                if (COUNT && tid < 6) s_cnt[j][tid] = 0ull;
                if (vq[j]) {
                    if (tid == 0) spill_base[(int64_t)(j * 2 + rd) * qa.vmax] = s;
                    ns[j] = 1;
                }
            }
            if (qs[0] < 0 && qs[1] < 0) break;
            __syncthreads();   // slots initialised before the round reads them
        }

        const int wr = R & 1, rd = wr ^ 1;
        int32_t *const it_rd = items + rd * icap;
        int32_t *const it_wr = items + wr * icap;
        if (tid == 0) {
            const int nx = cs == 2 ? 0 : cs + 1;
            s_res[nx] = 0u;
            s_spill[nx][0] = 0;
            s_spill[nx][1] = 0;
        }

        // Relax type t of tail u for slot j (Algorithm 3 with Algorithm 6).
        // Relax type t of tail u for slot j (Algorithm 3 with Algorithm 6): entry and type
        // record loaded together, e[v] read beside the further APs, as in eat_cta_kernel.
        auto relax = [&](int j, int32_t e_u, int32_t k, int32_t t) {
            int4 ca = make_int4(0, 0, 0, 0), cb = ca;
            if (k < N.y) load_entry(entry_at(N, k, t), ca, cb);
            const int4 tr = __ldg(N.tr + t);             // {v, lambda|d, row of v, last}
            if (COUNT) pc.add(j, 1, 1);
            if (e_u > tr.w) return;                      // no departure left (Section III-D)
            int32_t *const a = smem + j * vpad;
            const int32_t v = tr.x;
            const int32_t ev = load_arr(a, v, true);
            int32_t n, x, aps = 0;
            entry_aps(cb, n, x);
            const int32_t tc = cluster_lookup(ca, cb, n, x, cluster_base(N, k), e_u, N.apx, aps);
            if (COUNT) {
                pc.add(j, 2, 1);
                pc.add(j, 3, 1);
                pc.add(j, 4, aps);
            }
            const int32_t cand = tc + (tr.y & 0xffffff);
            if (cand >= ev) return;
            atomicMin(a + v, cand);                        // result not waited for, as above
            if (COUNT) pc.add(j, 5, 1);
            int32_t d = (int32_t)((uint32_t)tr.y >> 24);
            if (d == kCountOverflow) d = __ldg(N.row_ptr + v + 1) - tr.z;
            if (d <= 0) return;
            uint32_t *const pmask = masks + (j * 2 + wr) * qa.mask_words;
            const uint32_t bit = 1u << (v & 31);
            if (atomicOr(pmask + (v >> 5), bit) & bit) return;
            const uint32_t before = atomicAdd(&s_res[cs], (uint32_t)d << (j ? 16 : 0));
            const uint32_t lo = before & 0xffffu, hi = before >> 16;
            if (lo + hi + (uint32_t)d <= (uint32_t)icap) {
                const int32_t pos = j ? icap - (int32_t)hi - d : (int32_t)lo;
                const int32_t hv = (v << 16) | tr.z;
                it_wr[pos] = hv | kFirstItem;
                for (int32_t jj = 1; jj < d; ++jj) it_wr[pos + jj] = hv + jj;
            } else {
                if (lo + hi <= (uint32_t)icap) s_cross[cs] = before;   // the first that failed
                spill_base[(int64_t)(j * 2 + wr) * qa.vmax + atomicAdd(&s_spill[cs][j], 1)] = v;
            }
        };

        // One thread per (stop, type) item; slot 1's items sit at the buffer's end.
        const int32_t n0 = ni[0], nall = ni[0] + ni[1];
        const int32_t gap = icap - nall;
        for (int32_t i = tid; i < nall; i += nthr) {
            const int j = i >= n0;
            const int32_t raw = it_rd[j ? i + gap : i];
            const int32_t u = (raw >> 16) & 0x7fff;
            if (raw < 0) {
                atomicAnd(masks + (j * 2 + rd) * qa.mask_words + (u >> 5), ~(1u << (u & 31)));
                if (COUNT) pc.add(j, 0, 1);
            }
            const int32_t e_u = load_arr(smem + j * vpad, u, true);
            relax(j, e_u, cluster_slot(N, e_u), raw & 0xffff);
        }
        // Spilled stops of both slots: `vw` lanes per stop.
        const int32_t s0 = ns[0], sall = ns[0] + ns[1];
        for (int32_t i = sub; i < sall; i += nsub) {
            const int j = i >= s0;
            const int32_t u = __ldcg(spill_base + (int64_t)(j * 2 + rd) * qa.vmax + (j ? i - s0 : i));
            const int32_t beg = __ldg(N.row_ptr + u);
            const int32_t end = __ldg(N.row_ptr + u + 1);
            if (lane == 0) {
                atomicAnd(masks + (j * 2 + rd) * qa.mask_words + (u >> 5), ~(1u << (u & 31)));
                if (COUNT) pc.add(j, 0, 1);
            }
            const int32_t e_u = load_arr(smem + j * vpad, u, true);
            const int32_t k = cluster_slot(N, e_u);
            if (k >= N.y) {
                if (COUNT && lane == 0) pc.add(j, 1, end - beg);
                continue;
            }
            for (int32_t t = beg + lane; t < end; t += vw) relax(j, e_u, k, t);
        }
        __syncthreads();
        const uint32_t res = s_res[cs];
        const bool over = (res & 0xffffu) + (res >> 16) > (uint32_t)icap;
        const uint32_t okr = over ? s_cross[cs] : res;
        const int32_t nn[kSlots] = {(int32_t)(okr & 0xffffu), (int32_t)(okr >> 16)};
#pragma unroll
        for (int j = 0; j < kSlots; ++j) {
            if (qs[j] < 0) continue;
            rr[j] += ni[j] + ns[j] > 0;                    // a round with work for the slot
            ni[j] = nn[j];
            ns[j] = s_spill[cs][j];
            need[j] = ni[j] + ns[j] == 0 || rr[j] >= qa.max_rounds;
        }
        cs = cs == 2 ? 0 : cs + 1;
        ++R;
    }
}

// ------------------------------------------------------------------ asynchronous mode
//
// The same fixpoint without rounds.  The frontier is a bitmap of pending stops in
// shared memory.  Each warp works on its own: it reads 32 bitmap words (one per
// lane), every lane claims one pending stop (clears its bit, then reads e[u]), the
// warp spreads the claimed stops' (stop, type) pairs over its lanes and relaxes
// them; a lowered e[v] sets v's bit after the atomicMin, so a stop improved after
// it was read is claimed again (the invariant of Section III-B's double buffer,
// without the round barrier).  A work counter holds pending + claimed stops:
// a producer adds one before publishing a bit, a claimed stop is subtracted only
// after all its pushes, so the counter reaches zero exactly when no work is left.
// Every idle wait is capped (qa.idle_cap scans of 32 bitmap words in a row by one warp
// that find nothing while work is still counted, checked after each full pass); hitting
// the cap ends the query with EAT_ERR_NO_CONVERGENCE and the arrivals reached so far
// (upper bounds).

template <int NETS, int ARR>
__global__ void __launch_bounds__(1024, 1)
eat_async_kernel(const __grid_constant__ NetTable<NETS> nets, const QueryArgs qa) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ int32_t s_q;
    __shared__ int32_t s_work;
    __shared__ int32_t s_err;
    __shared__ unsigned long long s_cnt[6];

    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    uint32_t *const mask = (uint32_t *)(smem + qa.smem_mask_off);
    // Per-warp staging of claimed stops: row begin, exclusive item prefix, e[u], cluster.
    int32_t *const stage = smem + qa.smem_q_off + warp * (4 * 32);
    int32_t *const st_beg = stage, *const st_pre = stage + 32, *const st_e = stage + 64,
                   *const st_k = stage + 96;

    for (;;) {
        if (tid == 0) s_q = next_query(qa);
        if (tid < 6) s_cnt[tid] = 0;
        __syncthreads();
        const int q = s_q;
        if (q >= qa.n) break;

        const int ni = qa.net_idx == nullptr ? 0 : __ldg(qa.net_idx + q);
        const bool net_ok = (unsigned)ni < (unsigned)qa.n_nets;
        const NetDev &N = nets.net[net_ok ? ni : 0];
        const int32_t V = N.n_stops;
        const int64_t off = qa.arr_off ? __ldg(qa.arr_off + q) : (int64_t)q * V;
        int32_t *const out = qa.arr_out + off;
        const bool arr_shared = ARR == kArrShared || (ARR == kArrPerQuery && V <= qa.smem_arr_cap);
        // Arrivals: shared memory, else the block's scratch row (when the output is
        // host memory), else the output row itself.
        int32_t *const arr = arr_shared ? smem
                             : qa.arr_rows ? qa.arr_rows + (int64_t)blockIdx.x * qa.arr_rows_stride
                                           : out;
        const int32_t nwords = (V + 31) >> 5;
        const int32_t nchunks = (nwords + 31) >> 5;

        for (int32_t i = tid; i < V; i += nthr) arr[i] = kInf;
        for (int32_t i = tid; i < nwords; i += nthr) mask[i] = 0u;
        if (tid == 0) {
            s_work = 0;
            s_err = 0;
        }
        const int32_t s = __ldg(qa.src + q);
        const int32_t t_s = __ldg(qa.ts + q);
        const bool valid = net_ok && (unsigned)s < (unsigned)V;
        __syncthreads();
        if (tid == 0 && valid) {
            arr[s] = t_s;
            mask[s >> 5] = 1u << (s & 31);
            s_work = 1;
        }
        __syncthreads();

        int32_t c_vert = 0, c_types = 0, c_evals = 0, c_lookups = 0, c_aps = 0, c_relax = 0;
        int32_t chunk = nchunks > 0 ? warp % nchunks : 0;
        int32_t idle = 0, passes = 0;             // passes: empty chunk scans in a row
        bool go = valid;
        while (go) {
            // Claim up to one pending stop per lane from this chunk's 32 words.
            const int32_t word = chunk * 32 + lane;
            int32_t u = -1;
            if (word < nwords) {
                const uint32_t w = *((volatile uint32_t *)mask + word);
                if (w) {
                    const uint32_t bit = w & (0u - w);
                    if (atomicAnd(mask + word, ~bit) & bit) u = word * 32 + (__ffs(w) - 1);
                }
            }
            const uint32_t claimed = __ballot_sync(0xffffffffu, u >= 0);
            if (claimed == 0) {
                chunk = chunk + 1 == nchunks ? 0 : chunk + 1;
                ++passes;
                if (++idle >= nchunks) {          // a full pass found nothing
                    idle = 0;
                    int32_t stop = 0;
                    if (lane == 0) {
                        const int32_t wk = *((volatile int32_t *)&s_work);
                        const int32_t er = *((volatile int32_t *)&s_err);
                        stop = (wk == 0 || er) ? 1 : (passes >= qa.idle_cap ? 2 : 0);
                        if (stop == 2) atomicExch(&s_err, 1);
                    }
                    stop = __shfl_sync(0xffffffffu, stop, 0);
                    if (stop) break;
                    __nanosleep(200);
                }
                continue;
            }
            idle = 0;
            passes = 0;
            // Expand the claimed stops: read e[u] after the claim (fence), then the row.
            __threadfence_block();
            int32_t d = 0, beg = 0, e_u = 0, k = 0;
            if (u >= 0) {
                ++c_vert;
                e_u = load_arr(arr, u, arr_shared);
                k = cluster_slot(N, e_u);
                beg = __ldg(N.row_ptr + u);
                const int32_t end = __ldg(N.row_ptr + u + 1);
                if (k < N.y) d = end - beg;
                else c_types += end - beg;
            }
            int32_t incl = d;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
            st_beg[lane] = beg;
            st_pre[lane] = incl - d;
            st_e[lane] = e_u;
            st_k[lane] = k;
            __syncwarp();
            for (int32_t j = lane; j < total; j += 32) {
                // owner: the last lane whose exclusive prefix is <= j (lanes without
                // items share the next lane's prefix and sit before it)
                int32_t lo = 0, hi = 31;
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (st_pre[mid] <= j) lo = mid; else hi = mid - 1;
                }
                const int32_t t = st_beg[lo] + (j - st_pre[lo]);
                const int32_t eu = st_e[lo], kk = st_k[lo];
                ++c_types;
                int4 ca, cb;
                load_entry(entry_at(N, kk, t), ca, cb);
                const int4 tr = __ldg(N.tr + t);             // {v, lambda|d, row of v, last}
                if (eu > tr.w) continue;                     // no departure left
                ++c_lookups;
                ++c_evals;
                const int32_t v = tr.x;
                const int32_t ev = load_arr(arr, v, arr_shared);
                int32_t n, x;
                entry_aps(cb, n, x);
                const int32_t tc = cluster_lookup(ca, cb, n, x, cluster_base(N, kk), eu, N.apx, c_aps);
                const int32_t cand = tc + (tr.y & 0xffffff);
                if (cand >= ev) continue;
                const int32_t old = atomicMin(arr + v, cand);
                if (cand >= old) continue;
                ++c_relax;
                if (((uint32_t)tr.y >> 24) == 0) continue;  // v has no outgoing types
                const uint32_t bit = 1u << (v & 31);
                atomicAdd(&s_work, 1);                      // count before publishing
                __threadfence_block();
                if (atomicOr(mask + (v >> 5), bit) & bit) atomicAdd(&s_work, -1);
            }
            __syncwarp();
            // The claimed stops are done once all their pushes are published.
            __threadfence_block();
            if (lane == 0) atomicAdd(&s_work, -__popc(claimed));
        }
        __syncthreads();

        if (arr_shared || qa.arr_rows) copy_row(out, arr, V, arr_shared, tid, nthr);
        if (tid == 0 && qa.status)
            qa.status[q] = !valid ? EAT_ERR_INVALID : (s_err ? EAT_ERR_NO_CONVERGENCE : EAT_OK);
        if (qa.counters) {
            unsigned long long c[6] = {(unsigned long long)c_vert, (unsigned long long)c_types,
                                       (unsigned long long)c_evals, (unsigned long long)c_lookups,
                                       (unsigned long long)c_aps, (unsigned long long)c_relax};
#pragma unroll
            for (int j = 0; j < 6; ++j)
                for (int o = 16; o > 0; o >>= 1) c[j] += __shfl_down_sync(0xffffffffu, c[j], o);
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) atomicAdd(&s_cnt[j], c[j]);
            }
            __syncthreads();
            if (tid == 0) {
                eat_counters r;
                r.rounds = 0;                       // no rounds in this mode
                r.vertices = (int64_t)s_cnt[0];
                r.types = (int64_t)s_cnt[1];
                r.evals = (int64_t)s_cnt[2];
                r.lookups = (int64_t)s_cnt[3];
                r.aps = (int64_t)s_cnt[4];
                r.relaxed = (int64_t)s_cnt[5];
                qa.counters[q] = r;
            }
        }
        __syncthreads();
    }
}

// Start order of a batch: a counting sort of the query indices by t_s in 15-minute
// buckets (earliest first) in one block.  Queries started together then look up the
// same clusters of the network, and the longest (earliest) start first.
constexpr int kOrderBuckets = 4096;          // 15-minute buckets: 42 days
constexpr int kOrderThreads = 1024;

__device__ __forceinline__ int order_bucket(int32_t t) {
    return t <= 0 ? 0 : min(t / 900, kOrderBuckets - 1);
}

__global__ void __launch_bounds__(kOrderThreads)
eat_order_kernel(const int32_t *__restrict__ ts, int32_t n, int32_t *__restrict__ order) {
    __shared__ int32_t hist[kOrderBuckets];
    __shared__ int32_t wsum[kOrderThreads / 32];
    constexpr int kPer = kOrderBuckets / kOrderThreads;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b < kOrderBuckets; b += kOrderThreads) hist[b] = 0;
    __syncthreads();
    for (int32_t i = tid; i < n; i += kOrderThreads) atomicAdd(&hist[order_bucket(__ldg(ts + i))], 1);
    __syncthreads();
    // Exclusive prefix sum: thread tid owns buckets [kPer * tid, kPer * tid + kPer).
    int32_t loc[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        loc[k] = hist[kPer * tid + k];
        sum += loc[k];
    }
    int32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int32_t base = x - sum + (warp ? wsum[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        hist[kPer * tid + k] = base;
        base += loc[k];
    }
    __syncthreads();
    for (int32_t i = tid; i < n; i += kOrderThreads)
        order[atomicAdd(&hist[order_bucket(__ldg(ts + i))], 1)] = i;
}

__global__ void eat_next_departure_kernel(const NetDev N, const int32_t *types,
                                          const int32_t *times, int32_t n, int32_t *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = types[i];
    int32_t aps = 0;
    out[i] = ((unsigned)t < (unsigned)N.n_types) ? next_departure(N, t, times[i], aps) : kInf;
}

// ------------------------------------------------------------------ launchers

// ------------------------------------------------------------------ cluster mode
//
// One thread-block cluster of C blocks per query (grid = n * C; no persistent
// loop), for single queries and small batches that would leave most SMs idle.
// The arrivals and both frontier bitmaps are spread over the cluster's shared
// memory: stop v lives in block v mod C at slot v / C, and every block reads and
// lowers other blocks' entries through distributed shared memory.  Each block
// keeps its own (stop, type) item queues and pushes into them.  A round ends at a
// cluster barrier; after it every block sums all blocks' push counters, so all
// blocks take the same loop decisions and pass the same barriers.

template <int NETS>
__global__ void __launch_bounds__(1024, 1)
eat_cluster_kernel(const __grid_constant__ NetTable<NETS> nets, const QueryArgs qa) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ int32_t s_items[3];    // items this block reserved per round (rotating)
    __shared__ int32_t s_spill[3];    // stops this block spilled per round (rotating)
    __shared__ unsigned long long s_cnt[6];

    const int C = (int)cluster.num_blocks();
    const int me = (int)cluster.block_rank();
    const int qi = blockIdx.x / C;                    // the same for the whole cluster
    const int q = (qa.order && qi < qa.n) ? __ldg(qa.order + qi) : qi;
    if (q >= qa.n) return;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int vw = 1 << qa.vw_log2;
    const int lane = tid & (vw - 1);
    const int sub = tid >> qa.vw_log2;
    const int nsub = nthr >> qa.vw_log2;
    const int32_t icap = qa.qcap;

    int32_t *const item_base = smem + qa.smem_q_off;
    int32_t *const spill_base = qa.spill + (int64_t)blockIdx.x * qa.spill_stride;
    uint32_t *const mask0 = (uint32_t *)(smem + qa.smem_mask_off);
    uint32_t *const mask1 = mask0 + qa.mask_words;
    int32_t *const arr = smem;                        // this block's slots

    const NetDev &N = nets.net[0];
    const int32_t V = N.n_stops;
    const int32_t mine = me < V ? (V - me + C - 1) / C : 0;   // stops me, me + C, ...
    const int32_t mwords = (mine + 31) >> 5;
    int32_t *const out = qa.arr_out + (qa.arr_off ? __ldg(qa.arr_off + q) : (int64_t)q * V);
    // Arrival slot and bitmap word of stop v, in the block that holds it.
    auto arr_of = [&](int32_t v) { return cluster.map_shared_rank(arr + v / C, v % C); };
    auto word_of = [&](uint32_t *m, int32_t v) {
        return cluster.map_shared_rank(m + ((v / C) >> 5), v % C);
    };
    auto bit_of = [&](int32_t v) { return 1u << ((v / C) & 31); };

    // Algorithm 2 on this block's slots.
    if (tid < 6) s_cnt[tid] = 0;
    for (int32_t i = tid; i < mine; i += nthr) arr[i] = kInf;
    for (int32_t i = tid; i < mwords; i += nthr) {
        mask0[i] = 0u;
        mask1[i] = 0u;
    }
    if (tid < 3) {
        s_items[tid] = 0;
        s_spill[tid] = 0;
    }
    const int32_t s = __ldg(qa.src + q);
    const int32_t t_s = __ldg(qa.ts + q);
    const bool valid = (qa.net_idx == nullptr || __ldg(qa.net_idx + q) == 0) && (unsigned)s < (unsigned)V;
    __syncthreads();
    // The source is the frontier of "round -1" in the block that holds it.
    if (tid == 0 && valid && s % C == me) {
        arr[s / C] = t_s;
        spill_base[qa.vmax] = s;
        s_spill[2] = 1;
    }
    cluster.sync();

    int32_t n_items = 0, n_spill = s_spill[2];
    int32_t total = 0;
    for (int r = 0; r < C; ++r) total += *(volatile int32_t *)cluster.map_shared_rank(&s_spill[2], r);
    int32_t rounds = 0;
    int cs = 0;
    int32_t c_vert = 0, c_types = 0, c_evals = 0, c_lookups = 0, c_aps = 0, c_relax = 0;
    while (total > 0 && rounds < qa.max_rounds) {
        const int wr = rounds & 1, rd = wr ^ 1;
        int32_t *const iu_rd = item_base + (2 * rd) * icap;
        int32_t *const it_rd = iu_rd + icap;
        int32_t *const iu_wr = item_base + (2 * wr) * icap;
        int32_t *const it_wr = iu_wr + icap;
        const int32_t *const sp_rd = spill_base + (int64_t)rd * qa.vmax;
        int32_t *const sp_wr = spill_base + (int64_t)wr * qa.vmax;
        uint32_t *const pmask = wr ? mask1 : mask0;    // stops pushed this round
        uint32_t *const cmask = wr ? mask0 : mask1;    // stops pushed last round
        if (tid == 0) {
            const int nx = cs == 2 ? 0 : cs + 1;
            s_items[nx] = 0;
            s_spill[nx] = 0;
        }

        // Relax type t of tail u (Algorithm 3 with getConnection, Algorithm 6); on
        // success v joins this block's next frontier as items or as a spilled stop.
        auto relax = [&](int32_t e_u, int32_t k, int32_t t) {
            ++c_types;
            int4 ca, cb;
            load_entry(entry_at(N, k, t), ca, cb);
            const int4 tr = __ldg(N.tr + t);             // {v, lambda|d, row of v, last}
            if (e_u > tr.w) return;                      // no departure left (Section III-D)
            ++c_lookups;
            ++c_evals;
            int32_t n, x;
            entry_aps(cb, n, x);
            const int32_t tc = cluster_lookup(ca, cb, n, x, cluster_base(N, k), e_u, N.apx, c_aps);
            const int32_t v = tr.x;
            const int32_t cand = tc + (tr.y & 0xffffff);
            int32_t *const ev = arr_of(v);
            if (cand >= *(volatile int32_t *)ev) return;
            const int32_t old = atomicMin(ev, cand);
            if (cand >= old) return;
            ++c_relax;
            const int32_t row = tr.z;
            int32_t d = (int32_t)((uint32_t)tr.y >> 24);  // types leaving v
            if (d == kCountOverflow) d = __ldg(N.row_ptr + v + 1) - row;
            if (d <= 0) return;
            const uint32_t bit = bit_of(v);
            if (atomicOr(word_of(pmask, v), bit) & bit) return;   // already queued
            const int32_t base = atomicAdd(&s_items[cs], d);
            if (base + d <= icap) {
                iu_wr[base] = v | kFirstItem;
                it_wr[base] = row;
                for (int32_t j = 1; j < d; ++j) {
                    iu_wr[base + j] = v;
                    it_wr[base + j] = row + j;
                }
            } else {
                for (int32_t j = base; j < icap; ++j) iu_wr[j] = kNullItem;
                sp_wr[atomicAdd(&s_spill[cs], 1)] = v;
            }
        };

        for (int32_t i = tid; i < n_items; i += nthr) {
            const int32_t raw = iu_rd[i];
            if (raw == kNullItem) continue;
            const int32_t u = raw & 0x7fffffff;
            if (raw < 0) {                              // first item of u
                atomicAnd(word_of(cmask, u), ~bit_of(u));
                ++c_vert;
            }
            const int32_t e_u = *(volatile int32_t *)arr_of(u);
            const int32_t k = cluster_slot(N, e_u);
            if (k >= N.y) {
                ++c_types;
                continue;
            }
            relax(e_u, k, it_rd[i]);
        }
        for (int32_t i = sub; i < n_spill; i += nsub) {
            const int32_t u = __ldcg(sp_rd + i);
            const int32_t beg = __ldg(N.row_ptr + u);
            const int32_t end = __ldg(N.row_ptr + u + 1);
            if (lane == 0) {
                atomicAnd(word_of(cmask, u), ~bit_of(u));
                ++c_vert;
            }
            const int32_t e_u = *(volatile int32_t *)arr_of(u);
            const int32_t k = cluster_slot(N, e_u);
            if (k >= N.y) {
                if (lane == 0) c_types += end - beg;
                continue;
            }
            for (int32_t t = beg + lane; t < end; t += vw) relax(e_u, k, t);
        }
        cluster.sync();
        n_items = min(s_items[cs], icap);
        n_spill = s_spill[cs];
        total = 0;
        for (int r = 0; r < C; ++r) {
            total += min(*(volatile int32_t *)cluster.map_shared_rank(&s_items[cs], r), icap);
            total += *(volatile int32_t *)cluster.map_shared_rank(&s_spill[cs], r);
        }
        cs = cs == 2 ? 0 : cs + 1;
        ++rounds;
    }

    if (qa.counters) {
        unsigned long long c[6] = {(unsigned long long)c_vert, (unsigned long long)c_types,
                                   (unsigned long long)c_evals, (unsigned long long)c_lookups,
                                   (unsigned long long)c_aps, (unsigned long long)c_relax};
#pragma unroll
        for (int j = 0; j < 6; ++j)
            for (int o = 16; o > 0; o >>= 1) c[j] += __shfl_down_sync(0xffffffffu, c[j], o);
        if ((tid & 31) == 0) {
#pragma unroll
            for (int j = 0; j < 6; ++j) atomicAdd(&s_cnt[j], c[j]);
        }
    }
    cluster.sync();                                   // every block's slots and counters final
    // Block b writes the contiguous part [V b / C, V (b + 1) / C) of the row.
    const int32_t lo = (int32_t)((int64_t)V * me / C), hi = (int32_t)((int64_t)V * (me + 1) / C);
    for (int32_t i = lo + tid; i < hi; i += nthr) out[i] = *arr_of(i);
    if (me == 0 && tid == 0) {
        if (qa.status)
            qa.status[q] = !valid ? EAT_ERR_INVALID : (total > 0 ? EAT_ERR_NO_CONVERGENCE : EAT_OK);
        if (qa.counters) {
            eat_counters r{};
            r.rounds = rounds;
            for (int b = 0; b < C; ++b) {
                const unsigned long long *sc = cluster.map_shared_rank(s_cnt, b);
                r.vertices += (int64_t)sc[0];
                r.types += (int64_t)sc[1];
                r.evals += (int64_t)sc[2];
                r.lookups += (int64_t)sc[3];
                r.aps += (int64_t)sc[4];
                r.relaxed += (int64_t)sc[5];
            }
            qa.counters[q] = r;
        }
    }
    cluster.sync();                                   // block 0 is done reading the others
}

template <int NETS, bool COUNT>
static const void *cta_kernel_ptr(int mem) {
    switch (mem) {
    case 0: return (const void *)eat_cta_kernel<NETS, kArrShared, true, false, false, COUNT>;
    case 1: return (const void *)eat_cta_kernel<NETS, kArrGlobal, true, false, false, COUNT>;
    case 3: return (const void *)eat_cta_kernel<NETS, kArrPerQuery, true, false, false, COUNT>;
    default: return (const void *)eat_cta_kernel<NETS, kArrGlobal, false, false, false, COUNT>;
    }
}

const void *cta_kernel(int nets, int mem, bool pack, bool count, bool hz) {
    if (pack) {
        if (hz)
            return count ? (const void *)eat_cta_kernel<1, kArrShared, true, true, false, true, true>
                         : (const void *)eat_cta_kernel<1, kArrShared, true, true, false, false, true>;
        return count ? (const void *)eat_cta_kernel<1, kArrShared, true, true, false, true, false>
                     : (const void *)eat_cta_kernel<1, kArrShared, true, true, false, false, false>;
    }
    if (count) return nets == 1 ? cta_kernel_ptr<1, true>(mem) : cta_kernel_ptr<EAT_MAX_NETS, true>(mem);
    return nets == 1 ? cta_kernel_ptr<1, false>(mem) : cta_kernel_ptr<EAT_MAX_NETS, false>(mem);
}

template <int NETS>
static const void *async_kernel_ptr(int mem) {
    switch (mem) {
    case 0: return (const void *)eat_async_kernel<NETS, kArrShared>;
    case 3: return (const void *)eat_async_kernel<NETS, kArrPerQuery>;
    default: return (const void *)eat_async_kernel<NETS, kArrGlobal>;
    }
}

const void *async_kernel(int nets, int mem) {
    return nets == 1 ? async_kernel_ptr<1>(mem) : async_kernel_ptr<EAT_MAX_NETS>(mem);
}

template <int NETS>
static cudaError_t launch_async_t(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem,
                                  int grid, int block, size_t smem, cudaStream_t st) {
    NetTable<NETS> tab;
    for (int i = 0; i < n_nets && i < NETS; ++i) tab.net[i] = nets[i];
    for (int i = n_nets; i < NETS; ++i) tab.net[i] = NetDev{};
    switch (mem) {
    case 0: eat_async_kernel<NETS, kArrShared><<<grid, block, smem, st>>>(tab, qa); break;
    case 3: eat_async_kernel<NETS, kArrPerQuery><<<grid, block, smem, st>>>(tab, qa); break;
    default: eat_async_kernel<NETS, kArrGlobal><<<grid, block, smem, st>>>(tab, qa); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_async(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                         int block, size_t smem, cudaStream_t st) {
    if (n_nets == 1) return launch_async_t<1>(nets, n_nets, qa, mem, grid, block, smem, st);
    return launch_async_t<EAT_MAX_NETS>(nets, n_nets, qa, mem, grid, block, smem, st);
}

template <int NETS, bool COUNT>
static cudaError_t launch_cta_t(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem,
                                int grid, int block, size_t smem, cudaStream_t st) {
    NetTable<NETS> tab;
    for (int i = 0; i < n_nets && i < NETS; ++i) tab.net[i] = nets[i];
    for (int i = n_nets; i < NETS; ++i) tab.net[i] = NetDev{};
    switch (mem) {
    case 0: eat_cta_kernel<NETS, kArrShared, true, false, false, COUNT><<<grid, block, smem, st>>>(tab, qa); break;
    case 1: eat_cta_kernel<NETS, kArrGlobal, true, false, false, COUNT><<<grid, block, smem, st>>>(tab, qa); break;
    case 3: eat_cta_kernel<NETS, kArrPerQuery, true, false, false, COUNT><<<grid, block, smem, st>>>(tab, qa); break;
    default: eat_cta_kernel<NETS, kArrGlobal, false, false, false, COUNT><<<grid, block, smem, st>>>(tab, qa); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_cta(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                       int block, size_t smem, cudaStream_t st, bool pack) {
    const bool count = qa.counters != nullptr;
    if (pack) {
        NetTable<1> tab;
        tab.net[0] = nets[0];
        const bool hz = qa.horizon > 0;
        if (count && hz) eat_cta_kernel<1, kArrShared, true, true, false, true, true><<<grid, block, smem, st>>>(tab, qa);
        else if (count) eat_cta_kernel<1, kArrShared, true, true, false, true, false><<<grid, block, smem, st>>>(tab, qa);
        else if (hz) eat_cta_kernel<1, kArrShared, true, true, false, false, true><<<grid, block, smem, st>>>(tab, qa);
        else eat_cta_kernel<1, kArrShared, true, true, false, false, false><<<grid, block, smem, st>>>(tab, qa);
        return cudaGetLastError();
    }
    if (n_nets == 1)
        return count ? launch_cta_t<1, true>(nets, n_nets, qa, mem, grid, block, smem, st)
                     : launch_cta_t<1, false>(nets, n_nets, qa, mem, grid, block, smem, st);
    return count ? launch_cta_t<EAT_MAX_NETS, true>(nets, n_nets, qa, mem, grid, block, smem, st)
                 : launch_cta_t<EAT_MAX_NETS, false>(nets, n_nets, qa, mem, grid, block, smem, st);
}

const void *ring_kernel(int mem) {
    switch (mem) {
    case 0: return (const void *)eat_cta_kernel<EAT_MAX_NETS, kArrShared, true, false, true>;
    case 3: return (const void *)eat_cta_kernel<EAT_MAX_NETS, kArrPerQuery, true, false, true>;
    default: return (const void *)eat_cta_kernel<EAT_MAX_NETS, kArrGlobal, true, false, true>;
    }
}

cudaError_t launch_ring(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                        int block, size_t smem, cudaStream_t st) {
    NetTable<EAT_MAX_NETS> tab;
    for (int i = 0; i < n_nets && i < EAT_MAX_NETS; ++i) tab.net[i] = nets[i];
    for (int i = n_nets; i < EAT_MAX_NETS; ++i) tab.net[i] = NetDev{};
    switch (mem) {
    case 0: eat_cta_kernel<EAT_MAX_NETS, kArrShared, true, false, true><<<grid, block, smem, st>>>(tab, qa); break;
    case 3: eat_cta_kernel<EAT_MAX_NETS, kArrPerQuery, true, false, true><<<grid, block, smem, st>>>(tab, qa); break;
    default: eat_cta_kernel<EAT_MAX_NETS, kArrGlobal, true, false, true><<<grid, block, smem, st>>>(tab, qa); break;
    }
    return cudaGetLastError();
}

const void *pair_kernel(bool count) {
    return count ? (const void *)eat_pair_kernel<true> : (const void *)eat_pair_kernel<false>;
}

cudaError_t launch_pair(const NetDev &net, const QueryArgs &qa, int grid, int block, size_t smem,
                        cudaStream_t st) {
    NetTable<1> tab;
    tab.net[0] = net;
    if (qa.counters) eat_pair_kernel<true><<<grid, block, smem, st>>>(tab, qa);
    else eat_pair_kernel<false><<<grid, block, smem, st>>>(tab, qa);
    return cudaGetLastError();
}

const void *cluster_kernel() { return (const void *)eat_cluster_kernel<1>; }

cudaError_t launch_cluster(const NetDev &net, const QueryArgs &qa, int cluster, int grid,
                           int block, size_t smem, cudaStream_t st) {
    NetTable<1> tab;
    tab.net[0] = net;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, eat_cluster_kernel<1>, tab, qa);
}

cudaError_t launch_order(const int32_t *ts, int32_t n, int32_t *order, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    eat_order_kernel<<<1, kOrderThreads, 0, st>>>(ts, n, order);
    return cudaGetLastError();
}

cudaError_t launch_next_departure(const NetDev &N, const int32_t *types, const int32_t *times,
                                  int32_t n, int32_t *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    const int grid = (n + block - 1) / block;
    eat_next_departure_kernel<<<grid, block, 0, st>>>(N, types, times, n, out);
    return cudaGetLastError();
}

}  // namespace eat
