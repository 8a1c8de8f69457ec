// sm_103a kernels for earliest-arrival-time queries (Cluster-AP fixpoint).
//
// Per query (Algorithms 2-5 with the Cluster-AP lookup of Section III-D):
//   init     e[] = INF, e[s] = t_s, frontier = {s}                 (Algorithm 2)
//   round    for every stop u of the frontier and every connection type
//            (u, v, lambda) leaving u: find the first departure t_c >= e[u]
//            (clusters + APs, Algorithm 6), and if t_c + lambda < e[v] lower
//            e[v] with atomicMin and put v on the next frontier     (Algorithm 3)
//   stop     when a round puts nobody on the next frontier.
// The frontier replaces the paper's active[]/nextactive[] flags (Section IV-B):
// a stop joins the next frontier only after its e[] was lowered, through a
// test-and-set on a per-query bitmap, so each stop appears at most once per
// round; atomicMin resolves concurrent lowerings (Section IV-C).
//
// CTA mode: one thread block owns one query at a time (persistent blocks take
// queries from an atomic counter).  Rounds are separated by block barriers, so
// there is no grid-wide synchronisation and no spin-wait anywhere.  The arrival
// row lives in shared memory when it fits (SMEM_ARR), otherwise in the output
// row in global memory; the bitmap lives in shared memory when it fits.
#include <cuda_runtime.h>

#include "eat_launch.h"

namespace eat {

constexpr int kInf = INT32_MAX;


// Least departure >= e of a type whose first departure is < e and last is >= e:
// scan the APs of e's cluster (Algorithm 6, restricted to one cluster as in
// Section III-D); if that cluster has no departure >= e, the first AP of the
// next non-empty cluster starts with the answer.
__device__ __forceinline__ int32_t cluster_ap_lookup(const NetDev &N, int32_t cl_base, int32_t e,
                                                     int32_t &aps) {
    const int32_t k = (e - N.t0) / N.width;
    const int32_t lo = __ldg(N.cl + cl_base + k);
    const int32_t hi = __ldg(N.cl + cl_base + k + 1);
    int32_t tc = kInf;
    for (int32_t a = lo; a < hi; ++a) {
        const uint2 r = __ldg(N.ap + a);
        ++aps;
        const int32_t start = (int32_t)r.x;
        if (start >= tc) break;              // APs are ordered by first term
        if (e <= start) { tc = start; break; }
        const int32_t step = (int32_t)(r.y >> 16);
        const int32_t last = start + ((int32_t)(r.y & 0xffffu) - 1) * step;
        if (e <= last) {                      // start < e <= last: step >= 1
            const int32_t i = (e - start + step - 1) / step;
            tc = min(tc, start + i * step);
        }
    }
    if (tc == kInf) {
        tc = (int32_t)__ldg(N.ap + hi).x;
        ++aps;
    }
    return tc;
}

// getConnection for type t at time e: least departure >= e, or kInf.
__device__ __forceinline__ int32_t next_departure(const NetDev &N, int32_t t, int32_t e,
                                                  int32_t &aps) {
    const int4 ty = __ldg(N.ty + t);
    if (e > ty.w) return kInf;
    if (e <= ty.z) return ty.z;
    return cluster_ap_lookup(N, __ldg(N.cl_base + t), e, aps);
}

template <bool SMEM_ARR>
__device__ __forceinline__ int32_t load_arr(const int32_t *arr, int32_t i) {
    if (SMEM_ARR) return *((const volatile int32_t *)arr + i);
    return __ldcg(arr + i);
}

template <int NETS, bool SMEM_ARR, bool SMEM_MASK>
__global__ void __launch_bounds__(1024, 1)
eat_cta_kernel(const __grid_constant__ NetTable<NETS> nets, const QueryArgs qa) {
    extern __shared__ __align__(16) int32_t smem[];
    __shared__ int32_t s_q;
    __shared__ int32_t s_tail[2];
    __shared__ unsigned long long s_cnt[6];

    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int vw = 1 << qa.vw_log2;
    const int lane = tid & (vw - 1);
    const int sub = tid >> qa.vw_log2;
    const int nsub = nthr >> qa.vw_log2;
    int32_t *const q_base = qa.queues + (int64_t)blockIdx.x * qa.queue_stride;

    for (;;) {
        if (tid == 0) s_q = atomicAdd(qa.work, 1);
        if (tid < 6) s_cnt[tid] = 0;
        __syncthreads();
        const int q = s_q;
        if (q >= qa.n) break;

        const int ni = (NETS == 1 || qa.net_idx == nullptr) ? 0 : __ldg(qa.net_idx + q);
        const bool net_ok = (unsigned)ni < (unsigned)qa.n_nets;
        const NetDev &N = nets.net[net_ok ? ni : 0];
        const int32_t V = N.n_stops;
        const int64_t off = qa.arr_off ? __ldg(qa.arr_off + q) : (int64_t)q * V;
        int32_t *const out = qa.arr_out + off;
        int32_t *const arr = SMEM_ARR ? smem : out;
        const int32_t vpad = (V + 3) & ~3;
        uint32_t *const mask = SMEM_MASK ? (uint32_t *)(SMEM_ARR ? smem + vpad : smem)
                                         : qa.gmask + (int64_t)blockIdx.x * qa.mask_stride;
        const int32_t nwords = (V + 31) >> 5;
        int32_t *qa_ = q_base;
        int32_t *qb_ = q_base + V;

        // Algorithm 2: every stop passive at infinity.
        for (int32_t i = tid; i < V; i += nthr) arr[i] = kInf;
        for (int32_t i = tid; i < nwords; i += nthr) mask[i] = 0u;
        if (tid == 0) { s_tail[0] = 0; s_tail[1] = 0; }
        const int32_t s = __ldg(qa.src + q);
        const int32_t t_s = __ldg(qa.ts + q);
        const bool valid = net_ok && (unsigned)s < (unsigned)V;
        __syncthreads();
        if (tid == 0 && valid) {
            arr[s] = t_s;
            qa_[0] = s;
        }
        __syncthreads();

        int32_t F = valid ? 1 : 0;
        int32_t rounds = 0;
        int p = 0;
        int32_t c_vert = 0, c_types = 0, c_evals = 0, c_lookups = 0, c_aps = 0, c_relax = 0;
        while (F > 0 && rounds < qa.max_rounds) {
            // The stops of this frontier may join the next one again.
            for (int32_t i = tid; i < F; i += nthr) {
                const int32_t u = __ldcg(qa_ + i);
                atomicAnd(mask + (u >> 5), ~(1u << (u & 31)));
            }
            __syncthreads();
            for (int32_t i = sub; i < F; i += nsub) {
                const int32_t u = __ldcg(qa_ + i);
                const int32_t e_u = load_arr<SMEM_ARR>(arr, u);
                const int32_t beg = __ldg(N.row_ptr + u);
                const int32_t end = __ldg(N.row_ptr + u + 1);
                c_vert += (lane == 0);
                for (int32_t t = beg + lane; t < end; t += vw) {
                    ++c_types;
                    const int4 ty = __ldg(N.ty + t);   // {v, lambda, first, last}
                    if (e_u > ty.w) continue;           // no departure left (Section IV-D)
                    const int32_t v = ty.x, lam = ty.y;
                    ++c_evals;
                    const int32_t e_v = load_arr<SMEM_ARR>(arr, v);
                    if (max(e_u, ty.z) + lam >= e_v) continue;   // cannot improve e[v]
                    int32_t tc = ty.z;
                    if (e_u > ty.z) {
                        ++c_lookups;
                        tc = cluster_ap_lookup(N, __ldg(N.cl_base + t), e_u, c_aps);
                    }
                    const int32_t cand = tc + lam;
                    if (cand < e_v) {
                        const int32_t old = atomicMin(arr + v, cand);
                        if (cand < old) {
                            ++c_relax;
                            const uint32_t bit = 1u << (v & 31);
                            if (!(atomicOr(mask + (v >> 5), bit) & bit)) {
                                const int32_t pos = atomicAdd(&s_tail[p], 1);
                                qb_[pos] = v;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            F = s_tail[p];
            if (tid == 0) s_tail[p ^ 1] = 0;
            int32_t *tmp = qa_; qa_ = qb_; qb_ = tmp;
            p ^= 1;
            ++rounds;
        }

        if (SMEM_ARR) {
            __syncthreads();
            for (int32_t i = tid; i < V; i += nthr) out[i] = arr[i];
        }
        if (tid == 0 && qa.status)
            qa.status[q] = !valid ? EAT_ERR_INVALID : (F > 0 ? EAT_ERR_NO_CONVERGENCE : EAT_OK);
        if (qa.counters) {
            unsigned long long c[6] = {(unsigned long long)c_vert, (unsigned long long)c_types,
                                       (unsigned long long)c_evals, (unsigned long long)c_lookups,
                                       (unsigned long long)c_aps, (unsigned long long)c_relax};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_down_sync(0xffffffffu, c[k], o);
            if ((tid & 31) == 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) atomicAdd(&s_cnt[k], c[k]);
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

__global__ void eat_next_departure_kernel(const NetDev N, const int32_t *types,
                                          const int32_t *times, int32_t n, int32_t *out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t t = types[i];
    int32_t aps = 0;
    out[i] = ((unsigned)t < (unsigned)N.n_types) ? next_departure(N, t, times[i], aps) : kInf;
}

// ------------------------------------------------------------------ launchers

enum MemKind { kArrSmem = 0, kArrGlobalMaskSmem = 1, kArrGlobalMaskGlobal = 2 };

template <int NETS>
static const void *cta_kernel_ptr(int mem) {
    switch (mem) {
    case kArrSmem: return (const void *)eat_cta_kernel<NETS, true, true>;
    case kArrGlobalMaskSmem: return (const void *)eat_cta_kernel<NETS, false, true>;
    default: return (const void *)eat_cta_kernel<NETS, false, false>;
    }
}

const void *cta_kernel(int nets, int mem) {
    return nets == 1 ? cta_kernel_ptr<1>(mem) : cta_kernel_ptr<EAT_MAX_NETS>(mem);
}

template <int NETS>
static cudaError_t launch_cta_t(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem,
                                int grid, int block, size_t smem, cudaStream_t st) {
    NetTable<NETS> tab;
    for (int i = 0; i < n_nets && i < NETS; ++i) tab.net[i] = nets[i];
    for (int i = n_nets; i < NETS; ++i) tab.net[i] = NetDev{};
    switch (mem) {
    case kArrSmem:
        eat_cta_kernel<NETS, true, true><<<grid, block, smem, st>>>(tab, qa);
        break;
    case kArrGlobalMaskSmem:
        eat_cta_kernel<NETS, false, true><<<grid, block, smem, st>>>(tab, qa);
        break;
    default:
        eat_cta_kernel<NETS, false, false><<<grid, block, smem, st>>>(tab, qa);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_cta(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                       int block, size_t smem, cudaStream_t st) {
    if (n_nets == 1) return launch_cta_t<1>(nets, n_nets, qa, mem, grid, block, smem, st);
    return launch_cta_t<EAT_MAX_NETS>(nets, n_nets, qa, mem, grid, block, smem, st);
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
