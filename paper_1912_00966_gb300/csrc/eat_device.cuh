// Device functions of the Cluster-AP lookup shared by the query kernels
// (eat_kernels.cu) and the topology-driven variants (eat_ladder.cu).
#pragma once

#include <cuda_runtime.h>

#include "eat_internal.h"

namespace eat {

constexpr int32_t kInf = INT32_MAX;

// ceil(a / b) for 1 <= a, b < 2^16 without an integer divide: a fast float
// quotient (a few ulp of error, i.e. well under 1 for quotients < 2^16) rounded
// down, then made exact with the integer remainder.
__device__ __forceinline__ int32_t ceil_div_small(int32_t a, int32_t b) {
    int32_t q = __float2int_rz(__fdividef((float)a, (float)b));
    int32_t r = a - q * b;
    if (r < 0) { --q; r += b; }
    else if (r >= b) { ++q; r -= b; }
    return q + (r > 0);
}

// Least term >= e of the AP {start, sc = difference << 16 | terms}, or kInf.
// Only a many-term AP that straddles e needs arithmetic (Algorithm 6's
// ceil((e - start) / difference)); e - start < cluster width < 2^16 there.
__device__ __forceinline__ int32_t ap_candidate(int32_t start, uint32_t sc, int32_t e) {
    if (e <= start) return start;
    const int32_t cnt = (int32_t)(sc & 0xffffu);
    if (cnt <= 1) return kInf;
    const int32_t step = (int32_t)(sc >> 16);
    if (e > start + (cnt - 1) * step) return kInf;
    return start + ceil_div_small(e - start, step) * step;
}

// getConnectionFromAPs (Algorithm 6) over the APs of one cluster entry, with the
// Cluster-AP fallback of Section II-D: if the cluster has no departure >= e, the
// answer is the first departure of the next non-empty cluster (`next`).
// a = {rel0 | rel1 << 16, sc0, sc1, next}, b = {x/2 | n << 24, rel2 | rel3 << 16, sc2,
// sc3}; n APs, the fifth and later at apx[x..]; base is the cluster's start time.
// APs are ordered by first term, so the scan stops at the first start >= the best
// candidate so far.
__device__ __forceinline__ int32_t cluster_lookup(const int4 a, const int4 b, int32_t n, int32_t x,
                                                  int32_t base, int32_t e,
                                                  const uint2 *__restrict__ apx, int32_t &aps) {
    int32_t tc = kInf;
    if (n > 0) {
        ++aps;
        tc = ap_candidate(base + (a.x & 0xffff), (uint32_t)a.y, e);
        const int32_t s1 = base + (int32_t)((uint32_t)a.x >> 16);
        if (n > 1 && s1 < tc) {
            ++aps;
            tc = min(tc, ap_candidate(s1, (uint32_t)a.z, e));
            const int32_t s2 = base + (b.y & 0xffff);
            if (n > 2 && s2 < tc) {
                ++aps;
                tc = min(tc, ap_candidate(s2, (uint32_t)b.z, e));
                const int32_t s3 = base + (int32_t)((uint32_t)b.y >> 16);
                if (n > 3 && s3 < tc) {
                    ++aps;
                    tc = min(tc, ap_candidate(s3, (uint32_t)b.w, e));
                    // Further APs: batches of 8 loaded together (the list is 16-byte
                    // aligned and padded to an even length), one L2 round trip a batch.
                    // A count of 255 means the true count heads the list in two slots.
                    int32_t m = n - kInlineAps;
                    const uint2 *lst = apx + x;
                    if (n == kCountOverflow) {
                        m = (int32_t)__ldg(lst).x - kInlineAps;
                        lst += 2;
                    }
                    const uint4 *p = reinterpret_cast<const uint4 *>(lst);
                    for (int32_t j = 0; j < m; j += 8) {
                        uint4 r[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            r[q] = (j + 2 * q < m) ? __ldg(p + (j >> 1) + q) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (j + 2 * q < m) tc = min(tc, ap_candidate((int32_t)r[q].x, r[q].y, e));
                            if (j + 2 * q + 1 < m) tc = min(tc, ap_candidate((int32_t)r[q].z, r[q].w, e));
                        }
                        aps += min(8, m - j);
                        if (j + 8 < m && (int32_t)r[3].z >= tc) break;   // later starts are larger
                    }
                }
            }
        }
    }
    return tc == kInf ? a.w : tc;
}

// Count and index of a cluster entry's APs (b = {x/2 | n << 24, ...}); a count of 255
// stands for 255 or more (cluster_lookup then reads the true count from the list).
__device__ __forceinline__ void entry_aps(const int4 b, int32_t &n, int32_t &x) {
    n = (int32_t)((uint32_t)b.x >> 24);
    x = (b.x & 0xffffff) * 2;
}

// Cluster slot of time e relative to the first stored cluster; e before the first
// cluster maps to slot 0 (every departure is then >= e), and a result >= y means
// no departure at or after e exists in the network.
__device__ __forceinline__ int32_t cluster_slot(const NetDev &N, int32_t e) {
    const int64_t d = (int64_t)e - N.t0;
    if (d < 0) return 0;
    int32_t q;
    if (d < (1 << 22)) {       // float quotient, exact after one remainder step
        const int32_t di = (int32_t)d;
        q = __float2int_rz((float)di * N.inv_width);
        const int32_t r = di - q * N.width;
        if (r < 0) --q;
        else if (r >= N.width) ++q;
    } else {
        q = (int32_t)((uint32_t)d / (uint32_t)N.width);
    }
    const int32_t k = q - N.k_min;
    return k < 0 ? 0 : k;
}

// Start time of stored cluster slot k.
__device__ __forceinline__ int32_t cluster_base(const NetDev &N, int32_t k) {
    return N.t0 + (N.k_min + k) * N.width;
}

// One 32-byte cluster entry in a single 256-bit load (sm_100 and later), read
// through the non-coherent path: the entries never change during a query.
__device__ __forceinline__ void load_entry(const int4 *c, int4 &a, int4 &b) {
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
        : "l"(c));
}

// Cluster entry of type t for stored cluster slot k (cluster-major table).
__device__ __forceinline__ const int4 *entry_at(const NetDev &N, int32_t k, int32_t t) {
    return N.ce + 2 * ((int64_t)k * N.n_types + t);
}

// getConnection of type t at time e: least departure >= e, or kInf (none after the
// type's last departure, kept in its type record).
__device__ __forceinline__ int32_t next_departure(const NetDev &N, int32_t t, int32_t e,
                                                  int32_t &aps) {
    if (e > __ldg(&N.tr[t].w)) return kInf;
    const int32_t k = cluster_slot(N, e);
    if (k >= N.y) return kInf;
    int4 a, b;
    load_entry(entry_at(N, k, t), a, b);
    int32_t n, x;
    entry_aps(b, n, x);
    return cluster_lookup(a, b, n, x, cluster_base(N, k), e, N.apx, aps);
}

}  // namespace eat
