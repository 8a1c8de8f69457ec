// Internal declarations shared by libeat's translation units (not installed).
#pragma once

#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include <vector_types.h>

#include "eat.h"

namespace eat {

// Device-side descriptor of one resident network (plain pointers into one blob).
//
// Device layout (derived from the logical arrays of HostNet by build_fused):
//   tr[t]         16-byte record of connection type t: {v, lambda | d << 24, row_ptr[v],
//                 last departure}: head stop, duration, types leaving v (255 = read
//                 row_ptr), the head's first type, and the type's last departure
//   ce[k*T + t]   32-byte entry of type t for cluster k_min + k, for every cluster
//                 of the network (the paper's dense CL table, cluster-major so that
//                 lookups at nearby times fall in one slab of T entries), read in
//                 one load:
//                   int4 {rel0 | rel1 << 16, sc0, sc1, next}
//                   int4 {x/2 | n << 24, rel2 | rel3 << 16, sc2, sc3}
//                 the cluster's n APs: the first four inline with first terms
//                 base + rel (base = t0 + (k_min + k) * width) and
//                 sc = (difference << 16) | terms, the others at apx[x ..] (x even);
//                 n = 255 means more: the true count heads the list in two slots;
//                 next = first departure of the next non-empty cluster (INF if none)
//   apx[]         uint2 {first term, sc} of the fifth and later APs of a cluster
//   row_ptr[V+1]  types leaving stop u are row_ptr[u] .. row_ptr[u+1]-1
constexpr int32_t kCountOverflow = 255;
constexpr int32_t kMaxDuration = 1 << 24;
constexpr int32_t kInlineAps = 4;

struct NetDev {
    const int32_t *row_ptr;   // [V + 1] types by tail stop
    const int4 *tr;           // [T] type records
    const int4 *ce;           // [2 * y * T], cluster-major
    const uint2 *apx;         // [n_apx]
    int32_t n_stops;
    int32_t n_types;
    int32_t t0;
    int32_t width;            // cluster width (seconds)
    float inv_width;          // 1 / width, for the cluster index of times < 2^22 s
    int32_t k_min;            // first cluster index stored
    int32_t y;                // clusters stored per type
};

// Up to NETS networks passed by value as a kernel parameter.
template <int NETS>
struct NetTable {
    NetDev net[NETS];
};

// Host copy of the built arrays (kept for eat_net_host_view).
struct HostNet {
    int32_t n_stops = 0, n_types = 0, n_edges = 0, width = 3600, t0 = 0;
    int32_t max_clusters = 0, max_out_types = 0;
    int64_t n_conn = 0;
    int64_t n_shortcuts = 0;
    std::vector<int32_t> row_ptr;    // V + 1
    std::vector<int32_t> type_rec;   // 4 T
    std::vector<int32_t> type_cl;    // T
    std::vector<int32_t> cl;         // n_cl
    std::vector<uint32_t> ap;        // 2 n_ap
    // Device layout (see NetDev).
    int32_t k_min = 0, y = 1;
    std::vector<int32_t> tr;         // 4 T
    std::vector<int32_t> ce;         // 8 T y
    std::vector<uint32_t> apx;       // 2 n_apx
};

}  // namespace eat

struct eat_net {
    eat::HostNet host;
    int32_t device = -1;
    void *blob = nullptr;            // one cudaMalloc holding every array
    int64_t blob_bytes = 0;
    eat::NetDev dev{};
    // Internal workspace and staging buffers (eat_query, NULL-workspace batches).
    mutable std::mutex ws_lock;
    mutable void *ws = nullptr;
    mutable size_t ws_bytes = 0;
    mutable void *stage = nullptr;
    mutable size_t stage_bytes = 0;
    // Launch shape chosen by eat_autotune per batch-size class (log2 of n), packed as
    // block | vwarp << 16 | mode << 24 | horizon << 32 (0 = none) so that a query call
    // on another thread reads one whole shape.
    mutable std::atomic<uint64_t> tuned[32] = {};
};

namespace eat {

// Thread-local error message helpers (eat_api.cu).
int fail(int code, const std::string &msg);
void clear_error();

// Host preprocessing (eat_build.cpp): fills `h` from the connections.
int build_host(const eat_connections *c, int32_t width, int32_t t0, HostNet &h);

// Sub-trips (eat_build.cpp): the connections plus one artificial connection per
// sub-trip of >= 2 connections (Section II-G), as new SoA arrays.
int add_subtrips(const eat_connections *c, int32_t scheme, std::vector<int32_t> &u,
                 std::vector<int32_t> &v, std::vector<int32_t> &dep, std::vector<int32_t> &dur,
                 int64_t &n_added);

// Logical arrays from pre-encoded types / clusters / APs (eat_build.cpp).
int build_host_csr(const eat_csr_input *in, int32_t width, int32_t t0, HostNet &h);

// Device layout from the logical arrays (eat_build.cpp).
int build_fused(HostNet &h);

// Greedy AP cover of sorted unique values (eat_build.cpp); appends (first, step, terms).
void ap_cover(const int32_t *vals, int32_t n, int32_t width_hint,
              std::vector<uint32_t> &out_ap);

// Greedy AP cover of any sorted unique values (eat_build.cpp); appends
// (first, difference, terms) as three int32 per AP.
void ap_cover_wide(const int32_t *vals, int32_t n, std::vector<int32_t> &out);

}  // namespace eat
