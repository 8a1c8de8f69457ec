// Internal declarations shared by libeat's translation units (not installed).
#pragma once

#include <stdint.h>
#include <stddef.h>

#include <mutex>
#include <string>
#include <vector>

#include <vector_types.h>

#include "eat.h"

namespace eat {

// Device-side descriptor of one resident network (plain pointers into one blob).
struct NetDev {
    const int32_t *row_ptr;   // [V + 1] types by tail stop
    const int4 *ty;           // [T] {v, lambda, first departure, last departure}
    const int32_t *cl_base;   // [T] cluster k of type t starts at cl[cl_base[t] + k]
    const int32_t *cl;        // [n_cl]
    const uint2 *ap;          // [n_ap] {first term, (difference << 16) | terms}
    int32_t n_stops;
    int32_t n_types;
    int32_t t0;
    int32_t width;            // cluster width (seconds)
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
    std::vector<int32_t> row_ptr;    // V + 1
    std::vector<int32_t> type_rec;   // 4 T
    std::vector<int32_t> type_cl;    // T
    std::vector<int32_t> cl;         // n_cl
    std::vector<uint32_t> ap;        // 2 n_ap
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
};

namespace eat {

// Thread-local error message helpers (eat_api.cu).
int fail(int code, const std::string &msg);
void clear_error();

// Host preprocessing (eat_build.cpp): fills `h` from the connections.
int build_host(const eat_connections *c, int32_t width, int32_t t0, HostNet &h);

// Greedy AP cover of sorted unique values (eat_build.cpp); appends (first, step, terms).
void ap_cover(const int32_t *vals, int32_t n, int32_t width_hint,
              std::vector<uint32_t> &out_ap);

}  // namespace eat
