// Kernel argument block and launchers shared by eat_kernels.cu and eat_api.cu.
#pragma once

#include <cuda_runtime.h>

#include "eat_internal.h"

namespace eat {

// One request of the serving ring (page-locked host memory that the GPU reads and
// writes in place): the host dispatcher fills net, src, ts, row and clears done before
// it publishes the ring's tail; the block that ran the request writes the result row,
// then status, then done = 1 (a system-scope release).
struct RingEntry {
    int32_t net, src, ts, row;   // network index, source, departure, result row slot
    int32_t status;              // eat_status of the request
    int32_t done;                // 1 once the row and the status are in place
    int64_t seq;                 // ring position of the request (host bookkeeping)
};

// Ring-mode arguments: persistent blocks claim requests [head, tail) one at a time.
struct RingArgs {
    RingEntry *ring;             // [mask + 1] entries (device address of host memory)
    const int64_t *tail;         // requests published by the host (host memory)
    const int32_t *stop;         // nonzero: a block that finds no request leaves (host memory)
    unsigned long long *head;    // requests claimed so far (device memory, CAS)
    int64_t row_stride;          // ints per result row of the pool at arr_out
    int32_t mask;                // ring capacity - 1 (a power of two)
    int32_t idle_iters;          // polls (2 us apart, 20 us after the first 512) before an
                                 // idle block leaves
};

struct QueryArgs {
    const int32_t *net_idx;    // [n] or nullptr (single network)
    const int32_t *src;        // [n]
    const int32_t *ts;         // [n]
    const int64_t *arr_off;    // [n] or nullptr (row q at q * n_stops)
    int32_t *arr_out;
    int32_t *spill;            // [slots][spill_stride]: spilled frontier stops (2 x vmax)
    uint32_t *gmask;           // [slots][mask_stride]: both bitmaps when not in shared memory
    int32_t *work;             // query counter (zeroed before launch)
    int32_t *status;           // [n] or nullptr
    eat_counters *counters;    // [n] or nullptr
    int64_t spill_stride;      // ints per slot (>= 2 * vmax)
    int64_t mask_stride;       // words per slot (>= 2 * mask_words) when global
    int32_t n;
    int32_t n_nets;
    int32_t max_rounds;
    int32_t vw_log2;           // lanes per active stop = 1 << vw_log2
    int32_t vmax;              // largest n_stops in the launch
    int32_t qcap;              // shared-memory (stop, type) items per buffer
    int32_t mask_words;        // words per bitmap (padded)
    int32_t smem_mask_off;     // int offset of the bitmaps in dynamic shared memory
    int32_t smem_q_off;        // int offset of the item buffers in dynamic shared memory
    int32_t smem_arr_cap;      // per-query placement: arrivals shared when n_stops <= this
    int32_t *arr_rows;         // [grid][arr_rows_stride]: a block's arrivals when they are not
                               // in shared memory and arr_out is host memory, or nullptr
    int64_t arr_rows_stride;   // ints per block row
    const int32_t *order;      // [n]: the i-th query handed out is order[i], or nullptr (i)
    int32_t idle_cap;          // round-free mode: empty 32-word bitmap scans in a row per warp
    RingArgs rg;               // ring mode only
    int32_t edge;              // EAT_MODE_EDGE: warp min per head stop, stops with >= vwarp
                               // types expanded whole by a sub-warp
    int32_t horizon;           // seconds, 0 = none: stops lowered to an arrival at or after
                               // the horizon wait (per-query kernel); with one,
                               // spill_stride >= 4 * vmax + mask_words
};

// mem: 0 = arrivals and bitmaps in shared memory, 1 = arrivals global / bitmaps
// shared, 2 = both global, 3 = bitmaps shared and arrivals shared per query when
// the query's network fits.  nets: 1 or EAT_MAX_NETS (kernel table size).
// pack: one int32 per item (one network of at most 32,767 stops and 65,535 types,
// arrivals and bitmaps in shared memory).
// count: the instantiation that fills qa.counters (launch_cta picks it when counters are
// given); hz: with pack, the instantiation that honours qa.horizon (launch_cta picks it
// when qa.horizon > 0; the others always honour it).
const void *cta_kernel(int nets, int mem, bool pack = false, bool count = false, bool hz = false);
cudaError_t launch_cta(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                       int block, size_t smem, cudaStream_t st, bool pack = false);
// Ring mode of the per-query kernel (serving): persistent blocks take requests from
// qa.rg until the host's stop flag is set and no request is left, or until they find
// none for rg.idle_iters polls; mem 0, 1 or 3; rows go to arr_out + row * row_stride,
// arrivals not in shared memory live in the block's arr_rows row meanwhile.
const void *ring_kernel(int mem);
cudaError_t launch_ring(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                        int block, size_t smem, cudaStream_t st);
// Asynchronous (round-free) kernel; mem 0, 1 or 3 as above (bitmap always shared).
const void *async_kernel(int nets, int mem);
cudaError_t launch_async(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                         int block, size_t smem, cudaStream_t st);
// Cluster mode: one cluster of `cluster` blocks per query on one network; grid =
// n * cluster; arrivals and bitmaps spread over the cluster's shared memory.
const void *cluster_kernel();
cudaError_t launch_cluster(const NetDev &net, const QueryArgs &qa, int cluster, int grid,
                           int block, size_t smem, cudaStream_t st);
// Paired mode: two queries per block on one network of at most 32,767 stops and
// 65,535 types; both arrival rows and bitmaps in shared memory (smem_arr_cap = ints
// per row, bitmaps [slot][buffer]), spill queues [slot][buffer][vmax] per block;
// count: the instantiation that fills qa.counters.
const void *pair_kernel(bool count = false);
cudaError_t launch_pair(const NetDev &net, const QueryArgs &qa, int grid, int block, size_t smem,
                        cudaStream_t st);
// Serving ring (eat_server.cu): launch shape of the ring kernel for these networks,
// and its launch with the caller's buffers.
struct RingLaunch {
    int mem = 0, block = 0, grid = 0;
    size_t smem = 0;
    size_t ws_bytes = 0;          // device workspace (spill queues of every block)
    size_t rows_bytes = 0;        // device rows for arrivals kept out of shared memory
    int64_t rows_stride = 0;      // ints per such row
    int32_t vmax = 0;
    int32_t vw_log2 = 3, qcap = 0, mask_words = 0, smem_mask_off = 0, smem_q_off = 0;
    int32_t smem_arr_cap = 0;
    int64_t spill_stride = 0;
};
int ring_setup(const eat_net *const *nets, int n_nets, RingLaunch &rl);
int ring_launch(const eat_net *const *nets, int n_nets, const RingLaunch &rl, void *ws,
                int32_t *arr_rows, int32_t *pool, const RingArgs &rg, cudaStream_t st);
// order[0..n) = query indices sorted by t_s (15-minute buckets, earliest first; one
// block, counting sort; the order inside a bucket is not fixed).
cudaError_t launch_order(const int32_t *ts, int32_t n, int32_t *order, cudaStream_t st);
cudaError_t launch_next_departure(const NetDev &N, const int32_t *types, const int32_t *times,
                                  int32_t n, int32_t *out, cudaStream_t st);

}  // namespace eat
