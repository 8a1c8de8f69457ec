// Kernel argument block and launchers shared by eat_kernels.cu and eat_api.cu.
#pragma once

#include <cuda_runtime.h>

#include "eat_internal.h"

namespace eat {

struct QueryArgs {
    const int32_t *net_idx;    // [n] or nullptr (single network)
    const int32_t *src;        // [n]
    const int32_t *ts;         // [n]
    const int64_t *arr_off;    // [n] or nullptr (row q at q * n_stops)
    int32_t *arr_out;
    int32_t *queues;           // [slots][queue_stride]
    uint32_t *gmask;           // [slots][mask_stride] when the bitmap is global
    int32_t *work;             // query counter (zeroed before launch)
    int32_t *status;           // [n] or nullptr
    eat_counters *counters;    // [n] or nullptr
    int64_t queue_stride;      // ints per slot (>= 2 * max n_stops)
    int64_t mask_stride;       // words per slot
    int32_t n;
    int32_t n_nets;
    int32_t max_rounds;
    int32_t vw_log2;           // lanes per active stop = 1 << vw_log2
};

// mem: 0 = arrivals and bitmap in shared memory, 1 = arrivals global / bitmap
// shared, 2 = both global.  nets: 1 or EAT_MAX_NETS (kernel table size).
const void *cta_kernel(int nets, int mem);
cudaError_t launch_cta(const NetDev *nets, int n_nets, const QueryArgs &qa, int mem, int grid,
                       int block, size_t smem, cudaStream_t st);
cudaError_t launch_next_departure(const NetDev &N, const int32_t *types, const int32_t *times,
                                  int32_t n, int32_t *out, cudaStream_t st);

}  // namespace eat
