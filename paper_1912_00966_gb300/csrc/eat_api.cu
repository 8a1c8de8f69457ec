// C ABI of libeat (declared in include/eat.h): build, free, inspection, queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "eat_internal.h"

#include "eat_launch.h"

namespace eat {

static thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

void clear_error() { g_err.clear(); }

static int cuda_fail(cudaError_t e, const char *what) {
    return fail(EAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Restores the calling thread's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of a device other than dev (the kernels would read or write a foreign
// address); host, managed and NULL pointers are not foreign.
static bool foreign_ptr(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device != dev;
}

static int foreign_fail() {
    return fail(EAT_ERR_INVALID, "a buffer is device memory of another device than the network's");
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device address of page-locked host memory that the GPU may read and write in place
// (mapped pinned memory, reached over NVLink-C2C on Grace systems), else nullptr.
static void *mapped_host_ptr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// ------------------------------------------------------------------ launch planning

struct DeviceInfo {
    int sms = 0;
    size_t smem_optin = 0;        // per block
    size_t smem_per_sm = 0;
    size_t reserve = 2048;        // static __shared__ of the kernel + per-block reservation
    bool init = false;
};

static std::mutex g_dev_lock;
static DeviceInfo g_dev[64];

static int device_info(int dev, DeviceInfo &out) {
    if (dev < 0 || dev >= 64) return fail(EAT_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_dev_lock);
    DeviceInfo &d = g_dev[dev];
    if (!d.init) {
        int v = 0;
        cudaError_t e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
        d.sms = v;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(smem optin)");
        d.smem_optin = (size_t)v;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(smem per SM)");
        d.smem_per_sm = (size_t)v;
        // Allow every CTA kernel the full opt-in shared memory (once per device).
        DeviceGuard guard(dev);
        for (int nets : {1, EAT_MAX_NETS})
            for (int mem = 0; mem < 4; ++mem)
                for (const void *k : {cta_kernel(nets, mem), cta_kernel(nets, mem, false, true),
                                      async_kernel(nets, mem), cluster_kernel(), cta_kernel(1, 0, true),
                                      cta_kernel(1, 0, true, true), cta_kernel(1, 0, true, false, true),
                                      cta_kernel(1, 0, true, true, true), pair_kernel(false), pair_kernel(true),
                                      ring_kernel(mem)}) {
                    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(d.smem_optin - d.reserve));
                    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
                }
        d.init = true;
    }
    out = d;
    return EAT_OK;
}

// Launch plan of the CTA kernel for queries on networks of at most vmax stops.
struct Plan {
    int mem = 0;                  // 0 shared arrivals + bitmaps, 1 shared bitmaps, 2 none shared
    int block = 512;
    int vw_log2 = 3;
    int grid = 0;
    size_t smem = 0;              // dynamic shared memory bytes
    int32_t vmax = 0;
    int32_t qcap = 0;             // shared-memory (stop, type) items per buffer
    int32_t mask_words = 0;       // words per bitmap
    int32_t smem_mask_off = 0;    // int offsets into dynamic shared memory
    int32_t smem_q_off = 0;
    int32_t smem_arr_cap = 0;     // mem 3: arrivals shared for networks up to this size
    int64_t spill_stride = 0;     // ints per persistent block
    int64_t mask_stride = 0;      // words per persistent block (global bitmaps only)
    size_t ws_bytes = 0;
    size_t off_spill = 0, off_mask = 0;
    int nets = 1;
    bool async = false;           // round-free kernel (EAT_MODE_ASYNC)
    int cluster = 0;              // blocks per query in cluster mode (EAT_MODE_CLUSTER), else 0
    bool pack = false;            // one int32 per queued item (small networks, shared arrivals)
    bool pair = false;            // two queries per block (EAT_MODE_PAIR)
    bool edge = false;            // warp min per head stop, degree-chosen mapping (EAT_MODE_EDGE)
    bool order = false;           // queries start by t_s (EAT_ORDER_BY_TIME): order array at off_order
    size_t off_order = 0;
    int32_t horizon = 0;          // seconds (eat_query_opts.horizon resolved), 0 = none
};

static constexpr size_t kWsHeader = 256;   // work counter + internal status / counters
static constexpr int32_t kDefaultIdleCap = 1 << 24;   // round-free mode's wait limit (full scans)
static constexpr size_t kQueueEntryBytes = 16;  // (stop, type) item x 2 buffers

// Default round cap: n_stops + 1 rounds always reach the fixpoint (every productive round
// fixes one more stop); with a horizon, each move of the horizon can add one round in
// which only stops released from waiting are expanded, at most n_stops of them.
static int32_t default_round_cap(int32_t vmax, int32_t horizon) {
    const int64_t cap = horizon > 0 ? 2 * (int64_t)vmax + 2 : (int64_t)vmax + 1;
    return (int32_t)std::min<int64_t>(cap, INT32_MAX);
}

// Plan of the round-free kernel: arrivals (shared when they fit), one bitmap and
// a 512-byte staging area per warp in shared memory; no spill queues.
static int make_async_plan(int dev, const DeviceInfo &d, int32_t vmax, int32_t n, int n_nets,
                           const eat_query_opts *o, Plan &p, int32_t vmin) {
    p.async = true;
    const size_t words = ((size_t)vmax + 31) / 32;
    p.mask_words = (int32_t)align_up(words, 4);
    const size_t arr_bytes = align_up((size_t)vmax, 4) * 4;
    const size_t stage_bytes = (size_t)(p.block / 32) * 128 * 4;
    const size_t limit = d.smem_optin - d.reserve;
    const size_t half = d.smem_per_sm / 2 - d.reserve;
    const int place = o ? o->placement : EAT_PLACE_AUTO;
    const size_t fixed = (size_t)p.mask_words * 4 + stage_bytes;
    if (fixed > limit) return fail(EAT_ERR_INVALID, "bitmap does not fit in shared memory");
    p.smem_arr_cap = 0;
    if (place == EAT_PLACE_GLOBAL) return fail(EAT_ERR_INVALID, "asynchronous mode keeps the bitmap in shared memory");
    if (place == EAT_PLACE_SHARED) {
        if (arr_bytes + fixed > limit) return fail(EAT_ERR_INVALID, "arrivals do not fit in shared memory");
        p.mem = 0;
    } else if (place == EAT_PLACE_GLOBAL_ARR) {
        p.mem = 1;
    } else if (arr_bytes + fixed <= half || (n_nets == 1 && arr_bytes + fixed <= limit)) {
        p.mem = 0;
    } else if (vmin < vmax && fixed + (size_t)vmin * 4 <= half) {
        p.mem = 3;
        p.smem_arr_cap = (int32_t)std::min<size_t>((half - fixed) / 4 & ~(size_t)3, (size_t)vmax);
    } else {
        p.mem = 1;
    }
    p.smem_mask_off = p.mem == 0 ? (int32_t)(arr_bytes / 4) : p.mem == 3 ? p.smem_arr_cap : 0;
    p.smem_q_off = p.smem_mask_off + p.mask_words;
    p.smem = (size_t)p.smem_q_off * 4 + stage_bytes;
    p.qcap = 0;
    int per_sm = 0;
    cudaError_t e;
    {
        DeviceGuard guard(dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, async_kernel(p.nets, p.mem),
                                                          p.block, p.smem);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(EAT_ERR_INVALID, "kernel does not fit on an SM with this block size");
    p.grid = (int)std::min<int64_t>((int64_t)std::max(n, 1), (int64_t)per_sm * d.sms);
    p.spill_stride = 0;
    p.mask_stride = 0;
    p.off_spill = kWsHeader;
    p.off_mask = kWsHeader;
    p.ws_bytes = kWsHeader;
    return EAT_OK;
}

static constexpr int kCluster = 8;   // blocks per query in cluster mode (portable maximum)

// Plan of the cluster kernel: one cluster of kCluster blocks per query, each block
// holding every kCluster-th arrival and its bits of both bitmaps, plus its own item
// queues; the rest of a block's shared memory goes to the queues.
static int make_cluster_plan(int dev, const DeviceInfo &d, int32_t vmax, int32_t n,
                             const eat_query_opts *o, Plan &p) {
    const int C = (o && o->cluster) ? o->cluster : kCluster;
    if (C != 2 && C != 4 && C != 8) return fail(EAT_ERR_INVALID, "cluster must be 2, 4 or 8");
    p.cluster = C;
    p.mem = 0;
    p.async = false;
    p.nets = 1;
    const size_t slice = ((size_t)vmax + C - 1) / C;
    p.mask_words = (int32_t)align_up((slice + 31) / 32, 4);
    const size_t arr_bytes = align_up(slice, 4) * 4;
    const size_t base = arr_bytes + 2 * (size_t)p.mask_words * 4;
    const size_t limit = d.smem_optin - d.reserve;
    const size_t qmin = 256;
    if (base + kQueueEntryBytes * qmin > limit)
        return fail(EAT_ERR_INVALID, "arrivals do not fit in the shared memory of one cluster");
    size_t cap = std::min((limit - base) / kQueueEntryBytes, std::max((size_t)vmax, qmin));
    if (cap >= 64) cap &= ~(size_t)31;
    p.qcap = (int32_t)std::max(cap, qmin);
    p.smem_mask_off = (int32_t)(arr_bytes / 4);
    p.smem_q_off = p.smem_mask_off + 2 * p.mask_words;
    p.smem = base + kQueueEntryBytes * (size_t)p.qcap;
    p.grid = std::max(n, 1) * C;
    p.spill_stride = (int64_t)align_up((size_t)vmax * 2, 64);
    p.mask_stride = 0;
    p.off_spill = kWsHeader;
    p.off_mask = p.off_spill + (size_t)p.grid * (size_t)p.spill_stride * 4;
    p.ws_bytes = p.off_mask;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3((unsigned)p.block);
    cfg.dynamicSmemBytes = p.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cudaError_t e;
    {
        DeviceGuard guard(dev);
        e = cudaOccupancyMaxActiveClusters(&clusters, cluster_kernel(), &cfg);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EAT_ERR_INVALID, std::string("cluster launch not possible: ") + cudaGetErrorString(e));
    }
    if (clusters < 1) return fail(EAT_ERR_INVALID, "no cluster fits the device with this block size");
    return EAT_OK;
}

static constexpr int32_t kWideMinStops = 8192;   // 1,024-thread blocks for any batch from this size

// Plan of the paired kernel: two arrival rows, four bitmaps (two per query) and the
// shared item buffers (one int32 per item) in one block's shared memory.  Returns
// EAT_ERR_INVALID when the network is not small enough.
static int make_pair_plan(int dev, const DeviceInfo &d, int32_t vmax, int32_t n,
                          const eat_net *net, Plan &p) {
    if (!net || vmax > 32767 || net->host.n_types > 65535)
        return fail(EAT_ERR_INVALID, "paired mode needs one network of at most 32,767 stops and 65,535 types");
    p.pair = true;
    p.pack = true;
    p.mem = 0;
    p.async = false;
    p.nets = 1;
    const size_t vpad = align_up((size_t)std::max(vmax, 1), 4);
    p.mask_words = (int32_t)align_up(((size_t)vmax + 31) / 32, 4);
    const size_t base = 2 * vpad * 4 + 4 * (size_t)p.mask_words * 4;
    const size_t limit = d.smem_optin - d.reserve;
    const size_t qmin = 512;
    if (base + 8 * qmin > limit)
        return fail(EAT_ERR_INVALID, "two arrival rows do not fit in one block's shared memory");
    size_t cap = std::min((limit - base) / 8, 2 * (size_t)std::max(vmax, 1));
    if (cap >= 64) cap &= ~(size_t)31;
    p.qcap = (int32_t)std::max(cap, qmin);
    p.smem_arr_cap = (int32_t)vpad;
    p.smem_mask_off = (int32_t)(2 * vpad);
    p.smem_q_off = p.smem_mask_off + 4 * p.mask_words;
    p.smem = base + 8 * (size_t)p.qcap;
    int per_sm = 0;
    cudaError_t e;
    {
        DeviceGuard guard(dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_kernel(), p.block, p.smem);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(EAT_ERR_INVALID, "kernel does not fit on an SM with this block size");
    p.grid = (int)std::min<int64_t>((int64_t)std::max(n, 1), (int64_t)per_sm * d.sms);
    p.spill_stride = (int64_t)align_up((size_t)vmax * 4, 64);
    p.mask_stride = 0;
    p.off_spill = kWsHeader;
    p.off_mask = p.off_spill + (size_t)p.grid * (size_t)p.spill_stride * 4;
    p.ws_bytes = p.off_mask;
    return EAT_OK;
}

static int make_plan_core(int dev, int32_t vmax, int32_t n, int n_nets, const eat_query_opts *o,
                          Plan &p, int32_t vmin, const eat_net *tuned, bool own_workspace) {
    if (vmin < 0) vmin = vmax;
    DeviceInfo d;
    int rc = device_info(dev, d);
    if (rc) return rc;
    p.nets = n_nets == 1 ? 1 : EAT_MAX_NETS;
    p.vmax = vmax;
    int tb = 0, tv = 0, tm = 0, th = 0;
    if (tuned && n > 0) {
        int cls = 0;
        while (cls < 31 && (1 << (cls + 1)) <= n) ++cls;
        const uint64_t sh = tuned->tuned[cls].load(std::memory_order_relaxed);
        tb = (int)(sh & 0xffffu);
        tv = (int)((sh >> 16) & 0xffu);
        tm = (int)((sh >> 24) & 0xffu);
        th = (int)(uint32_t)(sh >> 32);
    }
    // Default shape: a 1,024-thread block per query when the batch has at most one query
    // per SM, or on one network of 8,192 stops or more (there the batch starts in order
    // of t_s, so the longest queries run first and the later ones fill the blocks that
    // free up: city 0.70 ms per 256-query step against 0.88 ms for two 512-thread
    // blocks per SM); fuller batches on small networks, and batches over several
    // networks (mostly small ones: the ragged batch of 64 networks took 4.59 ms with
    // 1,024 threads against 2.71 ms with 512), run two 512-thread blocks per SM.
    // A tuned shape or opts->block overrides.
    p.block = (o && o->block) ? o->block
              : (tb ? tb
                    : (n >= 1 && (n <= d.sms || (n_nets == 1 && vmax >= kWideMinStops)) ? 1024 : 512));
    if (p.block < 64 || p.block > 1024 || p.block % 32)
        return fail(EAT_ERR_INVALID, "block must be a multiple of 32 in 64..1024");
    int vw = (o && o->vwarp) ? o->vwarp : (tv ? tv : 8);
    int l = 0;
    while ((1 << l) < vw) ++l;
    if ((1 << l) != vw || vw > 32) return fail(EAT_ERR_INVALID, "vwarp must be 1, 2, 4, 8, 16 or 32");
    p.vw_log2 = l;
    if (o && (o->mode < EAT_MODE_AUTO || o->mode > EAT_MODE_EDGE))
        return fail(EAT_ERR_INVALID, "mode must be one of EAT_MODE_*");
    p.edge = (o && o->mode == EAT_MODE_EDGE) ||
             (tm == EAT_MODE_EDGE && !(o && o->mode != EAT_MODE_AUTO));
    const int32_t oh = o ? o->horizon : 0;
    if (oh > 0 && (o->mode == EAT_MODE_PAIR || o->mode == EAT_MODE_ASYNC || o->mode == EAT_MODE_CLUSTER))
        return fail(EAT_ERR_INVALID, "a horizon needs the per-query kernel's rounds (EAT_MODE_CTA or EAT_MODE_EDGE)");
    if (o && o->mode == EAT_MODE_PAIR) {
        if (n_nets != 1) return fail(EAT_ERR_INVALID, "paired mode serves one network per launch");
        if (o->placement != EAT_PLACE_AUTO && o->placement != EAT_PLACE_SHARED)
            return fail(EAT_ERR_INVALID, "paired mode keeps arrivals in shared memory");
        if (!o->block) p.block = 1024;
        return make_pair_plan(dev, d, vmax, n, tuned, p);
    }
    if (o && o->mode == EAT_MODE_CLUSTER) {
        if (n_nets != 1) return fail(EAT_ERR_INVALID, "cluster mode serves one network per launch");
        if (o->placement != EAT_PLACE_AUTO && o->placement != EAT_PLACE_SHARED)
            return fail(EAT_ERR_INVALID, "cluster mode keeps arrivals in shared memory");
        if (!own_workspace) return fail(EAT_ERR_INVALID, "cluster mode is not available here");
        return make_cluster_plan(dev, d, vmax, n, o, p);
    }
    // The round cap and the horizon need the per-query kernel's rounds.
    const bool rounds_needed = o && (o->max_rounds > 0 || o->horizon > 0);
    if ((o && o->mode == EAT_MODE_ASYNC) ||
        (tm == EAT_MODE_ASYNC && !rounds_needed && (!o || o->mode == EAT_MODE_AUTO)))
        return make_async_plan(dev, d, vmax, n, n_nets, o, p, vmin);
    const int place = o ? o->placement : EAT_PLACE_AUTO;
    if (place < EAT_PLACE_AUTO || place > EAT_PLACE_GLOBAL)
        return fail(EAT_ERR_INVALID, "placement must be one of EAT_PLACE_*");
    // The paired mode when the autotuner chose it for this batch size (never by default:
    // with the batch started in order of t_s, one query per 1,024-thread block is faster
    // on the city network, 0.70 against 0.79 ms per 256-query step).
    const bool explicit_block = o && o->block;
    if ((!o || o->mode == EAT_MODE_AUTO) && own_workspace && n_nets == 1 && tuned &&
        (place == EAT_PLACE_AUTO || place == EAT_PLACE_SHARED) && !explicit_block &&
        tm == EAT_MODE_PAIR && oh <= 0) {
        Plan q = p;
        q.block = tb ? tb : 1024;
        if (make_pair_plan(dev, d, vmax, n, tuned, q) == EAT_OK) {
            p = q;
            return EAT_OK;
        }
        clear_error();                       // network too large: the per-query kernel
    }

    const size_t words = ((size_t)vmax + 31) / 32;
    p.mask_words = (int32_t)align_up(words, 4);
    const size_t arr_bytes = align_up((size_t)vmax, 4) * 4;
    const size_t mask_bytes = 2 * (size_t)p.mask_words * 4;
    const size_t qmin = std::min<size_t>((size_t)std::max(vmax, 1), 256);
    const size_t limit = d.smem_optin - d.reserve;
    auto base = [&](int mem) { return (mem == 0 ? arr_bytes : 0) + (mem <= 1 ? mask_bytes : 0); };
    auto fits = [&](int mem) { return base(mem) + kQueueEntryBytes * qmin <= limit; };
    if (place == EAT_PLACE_SHARED && !fits(0))
        return fail(EAT_ERR_INVALID, "arrivals do not fit in shared memory");
    if (place == EAT_PLACE_GLOBAL_ARR && !fits(1))
        return fail(EAT_ERR_INVALID, "bitmaps do not fit in shared memory");
    // A batch over networks of uneven size whose largest arrival row would cost
    // more than half an SM's shared memory keeps arrivals in shared memory only
    // for the networks that fit half an SM (two blocks per SM stay resident).
    const size_t half = d.smem_per_sm / 2 - d.reserve;
    p.smem_arr_cap = 0;
    if (place == EAT_PLACE_AUTO && vmin < vmax && base(0) + kQueueEntryBytes * qmin > half &&
        fits(1)) {
        const size_t room = half - base(1) - kQueueEntryBytes * 1024;
        const int32_t cap = (int32_t)std::min<size_t>(room / 4 & ~(size_t)3, (size_t)vmax);
        if (cap >= vmin) {
            p.mem = 3;
            p.smem_arr_cap = cap;
        }
    }
    if (p.mem == 3) {
    } else if (place == EAT_PLACE_SHARED || (place == EAT_PLACE_AUTO && fits(0))) p.mem = 0;
    else if (place == EAT_PLACE_GLOBAL_ARR || (place == EAT_PLACE_AUTO && fits(1))) p.mem = 1;
    else p.mem = 2;

    // Items take one int32 instead of two on one network small enough for the packed
    // form (twice the queue in the same shared memory).
    p.pack = p.mem == 0 && n_nets == 1 && tuned && vmax <= 32767 && tuned->host.n_types <= 65535;
    p.horizon = oh > 0 ? oh : (oh == 0 ? th : 0);
    const size_t qbytes = p.pack ? kQueueEntryBytes / 2 : kQueueEntryBytes;
    // Largest queue capacity that keeps the most blocks per SM the threads and the
    // registers allow (shared memory is the only other limit, and the one sized here).
    const size_t b0 = p.mem == 3 ? base(1) + (size_t)p.smem_arr_cap * 4 : base(p.mem);
    int reg_blocks = 0;
    {
        DeviceGuard guard(dev);
        const void *k = cta_kernel(p.nets, p.mem, p.pack, false, p.horizon > 0);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&reg_blocks, k, p.block, 0) != cudaSuccess) {
            cudaGetLastError();
            reg_blocks = 0;
        }
    }
    const int max_blocks = std::max(1, std::min(2048 / p.block, reg_blocks > 0 ? reg_blocks : 2048));
    p.qcap = (int32_t)qmin;
    for (int b = max_blocks; b >= 1; --b) {
        const size_t budget = std::min(limit, d.smem_per_sm / (size_t)b - d.reserve);
        if (d.smem_per_sm / (size_t)b < d.reserve || b0 + qbytes * qmin > budget) continue;
        size_t cap = (budget - b0) / qbytes;
        cap = std::min(cap, (size_t)std::max(vmax, 1));
        if (cap >= 64) cap &= ~(size_t)31;
        p.qcap = (int32_t)std::max(cap, qmin);
        break;
    }
    p.smem_mask_off = p.mem == 0 ? (int32_t)(arr_bytes / 4) : p.mem == 3 ? p.smem_arr_cap : 0;
    p.smem_q_off = p.smem_mask_off + (p.mem != 2 ? 2 * p.mask_words : 0);
    p.smem = b0 + qbytes * (size_t)p.qcap;

    int per_sm = 0;
    cudaError_t e;
    {
        DeviceGuard guard(dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, cta_kernel(p.nets, p.mem, p.pack, false, p.horizon > 0), p.block, p.smem);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(EAT_ERR_INVALID, "kernel does not fit on an SM with this block size");
    p.grid = (int)std::min<int64_t>((int64_t)std::max(n, 1), (int64_t)per_sm * d.sms);
    // With a horizon a block also keeps two lists of waiting stops and their bitmap.
    p.spill_stride = p.horizon > 0 ? (int64_t)align_up((size_t)vmax * 4 + (size_t)p.mask_words, 64)
                                   : (int64_t)align_up((size_t)vmax * 2, 64);
    p.mask_stride = p.mem == 2 ? (int64_t)align_up(2 * (size_t)p.mask_words, 64) : 0;
    p.off_spill = kWsHeader;
    p.off_mask = p.off_spill + (size_t)p.grid * (size_t)p.spill_stride * 4;
    p.ws_bytes = p.off_mask + (size_t)p.grid * (size_t)p.mask_stride * 4;
    return EAT_OK;
}

// Launch plan for n queries; with a workspace of its own, a batch of more than one query
// also gets its start order (EAT_ORDER_BY_TIME) at the end of the workspace.
static int make_plan(int dev, int32_t vmax, int32_t n, int n_nets, const eat_query_opts *o,
                     Plan &p, int32_t vmin = -1, const eat_net *tuned = nullptr,
                     bool own_workspace = true) {
    const int order = o ? o->order : EAT_ORDER_AUTO;
    if (order < EAT_ORDER_AUTO || order > EAT_ORDER_AS_GIVEN)
        return fail(EAT_ERR_INVALID, "order must be one of EAT_ORDER_*");
    int rc = make_plan_core(dev, vmax, n, n_nets, o, p, vmin < 0 ? vmax : vmin, tuned, own_workspace);
    if (rc) return rc;
    // Automatic, on one network: sorted when some queries must wait for a free block
    // (they then start longest first) and in the paired mode (an early query shares its
    // block with a late one); a batch that starts all at once gains nothing for the
    // sort's launch.  Batches over several networks keep index order (measured only so).
    const bool waits = p.cluster == 0 && !p.pair && n > p.grid;
    if (own_workspace && n > 1 &&
        (order == EAT_ORDER_BY_TIME ||
         (order == EAT_ORDER_AUTO && n_nets == 1 && (waits || p.pair)))) {
        p.order = true;
        p.off_order = align_up(p.ws_bytes, 256);
        p.ws_bytes = p.off_order + align_up((size_t)n * 4, 256);
    }
    return EAT_OK;
}

// Kernel arguments for a plan; `grid` persistent blocks share the scratch at `ws`.
static QueryArgs make_args(const Plan &p, int grid, char *ws, const int32_t *net_idx,
                           const int32_t *src, const int32_t *ts, int32_t n, int n_nets,
                           int32_t *arr_out, const int64_t *arr_off, int32_t max_rounds,
                           int32_t *status, eat_counters *counters) {
    QueryArgs qa;
    qa.net_idx = net_idx;
    qa.src = src;
    qa.ts = ts;
    qa.arr_off = arr_off;
    qa.arr_out = arr_out;
    qa.spill = (int32_t *)(ws + kWsHeader);
    qa.gmask = (uint32_t *)(ws + kWsHeader + (size_t)grid * (size_t)p.spill_stride * 4);
    qa.work = (int32_t *)ws;
    qa.status = status;
    qa.counters = counters;
    qa.spill_stride = p.spill_stride;
    qa.mask_stride = p.mask_stride;
    qa.n = n;
    qa.n_nets = n_nets;
    qa.max_rounds = max_rounds;
    qa.vw_log2 = p.vw_log2;
    qa.vmax = p.vmax;
    qa.qcap = p.qcap;
    qa.mask_words = p.mask_words;
    qa.smem_mask_off = p.smem_mask_off;
    qa.smem_q_off = p.smem_q_off;
    qa.smem_arr_cap = p.smem_arr_cap;
    qa.arr_rows = nullptr;
    qa.arr_rows_stride = 0;
    qa.order = p.order ? (const int32_t *)(ws + p.off_order) : nullptr;
    qa.idle_cap = kDefaultIdleCap;
    qa.rg = RingArgs{};
    qa.edge = p.edge ? 1 : 0;
    qa.horizon = p.horizon;
    return qa;
}

// Per-block arrival rows needed when a plan keeps some arrivals out of shared memory
// and the output rows are host memory (0 when every query's arrivals are shared).
static size_t arr_rows_bytes(const Plan &p) {
    return p.mem == 0 ? 0 : (size_t)p.grid * align_up((size_t)p.vmax, 64) * 4;
}

static int ensure_buffer(void *&buf, size_t &cap, size_t need) {
    if (cap >= need) return EAT_OK;
    if (buf) cudaFree(buf);
    buf = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EAT_ERR_OOM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
    }
    cap = need;
    return EAT_OK;
}

// Runs a batch whose buffers are all device memory.
static int run_batch(const eat_net *const *nets, int n_nets, const int32_t *net_idx,
                     const int32_t *src, const int32_t *ts, int32_t n, int32_t *arr_out,
                     const int64_t *arr_off, void *ws, size_t ws_bytes,
                     const eat_query_opts *o, cudaStream_t st, int32_t *status_override,
                     eat_counters *counters_override, int32_t *arr_rows = nullptr,
                     size_t arr_rows_size = 0) {
    const int dev = nets[0]->device;
    int32_t vmax = 0, vmin = INT32_MAX;
    for (int i = 0; i < n_nets; ++i) {
        vmax = std::max(vmax, nets[i]->host.n_stops);
        vmin = std::min(vmin, nets[i]->host.n_stops);
    }
    Plan p;
    int rc = make_plan(dev, vmax, n, n_nets, o, p, vmin, n_nets == 1 ? nets[0] : nullptr);
    if (rc) return rc;
    if (ws_bytes < p.ws_bytes)
        return fail(EAT_ERR_WORKSPACE, "workspace of " + std::to_string(ws_bytes) +
                                           " bytes, need " + std::to_string(p.ws_bytes));
    if (n == 0) return EAT_OK;
    const int32_t cap = (o && o->max_rounds > 0) ? o->max_rounds : default_round_cap(vmax, p.horizon);
    QueryArgs qa = make_args(p, p.grid, (char *)ws, net_idx, src, ts, n, n_nets, arr_out, arr_off,
                             cap, status_override ? status_override : (o ? o->status : nullptr),
                             counters_override ? counters_override : (o ? o->counters : nullptr));
    if (o && o->idle_cap > 0) qa.idle_cap = o->idle_cap;
    if (arr_rows && p.mem != 0) {
        if (arr_rows_size < arr_rows_bytes(p)) return fail(EAT_ERR_INVALID, "arrival rows too small");
        qa.arr_rows = arr_rows;
        qa.arr_rows_stride = (int64_t)align_up((size_t)p.vmax, 64);
    }
    DeviceGuard guard(dev);
    cudaError_t e = cudaMemsetAsync(qa.work, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (p.order) {
        e = launch_order(ts, n, (int32_t *)((char *)ws + p.off_order), st);
        if (e != cudaSuccess) return cuda_fail(e, "start-order kernel launch");
    }
    NetDev devs[EAT_MAX_NETS];
    for (int i = 0; i < n_nets; ++i) devs[i] = nets[i]->dev;
    e = p.cluster ? launch_cluster(devs[0], qa, p.cluster, p.grid, p.block, p.smem, st)
        : p.pair  ? launch_pair(devs[0], qa, p.grid, p.block, p.smem, st)
        : p.async ? launch_async(devs, n_nets, qa, p.mem, p.grid, p.block, p.smem, st)
                  : launch_cta(devs, n_nets, qa, p.mem, p.grid, p.block, p.smem, st, p.pack);
    if (e != cudaSuccess) return cuda_fail(e, "query kernel launch");
    return EAT_OK;
}

// Launch shape of the serving ring kernel: the round-based per-query kernel with the
// default shape of a full batch over these networks (all blocks the SMs hold),
// frontier bitmaps in shared memory.
int ring_setup(const eat_net *const *nets, int n_nets, RingLaunch &rl) {
    int32_t vmax = 0, vmin = INT32_MAX;
    for (int i = 0; i < n_nets; ++i) {
        vmax = std::max(vmax, nets[i]->host.n_stops);
        vmin = std::min(vmin, nets[i]->host.n_stops);
    }
    DeviceInfo d;
    int rc = device_info(nets[0]->device, d);
    if (rc) return rc;
    eat_query_opts o{};
    o.mode = EAT_MODE_CTA;
    Plan p;
    rc = make_plan(nets[0]->device, vmax, 4 * d.sms, n_nets, &o, p, vmin, nullptr, false);
    if (rc) return rc;
    if (p.mem == 2)
        return fail(EAT_ERR_INVALID, "ring admission keeps the frontier bitmaps in shared memory; "
                                     "these networks are too large (use EAT_ADMIT_BATCH)");
    int per_sm = 0;
    {
        DeviceGuard guard(nets[0]->device);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ring_kernel(p.mem),
                                                                      p.block, p.smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    }
    if (per_sm < 1) return fail(EAT_ERR_INVALID, "ring kernel does not fit on an SM");
    rl.mem = p.mem;
    rl.block = p.block;
    rl.grid = per_sm * d.sms;
    rl.smem = p.smem;
    rl.vmax = p.vmax;
    rl.vw_log2 = p.vw_log2;
    rl.qcap = p.qcap;
    rl.mask_words = p.mask_words;
    rl.smem_mask_off = p.smem_mask_off;
    rl.smem_q_off = p.smem_q_off;
    rl.smem_arr_cap = p.smem_arr_cap;
    rl.spill_stride = p.spill_stride;
    rl.ws_bytes = kWsHeader + (size_t)rl.grid * (size_t)p.spill_stride * 4;
    rl.rows_stride = p.mem == 0 ? 0 : (int64_t)align_up((size_t)p.vmax, 64);
    rl.rows_bytes = (size_t)rl.grid * (size_t)rl.rows_stride * 4;
    return EAT_OK;
}

int ring_launch(const eat_net *const *nets, int n_nets, const RingLaunch &rl, void *ws,
                int32_t *arr_rows, int32_t *pool, const RingArgs &rg, cudaStream_t st) {
    Plan p;
    p.mem = rl.mem;
    p.block = rl.block;
    p.vw_log2 = rl.vw_log2;
    p.vmax = rl.vmax;
    p.qcap = rl.qcap;
    p.mask_words = rl.mask_words;
    p.smem_mask_off = rl.smem_mask_off;
    p.smem_q_off = rl.smem_q_off;
    p.smem_arr_cap = rl.smem_arr_cap;
    p.spill_stride = rl.spill_stride;
    p.mask_stride = 0;
    QueryArgs qa = make_args(p, rl.grid, (char *)ws, nullptr, nullptr, nullptr, 0, n_nets, pool,
                             nullptr, default_round_cap(rl.vmax, p.horizon), nullptr, nullptr);
    qa.rg = rg;
    if (rl.mem != 0) {
        qa.arr_rows = arr_rows;
        qa.arr_rows_stride = rl.rows_stride;
    }
    NetDev devs[EAT_MAX_NETS];
    for (int i = 0; i < n_nets; ++i) devs[i] = nets[i]->dev;
    DeviceGuard guard(nets[0]->device);
    cudaError_t e = launch_ring(devs, n_nets, qa, rl.mem, rl.grid, rl.block, rl.smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "ring kernel launch");
    return EAT_OK;
}

}  // namespace eat

using namespace eat;

extern "C" {

const char *eat_last_error(void) { return g_err.c_str(); }

int32_t eat_version(void) { return 100; }

}  // extern "C"

namespace eat {

// Upload a built network (logical arrays already in net->host) to its device.
static int upload(eat_net *net) {
    int rc = build_fused(net->host);
    if (rc) return rc;
    if (net->device < 0) return EAT_OK;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || net->device >= count) {
        cudaGetLastError();
        return fail(EAT_ERR_NO_DEVICE, "no CUDA device " + std::to_string(net->device));
    }
    const HostNet &h = net->host;
    size_t off_row = 0;
    size_t off_tr = align_up(off_row + ((size_t)h.n_stops + 1) * 4, 256);
    size_t off_ce = align_up(off_tr + h.tr.size() * 4, 256);
    size_t off_apx = align_up(off_ce + h.ce.size() * 4, 256);
    size_t total = align_up(off_apx + h.apx.size() * 4 + 16, 256);
    DeviceGuard guard(net->device);
    if (!guard.ok) return fail(EAT_ERR_NO_DEVICE, "cudaSetDevice failed");
    e = cudaMalloc(&net->blob, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        net->blob = nullptr;
        return fail(EAT_ERR_OOM, "cudaMalloc of the network failed");
    }
    net->blob_bytes = (int64_t)total;
    char *b = (char *)net->blob;
    struct Piece { size_t off; const void *src; size_t bytes; } pieces[] = {
        {off_row, h.row_ptr.data(), h.row_ptr.size() * 4},
        {off_tr, h.tr.data(), h.tr.size() * 4},
        {off_ce, h.ce.data(), h.ce.size() * 4},
        {off_apx, h.apx.data(), h.apx.size() * 4},
    };
    for (const Piece &pc : pieces) {
        if (!pc.bytes) continue;
        e = cudaMemcpy(b + pc.off, pc.src, pc.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy of the network");
    }
    NetDev &d = net->dev;
    d.row_ptr = (const int32_t *)(b + off_row);
    d.tr = (const int4 *)(b + off_tr);
    d.ce = (const int4 *)(b + off_ce);
    d.apx = (const uint2 *)(b + off_apx);
    d.n_stops = h.n_stops;
    d.n_types = h.n_types;
    d.t0 = h.t0;
    d.width = h.width;
    d.inv_width = 1.0f / (float)h.width;
    d.k_min = h.k_min;
    d.y = h.y;
    return EAT_OK;
}

}  // namespace eat

extern "C" {

int eat_build(const eat_connections *conn, const eat_build_opts *opts, eat_net **out) {
    clear_error();
    if (!out) return fail(EAT_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (!conn) return fail(EAT_ERR_INVALID, "conn must not be NULL");
    eat_build_opts o{};
    if (opts) o = *opts;
    const int32_t width = o.cluster_width ? o.cluster_width : 3600;
    eat_net *net = new (std::nothrow) eat_net();
    if (!net) return fail(EAT_ERR_OOM, "host allocation failed");
    int rc = EAT_OK;
    if (o.subtrips != EAT_SUBTRIPS_NONE) {
        // Check the plain input first so that errors name the caller's connections.
        eat_connections plain = *conn;
        plain.trip = nullptr;
        eat::HostNet scratch;
        rc = build_host(&plain, width, o.t0, scratch);
        std::vector<int32_t> u, v, dep, dur;
        int64_t added = 0;
        if (!rc) rc = add_subtrips(conn, o.subtrips, u, v, dep, dur, added);
        if (!rc) {
            eat_connections aug{conn->n_stops, (int64_t)u.size(), u.data(), v.data(), dep.data(),
                                dur.data(), nullptr};
            rc = build_host(&aug, width, o.t0, net->host);
            net->host.n_shortcuts = added;
        }
    } else {
        rc = build_host(conn, width, o.t0, net->host);
    }
    net->device = o.device;
    if (!rc) rc = upload(net);
    if (rc) {
        eat_free(net);
        return rc;
    }
    *out = net;
    return EAT_OK;
}

int eat_build_csr(const eat_csr_input *in, const eat_build_opts *opts, eat_net **out) {
    clear_error();
    if (!out) return fail(EAT_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (!in) return fail(EAT_ERR_INVALID, "input must not be NULL");
    eat_build_opts o{};
    if (opts) o = *opts;
    if (o.subtrips != EAT_SUBTRIPS_NONE)
        return fail(EAT_ERR_INVALID, "sub-trips need raw connections (use eat_build)");
    const int32_t width = o.cluster_width ? o.cluster_width : 3600;
    eat_net *net = new (std::nothrow) eat_net();
    if (!net) return fail(EAT_ERR_OOM, "host allocation failed");
    int rc = build_host_csr(in, width, o.t0, net->host);
    net->device = o.device;
    if (!rc) rc = upload(net);
    if (rc) {
        eat_free(net);
        return rc;
    }
    *out = net;
    return EAT_OK;
}

void eat_free(eat_net *net) {
    if (!net) return;
    if (net->device >= 0) {
        DeviceGuard guard(net->device);
        if (net->blob) cudaFree(net->blob);
        if (net->ws) cudaFree(net->ws);
        if (net->stage) cudaFree(net->stage);
    }
    delete net;
}

int eat_get_stats(const eat_net *net, eat_stats *out) {
    clear_error();
    if (!net || !out) return fail(EAT_ERR_INVALID, "NULL argument");
    const HostNet &h = net->host;
    out->n_stops = h.n_stops;
    out->n_types = h.n_types;
    out->n_edges = h.n_edges;
    out->cluster_width = h.width;
    out->t0 = h.t0;
    out->max_clusters = h.max_clusters;
    out->max_out_types = h.max_out_types;
    out->device = net->device;
    out->n_conn = h.n_conn;
    out->n_ap = (int64_t)h.ap.size() / 2;
    out->n_cl = (int64_t)h.cl.size();
    out->device_bytes = net->blob_bytes;
    out->k_min = h.k_min;
    out->y = h.y;
    out->n_ap_extra = (int64_t)h.apx.size() / 2;
    out->n_shortcuts = h.n_shortcuts;
    return EAT_OK;
}

int eat_net_host_view(const eat_net *net, eat_net_view *out) {
    clear_error();
    if (!net || !out) return fail(EAT_ERR_INVALID, "NULL argument");
    out->row_ptr = net->host.row_ptr.data();
    out->type_rec = net->host.type_rec.data();
    out->type_cl = net->host.type_cl.data();
    out->cl = net->host.cl.data();
    out->ap = net->host.ap.data();
    out->cluster_entries = net->host.ce.data();
    out->ap_extra = net->host.apx.data();
    out->type_records = net->host.tr.data();
    return EAT_OK;
}

size_t eat_workspace_bytes(const eat_net *const *nets, int32_t n_nets, int32_t n,
                           const eat_query_opts *opts) {
    clear_error();
    if (!nets || n_nets < 1 || n_nets > EAT_MAX_NETS || n < 0) return 0;
    int32_t vmax = 0, vmin = INT32_MAX;
    for (int i = 0; i < n_nets; ++i) {
        if (!nets[i] || nets[i]->device < 0 || nets[i]->device != nets[0]->device) return 0;
        vmax = std::max(vmax, nets[i]->host.n_stops);
        vmin = std::min(vmin, nets[i]->host.n_stops);
    }
    Plan p;
    if (make_plan(nets[0]->device, vmax, n, n_nets, opts, p, vmin, n_nets == 1 ? nets[0] : nullptr))
        return 0;
    return p.ws_bytes;
}

int eat_launch_shape(const eat_net *const *nets, int32_t n_nets, int32_t n,
                     const eat_query_opts *opts, eat_query_opts *shape) {
    clear_error();
    if (!nets || !shape || n_nets < 1 || n_nets > EAT_MAX_NETS || n < 0)
        return fail(EAT_ERR_INVALID, "invalid arguments");
    int32_t vmax = 0, vmin = INT32_MAX;
    for (int i = 0; i < n_nets; ++i) {
        if (!nets[i]) return fail(EAT_ERR_INVALID, "NULL network");
        if (nets[i]->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
        if (nets[i]->device != nets[0]->device) return fail(EAT_ERR_INVALID, "networks on different devices");
        vmax = std::max(vmax, nets[i]->host.n_stops);
        vmin = std::min(vmin, nets[i]->host.n_stops);
    }
    Plan p;
    int rc = make_plan(nets[0]->device, vmax, n, n_nets, opts, p, vmin, n_nets == 1 ? nets[0] : nullptr);
    if (rc) return rc;
    *shape = opts ? *opts : eat_query_opts{};
    shape->block = p.block;
    shape->vwarp = 1 << p.vw_log2;
    shape->mode = p.cluster ? EAT_MODE_CLUSTER : p.pair ? EAT_MODE_PAIR
                  : p.async ? EAT_MODE_ASYNC : p.edge ? EAT_MODE_EDGE : EAT_MODE_CTA;
    shape->cluster = p.cluster;
    shape->order = p.order ? EAT_ORDER_BY_TIME : EAT_ORDER_AS_GIVEN;
    shape->horizon = p.horizon > 0 ? p.horizon : -1;
    return EAT_OK;
}

int eat_query(const eat_net *net, int32_t s, int32_t t_s, int32_t *arr_out,
              eat_counters *counters) {
    clear_error();
    if (!net || !arr_out) return fail(EAT_ERR_INVALID, "NULL argument");
    if (net->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
    if (s < 0 || s >= net->host.n_stops) return fail(EAT_ERR_INVALID, "source out of range");
    if (foreign_ptr(arr_out, net->device)) return foreign_fail();
    std::lock_guard<std::mutex> g(net->ws_lock);
    Plan p;
    int rc = make_plan(net->device, net->host.n_stops, 1, 1, nullptr, p, -1, net);
    if (rc) return rc;
    DeviceGuard guard(net->device);
    // A page-locked host row is written in place; arrivals that do not fit in shared
    // memory then live in the device row below and are copied over at the end.
    const bool dev_out = is_device_ptr(arr_out);
    int32_t *const out_map = dev_out ? nullptr : (int32_t *)mapped_host_ptr(arr_out);
    const size_t rows = dev_out ? 0 : align_up((size_t)net->host.n_stops * 4, 256);
    rc = ensure_buffer(net->ws, net->ws_bytes, p.ws_bytes + rows + 256);
    if (rc) return rc;
    char *w = (char *)net->ws;
    // Internal scratch after the plan's workspace: [src, t_s, status, pad][counters][row].
    int32_t *io = (int32_t *)(w + p.ws_bytes);
    eat_counters *cnt = (eat_counters *)(w + p.ws_bytes + 64);
    int32_t *const dev_row = (int32_t *)(w + p.ws_bytes + 256);
    int32_t *row = dev_out ? arr_out : out_map ? out_map : dev_row;
    int32_t h_io[2] = {s, t_s};
    cudaError_t e = cudaMemcpyAsync(io, h_io, sizeof(h_io), cudaMemcpyHostToDevice, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    const eat_net *nets[1] = {net};
    rc = run_batch(nets, 1, nullptr, io, io + 1, 1, row, nullptr, w, p.ws_bytes, nullptr, 0,
                   io + 2, cnt, out_map ? dev_row : nullptr, rows);
    if (rc) return rc;
    int32_t st_h = 0;
    e = cudaMemcpyAsync(&st_h, io + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, 0);
    if (e == cudaSuccess && counters)
        e = cudaMemcpyAsync(counters, cnt, sizeof(eat_counters), cudaMemcpyDeviceToHost, 0);
    if (e == cudaSuccess && !dev_out && !out_map)
        e = cudaMemcpyAsync(arr_out, row, (size_t)net->host.n_stops * 4, cudaMemcpyDeviceToHost, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cuda_fail(e, "eat_query");
    if (st_h == EAT_ERR_NO_CONVERGENCE) return fail(st_h, "round cap reached");
    if (st_h) return fail(st_h, "query failed");
    return EAT_OK;
}

int eat_query_batch_multi(const eat_net *const *nets, int32_t n_nets, const int32_t *net_idx,
                          const int32_t *sources, const int32_t *times, int32_t n,
                          int32_t *arr_out, const int64_t *arr_offsets, void *workspace,
                          size_t workspace_bytes, const eat_query_opts *opts, void *stream) {
    clear_error();
    if (!nets || n_nets < 1 || n_nets > EAT_MAX_NETS) return fail(EAT_ERR_INVALID, "bad nets");
    for (int i = 0; i < n_nets; ++i) {
        if (!nets[i]) return fail(EAT_ERR_INVALID, "NULL network");
        if (nets[i]->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
        if (nets[i]->device != nets[0]->device)
            return fail(EAT_ERR_INVALID, "all networks must be on one device");
    }
    if (n < 0) return fail(EAT_ERR_INVALID, "n must be >= 0");
    if (n > 0 && (!net_idx || !sources || !times || !arr_out || !arr_offsets))
        return fail(EAT_ERR_INVALID, "NULL query array");
    for (const void *b : {(const void *)net_idx, (const void *)sources, (const void *)times,
                          (const void *)arr_out, (const void *)arr_offsets, (const void *)workspace})
        if (foreign_ptr(b, nets[0]->device)) return foreign_fail();
    DeviceGuard guard(nets[0]->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev_in = n == 0 || is_device_ptr(sources);
    const bool dev_out = n == 0 || is_device_ptr(arr_out);
    if (n > 0 && (is_device_ptr(net_idx) != dev_in || is_device_ptr(times) != dev_in ||
                  is_device_ptr(arr_offsets) != dev_in))
        return fail(EAT_ERR_INVALID, "query arrays must all be host or all device memory");
    if (!dev_out && dev_in)
        return fail(EAT_ERR_INVALID, "a host arr_out needs host query arrays");
    if (dev_in) {
        if (!workspace) {
            std::lock_guard<std::mutex> g(nets[0]->ws_lock);
            size_t need = eat_workspace_bytes(nets, n_nets, n, opts);
            if (!need) return EAT_ERR_INVALID;
            int rc = ensure_buffer(nets[0]->ws, nets[0]->ws_bytes, need);
            if (rc) return rc;
            return run_batch(nets, n_nets, net_idx, sources, times, n, arr_out, arr_offsets,
                             nets[0]->ws, nets[0]->ws_bytes, opts, st, nullptr, nullptr);
        }
        return run_batch(nets, n_nets, net_idx, sources, times, n, arr_out, arr_offsets, workspace,
                         workspace_bytes, opts, st, nullptr, nullptr);
    }
    // Host query arrays: validate here, stage them (and a host arr_out) through device memory.
    int64_t out_elems = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (net_idx[i] < 0 || net_idx[i] >= n_nets) return fail(EAT_ERR_INVALID, "net_idx out of range");
        if (sources[i] < 0 || sources[i] >= nets[net_idx[i]]->host.n_stops)
            return fail(EAT_ERR_INVALID, "source out of range");
        if (arr_offsets[i] < 0) return fail(EAT_ERR_INVALID, "negative arr_offsets entry");
        out_elems = std::max(out_elems, arr_offsets[i] + nets[net_idx[i]]->host.n_stops);
    }
    std::lock_guard<std::mutex> g(nets[0]->ws_lock);
    // A page-locked (mapped) arr_out is written in place by the kernel, with per-block
    // device rows for arrivals that do not fit in shared memory; else rows are staged.
    int32_t *out_map = dev_out ? nullptr : (int32_t *)mapped_host_ptr(arr_out);
    size_t rows_bytes = 0;
    if (out_map) {
        int32_t vmax = 0, vmin = INT32_MAX;
        for (int i = 0; i < n_nets; ++i) {
            vmax = std::max(vmax, nets[i]->host.n_stops);
            vmin = std::min(vmin, nets[i]->host.n_stops);
        }
        Plan p;
        if (make_plan(nets[0]->device, vmax, n, n_nets, opts, p, vmin, n_nets == 1 ? nets[0] : nullptr)) {
            clear_error();
            out_map = nullptr;
        } else {
            rows_bytes = arr_rows_bytes(p);
        }
    }
    const size_t in_bytes = align_up((size_t)n * 4, 256) * 3 + align_up((size_t)n * 8, 256);
    const size_t out_bytes = dev_out ? 0 : out_map ? rows_bytes : (size_t)out_elems * 4;
    int rc = ensure_buffer(nets[0]->stage, nets[0]->stage_bytes, in_bytes + out_bytes);
    if (rc) return rc;
    char *sb = (char *)nets[0]->stage;
    int32_t *d_idx = (int32_t *)sb;
    int32_t *d_src = (int32_t *)(sb + align_up((size_t)n * 4, 256));
    int32_t *d_ts = (int32_t *)(sb + 2 * align_up((size_t)n * 4, 256));
    int64_t *d_off = (int64_t *)(sb + 3 * align_up((size_t)n * 4, 256));
    cudaError_t e = cudaMemcpyAsync(d_idx, net_idx, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_src, sources, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ts, times, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, arr_offsets, (size_t)n * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    void *ws = workspace;
    size_t wsb = workspace_bytes;
    if (!ws) {
        size_t need = eat_workspace_bytes(nets, n_nets, n, opts);
        if (!need) return EAT_ERR_INVALID;
        rc = ensure_buffer(nets[0]->ws, nets[0]->ws_bytes, need);
        if (rc) return rc;
        ws = nets[0]->ws;
        wsb = nets[0]->ws_bytes;
    }
    int32_t *out_d = dev_out ? arr_out : out_map ? out_map : (int32_t *)(sb + in_bytes);
    rc = run_batch(nets, n_nets, d_idx, d_src, d_ts, n, out_d, d_off, ws, wsb, opts, st,
                   nullptr, nullptr, rows_bytes ? (int32_t *)(sb + in_bytes) : nullptr, rows_bytes);
    if (rc) return rc;
    if (!dev_out && !out_map)
        e = cudaMemcpyAsync(arr_out, out_d, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "eat_query_batch_multi");
    return EAT_OK;
}

int eat_query_batch(const eat_net *net, const int32_t *sources, const int32_t *times, int32_t n,
                    int32_t *arr_out, void *workspace, size_t workspace_bytes,
                    const eat_query_opts *opts, void *stream) {
    clear_error();
    if (!net) return fail(EAT_ERR_INVALID, "NULL network");
    if (net->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
    if (n < 0) return fail(EAT_ERR_INVALID, "n must be >= 0");
    if (n == 0) return EAT_OK;
    if (!sources || !times || !arr_out) return fail(EAT_ERR_INVALID, "NULL query array");
    for (const void *b : {(const void *)sources, (const void *)times, (const void *)arr_out,
                          (const void *)workspace})
        if (foreign_ptr(b, net->device)) return foreign_fail();
    DeviceGuard guard(net->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool d_src = is_device_ptr(sources), d_ts = is_device_ptr(times), d_out = is_device_ptr(arr_out);
    const eat_net *nets[1] = {net};
    if (d_src && d_ts && d_out) {
        if (!workspace) {
            std::lock_guard<std::mutex> g(net->ws_lock);
            size_t need = eat_workspace_bytes(nets, 1, n, opts);
            if (!need) return EAT_ERR_INVALID;
            int rc = ensure_buffer(net->ws, net->ws_bytes, need);
            if (rc) return rc;
            return run_batch(nets, 1, nullptr, sources, times, n, arr_out, nullptr, net->ws,
                             net->ws_bytes, opts, st, nullptr, nullptr);
        }
        return run_batch(nets, 1, nullptr, sources, times, n, arr_out, nullptr, workspace,
                         workspace_bytes, opts, st, nullptr, nullptr);
    }
    // At least one host buffer.  Page-locked (mapped) host buffers are used in place:
    // the kernel reads the queries and writes each converged row straight to host
    // memory, so the rows travel while other queries still run (arrivals that do not
    // fit in shared memory live in a per-block device row meanwhile).  Other host
    // buffers are staged through device memory.  Either way the call returns after
    // the rows are in arr_out.
    if (!d_src)
        for (int32_t i = 0; i < n; ++i)
            if (sources[i] < 0 || sources[i] >= net->host.n_stops)
                return fail(EAT_ERR_INVALID, "source out of range");
    std::lock_guard<std::mutex> g(net->ws_lock);
    int32_t *out_map = d_out ? nullptr : (int32_t *)mapped_host_ptr(arr_out);
    size_t rows_bytes = 0;                       // per-block arrival rows (host rows only)
    if (out_map) {
        Plan p;
        if (make_plan(net->device, net->host.n_stops, n, 1, opts, p, -1, net) != EAT_OK) {
            clear_error();
            out_map = nullptr;
        } else {
            rows_bytes = arr_rows_bytes(p);
        }
    }
    const int32_t *src_map = (out_map && !d_src) ? (const int32_t *)mapped_host_ptr(sources) : nullptr;
    const int32_t *ts_map = (out_map && !d_ts) ? (const int32_t *)mapped_host_ptr(times) : nullptr;
    const bool direct_out = d_out || out_map;
    const size_t in_bytes = align_up((size_t)n * 4, 256);
    const size_t out_bytes = (size_t)n * (size_t)net->host.n_stops * 4;
    int rc = ensure_buffer(net->stage, net->stage_bytes,
                           2 * in_bytes + (direct_out ? rows_bytes : out_bytes));
    if (rc) return rc;
    char *sb = (char *)net->stage;
    const int32_t *src_d = d_src ? sources : src_map ? src_map : (const int32_t *)sb;
    const int32_t *ts_d = d_ts ? times : ts_map ? ts_map : (const int32_t *)(sb + in_bytes);
    int32_t *out_d = d_out ? arr_out : out_map ? out_map : (int32_t *)(sb + 2 * in_bytes);
    cudaError_t e = cudaSuccess;
    if (!d_src && !src_map)
        e = cudaMemcpyAsync((void *)src_d, sources, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !d_ts && !ts_map)
        e = cudaMemcpyAsync((void *)ts_d, times, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    void *ws = workspace;
    size_t wsb = workspace_bytes;
    if (!ws) {
        size_t need = eat_workspace_bytes(nets, 1, n, opts);
        if (!need) return EAT_ERR_INVALID;
        rc = ensure_buffer(net->ws, net->ws_bytes, need);
        if (rc) return rc;
        ws = net->ws;
        wsb = net->ws_bytes;
    }
    rc = run_batch(nets, 1, nullptr, src_d, ts_d, n, out_d, nullptr, ws, wsb, opts, st, nullptr,
                   nullptr, rows_bytes ? (int32_t *)(sb + 2 * in_bytes) : nullptr, rows_bytes);
    if (rc) return rc;
    if (!direct_out) e = cudaMemcpyAsync(arr_out, out_d, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "eat_query_batch");
    return EAT_OK;
}

int eat_next_departure(const eat_net *net, const int32_t *types, const int32_t *times, int32_t n,
                       int32_t *out, void *stream) {
    clear_error();
    if (!net) return fail(EAT_ERR_INVALID, "NULL network");
    if (net->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
    if (n < 0) return fail(EAT_ERR_INVALID, "n must be >= 0");
    if (n == 0) return EAT_OK;
    if (!types || !times || !out) return fail(EAT_ERR_INVALID, "NULL argument");
    for (const void *b : {(const void *)types, (const void *)times, (const void *)out})
        if (foreign_ptr(b, net->device)) return foreign_fail();
    DeviceGuard guard(net->device);
    cudaError_t e = launch_next_departure(net->dev, types, times, n, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "next-departure kernel launch");
    return EAT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ autotuning

namespace eat {

struct TuneCand {
    int m, b, v, ord;            // mode, block, vwarp, start order (EAT_ORDER_*)
    int h;                       // horizon (s), 0 = none
    std::vector<float> ms;
};

static eat_query_opts cand_opts(const TuneCand &cd) {
    eat_query_opts o{};
    o.block = cd.b;
    o.vwarp = cd.v;
    o.mode = cd.m;
    o.order = cd.ord;
    o.horizon = cd.h > 0 ? cd.h : -1;    // none, not a horizon tuned earlier
    return o;
}

// Times every candidate with run(opts, workspace, rows) on `st` in nine rounds over
// all candidates (so that slow drift of the clock affects all alike): round 0 warms
// up, rounds 1..8 are timed with CUDA events, each after a write of twice the L2
// size so that every timing starts with the networks out of cache.  The earliest
// candidate whose median is within 5 % of the least median wins (closer differences
// are within the spread between batches of one workload), so that repeated tuning
// settles on one shape.  Allocates its scratch (workspace, rows, flush buffer) for
// the duration of the call.
template <class Run>
static int time_candidates(int dev, std::vector<TuneCand> &cands, size_t ws_need, size_t rows_bytes,
                           cudaStream_t st, const Run &run, TuneCand &best) {
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const size_t flush_bytes = std::max<size_t>(2 * (size_t)std::max(l2, 0), 64u << 20);
    void *ws = nullptr, *rows = nullptr, *flush = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&ws, std::max<size_t>(ws_need, 256));
    if (e == cudaSuccess) e = cudaMalloc(&rows, std::max<size_t>(rows_bytes, 256));
    if (e == cudaSuccess) e = cudaMalloc(&flush, flush_bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = EAT_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = fail(EAT_ERR_OOM, std::string("autotune scratch: ") + cudaGetErrorString(e));
    }
    constexpr int kTimed = 8;
    for (int rep = 0; rep <= kTimed && !rc; ++rep) {
        for (TuneCand &cd : cands) {
            if (rep > 0) {
                e = cudaMemsetAsync(flush, rep & 0xff, flush_bytes, st);
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune timing");
                    break;
                }
            }
            const eat_query_opts o = cand_opts(cd);
            rc = run(o, ws, ws_need, (int32_t *)rows);
            if (rc) break;
            if (rep > 0) {
                float ms = 0.f;
                e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune timing");
                    break;
                }
                cd.ms.push_back(ms);
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ws) cudaFree(ws);
    if (rows) cudaFree(rows);
    if (flush) cudaFree(flush);
    if (rc) return rc;
    float least = 1e30f;
    for (TuneCand &cd : cands) {
        if (cd.ms.size() != (size_t)kTimed) continue;
        std::sort(cd.ms.begin(), cd.ms.end());
        cd.ms[0] = 0.5f * (cd.ms[kTimed / 2 - 1] + cd.ms[kTimed / 2]);   // median
        least = std::min(least, cd.ms[0]);
    }
    for (const TuneCand &cd : cands) {
        if (cd.ms.size() == (size_t)kTimed && cd.ms[0] <= least * 1.05f) {
            best = cd;
            return EAT_OK;
        }
    }
    return fail(EAT_ERR_INVALID, "no candidate was timed");
}

// Keeps the candidates that have a plan for these networks; ws_need = the largest
// workspace among them.
static int usable_candidates(const eat_net *const *nets, int n_nets, int32_t n,
                             std::vector<TuneCand> &cands, size_t &ws_need) {
    ws_need = 0;
    std::vector<TuneCand> usable;
    for (const TuneCand &cd : cands) {
        const eat_query_opts o = cand_opts(cd);
        const size_t need = eat_workspace_bytes(nets, n_nets, n, &o);
        if (!need) continue;
        ws_need = std::max(ws_need, need);
        usable.push_back(cd);
    }
    clear_error();
    if (usable.empty()) return fail(EAT_ERR_INVALID, "no launch shape fits these networks");
    cands.swap(usable);
    return EAT_OK;
}

}  // namespace eat

extern "C" int eat_autotune(eat_net *net, const int32_t *sources, const int32_t *times,
                            int32_t n, eat_query_opts *best, void *stream) {
    clear_error();
    if (!net) return fail(EAT_ERR_INVALID, "NULL network");
    if (net->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
    if (n <= 0 || !sources || !times) return fail(EAT_ERR_INVALID, "empty sample");
    DeviceGuard guard(net->device);
    if (!is_device_ptr(sources) || !is_device_ptr(times))
        return fail(EAT_ERR_INVALID, "sample arrays must be device memory");
    if (foreign_ptr(sources, net->device) || foreign_ptr(times, net->device)) return foreign_fail();
    cudaStream_t st = (cudaStream_t)stream;
    const eat_net *nets[1] = {net};
    std::vector<TuneCand> cands;
    // Fixed order, the library's default shape first (rounds, vwarp 8, 1,024 threads on
    // networks of 8,192 stops or more, else 512): ties go to the earliest.
    DeviceInfo dinfo;
    int drc = device_info(net->device, dinfo);
    if (drc) return drc;
    std::vector<TuneCand> pairs;
    if (n > dinfo.sms) {
        eat_query_opts o{};
        o.mode = EAT_MODE_PAIR;
        if (eat_workspace_bytes(nets, 1, n, &o))
            for (int v : {8, 4, 16}) pairs.push_back({EAT_MODE_PAIR, 1024, v, EAT_ORDER_AUTO, 0, {}});
        else clear_error();                  // network too large for two rows per block
    }
    const bool wide = net->host.n_stops >= kWideMinStops || n <= dinfo.sms;
    for (int b : {wide ? 1024 : 512, wide ? 512 : 1024, 256}) {
        for (int v : {8, 4, 16, 2, 32}) cands.push_back({EAT_MODE_CTA, b, v, EAT_ORDER_AUTO, 0, {}});
        cands.push_back({EAT_MODE_ASYNC, b, 8, EAT_ORDER_AUTO, 0, {}});
        for (int v : {8, 32}) cands.push_back({EAT_MODE_EDGE, b, v, EAT_ORDER_AUTO, 0, {}});
    }
    cands.insert(cands.end(), pairs.begin(), pairs.end());
    // Horizons (1, 2, 4 and 12 hours) with the first two block sizes and vwarp 8.
    for (int b : {wide ? 1024 : 512, wide ? 512 : 1024})
        for (int h : {3600, 7200, 14400, 43200})
            cands.push_back({EAT_MODE_CTA, b, 8, EAT_ORDER_AUTO, h, {}});
    size_t ws_need = 0;
    int rc = usable_candidates(nets, 1, n, cands, ws_need);
    if (rc) return rc;
    TuneCand win{EAT_MODE_CTA, 512, 8, EAT_ORDER_AUTO, 0, {}};
    rc = time_candidates(net->device, cands, ws_need, (size_t)n * (size_t)net->host.n_stops * 4, st,
                         [&](const eat_query_opts &o, void *ws, size_t wsb, int32_t *rows) {
                             return run_batch(nets, 1, nullptr, sources, times, n, rows, nullptr,
                                              ws, wsb, &o, st, nullptr, nullptr);
                         },
                         win);
    if (rc) return rc;
    int cls = 0;
    while (cls < 31 && (1 << (cls + 1)) <= n) ++cls;
    net->tuned[cls].store((uint64_t)win.b | (uint64_t)win.v << 16 | (uint64_t)win.m << 24 |
                              (uint64_t)(uint32_t)win.h << 32,
                          std::memory_order_relaxed);
    if (best) {
        *best = eat_query_opts{};
        best->block = win.b;
        best->vwarp = win.v;
        best->mode = win.m;
        best->horizon = win.h > 0 ? win.h : -1;
    }
    return EAT_OK;
}

extern "C" int eat_autotune_multi(const eat_net *const *nets, int32_t n_nets, const int32_t *net_idx,
                                  const int32_t *sources, const int32_t *times, int32_t n,
                                  eat_query_opts *best, void *stream) {
    clear_error();
    if (!best) return fail(EAT_ERR_INVALID, "best must not be NULL");
    if (!nets || n_nets < 1 || n_nets > EAT_MAX_NETS) return fail(EAT_ERR_INVALID, "bad nets");
    for (int i = 0; i < n_nets; ++i) {
        if (!nets[i]) return fail(EAT_ERR_INVALID, "NULL network");
        if (nets[i]->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
        if (nets[i]->device != nets[0]->device)
            return fail(EAT_ERR_INVALID, "all networks must be on one device");
    }
    if (n <= 0 || !net_idx || !sources || !times) return fail(EAT_ERR_INVALID, "empty sample");
    const int dev = nets[0]->device;
    DeviceGuard guard(dev);
    if (!is_device_ptr(net_idx) || !is_device_ptr(sources) || !is_device_ptr(times))
        return fail(EAT_ERR_INVALID, "sample arrays must be device memory");
    for (const void *b : {(const void *)net_idx, (const void *)sources, (const void *)times})
        if (foreign_ptr(b, dev)) return foreign_fail();
    cudaStream_t st = (cudaStream_t)stream;
    // Output rows packed in query order: offsets from the sample's network indices.
    std::vector<int32_t> idx((size_t)n);
    cudaError_t e = cudaMemcpy(idx.data(), net_idx, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy of the sample's network indices");
    std::vector<int64_t> offs((size_t)n);
    int64_t total = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (idx[i] < 0 || idx[i] >= n_nets) return fail(EAT_ERR_INVALID, "net_idx out of range");
        offs[i] = total;
        total += nets[idx[i]]->host.n_stops;
    }
    int64_t *d_offs = nullptr;
    e = cudaMalloc(&d_offs, (size_t)n * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(EAT_ERR_OOM, "autotune scratch (row offsets)");
    }
    e = cudaMemcpy(d_offs, offs.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_offs);
        return cuda_fail(e, "cudaMemcpy of the row offsets");
    }
    // Candidates in a fixed order, the library's default for a batch over several
    // networks first (512 threads, vwarp 8, index order): block sizes 512, 1,024 and
    // 256, each with vwarp 8, 4, 16, 2, 32, the round-free mode and the edge mode, each
    // in index order and then in order of t_s; then horizons of 2 and 12 hours (512
    // threads, vwarp 8, in order of t_s).
    std::vector<TuneCand> cands;
    for (int ord : {EAT_ORDER_AS_GIVEN, EAT_ORDER_BY_TIME})
        for (int b : {512, 1024, 256}) {
            for (int v : {8, 4, 16, 2, 32}) cands.push_back({EAT_MODE_CTA, b, v, ord, 0, {}});
            cands.push_back({EAT_MODE_ASYNC, b, 8, ord, 0, {}});
            cands.push_back({EAT_MODE_EDGE, b, 8, ord, 0, {}});
        }
    for (int h : {7200, 43200}) cands.push_back({EAT_MODE_CTA, 512, 8, EAT_ORDER_BY_TIME, h, {}});
    size_t ws_need = 0;
    int rc = usable_candidates(nets, n_nets, n, cands, ws_need);
    TuneCand win{EAT_MODE_CTA, 512, 8, EAT_ORDER_AS_GIVEN, 0, {}};
    if (!rc)
        rc = time_candidates(dev, cands, ws_need, (size_t)total * 4, st,
                             [&](const eat_query_opts &o, void *ws, size_t wsb, int32_t *rows) {
                                 return run_batch(nets, n_nets, net_idx, sources, times, n, rows,
                                                  d_offs, ws, wsb, &o, st, nullptr, nullptr);
                             },
                             win);
    cudaFree(d_offs);
    if (rc) return rc;
    *best = eat_query_opts{};
    best->block = win.b;
    best->vwarp = win.v;
    best->mode = win.m;
    best->order = win.ord;
    best->horizon = win.h > 0 ? win.h : -1;
    return EAT_OK;
}

// ------------------------------------------------------------------ no-allocation entry point

// Fixed scratch for eat_query_batch_noalloc: the work counter (first 256 bytes)
// and the per-block frontier queues.  In host code this name is only a stand-in
// for the device array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[EAT_NOALLOC_SCRATCH_BYTES];

namespace eat {

static std::mutex g_noalloc_lock;
static void *g_noalloc_ptr[64];

// Looks up the scratch array's device address once per device (the device is
// current when this runs).
static int noalloc_scratch(int dev, void **out) {
    std::lock_guard<std::mutex> g(g_noalloc_lock);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return EAT_OK;
}

}  // namespace eat

extern "C" int eat_query_batch_noalloc(const eat_net *net, const int32_t *sources,
                                       const int32_t *times, int32_t n, int32_t *arr_out,
                                       const eat_query_opts *opts, void *stream) {
    clear_error();
    if (!net) return fail(EAT_ERR_INVALID, "NULL network");
    if (net->device < 0) return fail(EAT_ERR_NO_DEVICE, "network was built host-only");
    if (net->device >= 64) return fail(EAT_ERR_INVALID, "device ordinal out of range");
    if (n < 0) return fail(EAT_ERR_INVALID, "n must be >= 0");
    if (net->host.n_stops > EAT_NOALLOC_MAX_STOPS)
        return fail(EAT_ERR_INVALID, "network has " + std::to_string(net->host.n_stops) +
                                         " stops; the no-allocation scratch (16 MiB) serves at most " +
                                         std::to_string(EAT_NOALLOC_MAX_STOPS));
    if (n == 0) return EAT_OK;
    if (!sources || !times || !arr_out) return fail(EAT_ERR_INVALID, "NULL query array");
    DeviceGuard guard(net->device);
    if (!is_device_ptr(sources) || !is_device_ptr(times) || !is_device_ptr(arr_out))
        return fail(EAT_ERR_INVALID, "sources, times and arr_out must be device memory");
    for (const void *b : {(const void *)sources, (const void *)times, (const void *)arr_out})
        if (foreign_ptr(b, net->device)) return foreign_fail();
    Plan p;
    int rc = make_plan(net->device, net->host.n_stops, n, 1, opts, p, -1, net, false);
    if (rc) return rc;
    // Fewer persistent blocks so that their queue spill fits the fixed scratch.
    const size_t per_block = (size_t)p.spill_stride * 4 + (size_t)p.mask_stride * 4;
    const size_t fit = per_block ? (EAT_NOALLOC_SCRATCH_BYTES - kWsHeader) / per_block : (size_t)p.grid;
    if (fit < 1)
        return fail(EAT_ERR_INVALID, "network too large for the no-allocation scratch");
    const int grid = (int)std::min<size_t>((size_t)p.grid, fit);
    void *scratch = nullptr;
    rc = noalloc_scratch(net->device, &scratch);
    if (rc) return rc;
    const int32_t cap = (opts && opts->max_rounds > 0) ? opts->max_rounds
                                                       : default_round_cap(net->host.n_stops, p.horizon);
    QueryArgs qa = make_args(p, grid, (char *)scratch, nullptr, sources, times, n, 1, arr_out,
                             nullptr, cap, opts ? opts->status : nullptr,
                             opts ? opts->counters : nullptr);
    if (opts && opts->idle_cap > 0) qa.idle_cap = opts->idle_cap;
    cudaStream_t st = (cudaStream_t)stream;
    // The query counter must start at zero; the queues need no clearing.
    cudaError_t e = cudaMemsetAsync(qa.work, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(no-allocation scratch)");
    e = p.pair    ? launch_pair(net->dev, qa, grid, p.block, p.smem, st)
        : p.async ? launch_async(&net->dev, 1, qa, p.mem, grid, p.block, p.smem, st)
                  : launch_cta(&net->dev, 1, qa, p.mem, grid, p.block, p.smem, st, p.pack);
    if (e != cudaSuccess) return cuda_fail(e, "query kernel launch");
    return EAT_OK;
}
