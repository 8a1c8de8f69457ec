/*
 * eat.h -- C ABI of libeat: earliest-arrival-time (EAT) queries on public
 * transport timetables, computed on one NVIDIA GB300 (sm_103a) GPU.
 *
 * Method: "GPU Algorithm for Earliest Arrival Time Problem in Public Transport
 * Networks" (arXiv 1912.00966).
 *   - Problem (Section I and Section I-A, Preliminaries): a connection
 *     (u, v, t, lambda) leaves stop u at time t and reaches v at t + lambda.
 *     For a query (s, t_s), e[v] is the earliest arrival at v over
 *     time-respecting paths that leave s at or after t_s; e[s] = t_s.
 *   - Data structure (Section III-A): connections of one edge (u, v) with one
 *     duration form a connection type (Section II-B); each type's departures
 *     are split into clusters of `cluster_width` seconds (one hour in the
 *     paper, Section II-D) and each cluster is stored as arithmetic
 *     progressions (Section I-A, Arithmetic Progression Technique; Section II-C).
 *   - Query (Algorithms 2, 3 and 5 with the Cluster-AP lookup of Section II-D,
 *     the double-buffered activity of Section III-B and atomicMin of Section
 *     III-C): rounds relax the connection types whose tail stop improved in the
 *     previous round until no arrival changes.
 *
 * Conventions
 *   - Times are int32 seconds.  EAT_INF (INT32_MAX) marks an unreachable stop.
 *   - Stops are numbered 0 .. n_stops-1.
 *   - Every function returns EAT_OK (0) or one of the EAT_ERR_* codes;
 *     eat_last_error() returns a message for the calling thread's last error.
 *   - "device memory" means memory of the network's CUDA device (cudaMalloc,
 *     torch CUDA tensors); "host memory" is ordinary or pinned CPU memory.
 *     Entry points that accept either detect the kind with
 *     cudaPointerGetAttributes; a buffer in device memory of another device is
 *     refused with EAT_ERR_INVALID.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = the
 *     legacy default stream).
 */
#ifndef EAT_H
#define EAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EAT_INF INT32_MAX

enum eat_status {
    EAT_OK = 0,
    EAT_ERR_INVALID = 1,        /* bad argument or input data (message says which) */
    EAT_ERR_OOM = 2,            /* host or device allocation failed */
    EAT_ERR_CUDA = 3,           /* a CUDA runtime call failed (message has the CUDA error) */
    EAT_ERR_NO_CONVERGENCE = 4, /* a query hit its round cap before the fixpoint */
    EAT_ERR_NO_DEVICE = 5,      /* the network was built host-only, or no CUDA device */
    EAT_ERR_WORKSPACE = 6       /* the caller's workspace is smaller than required */
};

/* Opaque network: built once, immutable afterwards, resident on one GPU. */
typedef struct eat_net eat_net;

/* Input timetable: n_conn connections as four parallel int32 arrays in host
 * memory (Section I-A, Preliminaries).  Requirements, checked by eat_build:
 * 0 <= u, v < n_stops; 1 <= dur < 2^24; dep >= t0 (see eat_build_opts);
 * dep + dur < INT32_MAX.  Identical connections are merged.
 * `trip` (nullable) gives each connection's trip (vehicle run, Section II-G);
 * connections with a negative trip id belong to no trip.  The connections of a
 * trip, ordered by departure, must form a time-respecting chain (each one leaves
 * the stop the previous one reached, no earlier than it arrived). */
typedef struct {
    int32_t n_stops;
    int64_t n_conn;
    const int32_t *u;
    const int32_t *v;
    const int32_t *dep;
    const int32_t *dur;
    const int32_t *trip;
} eat_connections;

/* Sub-trip data enhancement (Section II-G). */
enum eat_subtrips {
    EAT_SUBTRIPS_NONE = 0,
    EAT_SUBTRIPS_SQRT_K = 1,     /* trip of k connections: sub-trips of round(sqrt(k)) */
    EAT_SUBTRIPS_SQRT_MEAN = 2   /* every trip: sub-trips of round(sqrt(mean trip length)) */
};

/* Build options.  Zero-initialise for the paper's defaults. */
typedef struct {
    int32_t cluster_width; /* seconds per cluster, 1..65535; 0 = 3600 (Section II-D) */
    int32_t t0;            /* start of cluster 0; departures must be >= t0; default 0 */
    int32_t device;        /* CUDA device ordinal; -1 = host-only build (inspection only) */
    int32_t subtrips;      /* EAT_SUBTRIPS_*; needs conn->trip */
} eat_build_opts;

/* Sizes of a built network. */
typedef struct {
    int32_t n_stops;
    int32_t n_types;        /* connection types C_{u,v,lambda} (Section II-B) */
    int32_t n_edges;        /* distinct (u, v) pairs with connections */
    int32_t cluster_width;
    int32_t t0;
    int32_t max_clusters;   /* y of Section III-A: clusters spanned by the widest type */
    int32_t max_out_types;  /* largest number of types leaving one stop */
    int32_t device;         /* -1 for a host-only build */
    int64_t n_conn;         /* connections after merging identical ones */
    int64_t n_ap;           /* AP records */
    int64_t n_cl;           /* cluster-offset entries */
    int64_t device_bytes;   /* bytes of the resident device copy */
    int32_t k_min;          /* device layout: first cluster index stored */
    int32_t y;              /* device layout: clusters stored per type (the paper's y) */
    int64_t n_ap_extra;     /* device layout: APs beyond the four kept in a cluster entry */
    int64_t n_shortcuts;    /* artificial sub-trip connections added (Section II-G) */
} eat_stats;

/* Read-only host view of the built arrays (Section III-A's CT[], CL[], AP[], in
 * this library's layout).  Valid until eat_free.
 *   row_ptr [n_stops + 1]: types leaving stop u are row_ptr[u] .. row_ptr[u+1]-1,
 *                          ordered by (v, lambda).
 *   type_rec[4 * n_types]: per type {v, lambda, first departure, last departure}.
 *   type_cl [n_types]:     cl_base; the APs of cluster k of the type are
 *                          ap[cl[cl_base + k]] .. ap[cl[cl_base + k + 1] - 1] for the
 *                          clusters k between the type's first and last departure;
 *                          a type's APs are contiguous and ordered by cluster, then
 *                          by first term.
 *   cl      [n_cl]
 *   ap      [2 * n_ap]:    per AP {first term, (difference << 16) | number of terms};
 *                          a one-term AP has difference 0. */
typedef struct {
    const int32_t *row_ptr;
    const int32_t *type_rec;
    const int32_t *type_cl;
    const int32_t *cl;
    const uint32_t *ap;
    /* The device layout, derived from the arrays above (Section III-A's CL stride y):
     *   cluster_entries[8 * y * n_types]  entry (t, k) for cluster k_min + k at
     *       record k * n_types + t (cluster-major), one 32-byte record:
     *       {rel0 | rel1 << 16, sc0, sc1, next, x/2 | n << 24, rel2 | rel3 << 16, sc2, sc3}:
     *       the cluster's n APs, the first four inline with first terms base + rel,
     *       base = t0 + (k_min + k) * cluster_width, and sc = difference << 16 | terms,
     *       the others at ap_extra[x ..] (n = 255: the count is the first of two header
     *       slots there); next = first departure of the next non-empty cluster,
     *       EAT_INF if none
     *   ap_extra[2 * n_ap_extra]
     *   type_records[4 * n_types]  per type {v, lambda | d << 24, row_ptr[v], last
     *       departure}: head stop, duration, types leaving v (255: see row_ptr) */
    const int32_t *cluster_entries;
    const uint32_t *ap_extra;
    const int32_t *type_records;
} eat_net_view;

/* Per-query work counters (optional output of the query calls). */
typedef struct {
    int64_t rounds;    /* relaxation rounds run (Algorithm 5's while loop) */
    int64_t vertices;  /* active stops expanded, summed over rounds (a stop with no
                          outgoing connection never needs expanding) */
    int64_t types;     /* connection types examined with an active tail: the
                          "connections processed" of Section IV-C */
    int64_t evals;     /* of the looked-up types, those with a departure at or after
                          e[u] (their e[v] is read) */
    int64_t lookups;   /* of the examined types, those whose cluster entry was read
                          (Section II-D); types >= lookups >= evals */
    int64_t aps;       /* AP records examined by the cluster lookup (Algorithm 6) */
    int64_t relaxed;   /* relaxations that lowered e[v] (Algorithm 3): candidates below
                          the e[v] read just before the atomic min, so a candidate whose
                          atomic lost to a lower one made meanwhile is counted too */
} eat_counters;

/* Query options.  Zero-initialise for defaults. */
typedef struct {
    int32_t max_rounds;      /* round cap; 0 = n_stops + 1 (always enough: every
                                productive round fixes at least one more stop), or
                                2 * n_stops + 2 with a horizon (each horizon step adds at
                                most one round to the n_stops + 1) */
    int32_t block;           /* threads per CTA: 0 = automatic (the tuned shape, else 1024
                                when the batch has at most one query per SM, runs in the
                                paired mode or is on one network of 8,192 stops or more,
                                else 512);
                                else 64..1024, multiple of 32 */
    int32_t vwarp;           /* lanes per active stop (1, 2, 4, 8, 16 or 32); 0 = automatic */
    int32_t mode;            /* EAT_MODE_* */
    int32_t placement;       /* EAT_PLACE_*: where a query's arrivals and frontier
                                bitmap live; 0 = automatic */
    int32_t cluster;         /* blocks per query in EAT_MODE_CLUSTER: 2, 4 or 8; 0 = 8 */
    int32_t order;           /* EAT_ORDER_*: the order in which a batch's queries start;
                                0 = automatic */
    int32_t idle_cap;        /* EAT_MODE_ASYNC only: a warp whose scans of 32 words of
                                the pending-stop bitmap find nothing this many times in a
                                row (checked after each full pass) while other warps still
                                hold work gives up the query, which then reports
                                EAT_ERR_NO_CONVERGENCE with upper bounds in its row;
                                0 = 2^24 (far beyond any wait of a correct run) */
    int32_t horizon;         /* seconds; the per-query kernel's rounds (EAT_MODE_CTA or
                                EAT_MODE_EDGE) expand a stop lowered to an arrival at or
                                after the horizon H only once no stop below H is left to
                                expand; H starts at t_s + horizon and then moves to the
                                earliest arrival still waiting + horizon.  The arrivals
                                are the same (the fixpoint does not depend on the order
                                of relaxations); stops first reached late by a path of
                                few connections are then expanded once, with an arrival
                                closer to their final one, instead of again each time a
                                later round improves them (Algorithms 4-5 expand every
                                improved stop in the next round).
                                0 = automatic (the value eat_autotune chose for this
                                batch size, else none); < 0 = none; > 0 with
                                EAT_MODE_PAIR, EAT_MODE_ASYNC or EAT_MODE_CLUSTER is
                                EAT_ERR_INVALID */
    int32_t *status;         /* optional [n] per-query eat_status, device memory */
    eat_counters *counters;  /* optional [n] per-query counters, device memory */
} eat_query_opts;

enum eat_placement {
    EAT_PLACE_AUTO = 0,
    EAT_PLACE_SHARED = 1,        /* arrivals and bitmap in shared memory (needs
                                    4 * n_stops + n_stops / 8 bytes to fit a CTA) */
    EAT_PLACE_GLOBAL_ARR = 2,    /* arrivals in the output row, bitmap in shared memory */
    EAT_PLACE_GLOBAL = 3         /* arrivals and bitmap in global memory */
};

enum eat_order {
    EAT_ORDER_AUTO = 0,      /* on one network: EAT_ORDER_BY_TIME when the batch has more
                                queries than the launch runs at once (some wait for a
                                free block) or runs in EAT_MODE_PAIR; otherwise, and for
                                batches over several networks, EAT_ORDER_AS_GIVEN */
    EAT_ORDER_BY_TIME = 1,   /* queries start in order of departure time t_s (15-minute
                                buckets, earliest first; a one-block device counting sort
                                before the launch, n int32 of workspace): the longest
                                queries start first, and queries running at the same time
                                read the same clusters of the network from L2 (measured:
                                large network 17.8 -> 14.0 ms per 1,024-query step, city
                                0.88 -> 0.70 ms per 256-query step with one 1,024-thread
                                block per query).  Results, status and counters stay at
                                each query's index */
    EAT_ORDER_AS_GIVEN = 2   /* queries start in index order (always in
                                eat_query_batch_noalloc and for a single query) */
};

enum eat_mode {
    EAT_MODE_AUTO = 0,  /* library picks */
    EAT_MODE_CTA = 1,   /* one thread block per query; rounds end at block barriers */
    EAT_MODE_CLUSTER = 2, /* one thread-block cluster of 8 blocks (on 8 SMs) per query, on
                           one network: the arrivals and frontier bitmaps are spread over
                           the cluster's shared memory (distributed shared memory) and a
                           round ends at a cluster barrier; arrivals up to about
                           440,000 stops.  Never chosen automatically: on GB300 the
                           distributed-shared-memory round trips and the cluster
                           barrier cost more per round than the extra blocks save (a
                           single city query 0.51-0.58 ms against 0.30 ms with one
                           1,024-thread block).  Not with eat_query_batch_noalloc */
    EAT_MODE_ASYNC = 3  /* one thread block per query, no rounds: warps claim pending stops
                           from a bitmap and relax their types as soon as they appear;
                           needs the bitmap (n_stops bits) in shared memory; the round cap
                           does not apply and counters.rounds is 0 */,
    EAT_MODE_PAIR = 4   /* two queries per 1,024-thread block sharing its rounds, on one
                           network of at most 32,767 stops and 65,535 connection types
                           whose two arrival rows fit in one block's shared memory: when
                           one query converges its threads go to the other and the slot
                           takes the next query.  EAT_MODE_AUTO uses it only where
                           eat_autotune chose it; never in eat_query_batch_noalloc
                           unless requested */,
    EAT_MODE_EDGE = 5   /* as EAT_MODE_CTA with two changes (the mapping chosen by degree
                           and the warp min of Section II-F's warps): a stop with at least
                           vwarp outgoing connection types is queued whole and expanded
                           by a sub-warp of vwarp lanes (the whole warp for vwarp 32)
                           instead of one item per type; and the lanes of a warp whose
                           types share a head stop v reduce their candidates with a warp
                           min, so that one lane per head stop reads e[v], lowers it and
                           pushes v.  EAT_MODE_AUTO uses it only where eat_autotune
                           chose it */
};

/* Error message of the calling thread's last failed call ("" if none). */
const char *eat_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t eat_version(void);

/*
 * eat_build -- preprocess a timetable into the Cluster-AP layout and upload it.
 * Section III-A (graph representation and preprocessing): group connections by
 * edge and duration into connection types (Section II-B), split each type by
 * departure time into clusters of cluster_width seconds (Section II-D), cover
 * each cluster by the greedy AP cover (Section I-A; Section II-C), order the
 * APs of a cluster by first term.  With opts->subtrips, each trip is first cut
 * into consecutive sub-trips and one artificial connection is added per
 * sub-trip of two or more connections, from its first stop at its first
 * departure to its last stop at its last arrival (Section II-G); earliest
 * arrival times are unchanged.
 *   conn  host arrays, read only during the call (copied).
 *   opts  may be NULL (defaults).
 *   out   receives a new network owned by the caller; release with eat_free.
 * Errors: EAT_ERR_INVALID (bad sizes, ids, durations, times, trips or options),
 * EAT_ERR_OOM, EAT_ERR_CUDA, EAT_ERR_NO_DEVICE.  On error *out is NULL.
 */
int eat_build(const eat_connections *conn, const eat_build_opts *opts, eat_net **out);

/* Pre-encoded input for eat_build_csr: the Cluster-AP structure itself (Section
 * III-A) for callers that encode their own timetable.  All arrays are host memory.
 *   row_ptr[n_stops + 1]   types leaving stop u are row_ptr[u] .. row_ptr[u+1]-1
 *                          (row_ptr[0] = 0, row_ptr[n_stops] = n_types)
 *   type_v[n_types], type_dur[n_types]   head stop and duration (1 .. 2^24-1) of each
 *                          connection type (Section II-B)
 *   type_cl_ptr[n_types + 1]   clusters of type t are type_cl_ptr[t] ..
 *                          type_cl_ptr[t+1]-1; every type has at least one
 *   cl_k[n_clusters]       cluster index k: the cluster holds departures in
 *                          [t0 + k * width, t0 + (k+1) * width) (Section II-D);
 *                          strictly increasing within a type
 *   cl_ap_ptr[n_clusters + 1]   APs of cluster c are cl_ap_ptr[c] .. cl_ap_ptr[c+1]-1;
 *                          every cluster has at least one
 *   ap_first[n_aps], ap_step[n_aps], ap_count[n_aps]   AP runs (Section I-A): terms
 *                          first, first + step, ..., first + (count-1) * step, all
 *                          inside the cluster's window; count >= 1, step >= 1 when
 *                          count >= 2, step and count <= 65535; ordered by first
 *                          term within a cluster */
typedef struct {
    int32_t n_stops;
    int32_t n_types;
    int64_t n_clusters;
    int64_t n_aps;
    const int32_t *row_ptr;
    const int32_t *type_v;
    const int32_t *type_dur;
    const int64_t *type_cl_ptr;
    const int32_t *cl_k;
    const int64_t *cl_ap_ptr;
    const int32_t *ap_first;
    const int32_t *ap_step;
    const int32_t *ap_count;
} eat_csr_input;

/*
 * eat_build_csr -- build a network from pre-encoded connection types, clusters
 * and AP runs (the layout of Section III-A) instead of raw connections.  The
 * input is validated and copied; opts->cluster_width and opts->t0 give the
 * cluster windows (opts->subtrips must be EAT_SUBTRIPS_NONE).  Queries behave
 * exactly as on a network built by eat_build from the connections the APs
 * expand to.  n_conn in eat_stats is the total number of AP terms.
 * Errors: EAT_ERR_INVALID (any inconsistency, with the first offending index),
 * EAT_ERR_OOM, EAT_ERR_CUDA, EAT_ERR_NO_DEVICE.  On error *out is NULL.
 */
int eat_build_csr(const eat_csr_input *in, const eat_build_opts *opts, eat_net **out);

/* Release a network and its device memory (no counterpart in the paper, which
 * keeps one network for a process).  NULL is ignored.  No query on the network may
 * be in flight. */
void eat_free(eat_net *net);

/* Sizes of a network: the counts of Section III-A's arrays (connection types,
 * clusters, AP tuples; y is the paper's CL stride) and of Table I's statistics for
 * the built network (stops, connections).  Named eat_get_stats because eat_stats is
 * the struct's name.  Errors: EAT_ERR_INVALID on NULL arguments. */
int eat_get_stats(const eat_net *net, eat_stats *out);

/* Host view of the built arrays (see eat_net_view).  Works for host-only builds. */
int eat_net_host_view(const eat_net *net, eat_net_view *out);

/*
 * eat_query -- one query (s, t_s), blocking (Algorithms 2-5, Section II-D).
 *   arr_out  [n_stops] int32, host or device memory: arr_out[v] = e[v],
 *            EAT_INF if v is unreachable; arr_out[s] = t_s.  Page-locked host
 *            memory is written in place when the arrivals fit in shared memory.
 *   counters optional (NULL), host memory.
 * Runs on the legacy default stream with the network's own workspace, so
 * concurrent eat_query calls on one network are serialised internally.
 * Errors: EAT_ERR_INVALID (s out of range, NULL arr_out), EAT_ERR_NO_DEVICE,
 * EAT_ERR_NO_CONVERGENCE (round cap hit; arr_out then holds upper bounds),
 * EAT_ERR_CUDA.
 */
int eat_query(const eat_net *net, int32_t s, int32_t t_s, int32_t *arr_out,
              eat_counters *counters);

/*
 * eat_workspace_bytes -- device workspace needed by eat_query_batch(_multi) for
 * n queries over the given networks with these options (opts may be NULL).
 * Returns 0 on invalid arguments.
 */
size_t eat_workspace_bytes(const eat_net *const *nets, int32_t n_nets, int32_t n,
                           const eat_query_opts *opts);

/*
 * eat_launch_shape -- the launch shape eat_query_batch(_multi) would use for n
 * queries over the given networks with these options (opts may be NULL): *shape
 * receives a copy of *opts with block, vwarp, mode (EAT_MODE_CTA, _CLUSTER,
 * _ASYNC, _PAIR or _EDGE, never _AUTO), cluster, order (EAT_ORDER_BY_TIME or
 * EAT_ORDER_AS_GIVEN, never _AUTO) and horizon (seconds, -1 for none, never 0)
 * filled in.  Nothing is launched.
 * Returns EAT_OK, or the error the batch call would report for these options.
 */
int eat_launch_shape(const eat_net *const *nets, int32_t n_nets, int32_t n,
                     const eat_query_opts *opts, eat_query_opts *shape);

/*
 * eat_query_batch -- n independent queries (sources[i], times[i]) on one
 * network, in one launch (batching across queries is this library's addition;
 * each query follows the same algorithm as eat_query).
 *   sources, times  [n] int32, host or device memory.
 *   arr_out         [n * n_stops] int32 row-major (row i = query i), host or
 *                   device memory.
 *   workspace       device memory of at least eat_workspace_bytes(&net, 1, n, opts)
 *                   bytes, or NULL to use the network's internal workspace (then
 *                   calls on one network must not overlap).
 *   opts            may be NULL.
 *   stream          cudaStream_t to run on.
 * If every buffer is device memory the call is asynchronous on `stream`.  If
 * any is host memory the call returns after the results are in arr_out: when
 * arr_out is page-locked host memory mapped for the device (cudaHostAlloc,
 * cudaHostRegister), the kernel writes each query's row into arr_out itself (and
 * reads page-locked sources/times in place), so the transfer overlaps the other
 * queries: as each query finishes, from shared memory or, for arrivals kept in a
 * device row of the block (networks too large for shared memory), from that row;
 * otherwise host buffers are staged through device memory with copies before and
 * after the launch.  Per-query round-cap failures are reported
 * only through opts->status (the return value covers launch errors).
 * Errors: EAT_ERR_INVALID, EAT_ERR_WORKSPACE, EAT_ERR_NO_DEVICE, EAT_ERR_CUDA,
 * EAT_ERR_OOM.
 */
int eat_query_batch(const eat_net *net, const int32_t *sources, const int32_t *times,
                    int32_t n, int32_t *arr_out, void *workspace, size_t workspace_bytes,
                    const eat_query_opts *opts, void *stream);

/*
 * eat_query_batch_multi -- n queries over several networks of uneven size in
 * one launch.  Query i runs on nets[net_idx[i]] and writes its
 * nets[net_idx[i]]->n_stops arrivals at arr_out + arr_offsets[i].
 *   nets         [n_nets] host array of networks, all on the same device,
 *                1 <= n_nets <= EAT_MAX_NETS.
 *   net_idx, sources, times  [n] int32; arr_offsets [n] int64 (element offsets);
 *                host or device memory, all of the same kind.
 *   arr_out      device memory large enough for every row, or host memory when
 *                the query arrays are host memory (then staged and copied back).
 * Asynchronous on `stream` when every buffer is device memory, else returns
 * after the rows are in arr_out.  One launch serves all queries: networks whose
 * arrival row fits half an SM's shared memory keep it there, larger ones use
 * their output row.  Other arguments as eat_query_batch.
 */
#define EAT_MAX_NETS 128
int eat_query_batch_multi(const eat_net *const *nets, int32_t n_nets, const int32_t *net_idx,
                          const int32_t *sources, const int32_t *times, int32_t n,
                          int32_t *arr_out, const int64_t *arr_offsets, void *workspace,
                          size_t workspace_bytes, const eat_query_opts *opts, void *stream);

/*
 * eat_next_departure -- the Cluster-AP lookup alone (getConnection with
 * getConnectionFromAPs, Algorithm 6, inside the hourly cluster of Section
 * II-D): for each i, out[i] = least departure >= times[i] of connection type
 * types[i], or EAT_INF if there is none.  Exposes the kernel's lookup for
 * testing.  types, times, out: [n] int32 device memory.  Asynchronous on stream.
 * Errors: EAT_ERR_INVALID (type index out of range), EAT_ERR_NO_DEVICE,
 * EAT_ERR_CUDA.
 */
int eat_next_departure(const eat_net *net, const int32_t *types, const int32_t *times,
                       int32_t n, int32_t *out, void *stream);

/*
 * eat_autotune -- choose the launch shape for this network by measurement (no
 * counterpart in the paper, which fixes one thread per type or per edge and
 * sweeps the virtual-warp size by hand, Section IV-B).  Candidates, in this
 * order: block sizes 512, 1024 and 256 threads, each with the round-based mode
 * and vwarp 8, 4, 16, 2, 32 lanes per spilled stop, then with the asynchronous
 * mode, then with EAT_MODE_EDGE and vwarp 8 and 32, as far as they fit the device
 * (1024 threads first on networks of 8,192 stops or more and for batches of at most
 * one query per SM, where it is the default); when n exceeds the SM count, then the
 * paired mode with vwarp 8, 4 and 16; then the round-based mode with the first two
 * block sizes, vwarp 8 and horizons of 1, 2, 4 and 12 hours (the other candidates run
 * with none).  They are run on the sample batch
 * sources/times (n queries, device memory) in nine rounds over all candidates:
 * the first warms up, the other eight are timed with CUDA events on `stream`,
 * each after a write of twice the L2 size so that every timing starts with the
 * network out of cache.  The earliest candidate whose median time is within 5 %
 * of the least median wins (closer differences are within the spread between
 * batches of one workload), and
 * is stored for batches of about n queries in the network; afterwards every
 * query call that leaves opts->block, opts->vwarp and opts->mode at 0 uses it
 * (a call with a round cap keeps the round-based mode), and every call that leaves
 * opts->horizon at 0 and runs the round-based kernel uses its horizon.  The tuned
 * shape (block, vwarp, mode, horizon: -1 for none) is written to *best (may be
 * NULL).  Blocks until done.  Allocates its own scratch (workspace, output rows and
 * the cache-flush buffer) for the duration of the call.  Errors: as eat_query_batch; EAT_ERR_INVALID if no shape fits.
 */
int eat_autotune(eat_net *net, const int32_t *sources, const int32_t *times, int32_t n,
                 eat_query_opts *best, void *stream);

/*
 * eat_autotune_multi -- choose the launch shape and start order of a batch over several
 * networks of uneven size (eat_query_batch_multi) by measurement; no counterpart in the
 * paper, as for eat_autotune.  Candidates, in this order: start order as given, then by
 * t_s (EAT_ORDER_AS_GIVEN, EAT_ORDER_BY_TIME); for each, block sizes 512, 1024 and 256
 * threads, each with the round-based mode and vwarp 8, 4, 16, 2, 32, then the
 * asynchronous mode, then EAT_MODE_EDGE with vwarp 8; then the round-based mode with 512
 * threads, vwarp 8, start by t_s and horizons of 2 and 12 hours (the others run with
 * none); shapes without a plan for these networks are skipped.  They run on
 * the sample batch (net_idx, sources, times: [n] int32 device memory; rows packed in
 * query order in a scratch buffer) and are timed as eat_autotune times them (nine rounds,
 * cold L2, median, earliest within 5 % wins).  Nothing is stored in the networks: the
 * caller passes *best (block, vwarp, mode, order and horizon filled in, the rest zero,
 * horizon -1 for none) as the
 * options of its eat_query_batch_multi calls.  Blocks until done; allocates its scratch
 * for the duration of the call.
 * Errors: EAT_ERR_INVALID (NULL best, bad networks or indices, host arrays, no shape
 * fits), EAT_ERR_NO_DEVICE, EAT_ERR_OOM, EAT_ERR_CUDA.
 */
int eat_autotune_multi(const eat_net *const *nets, int32_t n_nets, const int32_t *net_idx,
                       const int32_t *sources, const int32_t *times, int32_t n,
                       eat_query_opts *best, void *stream);

/* ------------------------------------------------------------------ serving
 * A request loop with continuous batching over resident networks (no
 * counterpart in the paper, which runs one query at a time; each request runs
 * the same algorithm as eat_query).  Requests for any of the server's networks
 * are queued by eat_server_submit and a dispatcher thread admits them to the GPU
 * as memory frees up.  When a request's row is in place it is copied to the
 * caller's arr_out and a result (tag, status, latency) is queued for
 * eat_server_poll.  Two admission modes (eat_server_opts.admission):
 *
 *   EAT_ADMIT_RING (default): one persistent launch of the per-query kernel (one
 *     query per thread block, all blocks the SMs hold) serves a ring of requests in
 *     page-locked host memory.  The dispatcher writes each admitted request into a
 *     free ring entry and publishes it; a block that finishes its query takes the
 *     next published request at once, while the launch runs, so a request that
 *     arrives while others are on the GPU starts as soon as one block is free.  The
 *     block writes the arrival row into the entry's row of a page-locked pool in
 *     place and marks the entry done.  The ring's capacity (requests on the GPU at
 *     once) is set by mem_budget (admission by memory: a request enters the ring
 *     only when an entry and its row are free), at most max_batch * max_inflight.
 *     The launch ends when the dispatcher has had no request in flight for about
 *     2 ms (it sets a stop flag that idle blocks read); a later request starts a
 *     new launch.  Every wait of a block is bounded (about 100 ms without a
 *     request, then it leaves).  Needs the networks' frontier bitmaps to fit in
 *     shared memory (up to about 900,000 stops).
 *   EAT_ADMIT_BATCH: a pool of slots, each a CUDA stream with pre-allocated device
 *     buffers for max_batch queries (the pool size set by mem_budget).  A free slot
 *     takes up to max_batch pending requests of any networks and runs them as one
 *     eat_query_batch_multi launch; batches started while others run overlap on the
 *     device, and a request that arrives while all slots run waits for a slot.
 * The networks must stay alive until eat_server_destroy. */
typedef struct eat_server eat_server;

enum eat_admission {
    EAT_ADMIT_RING = 0,
    EAT_ADMIT_BATCH = 1
};

typedef struct {
    int32_t max_batch;      /* EAT_ADMIT_BATCH: requests per launch; 0 = 256 */
    int32_t max_inflight;   /* EAT_ADMIT_BATCH: slots (concurrent launches); 0 = 4.
                               EAT_ADMIT_RING: ring capacity at most max_batch *
                               max_inflight, rounded down to a power of two */
    int32_t batch_wait_us;  /* EAT_ADMIT_BATCH: while another batch runs, wait up to this
                               long for a fuller batch; 0 = 200 */
    int32_t admission;      /* EAT_ADMIT_* */
    int64_t mem_budget;     /* device + pinned bytes for the slots or the ring; 0 = 1 GiB */
} eat_server_opts;

typedef struct {
    uint64_t tag;           /* the caller's tag from eat_server_submit */
    int32_t status;         /* eat_status of the query */
    int32_t net;            /* network index */
    int64_t latency_ns;     /* submit to result delivered */
} eat_server_result;

/* Counters since creation.  batches: launches (EAT_ADMIT_RING: ring launches);
 * batched_queries: requests admitted to the GPU; max_batch_seen: largest batch
 * (EAT_ADMIT_RING: most requests in the ring at once); max_inflight_seen: most
 * batches running at once (EAT_ADMIT_RING: most requests in the ring at once);
 * slots, slot_bytes: batch slots and bytes per slot (EAT_ADMIT_RING: ring capacity
 * and bytes per entry with its row); admitted_running: requests admitted while a
 * launch was already running (EAT_ADMIT_RING: entered the ring of a running
 * launch); base_bytes: see below.  mem_budget covers base_bytes + slots *
 * slot_bytes. */
typedef struct {
    int64_t submitted, completed, pending;
    int64_t batches, batched_queries;
    int64_t max_batch_seen, max_inflight_seen, max_pending_seen;
    int64_t slots, slot_bytes;
    int64_t last_error;
    int64_t admitted_running;
    int64_t base_bytes;     /* bytes held besides the slots or ring entries (EAT_ADMIT_RING:
                               the launch's workspace and device rows) */
} eat_server_stats;

/* Create a server for nets[0 .. n_nets-1] (same device, 1..EAT_MAX_NETS);
 * opts may be NULL.  Errors: EAT_ERR_INVALID, EAT_ERR_NO_DEVICE, EAT_ERR_OOM
 * (mem_budget holds no slot, or allocation failed). */
int eat_server_create(const eat_net *const *nets, int32_t n_nets, const eat_server_opts *opts,
                      eat_server **out);
/* Queue query (s, t_s) on network `net`; arr_out (host memory, n_stops int32)
 * receives the arrivals before the result is reported.  Never blocks on the GPU.
 * Errors: EAT_ERR_INVALID (bad network or source, server shutting down). */
int eat_server_submit(eat_server *sv, int32_t net, int32_t s, int32_t t_s, int32_t *arr_out,
                      uint64_t tag);
/* Move up to max finished results into results[], waiting up to timeout_us for
 * the first one; returns how many were moved. */
int32_t eat_server_poll(eat_server *sv, eat_server_result *results, int32_t max,
                        int32_t timeout_us);
/* Counters of the server since creation. */
int eat_server_get_stats(eat_server *sv, eat_server_stats *out);
/* Finish every queued request, then stop the dispatcher and free the slots.
 * Results not yet polled are discarded.  NULL is ignored. */
void eat_server_destroy(eat_server *sv);

/*
 * eat_query_batch_noalloc -- eat_query_batch for callers that cannot allocate
 * device memory.  The paper has no counterpart; this entry point exists for
 * users of the library, not for the method.
 *
 * Who needs it: code that is not allowed to call cudaMalloc and therefore
 * cannot provide the workspace eat_query_batch asks for -- for example a
 * plugin whose host application owns all device memory through its own
 * allocator or budget, or a serving loop that admits work against a fixed
 * memory reservation and must not grow it per call.  Such a caller still
 * passes its own input and output buffers; the frontier queues that
 * eat_query_batch keeps in the workspace live instead in one fixed scratch
 * array inside libeat (EAT_NOALLOC_SCRATCH_BYTES = 16 MiB), which every GPU
 * that loads the library holds until the process exits.
 *
 * Behaviour:
 *   - Same queries and results as eat_query_batch (same kernel); sources,
 *     times and arr_out must be device memory of the network's device.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device looks up the scratch array's device address
 *     (once per device, with that device current); make that first call before
 *     any stream capture on the device.
 *   - All calls share the one scratch array and it keeps the previous call's
 *     contents; the call clears what must start at zero.  Calls whose GPU work
 *     overlaps (on different streams or threads, for any network on the same
 *     device) race on the scratch and give wrong results: serialise them.
 *   - Limit: each persistent thread block needs 8 * n_stops bytes of the scratch
 *     (rounded up) for its frontier queue, plus n_stops / 4 bytes when the frontier
 *     bitmaps live in global memory (networks beyond about 900,000 stops), or
 *     16 * n_stops bytes in the paired mode (two queries per block); with a
 *     horizon, 16 * n_stops + n_stops / 8 bytes (the lists of waiting stops); the
 *     round-free mode needs none.  So the network may have at most 2,000,000 stops
 *     (about 1,000,000 with a horizon), and on large networks fewer blocks run at
 *     once while the other queries wait in the same launch.  Larger networks are
 *     rejected with EAT_ERR_INVALID.
 * Errors: EAT_ERR_INVALID (host buffers, network too large, bad options),
 * EAT_ERR_NO_DEVICE, EAT_ERR_CUDA.
 */
#define EAT_NOALLOC_SCRATCH_BYTES (16u << 20)
#define EAT_NOALLOC_MAX_STOPS 2000000
int eat_query_batch_noalloc(const eat_net *net, const int32_t *sources, const int32_t *times,
                            int32_t n, int32_t *arr_out, const eat_query_opts *opts,
                            void *stream);

/* ------------------------------------------------------------------------
 * Topology-driven variants (Section II-A to II-F), the paper's own execution
 * model, kept as a baseline and to show what each pruning step buys.
 *
 * One query at a time.  Each round one kernel visits every connection, type or
 * edge and works only on those whose tail stop is active, i.e. was improved in
 * the round before (Section III-B's active / nextactive pair, kept here as two
 * arrays of round stamps).  The host drives the rounds and reads the device's
 * "improved in round i" flag every `flag_every` rounds (Section IV-C: 1 = after
 * every round, as in Algorithms 4-5; about sqrt(d) = the reduced transfer of
 * Table V); the rounds run after convergence find nothing active.
 * ------------------------------------------------------------------------ */
typedef struct eat_ladder eat_ladder;

enum eat_variant {
    EAT_VAR_CONNECTION = 1,   /* Algorithm 4: one thread per connection; relax if its
                                 tail is active and e[u] <= t */
    EAT_VAR_TYPE = 2,         /* Algorithm 5: one thread per connection type; the
                                 earliest departure >= e[u] by linear search of the
                                 type's sorted departures (getConnection) */
    EAT_VAR_TYPE_AP = 3,      /* Section II-C: as 2, the departure from the type's
                                 whole-day AP tuples (Algorithm 6) */
    EAT_VAR_CLUSTER_AP = 4,   /* Section II-D: as 3 inside the cluster of e[u], else
                                 the next non-empty cluster's first departure */
    EAT_VAR_EDGE = 5,         /* Section II-E: one thread per edge (u, v), all its
                                 types by Cluster-AP */
    EAT_VAR_WARP = 6          /* Section II-F: one warp per edge, its types spread
                                 over the lanes, by Cluster-AP */
};

typedef struct {
    int32_t rounds;       /* rounds launched (including those after convergence) */
    int32_t flag_reads;   /* device-to-host copies of the flag */
} eat_ladder_stats;

/*
 * eat_ladder_build -- everything the variants read, on opts->device (>= 0):
 * the Cluster-AP network of eat_build (same options and errors) plus the
 * connections themselves (16 B each), every type's {tail, head, duration},
 * its sorted unique departures and its whole-day greedy AP cover (the cover
 * rule of Section I-A, as in the clusters, over all of the type's departures:
 * first term, difference and terms as int32), and the edges (runs of types
 * with the same tail and head).  Input arrays are copied.  Free with
 * eat_ladder_free.  Errors: as eat_build; EAT_ERR_NO_DEVICE for device < 0.
 */
int eat_ladder_build(const eat_connections *conn, const eat_build_opts *opts,
                     eat_ladder **out);
void eat_ladder_free(eat_ladder *l);

/*
 * eat_ladder_query -- one query (s, t_s) with `variant` (enum eat_variant),
 * blocking.  arr_out: [n_stops] int32, host or device memory, as eat_query.
 * flag_every >= 1: rounds between flag reads.  graph != 0: the flag_every
 * rounds between two reads are replayed as one CUDA graph (captured on first
 * use per variant and cadence and kept with the ladder; the round index then
 * lives on the device), else every round is its own launch.  stats may be
 * NULL.  Calls on one ladder are serialised internally.
 * Errors: EAT_ERR_INVALID (bad variant, s out of range, flag_every < 1),
 * EAT_ERR_NO_CONVERGENCE (more than n_stops + flag_every rounds), EAT_ERR_CUDA.
 */
int eat_ladder_query(eat_ladder *l, int32_t variant, int32_t s, int32_t t_s, int32_t flag_every,
                     int32_t graph, int32_t *arr_out, eat_ladder_stats *stats);

/*
 * eat_ladder_host_view -- the variants' host copies, valid until
 * eat_ladder_free: per type t, tail/head/duration at type_uvl[3t .. 3t+2];
 * departures dep[dep_ptr[t] .. dep_ptr[t+1]); whole-day APs
 * ap[3a .. 3a+2] = {first, difference, terms} for a in [ap_ptr[t], ap_ptr[t+1]);
 * edge e = types [edge_ptr[e], edge_ptr[e+1]).
 */
typedef struct {
    int32_t n_types, n_edges;
    int64_t n_dep, n_ap;
    const int32_t *type_uvl, *dep_ptr, *dep, *ap_ptr, *ap, *edge_ptr;
} eat_ladder_view;
int eat_ladder_host_view(const eat_ladder *l, eat_ladder_view *view);

#ifdef __cplusplus
}
#endif
#endif /* EAT_H */
