"""Benchmark: earliest-arrival-time queries per second on one GB300 (and N replicas).

Workload (default "large"): a 200,000-stop random geometric transit network (k = 5
nearest neighbours, 4,000 routes of 40-80 stops run both ways, headways 3-30 min,
10 % jittered trips, three duration bands), about 46 M connections, 1.8 GB on the
device; one step = one batch of 1,024 queries (random source with departures, t_s
uniform in 05:00-22:00), all relaxation rounds of all queries in one launch (the
launch shape by the library's autotuner unless given; the batch's queries cannot
all start at once, so the launch begins with the library's sort of the queries by
t_s, inside the timed region).  `--workload city` runs the 20,000-stop network
(about 3.6 M connections) with 256 queries per step.

Timing: W untimed warm-up steps, then K steps, each timed with CUDA events on the
launching stream; L2 is flushed (a 256 MB buffer is written) before every step,
outside the events; inputs are resident in device memory before timing starts.
`e2e` repeats the measurement through the C ABI with page-locked host buffers, so
each step includes moving the queries to the GPU and every arrival row back to host
memory (the kernel reads the queries and writes each converged row to host memory
in place).

Roofline: algorithmic bytes per launch come from the kernel's own per-query work
counters (stops expanded, types examined, AP records read, relaxations), taken in an
untimed pass over the same batches, times the fixed per-unit byte figures in BYTES
below.

`--impl reference` times the CPU oracle (connection scan, Algorithm 1) on the host
cores on the same queries instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

BATCH = 256
FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0

# Per-unit algorithmic bytes of the method's data structures: per expanded stop 8 B frontier
# entry + 4 B e[u] + 8 B row offsets; per examined type 16 B type record + 8 B pair of
# cluster offsets + 4 B read of e[v] (charged on every examined type, also those that
# stop early); per AP record examined 16 B; per relaxation 4 B atomic write + 8 B frontier
# push; per query 4 B x V initialisation + 4 B x V result row.
BYTES = {"vertices": 20, "types": 28, "aps": 16, "relaxed": 12}

# DRAM bytes per query of the timed kernel, from the ncu captures summarised in profiles/
# (the bench's own launches, dram__bytes_read.sum + dram__bytes_write.sum averaged over
# the 20 timed launches: 1,024 queries on the large network, 256 on the city network);
# keyed by the kernel source hash, the kernel's name, the block size, the horizon and the
# cluster width, so that another kernel or launch shape reports null until it is
# profiled again.
NCU_TRAFFIC_PER_QUERY = {
    "large": ("2de258fb4eb0b1dc", "eat_cta_kernel", 512, 3600, 600, 14555841037 / 1024),
    "city": ("2de258fb4eb0b1dc", "eat_cta_kernel", 1024, -1, 600, 135806746 / 256),
}
KERNEL_OF_MODE = {1: "eat_cta_kernel", 2: "eat_cluster_kernel", 3: "eat_async_kernel",
                  4: "eat_pair_kernel", 5: "eat_cta_kernel"}


def kernel_hash() -> str:
    """Hash of the sources the query kernels compile from."""
    h = hashlib.sha256()
    for f in ("eat_kernels.cu", "eat_device.cuh", "eat_launch.h", "eat_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1912_00966_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


RAGGED_QUERIES = 4096


def run_ours_ragged(args):
    """64 grid networks of 1k-50k stops, 4,096 queries per step in one launch."""
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    from paper_1912_00966_gb300 import eat

    tts = synth.ragged_grids(64)
    t_build = time.perf_counter()
    nets = [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=dev,
                          cluster_width=args.cluster_width) for t in tts]
    t_build = time.perf_counter() - t_build
    n_steps = args.warmup + args.steps
    Q = RAGGED_QUERIES
    qsets = rank_query_sets(tts, Q, n_steps, rank, 0xA0)
    Vs = np.array([t.n_stops for t in tts], np.int64)
    offs = [np.concatenate([[0], np.cumsum(Vs[q.net])[:-1]]).astype(np.int64) for q in qsets]
    total = max(int(Vs[q.net].sum()) for q in qsets)
    dq = [(torch.as_tensor(q.net).cuda(), torch.as_tensor(q.source).cuda(),
           torch.as_tensor(q.t_s).cuda(), torch.as_tensor(o).cuda()) for q, o in zip(qsets, offs)]
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((n_steps, Q, 7), dtype=torch.int64, device="cuda")
    status = torch.zeros((n_steps, Q), dtype=torch.int32, device="cuda")
    opts = dict(vwarp=args.vwarp, block=args.block, mode=args.mode, horizon=args.horizon,
                order=args.order)
    tuned = None
    if args.autotune and not (args.vwarp or args.block or args.mode or args.horizon):
        # Launch shape and start order chosen by the library's multi-network autotuner on
        # a sample batch (setup, untimed).
        sample = synth.random_queries(tts, Q, 0xA0 - 1)
        tuned = eat.eat_autotune_multi(nets, torch.as_tensor(sample.net).cuda(),
                                       torch.as_tensor(sample.source).cuda(),
                                       torch.as_tensor(sample.t_s).cuda())
        opts = dict(tuned)
    shape = eat.eat_launch_shape(nets, Q, **opts)
    ws = torch.empty(eat.eat_workspace_bytes(nets, Q, **opts), dtype=torch.uint8, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_steps)]

    # Work counters from an untimed pass over the same batches; the timed launches run
    # without counters, as in the single-network bench.
    for i in range(n_steps):
        ni, src, ts, of = dq[i]
        eat.eat_query_batch_multi(nets, ni, src, ts, out, of, workspace=ws, stream=stream,
                                  counters=cnt[i], **opts)
    torch.cuda.synchronize()

    def step(i):
        flush.fill_(i)
        a, b = evs[i]
        a.record(stream)
        ni, src, ts, of = dq[i]
        eat.eat_query_batch_multi(nets, ni, src, ts, out, of, workspace=ws, stream=stream,
                                  status=status[i], **opts)
        b.record(stream)

    with ClockSampler(dev) as clocks:
        clocks.wait_first()
        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.mark()
        for i in range(args.warmup, n_steps):
            step(i)
        torch.cuda.synchronize()
        time.sleep(0.06)
        clocks.stop_mark()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [evs[i][0].elapsed_time(evs[i][1]) for i in range(args.warmup, n_steps)]
    gpu_s = sum(step_ms) / 1e3
    if (status.cpu().numpy() != 0).any():
        raise SystemExit("bench: a query did not converge")
    c = cnt[args.warmup:].sum(dim=(0, 1)).cpu().numpy()
    names = eat.COUNTER_FIELDS
    tot = {n: int(c[k]) for k, n in enumerate(names)}
    alg_bytes = sum(BYTES[n] * tot[n] for n in BYTES) + sum(
        8 * int(Vs[q.net].sum()) for q in qsets[args.warmup:])
    per_launch = alg_bytes / args.steps
    mean_ms = gpu_s * 1e3 / args.steps
    kernel_name = KERNEL_OF_MODE[shape["mode"]]

    # End to end through the C ABI from pinned host buffers (rows copied back).
    hq = [(torch.as_tensor(q.net).pin_memory(), torch.as_tensor(q.source).pin_memory(),
           torch.as_tensor(q.t_s).pin_memory(), torch.as_tensor(o).pin_memory())
          for q, o in zip(qsets, offs)]
    out_h = torch.empty(total, dtype=torch.int32).pin_memory()
    e2e_t = []
    for i in range(n_steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eat.eat_query_batch_multi(nets, *hq[i][:3], out_h, hq[i][3], stream=stream, **opts)
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    d2h = float(np.mean([4 * int(Vs[q.net].sum()) for q in qsets[args.warmup:]]))

    # The same queries one at a time through eat_query (the plain single-query path).
    q0 = qsets[-1]
    plain_n = min(Q, args.plain_queries)
    for i in range(8):
        eat.eat_query(nets[q0.net[i]], int(q0.source[i]), int(q0.t_s[i]),
                      torch.empty(int(Vs[q0.net[i]]), dtype=torch.int32, device="cuda"))
    rows = {j: torch.empty(int(Vs[j]), dtype=torch.int32, device="cuda") for j in range(len(tts))}
    t0 = time.perf_counter()
    for i in range(plain_n):
        j = int(q0.net[i])
        eat.eat_query(nets[j], int(q0.source[i]), int(q0.t_s[i]), rows[j])
    plain_s = time.perf_counter() - t0

    gpu_s, e2e_s, plain_s = max_over_ranks([gpu_s, sum(e2e_t), plain_s], world)
    if rank != 0:
        return 0
    peak, peak_kind = measured_peak()
    achieved = per_launch / (mean_ms / 1e3) / 1e9

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        scs = [oracle.SortedConnections(t) for t in tts]
        threads = os.cpu_count() or 1
        done, spent, used = 0, 0.0, threads
        for q in qsets[args.warmup:]:
            for j in range(len(tts)):
                sel = np.nonzero(q.net == j)[0]
                if sel.size == 0:
                    continue
                t0 = time.perf_counter()
                _, used = oracle.csa_many(scs[j], q.source[sel], q.t_s[sel], threads)
                spent += time.perf_counter() - t0
                done += sel.size
            if spent >= args.cpu_budget:
                break
        cpu = {"value": done / spent, "unit": "queries/s", "cores": used, "kind": "oracle",
               "sample": f"{done} of the timed steps' queries (whole {Q}-query steps, grouped "
                         f"by network), connection scan on {used} threads, {spent:.1f} s"}

    n_q = Q * args.steps * world
    line = {
        "metric": "EAT queries/s (batched, ragged networks)",
        "value": n_q / gpu_s, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": gpu_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "ragged64: 64 grid networks, stops log-uniform in [1,000, "
                               "50,000], ceil(50 n / 1024) routes of 20 stops, headway 10-30 min",
                   "global_batch": Q, "n_stops_total": int(Vs.sum()),
                   "n_connections": int(sum(t.n_conn for t in tts)), "times": "int32 seconds",
                   "l2": "flushed before every step (256 MB write)", "parallelism": "replicas",
                   "method": "Cluster-AP fixpoint, one launch over all networks"},
        "e2e": {"value": n_q / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": 20 * Q,
                "d2h_bytes_per_step": d2h,
                "path": "blocking eat_query_batch_multi: query arrays staged to the device, "
                        "each converged row written by the kernel into the page-locked host "
                        "output in place (NVLink-C2C)"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_kind": f"{peak_kind} (burst copy)", "kernel": kernel_name,
                     "alg_bytes_per_launch": per_launch},
        "cpu_baseline": cpu,
        "sequential_plain_queries": {"value": plain_n / plain_s, "unit": "queries/s",
                                     "queries": plain_n},
        "launch_shape": {**{k: shape[k] for k in ("block", "vwarp", "mode", "order", "horizon")},
                         "chosen_by": "autotuner" if tuned else "library default or flags"},
        "cluster_width_s": args.cluster_width,
        "work_per_query": {n: tot[n] / (Q * args.steps) for n in names},
        "clocks": clocks.summary(), "kernel_hash": kernel_hash(), "build_s": t_build,
    }
    print(json.dumps(line))
    return 0


def run_serve(args):
    """Served queries: city network + 16 small grids resident; Poisson arrivals.  Rows of a
    1 % sample are kept and compared with the oracle after each rate's run, outside the
    submit/poll loop."""
    import torch
    import oracle
    from paper_1912_00966_gb300 import eat

    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    dev = torch.cuda.current_device()
    tts = [synth.city()] + [synth.small_grid(seed_offset=k) for k in range(16)]
    nets = [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=dev,
                          cluster_width=args.cluster_width) for t in tts]
    scs = {j: oracle.SortedConnections(t) for j, t in enumerate(tts)}   # before any timing
    results = []
    for rate in args.serve_rates:
        server = eat.Server(nets, max_batch=args.serve_batch, max_inflight=4,
                            batch_wait_us=args.serve_wait_us, admission=args.serve_admission)
        rng = np.random.default_rng(rate)
        n = int(rate * args.serve_seconds)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        qs = synth.random_queries(tts, n, 0x5E + rate)
        pool = {j: [np.empty(tts[j].n_stops, np.int32) for _ in range(64)] for j in range(len(tts))}
        inflight = {}
        kept = {}                     # the 1 % sample's rows, checked after the run
        lat, lag, bad_status = [], [], 0
        done = 0

        def drain(timeout_us):
            nonlocal done, bad_status
            for tag, status, net, l_ns in server.poll(timeout_us=timeout_us):
                buf = inflight.pop(tag)
                lat.append(l_ns / 1e6)
                if status != 0:
                    bad_status += 1
                if tag % 100 == 0:
                    kept[tag] = buf
                else:
                    pool[net].append(buf)
                done += 1

        t0 = time.perf_counter()
        i = 0
        while i < n:
            now = time.perf_counter() - t0
            while i < n and arrivals[i] <= now:
                j = int(qs.net[i])
                if not pool[j]:
                    pool[j].append(np.empty(tts[j].n_stops, np.int32))
                buf = pool[j].pop()
                inflight[i] = buf
                server.submit(j, int(qs.source[i]), int(qs.t_s[i]), buf, i)
                lag.append((time.perf_counter() - t0 - arrivals[i]) * 1e3)
                i += 1
            drain(0)
        while done < n:
            drain(5000)
        wall = time.perf_counter() - t0
        st = server.stats()
        server.close()
        mismatches = 0
        for tag, buf in kept.items():
            want = oracle.csa(scs[int(qs.net[tag])], int(qs.source[tag]), int(qs.t_s[tag]))
            mismatches += int(not np.array_equal(buf, want))
        results.append({
            "offered_qps": rate, "seconds": args.serve_seconds, "requests": n,
            "sustained_qps": n / wall, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(np.max(lat)),
            "submit_lag_p99_ms": float(np.percentile(lag, 99)),
            "launches": st["batches"], "admitted_into_running_launch": st["admitted_running"],
            "max_on_gpu": st["max_inflight_seen"], "ring_or_slots": st["slots"],
            "checked_vs_oracle": len(kept), "mismatches": mismatches, "bad_status": bad_status,
        })
    line = {
        "metric": "EAT serving latency and sustained queries/s", "unit": "ms / queries/s",
        "n_gpus": 1, "higher_is_better": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "serve: city20k network + 16 grid1024 networks resident; "
                               "Poisson arrivals, random network / source / t_s",
                   "admission": {0: "ring (requests join the running launch)",
                                 1: "batches per slot"}[args.serve_admission],
                   "max_batch": args.serve_batch, "slots": 4,
                   "batch_wait_us": args.serve_wait_us, "cluster_width_s": args.cluster_width},
        "rates": results, "kernel_hash": kernel_hash(),
    }
    print(json.dumps(line))
    return 0


def workload(name: str, seed_offset: int = 0):
    if name == "city":
        return synth.city(seed_offset=seed_offset), BATCH
    if name == "small":
        return synth.small_grid(seed_offset=seed_offset), BATCH
    if name == "large":
        return synth.large(seed_offset=seed_offset), 1024
    raise SystemExit(f"unknown workload {name}")


def describe(name, tt, batch):
    desc = {
        "city": "city20k: 20,000-stop geometric k=4 network, 400 routes x2 directions of 30-60 "
                "stops, headway 5-20 min, 20% jittered trips, 2 duration bands",
        "small": "grid1024: 32x32 grid, 50 routes of 20 stops, headway 10-30 min",
        "large": "large200k: 200,000-stop geometric k=5 network, 4,000 routes x2 of 40-80 "
                 "stops, headway 3-30 min, 10% jittered trips, 3 duration bands",
    }[name]
    return {"workload": desc, "global_batch": batch, "n_stops": int(tt.n_stops),
            "method": "Cluster-AP fixpoint, rounds inside one launch (launch_shape gives the kernel)",
            "n_connections": int(tt.n_conn), "times": "int32 seconds",
            "l2": "flushed before every step (256 MB write)", "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.02)

    def mark(self):
        self.start = len(self.lines)

    def stop_mark(self):
        self.end = len(self.lines)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = getattr(self, "start", 0)
        hi = max(getattr(self, "end", len(self.lines)), lo + 1)
        for line in self.lines[lo:hi]:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def rank_query_sets(nets, batch, n_steps, rank, base_seed):
    """This rank's query batches: every rank draws its own (weak scaling, replicas); the
    seeds of different ranks never meet for fewer than 1,000 steps."""
    return [synth.random_queries(nets, batch, base_seed + 1000 * rank + i) for i in range(n_steps)]


def max_over_ranks(values, world):
    """Element-wise maximum over ranks (the slowest replica sets the whole-job time)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_oracle_rate(tt, batches, budget_s, threads):
    """Time the oracle on whole 256-query batches until about budget_s seconds pass."""
    import oracle
    sc = oracle.SortedConnections(tt)
    done, t_used = 0, 0.0
    used = threads
    for src, ts in batches:
        t0 = time.perf_counter()
        _, used = oracle.csa_many(sc, src, ts, threads)
        t_used += time.perf_counter() - t0
        done += len(src)
        if t_used >= budget_s:
            break
    return done / t_used, used, done, t_used


def cpu_oracle_latency(tt, src, ts, budget_s, max_q=64):
    """The oracle one query at a time on one thread (the paper's serial baseline)."""
    import oracle
    sc = oracle.SortedConnections(tt)
    oracle.csa(sc, int(src[0]), int(ts[0]))
    done, t_used = 0, 0.0
    for i in range(min(max_q, len(src))):
        t0 = time.perf_counter()
        oracle.csa(sc, int(src[i]), int(ts[i]))
        t_used += time.perf_counter() - t0
        done += 1
        if t_used >= budget_s:
            break
    return 1e3 * t_used / done, done


LADDER_NAMES = {1: "Connection (Algorithm 4)", 2: "Connection-Type (Algorithm 5)",
                3: "Connection-Type-AP (Algorithm 6)", 4: "Cluster-AP (Section II-D)",
                5: "Edge (Section II-E)", 6: "Warps (Section II-F)"}


def run_ladder(args):
    """Single-query latency of the paper's topology-driven variants (Table II's ladder, on
    the synthetic city network), with the flag read after every round and every
    ceil(sqrt(d)) rounds (Section IV-C), each with one launch per round and with the rounds
    between flag reads replayed as a CUDA graph, beside the frontier-driven kernel and the
    oracle."""
    import torch
    from paper_1912_00966_gb300 import eat
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    tt = synth.city()
    V = tt.n_stops
    n_q = args.batch or 16
    qs = synth.random_queries(tt, n_q, 0xB0)
    t0 = time.perf_counter()
    lad = eat.eat_ladder_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur,
                               cluster_width=args.cluster_width, device=0)
    t_build = time.perf_counter() - t0
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0,
                        cluster_width=args.cluster_width)
    out = torch.empty(V, dtype=torch.int32, device="cuda")
    pairs = [(int(qs.source[i]), int(qs.t_s[i])) for i in range(n_q)]
    # Temporal depth of the sample: rounds with a flag read after every round, minus the
    # last round that finds nothing.
    depth = 0
    for s_, t_ in pairs:
        _, st = eat.eat_ladder_query(lad, eat.EAT_VAR_CLUSTER_AP, s_, t_, out=out, flag_every=1)
        depth = max(depth, st["rounds"] - 1)
    every_sqrt = max(1, int(np.ceil(np.sqrt(depth))))

    def timed(fn):
        fn(*pairs[0])
        torch.cuda.synchronize()
        t = time.perf_counter()
        extra = [fn(s_, t_) for s_, t_ in pairs]
        return 1e3 * (time.perf_counter() - t) / n_q, extra

    rows = []
    with ClockSampler(0) as clocks:
        clocks.wait_first()
        clocks.mark()
        for v in range(1, 7):
            for every in (1, every_sqrt):
                for graph in (False, True):
                    ms, st = timed(lambda s_, t_: eat.eat_ladder_query(
                        lad, v, s_, t_, out=out, flag_every=every, graph=graph)[1])
                    rows.append({"variant": LADDER_NAMES[v], "flag_every": every,
                                 "cuda_graph": graph, "ms_per_query": ms,
                                 "rounds_mean": float(np.mean([x["rounds"] for x in st])),
                                 "flag_reads_mean": float(np.mean([x["flag_reads"] for x in st]))})
        ms_front, _ = timed(lambda s_, t_: eat.eat_query(net, s_, t_, out))
        src_d = torch.as_tensor(qs.source).cuda()
        ts_d = torch.as_tensor(qs.t_s).cuda()
        rows_d = torch.empty(n_q * V, dtype=torch.int32, device="cuda")
        eat.eat_query_batch(net, src_d, ts_d, rows_d)
        torch.cuda.synchronize()
        t = time.perf_counter()
        eat.eat_query_batch(net, src_d, ts_d, rows_d)
        torch.cuda.synchronize()
        ms_batch = 1e3 * (time.perf_counter() - t) / n_q
        clocks.stop_mark()
    cpu_ms = None
    if not args.no_cpu_baseline:
        cpu_ms, _ = cpu_oracle_latency(tt, qs.source, qs.t_s, 10.0, max_q=n_q)
    for r in rows:
        r["speedup_vs_oracle_single_thread"] = None if cpu_ms is None else cpu_ms / r["ms_per_query"]
    line = {
        "metric": "EAT single-query latency by variant (the ladder of Section II, Table II)",
        "unit": "ms/query", "n_gpus": 1, "higher_is_better": False, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": describe("city", tt, n_q)["workload"], "queries": n_q,
                   "cluster_width_s": args.cluster_width, "temporal_depth_of_sample": depth,
                   "timing": "host wall clock around each blocking call; L2 not flushed"},
        "variants": rows,
        "frontier_kernel": {"eat_query_ms": ms_front, "eat_query_batch_ms_per_query": ms_batch},
        "oracle_single_thread_ms_per_query": cpu_ms,
        "ladder_build_s": t_build,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line))
    lad.close()
    return 0


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    tt, batch = workload(args.workload)
    batch = args.batch or batch
    # Each step runs the oracle on a bounded sample of the step's batch (its first
    # `sample` queries) so that the run ends within minutes: the connection scan takes
    # about 4 s for a whole 1,024-query batch of the large network on 16 host cores.
    sample = min(batch, args.ref_sample or (64 if args.workload == "large" else batch))
    batches = [(q.source[:sample], q.t_s[:sample]) for q in
               (synth.random_queries(tt, batch, 0xB0 + i) for i in range(args.warmup + args.steps))]
    import oracle
    sc = oracle.SortedConnections(tt)
    threads = os.cpu_count() or 1
    used = threads
    for src, ts in batches[:args.warmup]:
        oracle.csa_many(sc, src, ts, threads)
    times = []
    for src, ts in batches[args.warmup:]:
        t0 = time.perf_counter()
        _, used = oracle.csa_many(sc, src, ts, threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * len(times) / total
    line = {
        "impl": "reference", "metric": "EAT queries/s (batched)", "value": value,
        "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times) * batch / sample, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": describe(args.workload, tt, batch),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": used, "kind": "oracle",
                         "sample": (f"every query of each {batch}-query step" if sample == batch
                                    else f"the first {sample} queries of each {batch:,}-query step")
                                   + f", connection scan (Algorithm 1) on {used} host threads"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    from paper_1912_00966_gb300 import eat

    tt, batch = workload(args.workload)
    batch = args.batch or batch
    t_build = time.perf_counter()
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=dev, trip=tt.trip,
                        subtrips=args.subtrips, cluster_width=args.cluster_width)
    t_build = time.perf_counter() - t_build
    st = eat.eat_get_stats(net)
    V = tt.n_stops
    n_steps = args.warmup + args.steps
    qsets = rank_query_sets(tt, batch, n_steps, rank, 0xB0)
    src_d = [torch.as_tensor(q.source).cuda() for q in qsets]
    ts_d = [torch.as_tensor(q.t_s).cuda() for q in qsets]
    out = torch.empty(batch * V, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((n_steps, batch, 7), dtype=torch.int64, device="cuda")
    status = torch.zeros((n_steps, batch), dtype=torch.int32, device="cuda")
    opts = dict(vwarp=args.vwarp, block=args.block, mode=args.mode, horizon=args.horizon,
                order=args.order)
    tuned = None
    if args.autotune and not (args.vwarp or args.block or args.mode or args.horizon):
        # Launch shape chosen by the library's autotuner on a sample batch (setup, untimed).
        sample = synth.random_queries(tt, batch, 0xB0 - 1)
        tuned = eat.eat_autotune(net, torch.as_tensor(sample.source).cuda(),
                                 torch.as_tensor(sample.t_s).cuda())
    shape = eat.eat_launch_shape(net, batch, **opts)      # the shape the timed launches run
    ws = torch.empty(eat.eat_workspace_bytes(net, batch, **opts), dtype=torch.uint8, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_steps)]

    # Work counters of every step's batch come from an untimed pass over the same
    # queries: the timed launches run without counters (the paired kernel has a
    # separate counting build), and a query's counts vary only slightly between runs
    # (the order of relaxations within a round is not fixed).
    for i in range(n_steps):
        eat.eat_query_batch(net, src_d[i], ts_d[i], out, workspace=ws, stream=stream,
                            counters=cnt[i], **opts)
    torch.cuda.synchronize()

    def step(i):
        flush.fill_(i)
        a, b = evs[i]
        a.record(stream)
        eat.eat_query_batch(net, src_d[i], ts_d[i], out, workspace=ws, stream=stream,
                            status=status[i], **opts)
        b.record(stream)

    with ClockSampler(dev) as clocks:
        clocks.wait_first()
        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.mark()
        t_wall = time.perf_counter()
        for i in range(args.warmup, n_steps):
            step(i)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        time.sleep(0.06)
        clocks.stop_mark()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [evs[i][0].elapsed_time(evs[i][1]) for i in range(args.warmup, n_steps)]
    gpu_s = sum(step_ms) / 1e3
    if (status.cpu().numpy() != 0).any():
        raise SystemExit("bench: a query did not converge")
    c = cnt[args.warmup:].sum(dim=(0, 1)).cpu().numpy()
    names = eat.COUNTER_FIELDS
    tot = {n: int(c[k]) for k, n in enumerate(names)}
    alg_bytes = sum(BYTES[n] * tot[n] for n in BYTES) + 8 * V * batch * args.steps
    per_launch = alg_bytes / args.steps
    mean_ms = gpu_s * 1e3 / args.steps

    # The same queries end to end through the C ABI from pinned host buffers.
    src_h = [torch.as_tensor(q.source).pin_memory() for q in qsets]
    ts_h = [torch.as_tensor(q.t_s).pin_memory() for q in qsets]
    out_h = torch.empty(batch * V, dtype=torch.int32).pin_memory()
    for i in range(args.warmup):
        eat.eat_query_batch(net, src_h[i], ts_h[i], out_h, stream=stream, **opts)
    e2e_t = []
    for i in range(args.warmup, n_steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eat.eat_query_batch(net, src_h[i], ts_h[i], out_h, stream=stream, **opts)
        e2e_t.append(time.perf_counter() - t0)

    # The same steps on the network without sub-trips (Section II-G off), for comparison.
    base_ms = None
    if args.subtrips:
        net0 = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=dev,
                             cluster_width=args.cluster_width)
        ws0 = torch.empty(eat.eat_workspace_bytes(net0, batch, **opts), dtype=torch.uint8,
                          device="cuda")
        e0 = []
        for i in range(min(n_steps, args.warmup + 50)):
            flush.fill_(i)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eat.eat_query_batch(net0, src_d[i], ts_d[i], out, workspace=ws0, stream=stream, **opts)
            b.record(stream)
            e0.append((a, b))
        torch.cuda.synchronize()
        base_ms = statistics.mean(a.elapsed_time(b) for a, b in e0[args.warmup:])
        net0.close()

    # Plain single-query fixpoint (one blocking query at a time), for comparison.
    plain_n = min(64, batch)
    row = torch.empty(V, dtype=torch.int32, device="cuda")
    q0 = qsets[-1]
    for i in range(4):
        eat.eat_query(net, int(q0.source[i]), int(q0.t_s[i]), row)
    t0 = time.perf_counter()
    for i in range(plain_n):
        eat.eat_query(net, int(q0.source[i]), int(q0.t_s[i]), row)
    plain_s = time.perf_counter() - t0

    gpu_s, e2e_s, plain_s = max_over_ranks([gpu_s, sum(e2e_t), plain_s], world)
    if rank != 0:
        return 0

    peak, peak_kind = measured_peak()
    achieved = per_launch / (mean_ms / 1e3) / 1e9
    kernel_name = KERNEL_OF_MODE[shape["mode"]]
    h = kernel_hash()
    traffic = None
    key = (h, kernel_name, shape["block"], shape["horizon"], args.cluster_width)
    if args.workload in NCU_TRAFFIC_PER_QUERY and NCU_TRAFFIC_PER_QUERY[args.workload][:5] == key:
        traffic = NCU_TRAFFIC_PER_QUERY[args.workload][5] * batch

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, used, done, spent = cpu_oracle_rate(
            tt, [(q.source, q.t_s) for q in qsets[args.warmup:]], args.cpu_budget, threads)
        lat_ms, lat_n = cpu_oracle_latency(tt, qsets[args.warmup].source,
                                           qsets[args.warmup].t_s, 2.0)
        cpu = {"value": rate, "unit": "queries/s", "cores": used, "kind": "oracle",
               "sample": f"{done} of the timed steps' queries ({done // batch} whole "
                         f"{batch}-query batches), connection scan on {used} threads, "
                         f"{spent:.1f} s",
               "single_thread_ms_per_query": lat_ms,
               "single_thread_sample": f"first {lat_n} queries of the first timed step, "
                                       "one at a time on one thread"}

    n_q = batch * args.steps * world
    # Connections the connection scan would examine for the same queries (those
    # departing at or after t_s), per second of GPU time.
    dep_sorted = np.sort(tt.dep)
    csa_conn = 0
    for q in qsets[args.warmup:]:
        first = np.searchsorted(dep_sorted, q.t_s, side="left").astype(np.int64)
        csa_conn += int((len(dep_sorted) - first).sum())
    # Mean rounds per query of the timed batches (0 in the round-free mode).
    rounds_mean = tot["rounds"] / (batch * args.steps)
    line = {
        "metric": "EAT queries/s (batched)",
        "value": n_q / gpu_s,
        "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": gpu_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": describe(args.workload, tt, batch),
        "e2e": {"value": n_q / e2e_s, "unit": "queries/s",
                "h2d_bytes_per_step": 2 * 4 * batch, "d2h_bytes_per_step": 4 * V * batch,
                "path": "blocking eat_query_batch on page-locked host buffers: the kernel "
                        "reads the queries and writes each converged row into host memory in "
                        "place (NVLink-C2C); arrivals not in shared memory use a device row "
                        "per persistent block meanwhile"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} (burst copy)",
                     "kernel": kernel_name, "alg_bytes_per_launch": per_launch},
        "cpu_baseline": cpu,
        "connections_relaxed_per_s": tot["types"] / (gpu_s / world),
        "csa_equivalent_connections_per_s": csa_conn / (gpu_s / world),
        "subtrips": {0: "none", 1: "sqrt(k) per trip", 2: "sqrt(mean trip length)"}[args.subtrips],
        "cluster_width_s": args.cluster_width,
        "launch_shape": {**{k: shape[k] for k in ("block", "vwarp", "mode", "order", "horizon")},
                         "chosen_by": "autotuner" if tuned else "library default or flags"},
        "without_subtrips": None if base_ms is None else
            {"value": batch / (base_ms / 1e3), "unit": "queries/s", "ms_per_step": base_ms},
        "build_s": t_build,
        "plain_single_query": {"value": plain_n / plain_s, "unit": "queries/s",
                               "ms_per_query": 1e3 * plain_s / plain_n,
                               "rounds_mean": rounds_mean,
                               "us_per_round": (1e6 * plain_s / plain_n / rounds_mean
                                                if rounds_mean else None)},
        "work_per_query": {n: tot[n] / (batch * args.steps) for n in names},
        "network": {k: st[k] for k in ("n_types", "n_edges", "n_ap", "n_cl", "max_clusters",
                                       "device_bytes", "n_shortcuts", "y")},
        "clocks": clocks.summary(),
        "kernel_hash": h,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["city", "small", "large", "ragged", "serve", "ladder"])
    ap.add_argument("--serve-rates", type=int, nargs="+", default=[1000, 5000, 20000, 50000])
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-admission", type=int, default=0, choices=[0, 1],
                    help="serving: 0 ring (requests join the running launch), 1 batches per slot")
    ap.add_argument("--serve-batch", type=int, default=256)
    ap.add_argument("--serve-wait-us", type=int, default=200)
    ap.add_argument("--plain-queries", type=int, default=4096,
                    help="ragged workload: sequential single queries timed for comparison")
    ap.add_argument("--vwarp", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--mode", type=int, default=0,
                    help="0 auto, 1 rounds, 3 asynchronous, 4 paired, 5 edge min + degree mapping")
    ap.add_argument("--horizon", type=int, default=0,
                    help="seconds; 0 the tuned value (else none), -1 none (every improved stop "
                         "expanded next round, Algorithms 4-5)")
    ap.add_argument("--order", type=int, default=0,
                    help="start order of a batch: 0 automatic, 1 by t_s, 2 as given")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--cluster-width", type=int, default=600,
                    help="seconds per departure cluster (Section II-D uses one hour; Section IV-B finds narrower clusters faster)")
    ap.add_argument("--subtrips", type=int, default=0, choices=[0, 1, 2],
                    help="sub-trip shortcuts (Section II-G): 0 none, 1 sqrt(k), 2 sqrt(mean)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=0,
                    help="--impl reference: queries of each step the oracle runs (default: 64 "
                         "for the large workload, else the whole batch)")
    ap.add_argument("--batch", type=int, default=0,
                    help="queries per step (default: the workload's: 256, or 1,024 for large)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ragged":
        return run_ours_ragged(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "ladder":
        return run_ladder(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
