"""Autotuning of the query path: launch shape (in libeat, eat_autotune) and the cluster
width of the build (Section IV-B's cluster-size parameter, which needs a rebuild).

Everything here measures real launches through the C ABI on a caller's sample batch;
nothing is computed on the host.
"""
from __future__ import annotations

from . import eat


def tune_network(n_stops, u, v, dep, dur, sample_sources, sample_times,
                 widths=(3600, 1800, 900), device=0, repeats=3, **build_kw):
    """Build the network once per cluster width, tune each one's launch shape on the sample
    (device int32 tensors), time the tuned shape and keep the fastest network.

    Returns (net, report) where report lists {"cluster_width", "block", "vwarp", "ms"}."""
    import torch

    best, report = None, []
    n = int(sample_sources.shape[0])
    for w in widths:
        net = eat.eat_build(n_stops, u, v, dep, dur, cluster_width=w, device=device, **build_kw)
        shape = eat.eat_autotune(net, sample_sources, sample_times)
        out = torch.empty(n * net.stats["n_stops"], dtype=torch.int32, device="cuda")
        ws = torch.empty(eat.eat_workspace_bytes(net, n), dtype=torch.uint8, device="cuda")
        eat.eat_query_batch(net, sample_sources, sample_times, out, workspace=ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(repeats):
            eat.eat_query_batch(net, sample_sources, sample_times, out, workspace=ws)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / repeats
        report.append({"cluster_width": w, **shape, "ms": ms})
        if best is None or ms < best[1]:
            if best is not None:
                best[0].close()
            best = (net, ms)
        else:
            net.close()
    return best[0], report
