"""Serving loop (eat_server_*): continuous batching over resident networks.

Each result must be identical whether the query runs alone (eat_query) or in
the mix of a served stream, in both admission modes (a ring of requests served by
one running launch, or batches per slot), and what is in flight must respect the
memory budget.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00966_gb300 import eat as mod
    return mod


@pytest.fixture(scope="module")
def nets(eat):
    tts = [synth.city(), synth.small_grid()] + [synth.small_grid(seed_offset=k) for k in (1, 2, 3)]
    return tts, [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=0) for t in tts]


def _serve(eat, server, tts, qs, pace_s=0.0):
    """Submit every query (optionally spread over time) and poll until all are back."""
    outs = [np.full(tts[j].n_stops, -7, np.int32) for j in qs.net]
    got = {}

    def poller():
        while len(got) < len(qs):
            for tag, status, net, lat in server.poll(timeout_us=2000):
                got[tag] = (status, lat)

    th = threading.Thread(target=poller)
    th.start()
    for i in range(len(qs)):
        server.submit(int(qs.net[i]), int(qs.source[i]), int(qs.t_s[i]), outs[i], i)
        if pace_s and i % 16 == 0:
            time.sleep(pace_s)
    th.join(timeout=120)
    assert len(got) == len(qs)
    return outs, got


@pytest.mark.parametrize("admission", [0, 1])
def test_served_results_equal_alone(eat, nets, admission):
    tts, ns = nets
    server = eat.Server(ns, max_batch=64, max_inflight=4, admission=admission)
    qs = synth.random_queries(tts, 1500, 31)
    outs, got = _serve(eat, server, tts, qs)
    assert all(st == 0 for st, _ in got.values())
    for i in range(len(qs)):
        alone = eat.eat_query(ns[qs.net[i]], int(qs.source[i]), int(qs.t_s[i]))
        assert np.array_equal(outs[i], alone), i
    for i in range(0, len(qs), 97):
        want = oracle.csa(oracle.SortedConnections(tts[qs.net[i]]), int(qs.source[i]), int(qs.t_s[i]))
        assert np.array_equal(outs[i], want)
    st = server.stats()
    assert st["completed"] == len(qs) and st["batched_queries"] == len(qs)
    if admission == eat.EAT_ADMIT_BATCH:
        assert st["batches"] >= len(qs) // 64 and st["max_batch_seen"] <= 64
    else:
        assert st["slots"] == 256 and st["max_inflight_seen"] <= 256 and st["batches"] >= 1
    server.close()


def test_ring_admits_into_a_running_launch(eat, nets):
    """Ring admission: requests that arrive while the launch runs (paced submissions) enter
    its ring and are served by it; each row equals the row of the same query run alone and
    the oracle's.  A later burst after an idle gap starts a new launch."""
    tts, ns = nets
    server = eat.Server(ns, max_batch=16, max_inflight=4, admission=eat.EAT_ADMIT_RING)
    qs = synth.random_queries(tts, 800, 35)
    outs, got = _serve(eat, server, tts, qs, pace_s=0.0003)
    assert all(st == 0 for st, _ in got.values())
    st = server.stats()
    assert st["slots"] == 64 and st["max_inflight_seen"] <= 64
    assert st["admitted_running"] > 0
    for i in range(len(qs)):
        alone = eat.eat_query(ns[qs.net[i]], int(qs.source[i]), int(qs.t_s[i]))
        assert np.array_equal(outs[i], alone), i
    for i in range(0, len(qs), 41):
        want = oracle.csa(oracle.SortedConnections(tts[qs.net[i]]), int(qs.source[i]), int(qs.t_s[i]))
        assert np.array_equal(outs[i], want)
    launches = st["batches"]
    time.sleep(0.05)                                 # idle: the launch ends
    qs2 = synth.random_queries(tts, 100, 36)
    outs2, got2 = _serve(eat, server, tts, qs2)
    assert server.stats()["batches"] > launches
    for i in range(len(qs2)):
        assert np.array_equal(outs2[i], eat.eat_query(ns[qs2.net[i]], int(qs2.source[i]),
                                                        int(qs2.t_s[i])))
    server.close()


def test_paced_arrivals_overlap_and_match(eat, nets):
    tts, ns = nets
    server = eat.Server(ns, max_batch=32, max_inflight=3, batch_wait_us=100,
                        admission=eat.EAT_ADMIT_BATCH)
    qs = synth.random_queries(tts, 600, 32)
    outs, got = _serve(eat, server, tts, qs, pace_s=0.0005)
    for i in range(len(qs)):
        assert np.array_equal(outs[i], eat.eat_query(ns[qs.net[i]], int(qs.source[i]),
                                                       int(qs.t_s[i])))
    st = server.stats()
    assert st["slots"] == 3
    assert st["max_inflight_seen"] >= 2           # batches overlapped on the device
    server.close()


def test_ring_admission_by_memory(eat, nets):
    """The ring holds as many requests as the budget allows beyond the launch's
    workspace (rounded down to a power of two); no more are on the GPU at once."""
    tts, ns = nets
    with pytest.raises(eat.EatError) as ei:
        eat.Server(ns, mem_budget=1000, admission=eat.EAT_ADMIT_RING)
    assert ei.value.code == eat.EAT_ERR_OOM
    probe = eat.Server(ns, admission=eat.EAT_ADMIT_RING)
    pst = probe.stats()
    probe.close()
    budget = pst["base_bytes"] + 3 * pst["slot_bytes"] + pst["slot_bytes"] // 2
    server = eat.Server(ns, mem_budget=budget, admission=eat.EAT_ADMIT_RING)
    assert server.stats()["slots"] == 2
    qs = synth.random_queries(tts, 200, 34)
    outs, got = _serve(eat, server, tts, qs)
    assert server.stats()["max_inflight_seen"] <= 2
    for i in range(0, len(qs), 5):
        assert np.array_equal(outs[i], eat.eat_query(ns[qs.net[i]], int(qs.source[i]),
                                                       int(qs.t_s[i])))
    server.close()


def test_admission_by_memory(eat, nets):
    tts, ns = nets
    with pytest.raises(eat.EatError) as ei:
        eat.Server(ns, max_batch=32, mem_budget=1000, admission=eat.EAT_ADMIT_BATCH)
    assert ei.value.code == eat.EAT_ERR_OOM
    probe = eat.Server(ns, max_batch=32, max_inflight=1, admission=eat.EAT_ADMIT_BATCH)
    slot = probe.stats()["slot_bytes"]
    probe.close()
    server = eat.Server(ns, max_batch=32, max_inflight=8, mem_budget=slot + slot // 2,
                        admission=eat.EAT_ADMIT_BATCH)
    st = server.stats()
    assert st["slots"] == 1
    qs = synth.random_queries(tts, 300, 33)
    outs, got = _serve(eat, server, tts, qs)
    assert server.stats()["max_inflight_seen"] == 1
    for i in range(0, len(qs), 7):
        assert np.array_equal(outs[i], eat.eat_query(ns[qs.net[i]], int(qs.source[i]),
                                                       int(qs.t_s[i])))
    server.close()


@pytest.mark.parametrize("admission", [0, 1])
def test_invalid_submit_and_drain_on_close(eat, nets, admission):
    tts, ns = nets
    server = eat.Server(ns, max_batch=16, admission=admission)
    buf = np.empty(tts[0].n_stops, np.int32)
    with pytest.raises(eat.EatError):
        server.submit(len(ns), 0, 0, buf, 1)
    with pytest.raises(eat.EatError):
        server.submit(0, tts[0].n_stops, 0, buf, 1)
    outs = [np.full(tts[1].n_stops, -7, np.int32) for _ in range(50)]
    for i in range(50):
        server.submit(1, 0, 30000 + 60 * i, outs[i], i)
    server.close()                                  # drains the queue before stopping
    for i in range(50):
        assert np.array_equal(outs[i], eat.eat_query(ns[1], 0, 30000 + 60 * i))
