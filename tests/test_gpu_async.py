"""GPU parity of the round-free mode (EAT_MODE_ASYNC) against the oracle, bit-exact."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ASYNC = 3


@pytest.fixture(scope="module")
def eat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00966_gb300 import eat as mod
    return mod


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _run(eat, net, V, src, ts, **opts):
    n = len(src)
    out = torch.empty(n * V, dtype=torch.int32, device="cuda")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros((n, 7), dtype=torch.int64, device="cuda")
    eat.eat_query_batch(net, _dev(src), _dev(ts), out, status=status, counters=cnt,
                        mode=ASYNC, **opts)
    torch.cuda.synchronize()
    return out.view(n, V).cpu().numpy(), status.cpu().numpy(), cnt.cpu().numpy()


def _net(eat, tt, **kw):
    return eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0, **kw)


@pytest.mark.parametrize("seed", range(24))
def test_async_tiny_nets_all_sources(eat, seed):
    tt = synth.tiny_random(2 + seed % 13, 1 + (seed * 41) % 300, 700 + seed, t_max=300 + 40 * seed,
                           dur_max=1 + seed % 50)
    net = _net(eat, tt, cluster_width=[3600, 60, 7, 1][seed % 4])
    src = np.repeat(np.arange(tt.n_stops), 3).astype(np.int32)
    ts = np.random.default_rng(seed).integers(-5, int(tt.dep.max()) + 10, size=src.shape[0]).astype(np.int32)
    got, status, cnt = _run(eat, net, tt.n_stops, src, ts, block=[64, 256, 512][seed % 3])
    assert (status == 0).all()
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), src, ts, 8)
    assert np.array_equal(got, want)
    assert (cnt[:, 0] == 0).all()
    for i in range(0, len(src), 5):
        assert got[i].tolist() == oracle.brute.foremost_dijkstra(
            tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, int(src[i]), int(ts[i]))


@pytest.mark.parametrize("which,placement,block", [
    ("small", 0, 512), ("small", 2, 256), ("city", 0, 512), ("city", 2, 1024), ("city", 1, 512),
])
def test_async_batches(eat, which, placement, block):
    tt = synth.small_grid() if which == "small" else synth.city()
    net = _net(eat, tt, cluster_width=1800)
    q = synth.random_queries(tt, 256, 0xA5 + block)
    got, status, cnt = _run(eat, net, tt.n_stops, q.source, q.t_s, placement=placement, block=block)
    assert (status == 0).all()
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), q.source, q.t_s, 8)
    assert np.array_equal(got, want)
    again, _, _ = _run(eat, net, tt.n_stops, q.source, q.t_s, placement=placement, block=block)
    assert np.array_equal(again, got)


def test_async_ragged_multi_network(eat):
    tts = [synth.small_grid(), synth.grid_timetable(5000, 245, 77, force_stop0=False),
           synth.grid_timetable(60000, int(np.ceil(50 * 60000 / 1024)), 4242, force_stop0=False)]
    nets = [_net(eat, t) for t in tts]
    Q = 96
    qs = synth.random_queries(tts, Q, 19)
    sizes = np.array([tts[i].n_stops for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    out = torch.full((int(sizes.sum()),), -7, dtype=torch.int32, device="cuda")
    status = torch.full((Q,), -1, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_multi(nets, _dev(qs.net), _dev(qs.source), _dev(qs.t_s), out,
                              torch.as_tensor(offs).cuda(), status=status, mode=ASYNC)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    flat = out.cpu().numpy()
    for i in range(Q):
        tt = tts[qs.net[i]]
        want = oracle.csa(oracle.SortedConnections(tt), int(qs.source[i]), int(qs.t_s[i]))
        assert np.array_equal(flat[offs[i]:offs[i] + tt.n_stops], want), i


def test_async_large_network_all_rows(eat, large_tt, large_sc):
    """The round-free kernel on the 200,000-stop network: 512 queries, every row exact."""
    import os
    tt = large_tt
    net = _net(eat, tt)
    q = synth.random_queries(tt, 512, 0x1B)
    got, status, _ = _run(eat, net, tt.n_stops, q.source, q.t_s)
    assert (status == 0).all()
    want, _ = oracle.csa_many(large_sc, q.source, q.t_s, os.cpu_count() or 8)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, bad[:8]


def test_async_invalid_source_and_noalloc(eat):
    tt = synth.small_grid()
    net = _net(eat, tt)
    src = np.array([0, tt.n_stops, 7], np.int32)
    ts = np.full(3, 30000, np.int32)
    got, status, _ = _run(eat, net, tt.n_stops, src, ts)
    assert status.tolist() == [0, eat.EAT_ERR_INVALID, 0]
    assert (got[1] == 2**31 - 1).all()
    q = synth.random_queries(tt, 200, 4)
    ref = torch.empty(200 * tt.n_stops, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, _dev(q.source), _dev(q.t_s), ref)
    out = torch.empty_like(ref)
    eat.eat_query_batch_noalloc(net, _dev(q.source), _dev(q.t_s), out, mode=ASYNC)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_async_idle_cap_runs_out_with_upper_bounds(eat):
    """A tiny idle cap makes the round-free kernel's bounded waits run out (a warp that
    finds no pending stop while other warps still hold work gives up at once): the launch
    returns, every query reports EAT_OK or EAT_ERR_NO_CONVERGENCE, the rows of those that
    gave up are upper bounds of the oracle's, and the others are exact.  With the default
    cap every query converges."""
    tt = synth.city()
    net = _net(eat, tt)
    q = synth.random_queries(tt, 256, 0x1C)
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), q.source, q.t_s, 8)
    got, status, _ = _run(eat, net, tt.n_stops, q.source, q.t_s, idle_cap=1)
    assert set(status.tolist()) <= {eat.EAT_OK, eat.EAT_ERR_NO_CONVERGENCE}
    gave_up = status == eat.EAT_ERR_NO_CONVERGENCE
    assert gave_up.any()
    assert (got.astype(np.int64) >= want).all()
    assert np.array_equal(got[~gave_up], want[~gave_up])
    for i in np.nonzero(gave_up)[0][:4]:
        assert got[i, q.source[i]] == q.t_s[i]
    got, status, _ = _run(eat, net, tt.n_stops, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, want)
