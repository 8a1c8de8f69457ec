"""Autotuning and CUDA-graph capture of the batched query path (GPU)."""
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def test_autotune_picks_a_candidate_and_keeps_results(eat):
    tt = synth.city()
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0)
    q = synth.random_queries(tt, 128, 0xA7)
    src, ts = _dev(q.source), _dev(q.t_s)
    shape = eat.eat_autotune(net, src, ts)
    assert shape["block"] in (256, 512, 1024) and shape["vwarp"] in (2, 4, 8, 16, 32)
    assert shape["mode"] in (1, 3)
    out = torch.empty(128 * tt.n_stops, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, src, ts, out)            # uses the tuned shape
    torch.cuda.synchronize()
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), q.source, q.t_s, 8)
    assert np.array_equal(out.view(128, tt.n_stops).cpu().numpy(), want)


def test_tune_network_over_cluster_widths(eat):
    from paper_1912_00966_gb300.autotune import tune_network
    tt = synth.small_grid()
    q = synth.random_queries(tt, 64, 0xA8)
    net, report = tune_network(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, _dev(q.source),
                               _dev(q.t_s), widths=(3600, 900))
    assert {r["cluster_width"] for r in report} == {3600, 900}
    assert net.stats["cluster_width"] in (3600, 900)
    got = eat.eat_query(net, 0, 28800)
    assert np.array_equal(got, oracle.csa(oracle.SortedConnections(tt), 0, 28800))


def test_cuda_graph_capture_and_replay(eat):
    """The batched call is a memset and one kernel on the given stream, so it can be
    captured once and replayed on new inputs written into the same buffers."""
    tt = synth.city()
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0)
    n, V = 64, tt.n_stops
    src = torch.zeros(n, dtype=torch.int32, device="cuda")
    ts = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n * V, dtype=torch.int32, device="cuda")
    ws = torch.empty(eat.eat_workspace_bytes(net, n), dtype=torch.uint8, device="cuda")
    q0 = synth.random_queries(tt, n, 1)
    src.copy_(torch.as_tensor(q0.source))
    ts.copy_(torch.as_tensor(q0.t_s))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        eat.eat_query_batch(net, src, ts, out, workspace=ws, stream=s)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        eat.eat_query_batch(net, src, ts, out, workspace=ws, stream=s)
    sc = oracle.SortedConnections(tt)
    for seed in (2, 3, 4):
        q = synth.random_queries(tt, n, seed)
        src.copy_(torch.as_tensor(q.source))
        ts.copy_(torch.as_tensor(q.t_s))
        g.replay()
        torch.cuda.synchronize()
        want, _ = oracle.csa_many(sc, q.source, q.t_s, 8)
        assert np.array_equal(out.view(n, V).cpu().numpy(), want)


def test_autotune_multi_over_ragged_networks(eat):
    """eat_autotune_multi picks a shape and start order for a batch over networks of uneven
    size; a launch with that shape gives the oracle's rows."""
    tts = [synth.small_grid()] + [synth.grid_timetable(n, int(np.ceil(50 * n / 1024)), 600 + n,
                                                       force_stop0=False) for n in (2000, 9000)]
    nets = [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=0) for t in tts]
    Q = 512
    qs = synth.random_queries(tts, Q, 0xA9)
    shape = eat.eat_autotune_multi(nets, _dev(qs.net), _dev(qs.source), _dev(qs.t_s))
    assert shape["block"] in (256, 512, 1024) and shape["vwarp"] in (2, 4, 8, 16, 32)
    assert shape["mode"] in (1, 3)
    assert shape["order"] in (eat.EAT_ORDER_BY_TIME, eat.EAT_ORDER_AS_GIVEN)
    assert eat.eat_launch_shape(nets, Q, **shape)["order"] == shape["order"]
    sizes = np.array([tts[i].n_stops for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    out = torch.full((int(sizes.sum()),), -7, dtype=torch.int32, device="cuda")
    status = torch.full((Q,), -1, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_multi(nets, _dev(qs.net), _dev(qs.source), _dev(qs.t_s), out,
                              torch.as_tensor(offs).cuda(), status=status, **shape)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    flat = out.cpu().numpy()
    for j, tt in enumerate(tts):
        sel = np.nonzero(qs.net == j)[0]
        want, _ = oracle.csa_many(oracle.SortedConnections(tt), qs.source[sel], qs.t_s[sel], 8)
        for r, i in enumerate(sel):
            assert np.array_equal(flat[offs[i]:offs[i] + tt.n_stops], want[r]), (j, i)
    for order in (eat.EAT_ORDER_BY_TIME, eat.EAT_ORDER_AS_GIVEN):
        out2 = torch.full_like(out, -7)
        eat.eat_query_batch_multi(nets, _dev(qs.net), _dev(qs.source), _dev(qs.t_s), out2,
                                  torch.as_tensor(offs).cuda(), order=order)
        torch.cuda.synchronize()
        assert torch.equal(out, out2)
    with pytest.raises(eat.EatError):
        eat.eat_autotune_multi(nets, qs.net, qs.source, qs.t_s)        # host arrays
