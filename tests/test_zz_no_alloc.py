"""eat_query_batch_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (for example a plugin whose host application owns every device
allocation, or a serving loop held to a fixed memory reservation) cannot hand
eat_query_batch a workspace.  The no-allocation entry point runs the same kernel
with its frontier queues in a fixed scratch array inside libeat.  This file checks,
through the C ABI, that it returns exactly what eat_query_batch returns on two
calls in a row (the scratch keeps the previous call's contents, so the second call
shows it is cleared where it must be), and that it rejects what it cannot serve.

It is collected last on purpose and builds its own networks, so it passes both alone
in a fresh process and after the other GPU tests.
"""
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


@pytest.mark.parametrize("which", ["small", "city"])
def test_noalloc_matches_batch_on_two_calls(eat, which):
    tt = synth.small_grid() if which == "small" else synth.city()
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0)
    V = tt.n_stops
    for call, seed in enumerate((11, 12)):
        q = synth.random_queries(tt, 300, seed)
        src, ts = _dev(q.source), _dev(q.t_s)
        ref = torch.empty(300 * V, dtype=torch.int32, device="cuda")
        eat.eat_query_batch(net, src, ts, ref)
        got = torch.full((300 * V,), -1, dtype=torch.int32, device="cuda")
        status = torch.full((300,), -1, dtype=torch.int32, device="cuda")
        eat.eat_query_batch_noalloc(net, src, ts, got, status=status)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all(), call
        assert torch.equal(got, ref), call          # integers: exact, as every parity test here
    # and the last call against the oracle itself
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), q.source, q.t_s, 8)
    assert np.array_equal(got.view(300, V).cpu().numpy(), want)
    net.close()


@pytest.mark.parametrize("which,opts", [
    ("city", {"mode": 4}),          # paired mode: two queries per block, 16 bytes per stop
    ("city", {"mode": 3}),          # round-free mode: no spill queues
    ("small", {"placement": 3}),    # arrivals and bitmaps in global memory
])
def test_noalloc_other_layouts_match_batch_on_two_calls(eat, which, opts):
    """The scratch is laid out differently by the paired mode, the round-free mode and
    global bitmaps; each still returns what eat_query_batch returns, twice in a row."""
    tt = synth.small_grid() if which == "small" else synth.city()
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0)
    V = tt.n_stops
    for call, seed in enumerate((21, 22)):
        q = synth.random_queries(tt, 300, seed)
        src, ts = _dev(q.source), _dev(q.t_s)
        ref = torch.empty(300 * V, dtype=torch.int32, device="cuda")
        eat.eat_query_batch(net, src, ts, ref, **opts)
        got = torch.full((300 * V,), -1, dtype=torch.int32, device="cuda")
        status = torch.full((300,), -1, dtype=torch.int32, device="cuda")
        eat.eat_query_batch_noalloc(net, src, ts, got, status=status, **opts)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all(), call
        assert torch.equal(got, ref), call
    want, _ = oracle.csa_many(oracle.SortedConnections(tt), q.source, q.t_s, 8)
    assert np.array_equal(got.view(300, V).cpu().numpy(), want)
    net.close()


def test_noalloc_rejects_what_it_cannot_serve(eat):
    tt = synth.small_grid()
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0)
    q = synth.random_queries(tt, 4, 1)
    host_out = np.empty(4 * tt.n_stops, dtype=np.int32)
    with pytest.raises(eat.EatError) as ei:
        eat.eat_query_batch_noalloc(net, _dev(q.source), _dev(q.t_s), host_out)
    assert ei.value.code == eat.EAT_ERR_INVALID
    n = 2_000_001                                   # one stop beyond the stated limit
    big = eat.eat_build(n, [0], [1], [100], [10], device=0)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(eat.EatError) as ei:
        eat.eat_query_batch_noalloc(big, _dev([0]), _dev([0]), out)
    assert ei.value.code == eat.EAT_ERR_INVALID
    assert "no-allocation scratch" in str(ei.value)
    big.close()
    if torch.cuda.device_count() > 1:               # a buffer on another GPU is refused
        other = torch.empty(4 * tt.n_stops, dtype=torch.int32, device="cuda:1")
        with pytest.raises(eat.EatError) as ei:
            eat.eat_query_batch_noalloc(net, _dev(q.source), _dev(q.t_s), other)
        assert ei.value.code == eat.EAT_ERR_INVALID
    net.close()
