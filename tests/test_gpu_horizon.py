"""The horizon option of the per-query kernel (eat_query_opts.horizon) against the oracle.

With a horizon, a stop lowered to an arrival at or after the horizon waits until no stop
below it is left to expand, and the horizon then moves to the earliest waiting arrival
plus the step.  Only the order of relaxations changes, so every row must equal the
connection-scan oracle's (Algorithm 1) bit for bit: on tiny random networks (also
against brute force), the small grid (one-word items), the city network (arrivals in
shared memory, in global memory, bitmaps in global memory), with the degree-chosen edge
mode, for horizons from one minute (most stops wait) to far beyond the day (none
waits), with a round cap, through the no-allocation entry point and in a batch over
several networks of uneven size.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = 2**31 - 1
HORIZONS = [1, 60, 900, 7200, 43200, 10**9]


@pytest.fixture(scope="module")
def eat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00966_gb300 import eat as mod
    return mod


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).cuda()


class Net:
    def __init__(self, eat, tt, **kw):
        self.tt = tt
        self.V = tt.n_stops
        self.net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0, **kw)
        self.sc = oracle.SortedConnections(tt)

    def oracle_rows(self, src, ts):
        return oracle.csa_many(self.sc, src, ts, os.cpu_count() or 8)[0]

    def run(self, eat, src, ts, **opts):
        n = len(src)
        out = torch.full((n * self.V,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros((n, 7), dtype=torch.int64, device="cuda")
        eat.eat_query_batch(self.net, _dev(src), _dev(ts), out, status=status, counters=cnt, **opts)
        torch.cuda.synchronize()
        return out.view(n, self.V).cpu().numpy(), status.cpu().numpy(), cnt.cpu().numpy()


@pytest.fixture(scope="module")
def small(eat):
    return Net(eat, synth.small_grid())


@pytest.fixture(scope="module")
def city(eat):
    return Net(eat, synth.city(), cluster_width=600)


@pytest.mark.parametrize("seed", range(16))
def test_tiny_random_nets(eat, seed):
    tt = synth.tiny_random(2 + seed % 11, 1 + (seed * 53) % 250, 900 + seed, t_max=200 + 40 * seed,
                           dur_max=1 + seed % 40)
    case = Net(eat, tt, cluster_width=[3600, 60, 7][seed % 3])
    src = np.repeat(np.arange(tt.n_stops), 3).astype(np.int32)
    ts = np.random.default_rng(seed).integers(-5, int(tt.dep.max()) + 10, size=src.shape[0]).astype(np.int32)
    want = case.oracle_rows(src, ts)
    for h in (1, 17, 100):
        for placement in (0, 3):
            got, status, _ = case.run(eat, src, ts, horizon=h, placement=placement)
            assert (status == 0).all(), (h, placement)
            assert np.array_equal(got, want), (h, placement)
    for i in range(0, len(src), 5):
        assert np.array_equal(want[i], oracle.brute.foremost_dijkstra(
            tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, int(src[i]), int(ts[i])))


@pytest.mark.parametrize("horizon", HORIZONS)
def test_small_grid_one_word_items(eat, small, horizon):
    q = synth.random_queries(small.tt, 300, 0x40 + horizon % 97)
    got, status, _ = small.run(eat, q.source, q.t_s, horizon=horizon)
    assert (status == 0).all()
    assert np.array_equal(got, small.oracle_rows(q.source, q.t_s))


@pytest.mark.parametrize("placement", [0, 2, 3])
@pytest.mark.parametrize("horizon", HORIZONS)
def test_city_placements(eat, city, horizon, placement):
    q = synth.random_queries(city.tt, 96, 0x41 + placement)
    got, status, cnt = city.run(eat, q.source, q.t_s, horizon=horizon, placement=placement)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))
    assert (cnt[:, 0] <= 2 * city.V + 2).all()


def test_city_work_drops_with_horizon(eat, city):
    """Stops are expanded with arrivals closer to their final ones: fewer expansions than
    without a horizon, at least one per reached stop that has outgoing types."""
    q = synth.random_queries(city.tt, 128, 0x42)
    base, _, c0 = city.run(eat, q.source, q.t_s, horizon=-1)
    got, _, c1 = city.run(eat, q.source, q.t_s, horizon=3600)
    assert np.array_equal(got, base)
    assert c1[:, 1].sum() < c0[:, 1].sum()
    rp = eat.eat_net_host_view(city.net)["row_ptr"]
    has_out = rp[1:] > rp[:-1]
    assert (c1[:, 1] >= ((got < INF) & has_out).sum(axis=1)).all()


@pytest.mark.parametrize("vwarp", [8, 32])
def test_edge_mode_with_horizon(eat, city, vwarp):
    q = synth.random_queries(city.tt, 96, 0x43 + vwarp)
    got, status, _ = city.run(eat, q.source, q.t_s, mode=eat.EAT_MODE_EDGE, vwarp=vwarp, horizon=1800)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))


def test_round_cap_with_horizon(eat, small):
    """A cap below the rounds a query needs reports EAT_ERR_NO_CONVERGENCE, also when the
    cap falls while stops still wait beyond the horizon; capped rows are upper bounds."""
    q = synth.random_queries(small.tt, 64, 0x44)
    full, _, cnt = small.run(eat, q.source, q.t_s, horizon=600)
    for cap in (1, 5, 20):
        capped, status, _ = small.run(eat, q.source, q.t_s, horizon=600, max_rounds=cap)
        needs_more = cnt[:, 0] > cap
        assert needs_more.any()
        assert (status[needs_more] == eat.EAT_ERR_NO_CONVERGENCE).all(), cap
        assert (status[~needs_more] == 0).all(), cap
        assert np.array_equal(capped[~needs_more], full[~needs_more])
        assert (capped.astype(np.int64) >= full).all()


def test_horizon_needs_the_round_kernel(eat, small):
    src, ts = _dev([0]), _dev([30000])
    out = torch.empty(small.V, dtype=torch.int32, device="cuda")
    for mode in (eat.EAT_MODE_PAIR, eat.EAT_MODE_ASYNC, eat.EAT_MODE_CLUSTER):
        with pytest.raises(eat.EatError) as ei:
            eat.eat_query_batch(small.net, src, ts, out, mode=mode, horizon=600)
        assert ei.value.code == eat.EAT_ERR_INVALID
    assert eat.eat_launch_shape(small.net, 1, horizon=600)["horizon"] == 600
    assert eat.eat_launch_shape(small.net, 1, horizon=-1)["horizon"] == -1


def test_noalloc_with_horizon(eat, city):
    q = synth.random_queries(city.tt, 200, 0x45)
    n, V = 200, city.V
    got = torch.full((n * V,), -1, dtype=torch.int32, device="cuda")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_noalloc(city.net, _dev(q.source), _dev(q.t_s), got, status=status,
                                horizon=7200)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    assert np.array_equal(got.view(n, V).cpu().numpy(), city.oracle_rows(q.source, q.t_s))


def test_ragged_batch_with_horizon(eat):
    """Networks of uneven size in one launch (arrivals shared or global per query)."""
    tts = synth.ragged_grids(12)
    nets = [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=0, cluster_width=900) for t in tts]
    Q = 600
    qs = synth.random_queries(tts, Q, 0x46)
    sizes = np.array([tts[i].n_stops for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    for h in (900, 43200):
        out = torch.full((int(sizes.sum()),), -7, dtype=torch.int32, device="cuda")
        status = torch.full((Q,), -1, dtype=torch.int32, device="cuda")
        eat.eat_query_batch_multi(nets, _dev(qs.net), _dev(qs.source), _dev(qs.t_s), out,
                                  torch.as_tensor(offs).cuda(), status=status, horizon=h,
                                  placement=eat.EAT_PLACE_AUTO)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all()
        flat = out.cpu().numpy()
        for j, tt in enumerate(tts):
            sel = np.nonzero(qs.net == j)[0]
            if sel.size == 0:
                continue
            want = oracle.csa_many(oracle.SortedConnections(tt), qs.source[sel], qs.t_s[sel],
                                   os.cpu_count() or 8)[0]
            for r, i in enumerate(sel):
                assert np.array_equal(flat[offs[i]:offs[i] + tt.n_stops], want[r]), (h, j, i)
    for n in nets:
        n.close()


def test_autotuned_horizon_is_kept(eat, city):
    """eat_autotune may choose a horizon; the query calls then use it (and the rows stay
    the oracle's), and an explicit -1 turns it off."""
    net = eat.eat_build(city.tt.n_stops, city.tt.u, city.tt.v, city.tt.dep, city.tt.dur, device=0,
                        cluster_width=600)
    q = synth.random_queries(city.tt, 256, 0x47)
    shape = eat.eat_autotune(net, _dev(q.source), _dev(q.t_s))
    assert shape["horizon"] == -1 or shape["horizon"] in (3600, 7200, 14400, 43200)
    assert eat.eat_launch_shape(net, 256)["horizon"] == shape["horizon"]
    assert eat.eat_launch_shape(net, 256, horizon=-1)["horizon"] == -1
    out = torch.empty(256 * city.V, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, _dev(q.source), _dev(q.t_s), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.view(256, city.V).cpu().numpy(), city.oracle_rows(q.source, q.t_s))
    net.close()
