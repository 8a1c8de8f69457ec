"""Paired mode (EAT_MODE_PAIR): two queries share one 1,024-thread block and its rounds,
each slot taking the next query when its own converges.  Every result must equal the
oracle's, whatever the pairing, the queue size or the round cap."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAIR = 4


@pytest.fixture(scope="module")
def eat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00966_gb300 import eat as mod
    assert mod.EAT_MODE_PAIR == PAIR
    return mod


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).cuda()


class Case:
    def __init__(self, eat, tt, **kw):
        self.tt = tt
        self.net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0, **kw)
        self.sc = oracle.SortedConnections(tt)
        self.V = tt.n_stops

    def run(self, eat, src, ts, **opts):
        n = len(src)
        out = torch.full((n * self.V,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros((n, 7), dtype=torch.int64, device="cuda")
        eat.eat_query_batch(self.net, _dev(src), _dev(ts), out, status=status, counters=cnt, **opts)
        torch.cuda.synchronize()
        return out.view(n, self.V).cpu().numpy(), status.cpu().numpy(), cnt.cpu().numpy()

    def oracle_rows(self, src, ts):
        return oracle.csa_many(self.sc, src, ts, 8)[0]


@pytest.fixture(scope="module")
def small(eat):
    return Case(eat, synth.small_grid())


@pytest.fixture(scope="module")
def city(eat):
    return Case(eat, synth.city(), cluster_width=1800)


@pytest.mark.parametrize("n", [1, 151, 152, 153, 304, 305, 700])
def test_small_grid_batch_sizes(eat, small, n):
    """Fewer queries than blocks, one or two per block, and slots refilled from the
    counter; counters agree with the one-block-per-query kernel's rounds."""
    q = synth.random_queries(small.tt, n, 70 + n)
    got, status, cnt = small.run(eat, q.source, q.t_s, mode=PAIR)
    assert (status == 0).all()
    assert np.array_equal(got, small.oracle_rows(q.source, q.t_s))
    ref, _, cref = small.run(eat, q.source, q.t_s, mode=1)
    assert np.array_equal(got, ref)
    rounds, vert, types, evals, lookups, aps, relaxed = cnt.T
    assert (rounds >= 1).all() and (types >= lookups).all() and (lookups >= evals).all()
    assert (relaxed >= (got < 2**31 - 1).sum(axis=1) - 1).all()
    assert (vert >= 1).all()


@pytest.mark.parametrize("vwarp", [2, 8, 32])
def test_city_batch(eat, city, vwarp):
    q = synth.random_queries(city.tt, 200, 80 + vwarp)
    got, status, _ = city.run(eat, q.source, q.t_s, mode=PAIR, vwarp=vwarp)
    assert (status == 0).all()
    want = city.oracle_rows(q.source, q.t_s)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("block", [256, 512])
def test_city_smaller_blocks(eat, city, block):
    """Fewer threads per block: more items per thread and more spilled stops."""
    q = synth.random_queries(city.tt, 40, 90 + block)
    got, status, _ = city.run(eat, q.source, q.t_s, mode=PAIR, block=block)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))


@pytest.mark.parametrize("seed", range(16))
def test_tiny_nets_all_sources(eat, seed):
    """Tiny networks (queues of a few items that overflow into the spill queues) with
    every source, invalid sources mixed in."""
    tt = synth.tiny_random(2 + seed % 30, 1 + (seed * 41) % 400, 300 + seed, t_max=300 + 40 * seed,
                           dur_max=1 + seed % 50)
    case = Case(eat, tt, cluster_width=[3600, 60, 7, 1][seed % 4])
    src = np.concatenate([np.repeat(np.arange(tt.n_stops), 3), [-1, tt.n_stops]]).astype(np.int32)
    ts = np.random.default_rng(seed).integers(-5, int(tt.dep.max()) + 10, size=src.shape[0]).astype(np.int32)
    got, status, cnt = case.run(eat, src, ts, mode=PAIR)
    ok = (src >= 0) & (src < tt.n_stops)
    assert (status[ok] == 0).all()
    assert (status[~ok] == eat.EAT_ERR_INVALID).all()
    assert (got[~ok] == 2**31 - 1).all() and (cnt[~ok, 0] == 0).all()
    assert np.array_equal(got[ok], case.oracle_rows(src[ok], ts[ok]))


def test_round_cap(eat, small):
    q = synth.random_queries(small.tt, 300, 95)
    full, _, cnt = small.run(eat, q.source, q.t_s, mode=PAIR)
    for cap in (1, 3):
        capped, status, ccnt = small.run(eat, q.source, q.t_s, mode=PAIR, max_rounds=cap)
        needs_more = cnt[:, 0] > cap
        assert needs_more.any()
        assert (status[needs_more] == eat.EAT_ERR_NO_CONVERGENCE).all()
        assert (status[~needs_more] == 0).all()
        assert (ccnt[:, 0] <= cap).all()
        assert (capped.astype(np.int64) >= full).all()
        assert np.array_equal(capped[~needs_more], full[~needs_more])


def test_host_rows_and_noalloc(eat, city):
    """Page-locked host rows written in place, and the no-allocation entry point."""
    q = synth.random_queries(city.tt, 160, 96)
    want = city.oracle_rows(q.source, q.t_s)
    rows = torch.empty((160, city.V), dtype=torch.int32).pin_memory()
    eat.eat_query_batch(city.net, torch.as_tensor(q.source).pin_memory(),
                        torch.as_tensor(q.t_s).pin_memory(), rows, mode=PAIR)
    assert np.array_equal(rows.numpy(), want)
    out = torch.empty(160 * city.V, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_noalloc(city.net, _dev(q.source), _dev(q.t_s), out, mode=PAIR)
    torch.cuda.synchronize()
    assert np.array_equal(out.view(160, city.V).cpu().numpy(), want)


def test_rejected_where_not_available(eat, small):
    q = synth.random_queries(small.tt, 4, 97)
    out = torch.empty(4 * small.V, dtype=torch.int32, device="cuda")
    with pytest.raises(eat.EatError):
        eat.eat_query_batch(small.net, _dev(q.source), _dev(q.t_s), out, mode=PAIR,
                            placement=eat.EAT_PLACE_GLOBAL_ARR)
    other = eat.eat_build(small.tt.n_stops, small.tt.u, small.tt.v, small.tt.dep, small.tt.dur,
                          device=0)
    offs = np.arange(4, dtype=np.int64) * small.V
    with pytest.raises(eat.EatError):
        eat.eat_query_batch_multi([small.net, other], _dev([0, 1, 0, 1]), _dev(q.source), _dev(q.t_s),
                                  out, torch.as_tensor(offs).cuda(), mode=PAIR)
    big = synth.tiny_random(40000, 500, 98)                    # more stops than the packed items hold
    net = eat.eat_build(big.n_stops, big.u, big.v, big.dep, big.dur, device=0)
    outb = torch.empty(big.n_stops, dtype=torch.int32, device="cuda")
    with pytest.raises(eat.EatError):
        eat.eat_query_batch(net, _dev([0]), _dev([30000]), outb, mode=PAIR)


def test_launch_shape_defaults(eat, small, city):
    """Automatic shape: one 1,024-thread block per query for batches of at most one query
    per SM and on networks of 8,192 stops or more, two 512-thread blocks per SM for larger
    batches on small networks; the paired mode only when asked for (or tuned)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert eat.eat_launch_shape(city.net, sms + 1) == {"block": 1024, "vwarp": 8, "mode": 1, "cluster": 0,
                                                       "order": eat.EAT_ORDER_BY_TIME, "horizon": -1}
    assert eat.eat_launch_shape(small.net, sms + 1)["block"] == 512
    assert eat.eat_launch_shape(small.net, sms + 1, mode=PAIR)["mode"] == PAIR
    assert eat.eat_launch_shape(city.net, sms + 1, mode=PAIR)["block"] == 1024
    for case in (small, city):
        assert eat.eat_launch_shape(case.net, sms) == {"block": 1024, "vwarp": 8, "mode": 1, "cluster": 0,
                                                       "order": eat.EAT_ORDER_AS_GIVEN, "horizon": -1}
        assert eat.eat_launch_shape(case.net, 4 * sms, block=512)["mode"] == 1
        assert eat.eat_launch_shape(case.net, 4 * sms, mode=3)["mode"] == 3
    other = eat.eat_build(small.tt.n_stops, small.tt.u, small.tt.v, small.tt.dep, small.tt.dur,
                          device=0)
    assert eat.eat_launch_shape([small.net, other], 4 * sms)["mode"] == 1
    assert eat.eat_launch_shape([small.net, other], 4 * sms)["order"] == eat.EAT_ORDER_AS_GIVEN
    big = synth.tiny_random(40000, 500, 99)
    net = eat.eat_build(big.n_stops, big.u, big.v, big.dep, big.dur, device=0)
    assert eat.eat_launch_shape(net, 4 * sms)["mode"] == 1
    with pytest.raises(eat.EatError):
        eat.eat_launch_shape(net, 4 * sms, mode=PAIR)


def test_default_batch_and_autotune(eat, city):
    """The default call on a batch larger than the SM count (started in order of t_s) and
    the shape the tuner picks, paired or not, give the oracle's results."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = sms + 40
    q = synth.random_queries(city.tt, n, 0xA9)
    want = city.oracle_rows(q.source, q.t_s)
    got, status, _ = city.run(eat, q.source, q.t_s)
    assert (status == 0).all() and np.array_equal(got, want)
    net = eat.eat_build(city.tt.n_stops, city.tt.u, city.tt.v, city.tt.dep, city.tt.dur, device=0,
                        cluster_width=1800)
    shape = eat.eat_autotune(net, _dev(q.source), _dev(q.t_s))
    assert shape["mode"] in (1, 3, PAIR)
    assert eat.eat_launch_shape(net, n)["mode"] == shape["mode"]
    out = torch.empty(n * city.V, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, _dev(q.source), _dev(q.t_s), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.view(n, city.V).cpu().numpy(), want)


@pytest.mark.parametrize("mode", [0, 1, 3, PAIR])
def test_multi_entry_point_one_network(eat, small, mode):
    """eat_query_batch_multi over one network, in every mode that serves it: rows at
    caller offsets (here in reverse order), and a query naming a network that is not
    there is invalid."""
    n = 400
    q = synth.random_queries(small.tt, n, 0xAA)
    idx = np.zeros(n, np.int32)
    idx[::37] = 1
    idx[5] = -1
    offs = (np.arange(n, dtype=np.int64)[::-1] * small.V).copy()
    out = torch.full((n * small.V,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((n,), -9, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_multi([small.net], _dev(idx), _dev(q.source), _dev(q.t_s), out,
                              torch.as_tensor(offs).cuda(), status=status, mode=mode)
    torch.cuda.synchronize()
    rows = out.view(n, small.V).cpu().numpy()[::-1]
    st = status.cpu().numpy()
    ok = idx == 0
    assert (st[ok] == 0).all() and (st[~ok] == eat.EAT_ERR_INVALID).all()
    assert np.array_equal(rows[ok], small.oracle_rows(q.source[ok], q.t_s[ok]))
    assert (rows[~ok] == 2**31 - 1).all()


@pytest.mark.parametrize("mode", [0, 1, 3, PAIR])
def test_start_order_keeps_results_in_place(eat, city, mode):
    """Queries start in order of t_s by default (a device sort of the batch) or as given;
    rows, status and counters stay at each query's index either way."""
    q = synth.random_queries(city.tt, 300, 0xAB)
    want = city.oracle_rows(q.source, q.t_s)
    by_time, st0, c0 = city.run(eat, q.source, q.t_s, mode=mode)
    as_given, st1, c1 = city.run(eat, q.source, q.t_s, mode=mode, order=eat.EAT_ORDER_AS_GIVEN)
    assert (st0 == 0).all() and (st1 == 0).all()
    assert np.array_equal(by_time, want) and np.array_equal(as_given, want)
    relaxed_floor = (want < 2**31 - 1).sum(axis=1) - 1
    assert (c0[:, 6] >= relaxed_floor).all() and (c1[:, 6] >= relaxed_floor).all()
    n_ws = eat.eat_workspace_bytes(city.net, 300, mode=mode)
    assert n_ws >= eat.eat_workspace_bytes(city.net, 300, mode=mode, order=eat.EAT_ORDER_AS_GIVEN) + 1200
    with pytest.raises(eat.EatError):
        city.run(eat, q.source[:4], q.t_s[:4], order=7)
