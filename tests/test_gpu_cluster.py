"""Cluster mode (EAT_MODE_CLUSTER): one cluster of 8 blocks per query, arrivals and
frontier bitmaps spread over the cluster's distributed shared memory.  Every result must
equal the oracle's, as in the one-block-per-query kernel."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CLUSTER = 2


@pytest.fixture(scope="module")
def eat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00966_gb300 import eat as mod
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


@pytest.mark.parametrize("vwarp", [2, 8, 32])
def test_small_grid_batches(eat, small, vwarp):
    q = synth.random_queries(small.tt, 40, 50 + vwarp)        # 320 blocks: more than one wave
    got, status, cnt = small.run(eat, q.source, q.t_s, mode=CLUSTER, vwarp=vwarp)
    assert (status == 0).all()
    assert np.array_equal(got, small.oracle_rows(q.source, q.t_s))
    ref, _, cref = small.run(eat, q.source, q.t_s, mode=1)
    assert np.array_equal(got, ref)
    rounds, vert, types, evals, lookups, aps, relaxed = cnt.T
    assert (rounds >= 1).all() and (types >= lookups).all() and (lookups >= evals).all()
    assert (relaxed >= (got < 2**31 - 1).sum(axis=1) - 1).all()


@pytest.mark.parametrize("block", [256, 512, 1024])
def test_city_queries(eat, city, block):
    q = synth.random_queries(city.tt, 12, 60 + block)
    got, status, _ = city.run(eat, q.source, q.t_s, mode=CLUSTER, block=block)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))


@pytest.mark.parametrize("seed", range(12))
def test_tiny_nets_all_sources(eat, seed):
    """Networks with fewer stops than blocks in a cluster, and every source."""
    tt = synth.tiny_random(2 + seed % 10, 1 + (seed * 41) % 250, 300 + seed, t_max=300 + 40 * seed,
                           dur_max=1 + seed % 50)
    case = Case(eat, tt, cluster_width=[3600, 60, 7, 1][seed % 4])
    src = np.repeat(np.arange(tt.n_stops), 3).astype(np.int32)
    ts = np.random.default_rng(seed).integers(-5, int(tt.dep.max()) + 10, size=src.shape[0]).astype(np.int32)
    got, status, _ = case.run(eat, src, ts, mode=CLUSTER)
    assert (status == 0).all()
    assert np.array_equal(got, case.oracle_rows(src, ts))


def test_large_network_single_queries(eat):
    """200,000 stops: 25,000 arrivals per block; sampled against the oracle."""
    tt = synth.large()
    case = Case(eat, tt, cluster_width=1800)
    q = synth.random_queries(tt, 3, 61)
    got, status, _ = case.run(eat, q.source, q.t_s, mode=CLUSTER)
    assert (status == 0).all()
    for i in range(3):
        assert np.array_equal(got[i], oracle.csa(case.sc, int(q.source[i]), int(q.t_s[i])))


def test_round_cap_and_invalid_source(eat, small):
    q = synth.random_queries(small.tt, 16, 62)
    full, _, cnt = small.run(eat, q.source, q.t_s, mode=CLUSTER)
    capped, status, _ = small.run(eat, q.source, q.t_s, mode=CLUSTER, max_rounds=1)
    needs_more = cnt[:, 0] > 1
    assert needs_more.any()
    assert (status[needs_more] == eat.EAT_ERR_NO_CONVERGENCE).all()
    assert (capped.astype(np.int64) >= full).all()
    src = np.array([0, small.V, -3, 5], np.int32)
    ts = np.full(4, 30000, np.int32)
    got, status, _ = small.run(eat, src, ts, mode=CLUSTER)
    assert list(status) == [0, eat.EAT_ERR_INVALID, eat.EAT_ERR_INVALID, 0]
    assert np.array_equal(got[[0, 3]], small.oracle_rows(src[[0, 3]], ts[[0, 3]]))


def test_single_queries_and_host_rows(eat, city):
    """Single queries (eat_query, automatic shape) into device, pageable and page-locked
    rows agree with the cluster mode's batch into a page-locked buffer."""
    q = synth.random_queries(city.tt, 4, 63)
    want = city.oracle_rows(q.source, q.t_s)
    dev_row = torch.empty(city.V, dtype=torch.int32, device="cuda")
    pinned = torch.empty(city.V, dtype=torch.int32).pin_memory()
    for i in range(4):
        s, t = int(q.source[i]), int(q.t_s[i])
        assert np.array_equal(eat.eat_query(city.net, s, t), want[i])
        eat.eat_query(city.net, s, t, dev_row)
        assert np.array_equal(dev_row.cpu().numpy(), want[i])
        eat.eat_query(city.net, s, t, pinned)
        assert np.array_equal(pinned.numpy(), want[i])
    rows = torch.empty((4, city.V), dtype=torch.int32).pin_memory()
    eat.eat_query_batch(city.net, torch.as_tensor(q.source).pin_memory(),
                        torch.as_tensor(q.t_s).pin_memory(), rows, mode=CLUSTER)
    assert np.array_equal(rows.numpy(), want)


def test_rejected_where_not_available(eat, small):
    q = synth.random_queries(small.tt, 4, 64)
    out = torch.empty(4 * small.V, dtype=torch.int32, device="cuda")
    with pytest.raises(eat.EatError):
        eat.eat_query_batch_noalloc(small.net, _dev(q.source), _dev(q.t_s), out, mode=CLUSTER)
    with pytest.raises(eat.EatError):
        eat.eat_query_batch(small.net, _dev(q.source), _dev(q.t_s), out, mode=CLUSTER,
                            placement=eat.EAT_PLACE_GLOBAL_ARR)
    other = eat.eat_build(small.tt.n_stops, small.tt.u, small.tt.v, small.tt.dep, small.tt.dur,
                          device=0)
    offs = np.arange(4, dtype=np.int64) * small.V
    with pytest.raises(eat.EatError):
        eat.eat_query_batch_multi([small.net, other], _dev([0, 1, 0, 1]), _dev(q.source), _dev(q.t_s),
                                  out, torch.as_tensor(offs).cuda(), mode=CLUSTER)
