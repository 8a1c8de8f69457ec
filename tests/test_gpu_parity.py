"""GPU parity: libeat's CUDA path (through the C ABI) against the oracle, bit-exact.

Arrival times are int32, so every comparison is exact equality with the
connection-scan oracle (Algorithm 1) on the same seeded inputs; large cases are
compared on sampled queries and checked by the oracle's exactness certificate.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = 2**31 - 1


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
        if kw.get("subtrips"):
            kw.setdefault("trip", tt.trip)
        self.net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0, **kw)
        self.sc = oracle.SortedConnections(tt)
        self.V = tt.n_stops

    def oracle_rows(self, src, ts):
        out, _ = oracle.csa_many(self.sc, src, ts, 8)
        return out

    def run(self, eat, src, ts, **opts):
        n = len(src)
        out = torch.empty(n * self.V, dtype=torch.int32, device="cuda")
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros((n, 7), dtype=torch.int64, device="cuda")
        eat.eat_query_batch(self.net, _dev(src), _dev(ts), out, status=status, counters=cnt, **opts)
        torch.cuda.synchronize()
        return out.view(n, self.V).cpu().numpy(), status.cpu().numpy(), cnt.cpu().numpy()


@pytest.fixture(scope="module")
def small(eat):
    return Case(eat, synth.small_grid())


@pytest.fixture(scope="module")
def city(eat):
    return Case(eat, synth.city())


def test_smoke_entry(eat):
    import __graft_entry__
    __graft_entry__.smoke()


def test_single_query_edge_cases(eat, small):
    tt = small.tt
    unserved = int(np.setdiff1d(np.arange(tt.n_stops), np.concatenate([tt.u, tt.v]))[0])
    exact_dep = int(tt.dep[tt.u == 0].min())
    cases = [(0, 28800), (0, 0), (0, 200000), (unserved, 30000), (0, exact_dep),
             (0, exact_dep + 1), (0, -1000), (0, INF), (tt.n_stops - 1, 40000)]
    for s, t_s in cases:
        got = eat.eat_query(small.net, s, t_s)
        want = oracle.csa(small.sc, s, t_s)
        assert np.array_equal(got, want), (s, t_s)
        # device output buffer
        out = torch.empty(tt.n_stops, dtype=torch.int32, device="cuda")
        eat.eat_query(small.net, s, t_s, out)
        assert np.array_equal(out.cpu().numpy(), want)


def test_batch_small_random(eat, small):
    q = synth.random_queries(small.tt, 300, 21)
    got, status, cnt = small.run(eat, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, small.oracle_rows(q.source, q.t_s))
    rounds, vert, types, evals, lookups, aps, relaxed = cnt.T
    assert (rounds >= 1).all() and (rounds <= small.V + 1).all()
    assert (types >= lookups).all() and (lookups >= evals).all()
    reach = (got < INF).sum(axis=1)
    assert (relaxed >= reach - 1).all()
    rp = eat.eat_net_host_view(small.net)["row_ptr"]
    has_out = rp[1:] > rp[:-1]
    assert (vert >= ((got < INF) & has_out).sum(axis=1)).all()


def test_host_buffers_match_device(eat, small):
    q = synth.random_queries(small.tt, 40, 5)
    host = np.empty((40, small.V), dtype=np.int32)
    eat.eat_query_batch(small.net, q.source, q.t_s, host)
    pinned = torch.empty((40, small.V), dtype=torch.int32).pin_memory()
    eat.eat_query_batch(small.net, torch.as_tensor(q.source), torch.as_tensor(q.t_s), pinned)
    want = small.oracle_rows(q.source, q.t_s)
    assert np.array_equal(host, want)
    assert np.array_equal(pinned.numpy(), want)


@pytest.mark.parametrize("mode", [1, 3])
def test_pinned_host_rows_written_in_place(eat, city, mode):
    """Page-locked host queries and rows (the kernel reads and writes them in place)
    equal the oracle, also when the arrivals are kept in global memory (per-block
    device rows, copied to the host row at the end) and for a single eat_query into
    a page-locked row."""
    q = synth.random_queries(city.tt, 256, 0x9A + mode)
    src = torch.as_tensor(q.source).pin_memory()
    ts = torch.as_tensor(q.t_s).pin_memory()
    want = city.oracle_rows(q.source, q.t_s)
    rows = torch.full((256, city.V), -7, dtype=torch.int32).pin_memory()
    eat.eat_query_batch(city.net, src, ts, rows, mode=mode)
    assert np.array_equal(rows.numpy(), want)
    for placement in (eat.EAT_PLACE_GLOBAL_ARR, eat.EAT_PLACE_GLOBAL):
        if mode == 3 and placement == eat.EAT_PLACE_GLOBAL:
            continue                                   # the round-free mode keeps its bitmap shared
        rows.fill_(-7)
        eat.eat_query_batch(city.net, src, ts, rows, mode=mode, placement=placement)
        assert np.array_equal(rows.numpy(), want)
    one = torch.full((city.V,), -7, dtype=torch.int32).pin_memory()
    for i in (0, 77, 255):
        eat.eat_query(city.net, int(q.source[i]), int(q.t_s[i]), one)
        assert np.array_equal(one.numpy(), want[i])


@pytest.mark.parametrize("placement", [2, 3])
def test_host_rows_written_by_the_kernel(eat, city, placement):
    """Rows of queries whose arrivals live in a device row of the block are copied by the
    block (16-byte words) into page-locked host memory as each query converges: 1,000
    queries, so each block reuses its row several times; every row equals the oracle's,
    in a batch whose buffers are all host memory and in one that starts from device
    queries."""
    q = synth.random_queries(city.tt, 1000, 0x7C + placement)
    want = city.oracle_rows(q.source, q.t_s)
    rows = torch.full((1000, city.V), -7, dtype=torch.int32).pin_memory()
    eat.eat_query_batch(city.net, torch.as_tensor(q.source).pin_memory(),
                        torch.as_tensor(q.t_s).pin_memory(), rows, placement=placement)
    assert np.array_equal(rows.numpy(), want)
    rows.fill_(-7)
    eat.eat_query_batch(city.net, _dev(q.source), _dev(q.t_s), rows, placement=placement,
                        block=256)
    assert np.array_equal(rows.numpy(), want)


def test_ragged_batch_into_host_rows(eat):
    """Networks of uneven size, arrivals shared or in device rows per query, rows written
    into one page-locked host buffer (row offsets not all 16-byte aligned)."""
    import os
    tts = synth.ragged_grids(10, seed_offset=3)
    nets = [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=0) for t in tts]
    Q = 700
    qs = synth.random_queries(tts, Q, 0x7E)
    sizes = np.array([tts[i].n_stops for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes + 1)[:-1]]).astype(np.int64)   # odd gaps
    out = torch.full((int(offs[-1] + sizes[-1]),), -7, dtype=torch.int32).pin_memory()
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    eat.eat_query_batch_multi(nets, i32(qs.net), i32(qs.source), i32(qs.t_s), out, offs)
    flat = out.numpy()
    for j, tt in enumerate(tts):
        sel = np.nonzero(qs.net == j)[0]
        if sel.size == 0:
            continue
        want = oracle.csa_many(oracle.SortedConnections(tt), qs.source[sel], qs.t_s[sel],
                               os.cpu_count() or 8)[0]
        for r, i in enumerate(sel):
            assert np.array_equal(flat[offs[i]:offs[i] + tt.n_stops], want[r]), (j, i)
    for n in nets:
        n.close()


@pytest.mark.parametrize("seed", range(30))
def test_tiny_random_nets_all_sources(eat, seed):
    tt = synth.tiny_random(2 + seed % 13, 1 + (seed * 37) % 300, 500 + seed, t_max=300 + 50 * seed,
                           dur_max=1 + seed % 60)
    case = Case(eat, tt, cluster_width=[3600, 60, 7, 1][seed % 4])
    src = np.repeat(np.arange(tt.n_stops), 4).astype(np.int32)
    rng = np.random.default_rng(seed)
    ts = rng.integers(-5, int(tt.dep.max()) + 10, size=src.shape[0]).astype(np.int32)
    got, status, _ = case.run(eat, src, ts)
    assert (status == 0).all()
    want = case.oracle_rows(src, ts)
    assert np.array_equal(got, want)
    for i in range(0, len(src), 7):
        assert np.array_equal(got[i], oracle.brute.foremost_dijkstra(
            tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, int(src[i]), int(ts[i])))


@pytest.mark.parametrize("vwarp", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("block", [64, 256, 1024])
def test_mapping_variants(eat, city, vwarp, block):
    q = synth.random_queries(city.tt, 48, 100 + vwarp)
    got, status, _ = city.run(eat, q.source, q.t_s, vwarp=vwarp, block=block)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))


@pytest.mark.parametrize("placement", [1, 2, 3])
def test_memory_placements(eat, small, city, placement):
    for case in (small, city):
        q = synth.random_queries(case.tt, 64, 7 + placement)
        got, status, _ = case.run(eat, q.source, q.t_s, placement=placement)
        assert (status == 0).all()
        assert np.array_equal(got, case.oracle_rows(q.source, q.t_s))


def test_city_256_queries_default_launch(eat, city):
    """The benchmark's workload and launch configuration (256 queries, default options)."""
    q = synth.random_queries(city.tt, 256, 0xC17)
    got, status, cnt = city.run(eat, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))
    for i in range(0, 256, 64):
        assert oracle.certify(city.tt, int(q.source[i]), int(q.t_s[i]), got[i]) == (0, -1)


def test_repeatable(eat, city):
    q = synth.random_queries(city.tt, 128, 3)
    first, _, _ = city.run(eat, q.source, q.t_s)
    for _ in range(4):
        again, _, _ = city.run(eat, q.source, q.t_s)
        assert np.array_equal(first, again)


def test_monotone_in_departure_time(eat, city):
    s = int(synth.random_queries(city.tt, 1, 77).source[0])
    ts = np.arange(18000, 80000, 1800, dtype=np.int32)
    got, _, _ = city.run(eat, np.full(ts.shape, s, np.int32), ts)
    g = got.astype(np.int64)
    g[:, s] = 0
    assert (np.diff(g, axis=0) >= 0).all()


def test_round_cap_reports_no_convergence(eat, small):
    q = synth.random_queries(small.tt, 64, 8)
    full, _, cnt = small.run(eat, q.source, q.t_s)
    capped, status, _ = small.run(eat, q.source, q.t_s, max_rounds=1)
    needs_more = cnt[:, 0] > 1
    assert needs_more.any()
    assert (status[needs_more] == eat.EAT_ERR_NO_CONVERGENCE).all()
    assert (status[~needs_more] == 0).all()
    assert (capped.astype(np.int64) >= full).all()          # upper bounds only


def test_invalid_source_and_workspace(eat, small):
    src = np.array([0, small.V, -3, 5], np.int32)
    ts = np.full(4, 30000, np.int32)
    got, status, _ = small.run(eat, src, ts)
    assert status.tolist()[1:3] == [eat.EAT_ERR_INVALID] * 2
    assert (got[1] == INF).all() and (got[2] == INF).all()
    assert np.array_equal(got[[0, 3]], small.oracle_rows(src[[0, 3]], ts[[0, 3]]))
    with pytest.raises(eat.EatError) as ei:
        eat.eat_query(small.net, small.V, 0)
    assert ei.value.code == eat.EAT_ERR_INVALID
    need = eat.eat_workspace_bytes(small.net, 4)
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    out = torch.empty(4 * small.V, dtype=torch.int32, device="cuda")
    with pytest.raises(eat.EatError) as ei:
        eat.eat_query_batch(small.net, _dev(src), _dev(ts), out, workspace=ws)
    assert ei.value.code == eat.EAT_ERR_WORKSPACE
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    eat.eat_query_batch(small.net, _dev(src[[0, 3]]), _dev(ts[[0, 3]]), out, workspace=ws)
    torch.cuda.synchronize()


def test_empty_network_and_empty_batch(eat):
    net = eat.eat_build(5, [], [], [], [], device=0)
    got = eat.eat_query(net, 2, 100)
    assert got.tolist() == [INF, INF, 100, INF, INF]
    out = torch.empty(0, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, _dev([]), _dev([]), out)


def test_ragged_multi_network_batch(eat, small):
    nets = [small] + [Case(eat, synth.grid_timetable(n, int(np.ceil(50 * n / 1024)), 900 + n,
                                                       force_stop0=False)) for n in (1500, 3100, 7000)]
    Q = 200
    qs = synth.random_queries([c.tt for c in nets], Q, 42)
    sizes = np.array([nets[i].V for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    out = torch.full((int(sizes.sum()),), -7, dtype=torch.int32, device="cuda")
    status = torch.full((Q,), -1, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_multi([c.net for c in nets], _dev(qs.net), _dev(qs.source), _dev(qs.t_s),
                              out, torch.as_tensor(offs).cuda(), status=status)
    torch.cuda.synchronize()
    flat = out.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    for i in range(Q):
        c = nets[qs.net[i]]
        want = oracle.csa(c.sc, int(qs.source[i]), int(qs.t_s[i]))
        assert np.array_equal(flat[offs[i]:offs[i] + c.V], want), i
    # Host query arrays take the staged path and give the same rows.
    out2 = torch.full_like(out, -7)
    eat.eat_query_batch_multi([c.net for c in nets], qs.net, qs.source, qs.t_s, out2, offs)
    assert torch.equal(out, out2)


def _type_departures(case, eat):
    hv = eat.eat_net_host_view(case.net)
    types = oracle.connection_types(case.tt)
    keys = []
    for u in range(case.V):
        for t in range(hv["row_ptr"][u], hv["row_ptr"][u + 1]):
            v, lam = int(hv["type_rec"][t][0]), int(hv["type_rec"][t][1])
            keys.append(types[(u, v, lam)])
    return keys


@pytest.mark.parametrize("which", ["small", "city"])
def test_next_departure_lookup(eat, small, city, which):
    case = small if which == "small" else city
    deps = _type_departures(case, eat)
    rng = np.random.default_rng(3)
    pick = range(len(deps)) if which == "small" else rng.choice(len(deps), 1500, replace=False)
    T, E = [], []
    for t in pick:
        d = deps[t]
        probes = {d[0] - 1, d[0], d[0] + 1, d[-1] - 1, d[-1], d[-1] + 1, -5, INF - 1}
        for x in d[:: max(1, len(d) // 12)]:
            probes.update({x - 1, x, x + 1, x // 3600 * 3600, x // 3600 * 3600 - 1})
        probes.update(int(y) for y in rng.integers(d[0] - 100, d[-1] + 100, size=6))
        for e in probes:
            T.append(int(t))
            E.append(int(e))
    out = torch.empty(len(T), dtype=torch.int32, device="cuda")
    eat.eat_next_departure(case.net, _dev(T), _dev(E), out)
    got = out.cpu().numpy()
    want = np.array([oracle.next_departure(deps[t], e) for t, e in zip(T, E)], np.int64)
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("width", [60, 900, 7200, 65535])
def test_cluster_widths(eat, width):
    tt = synth.small_grid(seed_offset=5)
    case = Case(eat, tt, cluster_width=width, t0=min(width // 3, 17000))
    q = synth.random_queries(tt, 96, width)
    got, status, _ = case.run(eat, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, case.oracle_rows(q.source, q.t_s))


@pytest.mark.parametrize("width", [60, 200])
@pytest.mark.parametrize("placement", [2, 3])    # arrivals in global memory: two-word items
def test_more_than_255_cluster_slots(eat, width, placement):
    """More than 255 cluster slots, two-word queue items: rows equal the oracle's for
    queries whose arrivals pass through slot 255 and beyond (an earlier version used
    slot 255 as a 'none' marker in its items and skipped that slot's entry load)."""
    tt = synth.small_grid(seed_offset=7)
    case = Case(eat, tt, cluster_width=width)
    st = eat.eat_get_stats(case.net)
    assert st["y"] > 255
    q = synth.random_queries(tt, 192, 0x255 + width)
    slot255 = (st["k_min"] + 255) * width         # start of slot 255 (t0 = 0)
    assert (q.t_s < slot255).sum() >= 24          # many queries start before it
    got, status, _ = case.run(eat, q.source, q.t_s, placement=placement)
    assert (status == 0).all()
    assert np.array_equal(got, case.oracle_rows(q.source, q.t_s))


def test_city_at_300_second_clusters(eat):
    """The city network with 300-second clusters (about 285 slots), default launch."""
    tt = synth.city()
    case = Case(eat, tt, cluster_width=300)
    assert eat.eat_get_stats(case.net)["y"] > 255
    q = synth.random_queries(tt, 96, 0x300)
    got, status, _ = case.run(eat, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, case.oracle_rows(q.source, q.t_s))


def test_large_network_all_rows(eat, large_tt, large_sc):
    """200,000-stop network, about 46 M connections, 1,024 queries in one launch: every row
    equals the oracle's, with the library's default launch and 60-minute clusters, with
    10-minute clusters in the launch shape the autotuner picks (the benchmark's setup),
    and with 10-minute clusters and a 2-hour horizon."""
    import os
    tt = large_tt
    q = synth.random_queries(tt, 1024, 0x1A)
    want, _ = oracle.csa_many(large_sc, q.source, q.t_s, os.cpu_count() or 8)
    for width, tune, opts in ((3600, False, {}), (600, True, {}), (600, False, {"horizon": 7200})):
        net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0, cluster_width=width)
        if tune:
            sample = synth.random_queries(tt, 1024, 0x1A - 1)
            eat.eat_autotune(net, _dev(sample.source), _dev(sample.t_s))
        out = torch.empty(1024 * tt.n_stops, dtype=torch.int32, device="cuda")
        status = torch.full((1024,), -1, dtype=torch.int32, device="cuda")
        eat.eat_query_batch(net, _dev(q.source), _dev(q.t_s), out, status=status, **opts)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all()
        got = out.view(1024, tt.n_stops).cpu().numpy()
        bad = np.nonzero((got != want).any(axis=1))[0]
        assert bad.size == 0, (width, tune, opts, bad[:8])
        del out
        if tune:
            # the same batch from and into page-locked host memory (the end-to-end path:
            # each block copies its converged rows into the host buffer)
            host = torch.full((1024, tt.n_stops), -7, dtype=torch.int32).pin_memory()
            eat.eat_query_batch(net, torch.as_tensor(q.source).pin_memory(),
                                torch.as_tensor(q.t_s).pin_memory(), host)
            bad = np.nonzero((host.numpy() != want).any(axis=1))[0]
            assert bad.size == 0, ("host rows", bad[:8])
            del host
        net.close()
    for i in (0, 511, 1023):
        assert oracle.certify(tt, int(q.source[i]), int(q.t_s[i]), want[i]) == (0, -1)


def test_ragged_64_networks_4096_queries(eat):
    """The ragged workload at full size: 64 grid networks of 1,000-50,000 stops and 4,096
    queries over them in one eat_query_batch_multi launch (the benchmark's first timed
    batch, default launch shape); every row equals the oracle's."""
    import os
    tts = synth.ragged_grids(64)
    nets = [eat.eat_build(t.n_stops, t.u, t.v, t.dep, t.dur, device=0, cluster_width=600)
            for t in tts]
    Q = 4096
    qs = synth.random_queries(tts, Q, 0xA0 + 5)
    sizes = np.array([tts[i].n_stops for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    out = torch.full((int(sizes.sum()),), -7, dtype=torch.int32, device="cuda")
    status = torch.full((Q,), -1, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_multi(nets, _dev(qs.net), _dev(qs.source), _dev(qs.t_s), out,
                              torch.as_tensor(offs).cuda(), status=status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    flat = out.cpu().numpy()
    threads = os.cpu_count() or 8
    for j, tt in enumerate(tts):
        sel = np.nonzero(qs.net == j)[0]
        if sel.size == 0:
            continue
        want, _ = oracle.csa_many(oracle.SortedConnections(tt), qs.source[sel], qs.t_s[sel], threads)
        for r, i in enumerate(sel):
            assert np.array_equal(flat[offs[i]:offs[i] + tt.n_stops], want[r]), (j, i)
    for n in nets:
        n.close()


@pytest.mark.parametrize("scheme", [1, 2])
def test_subtrips_same_arrivals_fewer_rounds(eat, city, scheme):
    """Section II-G: with sub-trip shortcuts the arrivals equal the oracle's on the original
    timetable, and queries need fewer rounds."""
    enh = Case(eat, city.tt, subtrips=scheme)
    q = synth.random_queries(city.tt, 256, 0x5B + scheme)
    got, status, cnt = enh.run(eat, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, city.oracle_rows(q.source, q.t_s))
    _, _, base = city.run(eat, q.source, q.t_s)
    assert cnt[:, 0].mean() < 0.8 * base[:, 0].mean()
    assert cnt[:, 0].max() < base[:, 0].max()


def test_subtrips_small_grid_all_queries(eat, small):
    enh = Case(eat, small.tt, subtrips=1)
    q = synth.random_queries(small.tt, 300, 77)
    got, status, _ = enh.run(eat, q.source, q.t_s)
    assert (status == 0).all()
    assert np.array_equal(got, small.oracle_rows(q.source, q.t_s))
    for s_, t_ in [(0, 28800), (0, 0), (5, 86000)]:
        assert np.array_equal(eat.eat_query(enh.net, s_, t_), oracle.csa(small.sc, s_, t_))


def test_build_csr_network_parity(eat, city):
    """A network built from pre-encoded types, clusters and AP runs answers like eat_build's."""
    from test_build_host import csr_from_view
    host = eat.eat_build(city.tt.n_stops, city.tt.u, city.tt.v, city.tt.dep, city.tt.dur, device=-1)
    net = eat.eat_build_csr(**csr_from_view(host), device=0)
    q = synth.random_queries(city.tt, 128, 0xC5)
    out = torch.empty(128 * city.V, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, _dev(q.source), _dev(q.t_s), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.view(128, city.V).cpu().numpy(), city.oracle_rows(q.source, q.t_s))


def test_ragged_batch_with_per_query_placement(eat, small):
    """A 60,000-stop network next to small ones: one launch, arrivals in shared memory for
    the networks that fit and in the output row for the others; host output staged."""
    big_tt = synth.grid_timetable(60000, int(np.ceil(50 * 60000 / 1024)), 4242, force_stop0=False)
    nets = [small, Case(eat, synth.grid_timetable(5000, 245, 77, force_stop0=False)), Case(eat, big_tt)]
    Q = 120
    qs = synth.random_queries([c.tt for c in nets], Q, 9)
    sizes = np.array([nets[i].V for i in qs.net], np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    out = np.full(int(sizes.sum()), -7, dtype=np.int32)
    eat.eat_query_batch_multi([c.net for c in nets], qs.net, qs.source, qs.t_s, out, offs)
    for i in range(Q):
        c = nets[qs.net[i]]
        assert np.array_equal(out[offs[i]:offs[i] + c.V],
                              oracle.csa(c.sc, int(qs.source[i]), int(qs.t_s[i]))), i
    dev = torch.full((int(sizes.sum()),), -7, dtype=torch.int32, device="cuda")
    eat.eat_query_batch_multi([c.net for c in nets], _dev(qs.net), _dev(qs.source), _dev(qs.t_s), dev,
                              torch.as_tensor(offs).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), out)
    # Page-locked host output: written in place, the big network's arrivals in
    # per-block device rows meanwhile.
    pinned = torch.full((int(sizes.sum()),), -7, dtype=torch.int32).pin_memory()
    eat.eat_query_batch_multi([c.net for c in nets], qs.net, qs.source, qs.t_s, pinned, offs)
    assert np.array_equal(pinned.numpy(), out)


def test_lookup_through_count_overflow_header(eat):
    """A cluster of > 254 APs (its count in the AP-list header) still answers exactly."""
    vals = [sum(((i >> b) & 1) * 3 ** b for b in range(10)) for i in range(1024)]
    deps = np.array(sorted(vals), dtype=np.int32)
    z = np.zeros(deps.shape[0], np.int32)
    tt = synth.Timetable("dense", 2, z, z + 1, deps, z + 5, z, z)
    net = eat.eat_build(2, tt.u, tt.v, tt.dep, tt.dur, cluster_width=65535, device=0)
    times = np.concatenate([deps - 1, deps, deps + 1, [-3, 0, 70000]]).astype(np.int32)
    out = torch.empty(times.shape[0], dtype=torch.int32, device="cuda")
    eat.eat_next_departure(net, _dev(np.zeros_like(times)), _dev(times), out)
    want = [oracle.next_departure(deps.tolist(), int(e)) for e in times]
    assert out.cpu().numpy().tolist() == want
    for t_s in (0, 5000, 59000):
        got = eat.eat_query(net, 0, t_s)
        assert np.array_equal(got, oracle.csa(oracle.SortedConnections(tt), 0, t_s))


@pytest.mark.parametrize("vwarp", [1, 4, 8, 32])
@pytest.mark.parametrize("block", [256, 1024])
def test_edge_mode_matches_oracle(eat, small, city, vwarp, block):
    """EAT_MODE_EDGE (a sub-warp of vwarp lanes per stop with at least vwarp types, one
    relaxation per head stop after a warp min) gives the oracle's rows, on the packed
    (small networks) and two-word items alike, with any sub-warp size."""
    for case in (small, city):
        q = synth.random_queries(case.tt, 96, 300 + vwarp)
        got, status, cnt = case.run(eat, q.source, q.t_s, vwarp=vwarp, block=block,
                                    mode=eat.EAT_MODE_EDGE)
        assert (status == 0).all()
        assert np.array_equal(got, case.oracle_rows(q.source, q.t_s))
        for i in range(0, 96, 48):
            assert oracle.certify(case.tt, int(q.source[i]), int(q.t_s[i]), got[i]) == (0, -1)
    assert eat.eat_launch_shape(city.net, 96, mode=eat.EAT_MODE_EDGE)["mode"] == eat.EAT_MODE_EDGE


def test_edge_mode_large_and_placements(eat, large_tt, large_sc):
    """EAT_MODE_EDGE on the 200,000-stop network (arrivals in global memory) and with the
    arrivals and bitmaps forced into global memory on the city network."""
    import os
    tt = large_tt
    net = eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=0, cluster_width=1800)
    q = synth.random_queries(tt, 256, 0x1E)
    out = torch.empty(256 * tt.n_stops, dtype=torch.int32, device="cuda")
    status = torch.full((256,), -1, dtype=torch.int32, device="cuda")
    eat.eat_query_batch(net, _dev(q.source), _dev(q.t_s), out, status=status,
                        mode=eat.EAT_MODE_EDGE, vwarp=8)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    want, _ = oracle.csa_many(large_sc, q.source, q.t_s, os.cpu_count() or 8)
    assert np.array_equal(out.view(256, tt.n_stops).cpu().numpy(), want)
    net.close()


@pytest.mark.parametrize("seed", range(24))
def test_tiny_nets_two_word_items(eat, seed):
    """Two-word queue items (arrivals in global memory) on tiny random nets with narrow
    clusters: the pushed types are filtered by their last departure against the cluster of
    the new arrival, and a stop lowered into an earlier cluster after its push is pushed
    again from its first item; every row equals the oracle's and brute force."""
    tt = synth.tiny_random(3 + seed % 11, 20 + (seed * 53) % 400, 900 + seed, t_max=600 + 40 * seed,
                           dur_max=1 + seed % 90)
    case = Case(eat, tt, cluster_width=[30, 60, 120, 7][seed % 4])
    src = np.repeat(np.arange(tt.n_stops), 3).astype(np.int32)
    rng = np.random.default_rng(seed)
    ts = rng.integers(-5, int(tt.dep.max()) + 10, size=src.shape[0]).astype(np.int32)
    for placement in (eat.EAT_PLACE_GLOBAL_ARR, eat.EAT_PLACE_GLOBAL):
        got, status, _ = case.run(eat, src, ts, placement=placement, block=64)
        assert (status == 0).all()
        assert np.array_equal(got, case.oracle_rows(src, ts))
    for i in range(0, len(src), 5):
        assert np.array_equal(got[i], oracle.brute.foremost_dijkstra(
            tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, int(src[i]), int(ts[i])))
