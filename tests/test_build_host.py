"""libeat's host preprocessing (Section III-A layout) against the oracle's definitions (no GPU).

A host-only build (device = -1) exposes the built arrays; they must encode exactly
the oracle's connection types (Section II-B), cluster split (Section II-D) and
greedy AP cover (Section I-A), and the builder must reject invalid input.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle.ap_greedy import ap_cover, ap_expand
from paper_1912_00966_gb300 import eat

INF = 2**31 - 1


def _build(tt, **kw):
    return eat.eat_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=-1, **kw)


def _decode(net):
    """Per type (u, v, lambda) -> {cluster k: [(first, last, diff), ...]} from the host view."""
    hv = eat.eat_net_host_view(net)
    st = eat.eat_get_stats(net)
    out = {}
    rp, rec, clb, cl, ap = hv["row_ptr"], hv["type_rec"], hv["type_cl"], hv["cl"], hv["ap"]
    for u in range(st["n_stops"]):
        for t in range(rp[u], rp[u + 1]):
            v, lam, first, last = (int(x) for x in rec[t])
            W, t0 = st["cluster_width"], st["t0"]
            clusters = {}
            for k in range((first - t0) // W, (last - t0) // W + 1):
                lo, hi = int(cl[clb[t] + k]), int(cl[clb[t] + k + 1])
                aps = []
                for a in range(lo, hi):
                    start, packed = int(ap[a, 0]), int(ap[a, 1])
                    step, cnt = packed >> 16, packed & 0xFFFF
                    aps.append((start, start + (cnt - 1) * step, step))
                if aps:
                    clusters[k] = aps
            out[(u, v, lam)] = (first, last, clusters)
    return out, hv, st


@pytest.mark.parametrize("make,width,t0", [
    (synth.small_grid, 0, 0),
    (synth.small_grid, 900, 0),
    (synth.small_grid, 600, 17000),
    (lambda: synth.tiny_random(9, 400, 3, t_max=20000, dur_max=300), 3600, 0),
    (lambda: synth.tiny_random(5, 300, 4, t_max=500, dur_max=5), 7, 0),
])
def test_layout_matches_oracle(make, width, t0):
    tt = make()
    net = _build(tt, cluster_width=width, t0=t0)
    got, hv, st = _decode(net)
    W = width or 3600
    types = oracle.connection_types(tt)
    assert set(got) == set(types)
    assert st["n_types"] == len(types)
    assert st["n_conn"] == sum(len(d) for d in types.values())
    # types ordered by (u, v, lambda) inside each row
    keys = [(int(u), int(r[0]), int(r[1])) for u in range(st["n_stops"])
            for r in hv["type_rec"][hv["row_ptr"][u]:hv["row_ptr"][u + 1]]]
    assert keys == sorted(keys)
    for key, deps in types.items():
        first, last, clusters = got[key]
        assert first == deps[0] and last == deps[-1]
        want = oracle.cluster_sets(deps, width=W, t0=t0)
        assert set(clusters) == set(want)
        for k, vals in want.items():
            assert ap_expand(clusters[k]) == vals          # exact cover, no extra departures
            assert clusters[k] == ap_cover(vals)           # same greedy decisions
            starts = [a[0] for a in clusters[k]]
            assert starts == sorted(starts)


def test_duplicates_merged_and_stats():
    tt = synth.small_grid()
    twice = synth.Timetable("dup", tt.n_stops, np.concatenate([tt.u, tt.u]),
                            np.concatenate([tt.v, tt.v]), np.concatenate([tt.dep, tt.dep]),
                            np.concatenate([tt.dur, tt.dur]), np.concatenate([tt.trip, tt.trip]),
                            np.concatenate([tt.seq, tt.seq]))
    a = eat.eat_get_stats(_build(tt))
    b = eat.eat_get_stats(_build(twice))
    for k in ("n_types", "n_conn", "n_ap", "n_cl", "n_edges"):
        assert a[k] == b[k]
    assert a["n_conn"] == tt.n_conn


def test_paper_worked_example_through_builder():
    # Section II-C: departures 8:00, 8:15, ..., 18:00 on one type are a single AP
    # (8:00, 18:00, 15 min) when no cluster boundary cuts them.
    deps = np.arange(28800, 64801, 900, dtype=np.int32)
    n = deps.shape[0]
    z = np.zeros(n, np.int32)
    tt = synth.Timetable("ex", 2, z, z + 1, deps, z + 60, z, z)
    got, _, st = _decode(_build(tt, cluster_width=65535, t0=0))
    assert got[(0, 1, 60)][2] == {0: [(28800, 64800, 900)]}
    # With hourly clusters the same departures split into one AP per hour.
    got, _, _ = _decode(_build(tt))
    assert got[(0, 1, 60)][2][8] == [(28800, 31500, 900)]
    assert got[(0, 1, 60)][2][18] == [(64800, 64800, 0)]


@pytest.mark.parametrize("field,value,msg", [
    ("u", 10, "stop id"), ("v", -1, "stop id"), ("dur", 0, "duration"),
    ("dep", -5, "before t0"), ("dep", INF - 10, "overflow"),
])
def test_invalid_connections_rejected(field, value, msg):
    tt = synth.tiny_random(10, 50, 1)
    arrs = {f: getattr(tt, f).copy() for f in ("u", "v", "dep", "dur")}
    arrs[field][7] = value
    if field == "dep" and value > 0:
        arrs["dur"][7] = 20
    with pytest.raises(eat.EatError) as ei:
        eat.eat_build(10, arrs["u"], arrs["v"], arrs["dep"], arrs["dur"], device=-1)
    assert ei.value.code == eat.EAT_ERR_INVALID
    assert msg in str(ei.value)


def test_invalid_options_rejected():
    tt = synth.tiny_random(10, 50, 1)
    for kw in ({"cluster_width": 65536}, {"cluster_width": -3}):
        with pytest.raises(eat.EatError) as ei:
            _build(tt, **kw)
        assert ei.value.code == eat.EAT_ERR_INVALID
    with pytest.raises(eat.EatError) as ei:
        eat.eat_build(0, [], [], [], [], device=-1)
    assert ei.value.code == eat.EAT_ERR_INVALID
    with pytest.raises(eat.EatError) as ei:
        _build(tt, t0=10**6)
    assert ei.value.code == eat.EAT_ERR_INVALID


def test_empty_timetable_and_host_only_queries():
    net = eat.eat_build(4, [], [], [], [], device=-1)
    st = eat.eat_get_stats(net)
    assert st["n_types"] == 0 and st["n_ap"] == 0
    assert eat.eat_net_host_view(net)["row_ptr"].tolist() == [0, 0, 0, 0, 0]
    with pytest.raises(eat.EatError) as ei:
        eat.eat_query(net, 0, 0)
    assert ei.value.code == eat.EAT_ERR_NO_DEVICE


@pytest.mark.parametrize("make,width,t0", [
    (synth.small_grid, 0, 0),
    (synth.small_grid, 900, 1000),
    (lambda: synth.tiny_random(9, 400, 3, t_max=20000, dur_max=300), 3600, 0),
    (lambda: synth.tiny_random(5, 300, 4, t_max=500, dur_max=5), 7, 0),
    (lambda: synth.single_route(30000, 600, 40, [120, 60]), 1800, 0),
])
def test_device_cluster_entries_match_oracle(make, width, t0):
    """Every (type, cluster) entry of the device layout holds exactly the oracle's greedy
    cover of that cluster (first four APs inline, the rest in ap_extra, in order) and the
    first departure of the next non-empty cluster (INF if none); every type record holds
    the type's head, duration, the head's out-degree and first type, and the type's last
    departure."""
    tt = make()
    net = _build(tt, cluster_width=width, t0=t0)
    hv, st = eat.eat_net_host_view(net), eat.eat_get_stats(net)
    W = width or 3600
    types = oracle.connection_types(tt)
    rp, rec, ce, apx, tr = (hv[k] for k in ("row_ptr", "type_rec", "cluster_entries", "ap_extra",
                                            "type_records"))
    y, kmin = st["y"], st["k_min"]
    all_k = [(d - t0) // W for ds in types.values() for d in ds]
    assert kmin == min(all_k) and y == max(all_k) - kmin + 1

    def dec(start, sc):
        step, cnt = (sc >> 16) & 0xFFFF, sc & 0xFFFF
        return (int(start), int(start) + (cnt - 1) * step, step)

    for u in range(st["n_stops"]):
        for t in range(rp[u], rp[u + 1]):
            v, lam = int(rec[t][0]), int(rec[t][1])
            deps = types[(u, v, lam)]
            r = [int(x_) & 0xFFFFFFFF for x_ in tr[t]]
            assert (r[0], r[1] & 0xFFFFFF, r[2], r[3]) == (v, lam, rp[v], deps[-1])
            assert r[1] >> 24 == min(255, rp[v + 1] - rp[v])
            clusters = oracle.cluster_sets(deps, width=W, t0=t0)
            for kr in range(y):
                k = kmin + kr
                base = t0 + k * W
                e = [int(x_) & 0xFFFFFFFF for x_ in ce[t, kr]]
                n, x = e[4] >> 24, (e[4] & 0xFFFFFF) * 2
                if n == 255:
                    n, x = int(apx[x][0]), x + 2
                inline = [(e[0] & 0xFFFF, e[1]), (e[0] >> 16, e[2]), (e[5] & 0xFFFF, e[6]),
                          (e[5] >> 16, e[7])]
                got = [dec(base + rel, sc) for rel, sc in inline[:n]]
                for j in range(4, n):
                    got.append(dec(apx[x + j - 4][0], int(apx[x + j - 4][1])))
                assert got == ap_cover(clusters.get(k, []))
                later = [dd for dd in deps if (dd - t0) // W > k]
                assert e[3] == (min(later) if later else INF)


def test_count_overflow_header():
    """A cluster needing more than 254 APs keeps its count in the header of its AP list.
    Integers whose base-3 digits are all 0 or 1 contain no three-term arithmetic
    progression, so the greedy cover needs about one AP per two departures."""
    vals = [sum(((i >> b) & 1) * 3 ** b for b in range(10)) for i in range(1024)]
    deps = np.array(sorted(vals), dtype=np.int32)
    n = deps.shape[0]
    z = np.zeros(n, np.int32)
    tt = synth.Timetable("dense", 2, z, z + 1, deps, z + 5, z, z)
    net = _build(tt, cluster_width=65535)
    ce = eat.eat_net_host_view(net)["cluster_entries"]
    e4 = int(ce[0, 0, 4]) & 0xFFFFFFFF
    n_ap = eat.eat_get_stats(net)["n_ap"]
    assert n_ap >= 255 and e4 >> 24 == 255
    apx = eat.eat_net_host_view(net)["ap_extra"]
    assert int(apx[(e4 & 0xFFFFFF) * 2][0]) == n_ap


def test_long_duration_rejected():
    z = np.zeros(1, np.int32)
    with pytest.raises(eat.EatError) as ei:
        eat.eat_build(2, z, z + 1, z + 10, z + (1 << 24), device=-1)
    assert "2^24" in str(ei.value)


# ------------------------------------------------------------------ sub-trips (Section II-G)

def _expand_connections(net):
    """All connections (u, v, t, lambda) encoded by a built network, from its host view."""
    hv, st = eat.eat_net_host_view(net), eat.eat_get_stats(net)
    rp, rec, clb, cl, ap = hv["row_ptr"], hv["type_rec"], hv["type_cl"], hv["cl"], hv["ap"]
    W, t0 = st["cluster_width"], st["t0"]
    out = []
    for u in range(st["n_stops"]):
        for t in range(rp[u], rp[u + 1]):
            v, lam, first, last = (int(x) for x in rec[t])
            for a in range(cl[clb[t] + (first - t0) // W], cl[clb[t] + (last - t0) // W + 1]):
                start, packed = int(ap[a, 0]), int(ap[a, 1])
                step, cnt = packed >> 16, packed & 0xFFFF
                for m in range(cnt):
                    out.append((u, v, start + m * step, lam))
    return sorted(set(out))


def test_subtrips_on_one_route():
    # 9 connections per trip (stops 0..9): sqrt(9) = 3, so sub-trips 0-3, 3-6, 6-9.
    durs = [100, 200, 300, 50, 60, 70, 400, 10, 20]
    tt = synth.single_route(30000, 600, 5, durs)
    net = _build(tt, trip=tt.trip, subtrips=eat.EAT_SUBTRIPS_SQRT_K)
    st = eat.eat_get_stats(net)
    assert st["n_shortcuts"] == 3 * 5
    got = _expand_connections(net)
    cum = np.concatenate([[0], np.cumsum(durs)])
    for j in range(5):
        for a, b in ((0, 3), (3, 6), (6, 9)):
            assert (a, b, 30000 + 600 * j + int(cum[a]), int(cum[b] - cum[a])) in got
    assert len(got) == tt.n_conn + 15


def test_subtrips_mean_length_scheme():
    # Trips of 4 and 16 connections: mean 10, so sub-trips of round(sqrt(10)) = 3 everywhere.
    a = synth.single_route(1000, 1000, 1, [10] * 4, stops=np.arange(5))
    b = synth.single_route(2000, 1000, 1, [10] * 16, stops=np.arange(10, 27))
    cat = lambda f: np.concatenate([getattr(a, f), getattr(b, f)])
    trip = np.concatenate([a.trip, b.trip + 1])
    tt = synth.Timetable("two", 27, cat("u"), cat("v"), cat("dep"), cat("dur"), trip, cat("seq"))
    per_k = eat.eat_get_stats(_build(tt, trip=trip, subtrips=eat.EAT_SUBTRIPS_SQRT_K))
    mean = eat.eat_get_stats(_build(tt, trip=trip, subtrips=eat.EAT_SUBTRIPS_SQRT_MEAN))
    # sqrt(k): r = 2 for 4 (2 shortcuts), r = 4 for 16 (4 shortcuts); mean: r = 3 -> 1 + 5.
    assert per_k["n_shortcuts"] == 6
    assert mean["n_shortcuts"] == 6
    got = _expand_connections(_build(tt, trip=trip, subtrips=eat.EAT_SUBTRIPS_SQRT_MEAN))
    assert (0, 3, 1000, 30) in got and (3, 4, 1030, 10) in got and (10, 13, 2000, 30) in got


def test_subtrips_reject_broken_trips_and_missing_ids():
    tt = synth.small_grid()
    bad = tt.trip.copy()
    bad[5], bad[500] = bad[500], bad[5]            # two connections swap trips
    with pytest.raises(eat.EatError) as ei:
        _build(tt, trip=bad, subtrips=eat.EAT_SUBTRIPS_SQRT_K)
    assert ei.value.code == eat.EAT_ERR_INVALID and "trip" in str(ei.value)
    with pytest.raises(eat.EatError) as ei:
        _build(tt, subtrips=eat.EAT_SUBTRIPS_SQRT_K)
    assert ei.value.code == eat.EAT_ERR_INVALID
    with pytest.raises(eat.EatError):
        _build(tt, trip=tt.trip, subtrips=7)


@pytest.mark.parametrize("scheme", [1, 2])
def test_subtrips_leave_earliest_arrivals_unchanged(scheme):
    """Section II-G: the artificial connections ride the same vehicle, so the earliest
    arrival times of the enhanced timetable equal the original's (oracle on both)."""
    tt = synth.small_grid()
    net = _build(tt, trip=tt.trip, subtrips=scheme)
    conns = np.array(_expand_connections(net), dtype=np.int64)
    z = np.zeros(len(conns), np.int32)
    enh = synth.Timetable("enh", tt.n_stops, conns[:, 0].astype(np.int32), conns[:, 1].astype(np.int32),
                          conns[:, 2].astype(np.int32), conns[:, 3].astype(np.int32), z, z)
    assert len(conns) > tt.n_conn
    a, b = oracle.SortedConnections(tt), oracle.SortedConnections(enh)
    q = synth.random_queries(tt, 40, scheme)
    ra, _ = oracle.csa_many(a, q.source, q.t_s, 4)
    rb, _ = oracle.csa_many(b, q.source, q.t_s, 4)
    assert np.array_equal(ra, rb)


# ------------------------------------------------------------------ pre-encoded input (eat_build_csr)

def csr_from_view(net):
    """The pre-encoded (types, clusters, AP runs) arrays of a built network."""
    hv, st = eat.eat_net_host_view(net), eat.eat_get_stats(net)
    rp, rec, clb, cl, ap = hv["row_ptr"], hv["type_rec"], hv["type_cl"], hv["cl"], hv["ap"]
    W, t0 = st["cluster_width"], st["t0"]
    type_cl_ptr, cl_k, cl_ap_ptr, first, step, count = [0], [], [0], [], [], []
    for t in range(st["n_types"]):
        f, l = int(rec[t][2]), int(rec[t][3])
        for k in range((f - t0) // W, (l - t0) // W + 1):
            lo, hi = int(cl[clb[t] + k]), int(cl[clb[t] + k + 1])
            if hi == lo:
                continue
            cl_k.append(k)
            for a in range(lo, hi):
                first.append(int(ap[a, 0]))
                step.append(int(ap[a, 1]) >> 16)
                count.append(int(ap[a, 1]) & 0xFFFF)
            cl_ap_ptr.append(len(first))
        type_cl_ptr.append(len(cl_k))
    return dict(n_stops=st["n_stops"], row_ptr=rp, type_v=rec[:, 0], type_dur=rec[:, 1],
                type_cl_ptr=type_cl_ptr, cl_k=cl_k, cl_ap_ptr=cl_ap_ptr, ap_first=first,
                ap_step=step, ap_count=count)


@pytest.mark.parametrize("make,width", [(synth.small_grid, 3600), (synth.small_grid, 900),
                                        (lambda: synth.tiny_random(9, 400, 3, t_max=20000), 3600)])
def test_build_csr_round_trip(make, width):
    tt = make()
    a = _build(tt, cluster_width=width)
    b = eat.eat_build_csr(**csr_from_view(a), cluster_width=width, device=-1)
    va, vb = eat.eat_net_host_view(a), eat.eat_net_host_view(b)
    for k in ("row_ptr", "type_rec", "cl", "ap", "cluster_entries", "ap_extra", "type_records"):
        assert np.array_equal(va[k], vb[k]), k
    sa, sb = eat.eat_get_stats(a), eat.eat_get_stats(b)
    for k in ("n_types", "n_edges", "n_ap", "y", "k_min", "max_out_types"):
        assert sa[k] == sb[k], k


def test_build_csr_paper_example():
    # Section II-C: departures 8:00, 8:15, ..., 18:00 as one AP when one cluster spans them.
    net = eat.eat_build_csr(2, [0, 1, 1], [1], [60], [0, 1], [0], [0, 1], [28800], [900], [41],
                            cluster_width=65535, device=-1)
    st = eat.eat_get_stats(net)
    assert st["n_types"] == 1 and st["n_conn"] == 41 and st["n_ap"] == 1


@pytest.mark.parametrize("field,value,msg", [
    ("ap_first", [3599], "outside"), ("ap_count", [0], "count"), ("ap_step", [0], "difference"),
    ("type_dur", [0], "duration"), ("type_v", [5], "head stop"), ("row_ptr", [0, 2, 1], "row_ptr"),
    ("cl_k", [-1], "cluster index"),
])
def test_build_csr_rejects_bad_input(field, value, msg):
    args = dict(n_stops=2, row_ptr=[0, 1, 1], type_v=[1], type_dur=[60], type_cl_ptr=[0, 1],
                cl_k=[1], cl_ap_ptr=[0, 1], ap_first=[3600], ap_step=[600], ap_count=[6])
    eat.eat_build_csr(**args, device=-1)          # the unmodified input is valid
    args[field] = value
    with pytest.raises(eat.EatError) as ei:
        eat.eat_build_csr(**args, device=-1)
    assert ei.value.code == eat.EAT_ERR_INVALID and msg in str(ei.value)


def test_build_csr_rejects_unsorted_aps():
    args = dict(n_stops=2, row_ptr=[0, 1, 1], type_v=[1], type_dur=[60], type_cl_ptr=[0, 1],
                cl_k=[1], cl_ap_ptr=[0, 2], ap_first=[4000, 3700], ap_step=[0, 0], ap_count=[1, 1])
    with pytest.raises(eat.EatError) as ei:
        eat.eat_build_csr(**args, device=-1)
    assert "ordered" in str(ei.value)
