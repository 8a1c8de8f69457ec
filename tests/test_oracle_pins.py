"""Pins of the oracle to things other than itself (no GPU).

The connection-scan oracle (Algorithm 1) is checked against
  * two independent brute-force methods on tiny timetables (time-dependent
    Dijkstra; exhaustive enumeration of time-respecting paths),
  * the exactness certificate (feasibility + witness), which characterises the
    earliest-arrival vector without any scan order,
  * the closed form of a single route with constant headway,
  * monotonicity of arrivals in the departure time t_s,
and the pins themselves are shown to catch plausible mistakes planted in a CPU
copy of the scan (wrong comparison, dropped term, unsorted input).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import brute

INF = oracle.INF


def _sorted(tt):
    return oracle.SortedConnections(tt)


def _tiny_cases():
    cases = []
    for seed in range(60):
        n_stops = 2 + seed % 11
        n_conn = 1 + (seed * 7) % 200
        tt = synth.tiny_random(n_stops, n_conn, seed, t_max=120 + seed, dur_max=1 + seed % 40)
        cases.append(tt)
    return cases


@pytest.mark.parametrize("tt", _tiny_cases(), ids=lambda t: f"{t.n_stops}x{t.n_conn}")
def test_csa_matches_dijkstra_tiny(tt):
    sc = _sorted(tt)
    rng = np.random.default_rng(tt.n_conn)
    t_max = int(tt.dep.max()) + 5
    for s in range(tt.n_stops):
        for t_s in [0, int(rng.integers(0, t_max)), t_max, -7]:
            e = oracle.csa(sc, s, t_s)
            ref = brute.foremost_dijkstra(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, s, t_s)
            assert e.tolist() == ref
            assert oracle.certify(tt, s, t_s, e) == (0, -1)


@pytest.mark.parametrize("seed", range(25))
def test_csa_matches_exhaustive_paths(seed):
    tt = synth.tiny_random(2 + seed % 5, 4 + seed % 12, 1000 + seed, t_max=60, dur_max=15)
    sc = _sorted(tt)
    for s in range(tt.n_stops):
        for t_s in (0, 17, 40):
            e = oracle.csa(sc, s, t_s)
            ref = brute.exhaustive_paths(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, s, t_s)
            assert e.tolist() == ref


def test_special_cases():
    # lambda = 1 chains, identical departures, a source with no departures, t_s past the end.
    u = np.array([0, 1, 2, 0, 0, 3], np.int32)
    v = np.array([1, 2, 3, 2, 2, 0], np.int32)
    dep = np.array([10, 11, 12, 10, 10, 5], np.int32)
    dur = np.array([1, 1, 1, 5, 2, 1], np.int32)
    z = np.zeros(6, np.int32)
    tt = synth.Timetable("special", 5, u, v, dep, dur, z, z)
    sc = _sorted(tt)
    assert oracle.csa(sc, 0, 10).tolist() == [10, 11, 12, 13, INF]
    assert oracle.csa(sc, 0, 11).tolist() == [11, INF, INF, INF, INF]
    assert oracle.csa(sc, 4, 0).tolist() == [INF, INF, INF, INF, 0]   # isolated source
    assert oracle.csa(sc, 3, 5).tolist() == [6, 11, 12, 5, INF]        # departure exactly at t_s is usable
    assert oracle.csa(sc, 0, INF).tolist() == [INF] * 5


def test_special_case_chain_through_source_rejoin():
    # From 3 at t=5: reach 0 at 6, then 0->1 at 10 (arr 11), 1->2 at 11 (12), 0->2 at 10 (arr 12 via dur 2).
    u = np.array([0, 1, 2, 0, 0, 3], np.int32)
    v = np.array([1, 2, 3, 2, 2, 0], np.int32)
    dep = np.array([10, 11, 12, 10, 10, 5], np.int32)
    dur = np.array([1, 1, 1, 5, 2, 1], np.int32)
    z = np.zeros(6, np.int32)
    tt = synth.Timetable("special", 5, u, v, dep, dur, z, z)
    e = oracle.csa(_sorted(tt), 3, 4)
    assert e.tolist() == [6, 11, 12, 4, INF]


@pytest.mark.parametrize("first,headway,trips,durs", [
    (18000, 600, 30, [120, 300, 60, 600]),
    (0, 1, 50, [1, 1, 1]),
    (3600, 3599, 3, [5000]),
])
def test_closed_form_single_route(first, headway, trips, durs):
    """One route with trips every h from `first`: stop i>0 is reached at
    first + ceil(max(0, t_s - first)/h)*h + D_i if that trip exists, else never."""
    tt = synth.single_route(first, headway, trips, durs)
    sc = _sorted(tt)
    cum = np.concatenate([[0], np.cumsum(durs)])
    for t_s in [first - 100, first, first + 1, first + headway * (trips - 1), first + headway * trips,
                first + headway // 2 + 3]:
        e = oracle.csa(sc, 0, t_s)
        j = -(-max(0, t_s - first) // headway)
        for i in range(1, len(durs) + 1):
            want = first + j * headway + cum[i] if j <= trips - 1 else INF
            assert e[i] == want, (t_s, i)
        assert e[0] == t_s


def test_monotone_in_departure_time():
    tt = synth.small_grid()
    sc = _sorted(tt)
    prev = None
    for t_s in range(18000, 80000, 2400):
        e = oracle.csa(sc, 0, t_s).astype(np.int64)
        e[0] = 0  # e[s] = t_s by definition; compare the other stops
        if prev is not None:
            assert (e >= prev).all()
        prev = e


def test_small_grid_three_ways():
    tt = synth.small_grid()
    sc = _sorted(tt)
    q = synth.random_queries(tt, 6, 11)
    for s, t_s in [(0, 28800)] + list(zip(q.source.tolist(), q.t_s.tolist())):
        e = oracle.csa(sc, s, t_s)
        assert oracle.certify(tt, s, t_s, e) == (0, -1)
        ref = brute.foremost_dijkstra(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, s, t_s)
        assert e.tolist() == ref


def test_csa_many_matches_single_and_threads():
    tt = synth.small_grid()
    sc = _sorted(tt)
    q = synth.random_queries(tt, 20, 3)
    one, used1 = oracle.csa_many(sc, q.source, q.t_s, 1)
    many, used = oracle.csa_many(sc, q.source, q.t_s, 4)
    assert used1 == 1 and used >= 1
    assert (one == many).all()
    for i in range(20):
        assert (one[i] == oracle.csa(sc, q.source[i], q.t_s[i])).all()


# ------------------------------------------------------------------ the certificate's power

def test_certificate_rejects_perturbations():
    tt = synth.small_grid()
    sc = _sorted(tt)
    e = oracle.csa(sc, 0, 28800)
    reach = np.nonzero((e < INF) & (np.arange(tt.n_stops) != 0))[0]
    for x in reach[:20]:
        lower = e.copy(); lower[x] -= 1
        assert oracle.certify(tt, 0, 28800, lower)[0] == 3           # no witness
        higher = e.copy(); higher[x] += 1
        assert oracle.certify(tt, 0, 28800, higher)[0] in (2, 3)     # infeasible
        gone = e.copy(); gone[x] = INF
        assert oracle.certify(tt, 0, 28800, gone)[0] == 2
    unreach = np.nonzero(e == INF)[0]
    bad = e.copy(); bad[unreach[0]] = 99999
    assert oracle.certify(tt, 0, 28800, bad)[0] == 3
    src = e.copy(); src[0] = 28801
    assert oracle.certify(tt, 0, 28800, src)[0] == 1


# ------------------------------------------------------------------ mutation tests: planted mistakes

def _csa_py(n, u, v, dep, dur, s, t_s, mutate=None, sort=True):
    """A CPU copy of Algorithm 1 with an optional planted mistake."""
    order = np.argsort(dep, kind="stable") if sort else np.arange(len(dep))
    e = [INF] * n
    e[s] = t_s
    for i in order:
        a, b, t, lam = int(u[i]), int(v[i]), int(dep[i]), int(dur[i])
        if mutate == "strict_dep":
            ok = e[a] < t and t + lam < e[b]
        elif mutate == "no_tail_check":
            ok = t >= t_s and t + lam < e[b]
        elif mutate == "drop_lambda":
            ok = e[a] <= t and t < e[b]
            lam = 0
        elif mutate == "swap_uv":
            ok = e[b] <= t and t + lam < e[a]
            a, b = b, a
        else:
            ok = e[a] <= t and t + lam < e[b]
        if ok:
            e[b] = t + lam
    return e


@pytest.mark.parametrize("mutate,sort", [("strict_dep", True), ("no_tail_check", True),
                                          ("drop_lambda", True), ("swap_uv", True),
                                          (None, False)])
def test_pins_catch_planted_mistakes(mutate, sort):
    tt = synth.small_grid()
    caught = False
    for s, t_s in [(0, 28800), (0, 30000), (5, 40000)]:
        good = _csa_py(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, s, t_s)
        assert oracle.certify(tt, s, t_s, np.array(good, np.int32)) == (0, -1)
        bad = _csa_py(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, s, t_s, mutate=mutate, sort=sort)
        ref = brute.foremost_dijkstra(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, s, t_s)
        if bad != ref:
            assert oracle.certify(tt, s, t_s, np.array(bad, np.int32))[0] != 0
            caught = True
    assert caught
