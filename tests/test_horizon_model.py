"""A CPU model of the round schedule with a horizon (eat_query_opts.horizon), no GPU.

The per-query kernel relaxes, round by round, the connection types of the stops whose
arrival improved in the round before (Algorithms 3-5).  With a horizon step D it keeps a
horizon H (first t_s + D): a stop lowered to an arrival >= H waits instead of joining the
next frontier; when a round leaves no stop to expand, waiting stops whose arrival has
since dropped below H are dropped (that lowering queued them), H moves to the earliest
remaining arrival + D, and the stops below the new H are expanded next round.

This file runs that schedule in plain Python over the oracle's connection types and
getConnection (oracle.connection_types, oracle.next_departure) with rounds that read
the arrivals of the round before (the kernel reads them as they change; both reach the
fixpoint), and checks on small random networks, for steps from 1 s to beyond the day:
  * the arrivals equal the connection scan's (Algorithm 1) for every source and time,
  * the number of rounds stays within the kernel's default cap with a horizon, 2V + 2,
  * no stop that left the waiting list would ever have to wait again (the kernel's
    bitmap of stops that waited is never cleared within a query),
and that a planted mistake (releasing only the stops at the earliest waiting arrival,
not all below the new horizon, and never dropping the waiting list) is caught.
"""
import numpy as np
import pytest

import oracle
import synth

INF = 2**31 - 1


def _types_by_tail(tt):
    by_tail = {}
    for (u, v, lam), deps in oracle.connection_types(tt).items():
        by_tail.setdefault(u, []).append((v, lam, deps))
    return by_tail


def rounds_with_horizon(n_stops, by_tail, s, t_s, step, release_all=True):
    """Arrivals, rounds and the stops that waited, by the horizon schedule (step 0: none).
    Raises if a stop that already left the waiting list (released or dropped) would have
    to wait again: the kernel marks a stop that waited in a bitmap it never clears within
    a query, which is right only if that cannot happen."""
    e = [INF] * n_stops
    e[s] = t_s
    H = t_s + step if step > 0 and t_s < INF - step else INF
    frontier, waiting, waited, left = {s}, [], set(), set()
    rounds = 0
    while frontier:
        rounds += 1
        snapshot = list(e)
        nxt = set()
        for u in sorted(frontier):
            for v, lam, deps in by_tail.get(u, []):
                t_c = oracle.next_departure(deps, snapshot[u])
                if t_c == INF:
                    continue
                cand = t_c + lam
                if cand < e[v]:
                    e[v] = cand
                    if not by_tail.get(v):
                        continue                    # no types leave v: nothing to expand
                    if cand >= H:
                        if v in left:
                            raise AssertionError(f"stop {v} would wait a second time")
                        if v not in waited:
                            waited.add(v)
                            waiting.append(v)
                    else:
                        nxt.add(v)
        frontier = nxt
        if not frontier and waiting:
            keep = [v for v in waiting if e[v] >= H] if release_all else waiting
            left.update(v for v in waiting if v not in keep)
            if keep:
                lo = min(e[v] for v in keep)
                Hn = lo + step if lo < INF - step else INF
                if release_all:
                    frontier = {v for v in keep if e[v] < Hn}
                    waiting = [v for v in keep if e[v] >= Hn]
                    left.update(frontier)
                else:                               # planted mistake
                    frontier = {v for v in keep if e[v] == lo}
                    waiting = [v for v in keep if e[v] != lo and e[v] >= Hn]
                H = Hn
            else:
                left.update(waiting)
                waiting = []
    return np.array(e, dtype=np.int64), rounds, waited


def _cases():
    for seed in range(10):
        tt = synth.tiny_random(3 + seed % 7, 20 + 11 * seed, 700 + seed, t_max=400 + 60 * seed,
                               dur_max=5 + 7 * (seed % 4))
        yield seed, tt


@pytest.mark.parametrize("seed,tt", list(_cases()))
def test_same_fixpoint_within_the_round_cap(seed, tt):
    sc = oracle.SortedConnections(tt)
    by_tail = _types_by_tail(tt)
    rng = np.random.default_rng(seed)
    runs = with_waits = 0
    for s in range(tt.n_stops):
        for t_s in rng.integers(-5, int(tt.dep.max()) + 10, size=3).tolist():
            want = oracle.csa(sc, s, t_s).astype(np.int64)
            for step in (0, 1, 7, 30, 120, 10**6):
                got, rounds, waited = rounds_with_horizon(tt.n_stops, by_tail, s, t_s, step)
                assert np.array_equal(got, want), (s, t_s, step)
                assert rounds <= 2 * tt.n_stops + 2, (s, t_s, step, rounds)
                if step == 0:
                    assert rounds <= tt.n_stops + 1
                elif step <= 120:
                    runs += 1
                    with_waits += bool(waited)
    assert with_waits >= runs // 4          # the schedule is exercised, not bypassed


def test_small_grid_sample_and_waits_once():
    tt = synth.small_grid()
    sc = oracle.SortedConnections(tt)
    by_tail = _types_by_tail(tt)
    q = synth.random_queries(tt, 6, 0x51)
    n_waited = 0
    for s, t_s in zip(q.source.tolist(), q.t_s.tolist()):
        want = oracle.csa(sc, s, t_s).astype(np.int64)
        _, r0, _ = rounds_with_horizon(tt.n_stops, by_tail, s, t_s, 0)
        for step in (300, 3600):
            got, rounds, waited = rounds_with_horizon(tt.n_stops, by_tail, s, t_s, step)
            assert np.array_equal(got, want)
            assert rounds <= 2 * tt.n_stops + 2
            n_waited += len(waited)                   # (no stop waited twice: raised above)
        assert r0 <= tt.n_stops + 1
    assert n_waited > 100


def test_planted_release_mistake_is_caught():
    """Releasing only the stops at the earliest waiting arrival and forgetting the rest
    below the new horizon loses arrivals on some query of these networks."""
    caught = False
    for seed, tt in _cases():
        sc = oracle.SortedConnections(tt)
        by_tail = _types_by_tail(tt)
        for s in range(tt.n_stops):
            for t_s in (0, int(tt.dep.min())):
                want = oracle.csa(sc, s, t_s).astype(np.int64)
                got, _, _ = rounds_with_horizon(tt.n_stops, by_tail, s, t_s, 30, release_all=False)
                if not np.array_equal(got, want):
                    caught = True
                    break
            if caught:
                break
        if caught:
            break
    assert caught
