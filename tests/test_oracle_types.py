"""Pins of oracle.connection_types, the type partition of Section II-B (no GPU).

A connection type C_{u,v,lambda} holds the connections of one edge (u, v) that share
the duration lambda.  The oracle's partition is checked against
  * a hand-written timetable whose types are known by construction (two durations on
    one edge, a reverse edge, duplicate departures, departures out of order),
  * an invariant computed from the raw connections with plain Python sets: the
    (u, v, lambda, t) tuples of all types are exactly the distinct tuples of the
    input, each type's departures are strictly increasing, and every member of a
    type carries the type's key,
and two plausible mistakes planted in CPU copies (grouping by the edge alone; no
merge of identical departures) are shown to fail these pins.
"""
import numpy as np
import pytest

import oracle
import synth


def _tt(rows, n_stops):
    a = np.array(rows, np.int32)
    z = np.zeros(len(rows), np.int32)
    return synth.Timetable("types", n_stops, a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy(),
                           a[:, 3].copy(), z, z)


# (u, v, dep, dur): edge 0->1 with durations 60 and 90, its reverse 1->0, a duplicate
# departure (0->1 at 100, dur 60, twice), departures listed out of order, and an edge
# 2->1 whose duration equals one of 0->1's.
HAND = [
    (0, 1, 300, 60),
    (0, 1, 100, 60),
    (0, 1, 100, 60),
    (0, 1, 200, 90),
    (0, 1, 100, 90),
    (1, 0, 150, 60),
    (1, 0, 50, 60),
    (2, 1, 100, 60),
    (0, 1, 250, 60),
]
HAND_TYPES = {
    (0, 1, 60): [100, 250, 300],
    (0, 1, 90): [100, 200],
    (1, 0, 60): [50, 150],
    (2, 1, 60): [100],
}


def _check_invariant(tt, types):
    tuples = {(int(a), int(b), int(lam), int(t))
              for a, b, t, lam in zip(tt.u, tt.v, tt.dep, tt.dur)}
    got = set()
    total = 0
    for key, deps in types.items():
        assert len(key) == 3
        assert all(deps[i] < deps[i + 1] for i in range(len(deps) - 1)), key
        total += len(deps)
        for t in deps:
            got.add((key[0], key[1], key[2], int(t)))
    assert got == tuples
    assert total == len(tuples)
    # every connection's key names a type that holds its departure
    for a, b, t, lam in zip(tt.u, tt.v, tt.dep, tt.dur):
        assert int(t) in types[(int(a), int(b), int(lam))]


def test_hand_written_types():
    tt = _tt(HAND, 3)
    assert oracle.connection_types(tt) == HAND_TYPES


@pytest.mark.parametrize("seed", range(12))
def test_invariant_on_random_timetables(seed):
    tt = synth.tiny_random(2 + seed % 6, 5 + 13 * seed, 300 + seed, t_max=90, dur_max=1 + seed % 5)
    _check_invariant(tt, oracle.connection_types(tt))


def test_invariant_on_small_grid():
    tt = synth.small_grid()
    types = oracle.connection_types(tt)
    _check_invariant(tt, types)
    # the grid's routes give constant durations per edge: one type per edge
    assert len(types) == len({(int(a), int(b)) for a, b in zip(tt.u, tt.v)})


def test_invariant_on_city_duration_bands():
    # Peak-hour durations (x1.3) give edges with two types.
    tt = synth.city()
    sel = np.arange(0, tt.n_conn, 37)
    sub = synth.Timetable("city-sample", tt.n_stops, tt.u[sel], tt.v[sel], tt.dep[sel],
                          tt.dur[sel], tt.trip[sel], tt.seq[sel])
    types = oracle.connection_types(sub)
    _check_invariant(sub, types)
    edges = {(k[0], k[1]) for k in types}
    assert len(types) > len(edges)


# ------------------------------------------------------------------ planted mistakes

def _types_by_edge_only(tt):
    """Mistake: groups by (u, v) and keeps the first duration seen as the key."""
    out, lam_of = {}, {}
    for a, b, t, lam in zip(tt.u.tolist(), tt.v.tolist(), tt.dep.tolist(), tt.dur.tolist()):
        lam_of.setdefault((a, b), lam)
        out.setdefault((a, b), set()).add(t)
    return {(a, b, lam_of[(a, b)]): sorted(d) for (a, b), d in out.items()}


def _types_no_merge(tt):
    """Mistake: keeps identical departures of a type twice."""
    out = {}
    for a, b, t, lam in zip(tt.u.tolist(), tt.v.tolist(), tt.dep.tolist(), tt.dur.tolist()):
        out.setdefault((a, b, lam), []).append(t)
    return {k: sorted(d) for k, d in out.items()}


@pytest.mark.parametrize("mutant", [_types_by_edge_only, _types_no_merge])
def test_pins_catch_planted_mistakes(mutant):
    tt = _tt(HAND, 3)
    assert mutant(tt) != HAND_TYPES
    with pytest.raises(AssertionError):
        _check_invariant(tt, mutant(tt))
