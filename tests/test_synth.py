"""The seeded generators are deterministic and produce valid, transit-shaped timetables."""
import numpy as np

import synth

INT32_MAX = 2**31 - 1


def _valid(tt):
    assert tt.u.dtype == np.int32 and tt.dep.dtype == np.int32
    assert tt.u.min() >= 0 and tt.u.max() < tt.n_stops
    assert tt.v.min() >= 0 and tt.v.max() < tt.n_stops
    assert (tt.u != tt.v).all()
    assert tt.dur.min() >= 1
    assert tt.dep.min() >= 0
    assert (tt.dep.astype(np.int64) + tt.dur).max() < INT32_MAX


def test_small_grid_deterministic_and_shaped():
    a, b = synth.small_grid(), synth.small_grid()
    for f in ("u", "v", "dep", "dur", "trip"):
        assert (getattr(a, f) == getattr(b, f)).all()
    _valid(a)
    assert a.n_stops == 1024
    assert 40_000 < a.n_conn < 100_000
    assert (a.u == 0).any()                     # route 0 starts at stop 0
    assert 60 <= a.dur.min() and a.dur.max() <= 600
    # grid edges only: |du| is 1 (same row) or 32 (same column)
    d = np.abs(a.u.astype(np.int64) - a.v)
    assert set(np.unique(d).tolist()) <= {1, 32}


def test_trips_are_chains():
    tt = synth.small_grid()
    order = np.lexsort((tt.seq, tt.trip))
    u, v, dep, dur, trip = tt.u[order], tt.v[order], tt.dep[order], tt.dur[order], tt.trip[order]
    same = trip[1:] == trip[:-1]
    assert (v[:-1][same] == u[1:][same]).all()
    assert (dep[:-1][same] + dur[:-1][same] == dep[1:][same]).all()


def test_queries_deterministic():
    tt = synth.small_grid()
    q1 = synth.random_queries(tt, 50, 9)
    q2 = synth.random_queries(tt, 50, 9)
    assert (q1.source == q2.source).all() and (q1.t_s == q2.t_s).all()
    has_dep = set(tt.sources_with_departures().tolist())
    assert all(s in has_dep for s in q1.source.tolist())
    assert q1.t_s.min() >= 5 * 3600 and q1.t_s.max() <= 22 * 3600


def test_single_route_shape():
    tt = synth.single_route(100, 60, 4, [10, 20])
    _valid(tt)
    assert tt.n_conn == 8
    assert sorted(tt.dep.tolist()) == [100, 110, 160, 170, 220, 230, 280, 290]
