"""Seeded synthetic transit timetables shaped like the paper's GTFS workloads.

The paper measures on nine GTFS city feeds (Section IV, Table I).  Those feeds are
not available here, so these generators stand in for them: stops on a grid or a
random geometric graph, routes as random walks over that graph, trips that run
every h seconds along a route, and one connection (u, v, t, lambda) per trip and
route edge (Section I-A, Preliminaries: a connection leaves u at t and reaches v
at t + lambda).  Times are int32 seconds from 00:00 of the service day and may
run past 24 h (Section IV: some feeds cover more than a day).

This module only draws inputs.  It holds no part of the earliest-arrival
computation and is shared, unchanged, by the oracle side and the CUDA side.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 0xEA7
DAY_START = 5 * 3600      # first trip leaves its first stop no earlier than 05:00
DAY_END = 23 * 3600       # ... and no later than 23:00
QUERY_T_MIN = 5 * 3600    # query departure times are drawn from 05:00 ...
QUERY_T_MAX = 22 * 3600   # ... to 22:00


@dataclasses.dataclass
class Timetable:
    """A temporal graph G = (V, C) as structure-of-arrays int32 connections."""

    name: str
    n_stops: int
    u: np.ndarray      # int32 [C] departure stop
    v: np.ndarray      # int32 [C] arrival stop
    dep: np.ndarray    # int32 [C] departure time t (s)
    dur: np.ndarray    # int32 [C] duration lambda (s), >= 1
    trip: np.ndarray   # int32 [C] trip id (vehicle run) of the connection
    seq: np.ndarray    # int32 [C] position of the connection within its trip

    @property
    def n_conn(self) -> int:
        return int(self.u.shape[0])

    def sources_with_departures(self) -> np.ndarray:
        """Stops that have at least one outgoing connection."""
        return np.unique(self.u).astype(np.int32)


@dataclasses.dataclass
class QuerySet:
    """A batch of (network, source, departure time) queries."""

    net: np.ndarray      # int32 [Q] index into a list of timetables (0 for one net)
    source: np.ndarray   # int32 [Q]
    t_s: np.ndarray      # int32 [Q]

    def __len__(self) -> int:
        return int(self.source.shape[0])


# --------------------------------------------------------------------------- graphs

def grid_graph(n: int):
    """n stops on a ceil(sqrt(n))-wide grid (last row truncated), 4-neighbour edges.

    Returns a padded neighbour table nbr [n, 4] (-1 = none), degrees and positions."""
    w = int(math.ceil(math.sqrt(n)))
    ids = np.arange(n, dtype=np.int64)
    r, c = ids // w, ids % w
    cand = np.stack([ids - w, ids + w, ids - 1, ids + 1], axis=1)
    ok = np.stack([r > 0, ids + w < n, c > 0, (c < w - 1) & (ids + 1 < n)], axis=1)
    nbr = np.where(ok, cand, -1)
    pos = np.stack([c, r], axis=1).astype(np.float64)
    return nbr, ok.sum(axis=1), pos


def geometric_graph(n: int, k: int, rng: np.random.Generator):
    """n stops uniform in the unit square; each joined to its k nearest neighbours.

    The k-NN relation is symmetrised, so every edge is present in both directions.
    Returns a padded neighbour table nbr [n, dmax] (-1 = none), degrees and positions."""
    from scipy.spatial import cKDTree

    pts = rng.random((n, 2))
    _, idx = cKDTree(pts).query(pts, k=k + 1)
    a = np.repeat(np.arange(n), k)
    b = idx[:, 1:].reshape(-1)
    pairs = np.unique(np.concatenate([np.stack([a, b], 1), np.stack([b, a], 1)]), axis=0)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    deg = np.bincount(pairs[:, 0], minlength=n)
    dmax = int(deg.max())
    nbr = np.full((n, dmax), -1, dtype=np.int64)
    start = np.concatenate([[0], np.cumsum(deg)[:-1]])
    slot = np.arange(pairs.shape[0]) - start[pairs[:, 0]]
    nbr[pairs[:, 0], slot] = pairs[:, 1]
    return nbr, deg, pts


def random_walks(nbr, deg, lengths, starts, rng, pos=None, persistence=1.0):
    """One correlated random walk per route (a route keeps its heading, as bus lines do).

    At each step the next stop is the neighbour minimising
    -persistence * cos(turn angle) + U(0, 1), with stops already on the walk used only
    as a fallback.  lengths[r] is the number of stops of route r.  Returns an int64
    [R, Lmax] table of stop ids padded with -1."""
    R = len(lengths)
    L = int(lengths.max())
    path = np.full((R, L), -1, dtype=np.int64)
    path[:, 0] = starts
    dmax = nbr.shape[1]
    heading = rng.normal(size=(R, 2))
    for i in range(1, L):
        cur = path[:, i - 1]
        cand = nbr[cur]                                   # [R, dmax]
        key = rng.random((R, dmax))
        if pos is not None and persistence > 0:
            step = pos[np.maximum(cand, 0)] - pos[cur][:, None, :]
            norm = np.linalg.norm(step, axis=2) * np.linalg.norm(heading, axis=1)[:, None]
            cos = (step * heading[:, None, :]).sum(axis=2) / np.maximum(norm, 1e-12)
            key -= persistence * cos
        key[cand < 0] = 1e9                               # never pick padding
        seen = (cand[:, :, None] == path[:, None, :i]).any(axis=2)
        key[seen & (cand >= 0)] += 1e6                     # visited stops only as a fallback
        pick = cand[np.arange(R), key.argmin(axis=1)]
        live = i < lengths
        if pos is not None:
            heading = np.where(live[:, None], pos[pick] - pos[cur], heading)
        path[:, i] = np.where(live, pick, -1)
    return path


# --------------------------------------------------------------------------- timetables

def _undirected_durations(paths, rng, lo=60, hi=600):
    """Base duration per undirected stop pair, uniform int in [lo, hi], shared by all routes."""
    a = paths[:, :-1].reshape(-1)
    b = paths[:, 1:].reshape(-1)
    m = (a >= 0) & (b >= 0)
    lo_id, hi_id = np.minimum(a[m], b[m]), np.maximum(a[m], b[m])
    key = np.unique(lo_id * (1 << 32) + hi_id)
    val = rng.integers(lo, hi + 1, size=key.shape[0], dtype=np.int64)
    return key, val


def _band_duration(base, t, bands):
    """Apply the time-band duration rule: bands = list of (lo, hi, num, den)."""
    out = base.copy()
    for lo, hi, num, den in bands:
        sel = (t >= lo) & (t < hi)
        out[sel] = (num * base[sel] + den // 2) // den
    return out


def _timetable(name, n, paths, headway_min, jitter_frac, bands, rng) -> Timetable:
    """Runs trips along each route and emits one connection per trip and route edge.

    A trip's departure at stop i+1 equals its departure at stop i plus that edge's
    duration (no dwell), so a route edge sees exact arithmetic progressions of
    departures as long as the headway is constant and no jitter or band applies."""
    R, L = paths.shape
    key, val = _undirected_durations(paths, rng)
    hw = rng.integers(headway_min[0], headway_min[1] + 1, size=R) * 60
    ntrips = (DAY_END - DAY_START) // hw + 1
    trip_route = np.repeat(np.arange(R), ntrips)
    first = np.concatenate([[0], np.cumsum(ntrips)[:-1]])
    j = np.arange(trip_route.shape[0]) - first[trip_route]
    dep = DAY_START + j * hw[trip_route]
    if jitter_frac > 0:
        jit = rng.random(dep.shape[0]) < jitter_frac
        off = rng.integers(-180, 181, size=dep.shape[0])
        dep = dep + np.where(jit, off, 0)
    cu, cv, ct, cd, ctrip, cseq = [], [], [], [], [], []
    for i in range(L - 1):
        a = paths[trip_route, i]
        b = paths[trip_route, i + 1]
        live = (a >= 0) & (b >= 0)
        if not live.any():
            break
        a, b, t, tr = a[live], b[live], dep[live], np.nonzero(live)[0]
        k = np.minimum(a, b) * (1 << 32) + np.maximum(a, b)
        base = val[np.searchsorted(key, k)]
        d = _band_duration(base, t, bands)
        cu.append(a); cv.append(b); ct.append(t); cd.append(d); ctrip.append(tr)
        cseq.append(np.full(a.shape[0], i))
        dep = dep.copy()
        dep[live] = t + d
    cat = lambda xs: np.concatenate(xs).astype(np.int32)
    return Timetable(name, n, cat(cu), cat(cv), cat(ct), cat(cd), cat(ctrip), cat(cseq))


PEAK_BANDS = [(7 * 3600, 10 * 3600, 13, 10), (17 * 3600, 20 * 3600, 13, 10)]
OFFPEAK_BANDS = [(0, 6 * 3600, 8, 10), (21 * 3600, 1 << 30, 8, 10)]


def grid_timetable(n, n_routes, seed, route_len=20, headway_min=(10, 30),
                   force_stop0=True, name="grid") -> Timetable:
    """Grid network with routes as random walks (one direction), as in the small configuration."""
    rng = np.random.default_rng(seed)
    nbr, deg, pos = grid_graph(n)
    starts = rng.integers(0, n, size=n_routes)
    if force_stop0:
        starts[0] = 0
    lengths = np.full(n_routes, route_len)
    paths = random_walks(nbr, deg, lengths, starts, rng, pos)
    return _timetable(name, n, paths, headway_min, 0.0, [], rng)


def geometric_timetable(n, k, n_routes, route_len, headway_min, jitter_frac, bands,
                        seed, name="geometric") -> Timetable:
    """Random geometric k-NN network; routes run in both directions."""
    rng = np.random.default_rng(seed)
    nbr, deg, pos = geometric_graph(n, k, rng)
    starts = rng.integers(0, n, size=n_routes)
    lengths = rng.integers(route_len[0], route_len[1] + 1, size=n_routes)
    fwd = random_walks(nbr, deg, lengths, starts, rng, pos)
    back = np.full_like(fwd, -1)
    for r in range(n_routes):
        m = int(lengths[r])
        back[r, :m] = fwd[r, :m][::-1]
    paths = np.concatenate([fwd, back], axis=0)
    return _timetable(name, n, paths, headway_min, jitter_frac, bands, rng)


# --------------------------------------------------------------------------- configurations

def small_grid(seed_offset=0) -> Timetable:
    """1,024 stops on a 32x32 grid, 50 routes of 20 stops, headway 10-30 min."""
    return grid_timetable(1024, 50, SEED_BASE + 0 + seed_offset, name="grid1024")


def city(seed_offset=0) -> Timetable:
    """20,000 stops, geometric k=4, 400 routes of 30-60 stops both ways, headway 5-20 min,
    20% jittered trips, peak durations x1.3 in 07-10 and 17-20 h."""
    return geometric_timetable(20000, 4, 400, (30, 60), (5, 20), 0.20, PEAK_BANDS,
                               SEED_BASE + 1 + seed_offset, name="city20k")


def large(seed_offset=0) -> Timetable:
    """200,000 stops, geometric k=5, 4,000 routes of 40-80 stops both ways, headway 3-30 min,
    10% jittered trips, three duration bands (x1.3 peak, x0.8 early/late, x1 otherwise)."""
    return geometric_timetable(200000, 5, 4000, (40, 80), (3, 30), 0.10,
                               PEAK_BANDS + OFFPEAK_BANDS, SEED_BASE + 2 + seed_offset,
                               name="large200k")


def ragged_grids(n_nets=64, seed_offset=0):
    """Grid networks with stop counts log-uniform in [1,000, 50,000], route density as the
    small grid (ceil(50 n / 1024) routes of 20 stops)."""
    rng = np.random.default_rng(SEED_BASE + 3 + seed_offset)
    sizes = np.exp(rng.uniform(math.log(1000), math.log(50000), size=n_nets)).astype(np.int64)
    nets = []
    for i, n in enumerate(sizes):
        nets.append(grid_timetable(int(n), int(math.ceil(50 * n / 1024)),
                                   SEED_BASE + 1000 + 7 * i + seed_offset,
                                   force_stop0=False, name=f"grid{int(n)}"))
    return nets


def random_queries(nets, n_queries, seed, t_lo=QUERY_T_MIN, t_hi=QUERY_T_MAX) -> QuerySet:
    """Queries spread uniformly over nets; source uniform over stops with a departure;
    t_s uniform int in [t_lo, t_hi]."""
    if isinstance(nets, Timetable):
        nets = [nets]
    rng = np.random.default_rng(seed)
    net = rng.integers(0, len(nets), size=n_queries).astype(np.int32)
    src = np.empty(n_queries, dtype=np.int32)
    for i, tt in enumerate(nets):
        sel = np.nonzero(net == i)[0]
        cand = tt.sources_with_departures()
        src[sel] = cand[rng.integers(0, cand.shape[0], size=sel.shape[0])]
    ts = rng.integers(t_lo, t_hi + 1, size=n_queries).astype(np.int32)
    return QuerySet(net, src, ts)


def single_route(first_dep, headway, n_trips, durations, stops=None) -> Timetable:
    """One route, constant headway and per-edge durations: the closed-form case.

    Trip j leaves the first stop at first_dep + j*headway; stop i+1 is reached
    sum(durations[:i+1]) later."""
    durations = np.asarray(durations, dtype=np.int64)
    m = durations.shape[0]
    if stops is None:
        stops = np.arange(m + 1)
    stops = np.asarray(stops, dtype=np.int64)
    cum = np.concatenate([[0], np.cumsum(durations)])
    j = np.repeat(np.arange(n_trips), m)
    i = np.tile(np.arange(m), n_trips)
    dep = first_dep + j * headway + cum[i]
    c = lambda x: np.asarray(x, dtype=np.int32)
    return Timetable("route", int(stops.max()) + 1, c(stops[i]), c(stops[i + 1]), c(dep),
                     c(durations[i]), c(j), c(i))


def tiny_random(n_stops, n_conn, seed, t_max=200, dur_max=40) -> Timetable:
    """Unstructured random connections on a few stops, for brute-force checks."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n_stops, size=n_conn)
    v = (u + rng.integers(1, n_stops, size=n_conn)) % n_stops
    dep = rng.integers(0, t_max, size=n_conn)
    dur = rng.integers(1, dur_max + 1, size=n_conn)
    c = lambda x: np.asarray(x, dtype=np.int32)
    z = np.zeros(n_conn, dtype=np.int32)
    return Timetable("tiny", n_stops, c(u), c(v), c(dep), c(dur), z, z)


CONFIGS = {
    "small": small_grid,
    "city": city,
    "large": large,
}
