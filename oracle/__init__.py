"""Oracle for earliest arrival times: plain, slow, obviously correct CPU code.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares no
code, header, table or helper with the CUDA path (`paper_1912_00966_gb300`), and
neither side imports the other; both read the same seeded inputs from `synth`.

Contents, each following the paper:
  * `csa`, `csa_many`: the connection-scan algorithm, Algorithm 1 (C, csa.c).
  * `certify`: exactness certificate for an arrival vector (C, csa.c).
  * `brute.foremost_dijkstra`, `brute.exhaustive_paths`: independent brute force.
  * `ap_greedy.ap_cover`: greedy AP cover (Section I-A, Arithmetic Progression
    Technique).
  * `next_departure`: the plain definition of getConnection (Section II-B):
    t_c = min{ t : (u, v, t, lambda) in C_{u,v,lambda}, t >= e[u] }.
  * `cluster_sets`: the partition of a connection type into clusters by
    departure time, cluster k holding departures in [t0 + kW, t0 + (k+1)W)
    (Section II-D with W = 3600 and t0 = 0: departures in [k:00:00, k:59:59]).
  * `connection_types`: the partition of C into connection types C_{u,v,lambda}
    (Section II-B), each type's departures sorted and merged.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import ap_greedy, brute  # noqa: F401
from .build import build as _build_lib

INF = 2**31 - 1
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)


def _load():
    global _lib
    if _lib is None:
        path = _build_lib()
        lib = ctypes.CDLL(path)
        lib.oracle_csa.restype = None
        lib.oracle_csa.argtypes = [ctypes.c_int32, ctypes.c_int64] + [_i32p] * 4 + [
            ctypes.c_int32, ctypes.c_int32, _i32p]
        lib.oracle_csa_many.restype = ctypes.c_int32
        lib.oracle_csa_many.argtypes = [ctypes.c_int32, ctypes.c_int64] + [_i32p] * 6 + [
            ctypes.c_int64, _i32p, ctypes.c_int32]
        lib.oracle_certify.restype = ctypes.c_int32
        lib.oracle_certify.argtypes = [ctypes.c_int32, ctypes.c_int64] + [_i32p] * 4 + [
            ctypes.c_int32, ctypes.c_int32, _i32p, ctypes.POINTER(ctypes.c_uint8),
            ctypes.POINTER(ctypes.c_int64)]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_i32p)


class SortedConnections:
    """Connections of a timetable sorted by departure time, as Algorithm 1 requires.

    The sort is a library primitive (numpy's stable argsort on the departure)."""

    def __init__(self, tt):
        order = np.argsort(tt.dep, kind="stable")
        self.n_stops = int(tt.n_stops)
        self.u = np.ascontiguousarray(tt.u[order], dtype=np.int32)
        self.v = np.ascontiguousarray(tt.v[order], dtype=np.int32)
        self.dep = np.ascontiguousarray(tt.dep[order], dtype=np.int32)
        self.dur = np.ascontiguousarray(tt.dur[order], dtype=np.int32)

    @property
    def n_conn(self):
        return int(self.u.shape[0])


def csa(sc: SortedConnections, s: int, t_s: int) -> np.ndarray:
    """Earliest arrival times from (s, t_s) by the connection-scan algorithm (Algorithm 1)."""
    lib = _load()
    e = np.empty(sc.n_stops, dtype=np.int32)
    lib.oracle_csa(sc.n_stops, sc.n_conn, _p(sc.u), _p(sc.v), _p(sc.dep), _p(sc.dur),
                   int(s), int(t_s), _p(e))
    return e


def csa_many(sc: SortedConnections, sources, times, n_threads: int = 1):
    """Algorithm 1 for each (sources[q], times[q]); returns ([Q, V] arrivals, threads used)."""
    lib = _load()
    src = np.ascontiguousarray(sources, dtype=np.int32)
    ts = np.ascontiguousarray(times, dtype=np.int32)
    out = np.empty((src.shape[0], sc.n_stops), dtype=np.int32)
    used = lib.oracle_csa_many(sc.n_stops, sc.n_conn, _p(sc.u), _p(sc.v), _p(sc.dep),
                               _p(sc.dur), _p(src), _p(ts), src.shape[0], _p(out),
                               int(n_threads))
    return out, int(used)


def certify(tt, s: int, t_s: int, e) -> tuple[int, int]:
    """Check that e is exactly the earliest-arrival vector for (s, t_s) on timetable tt.

    Returns (code, where): code 0 = exact; 1 = e[s] != t_s; 2 = a connection with
    e[u] <= t has e[v] > t + lambda (index `where`); 3 = stop `where` has a finite
    e[] without a witness connection.  Connection order does not matter."""
    lib = _load()
    e = np.ascontiguousarray(e, dtype=np.int32)
    u = np.ascontiguousarray(tt.u, dtype=np.int32)
    v = np.ascontiguousarray(tt.v, dtype=np.int32)
    dep = np.ascontiguousarray(tt.dep, dtype=np.int32)
    dur = np.ascontiguousarray(tt.dur, dtype=np.int32)
    scratch = np.empty(tt.n_stops, dtype=np.uint8)
    bad = ctypes.c_int64(-1)
    code = lib.oracle_certify(int(tt.n_stops), int(u.shape[0]), _p(u), _p(v), _p(dep), _p(dur),
                              int(s), int(t_s), _p(e),
                              scratch.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              ctypes.byref(bad))
    return int(code), int(bad.value)


def connection_types(tt):
    """Partition C into connection types C_{u,v,lambda} (Section II-B): connections with
    the same endpoints and duration.  Returns {(u, v, lambda): sorted unique departures}."""
    key = np.stack([tt.u, tt.v, tt.dur], axis=1).astype(np.int64)
    order = np.lexsort((tt.dep, key[:, 2], key[:, 1], key[:, 0]))
    out = {}
    for i in order:
        k = (int(tt.u[i]), int(tt.v[i]), int(tt.dur[i]))
        out.setdefault(k, []).append(int(tt.dep[i]))
    return {k: sorted(set(d)) for k, d in out.items()}


def next_departure(departures, e_u: int) -> int:
    """getConnection's result (Section II-B): the least departure >= e_u of a type, or INF."""
    best = INF
    for t in departures:
        if t >= e_u and t < best:
            best = t
    return best


def cluster_sets(departures, width: int = 3600, t0: int = 0):
    """Split a type's departures into clusters: cluster k holds t with
    k*width <= t - t0 < (k+1)*width (Section II-D).  Returns {k: sorted list}."""
    out = {}
    for t in departures:
        out.setdefault((int(t) - t0) // width, []).append(int(t))
    return {k: sorted(v) for k, v in out.items()}
