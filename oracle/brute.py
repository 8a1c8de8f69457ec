"""Oracle (test infrastructure only): earliest arrival times by other routes than CSA.

Two independent brute-force methods for tiny timetables, used to pin the
connection-scan oracle:

  * `foremost_dijkstra`: the time-dependent Dijkstra of Bui-Xuan, Ferreira and
    Jarry (cited in Section I).  Waiting at a stop is allowed, so being at a stop
    earlier never hurts; the stop popped with the least time is final, and from
    stop x at time T every connection out of x with departure >= T is usable.
  * `exhaustive_paths`: enumerate every time-respecting path from s (Section I:
    each connection departs no earlier than the previous one arrives, the first
    one no earlier than t_s) and keep the least arrival per stop.

Both return a list of arrival times with INT32_MAX for unreachable stops and
e[s] = t_s.  Pure Python; tiny inputs only.
"""
from __future__ import annotations

import heapq

INF = 2**31 - 1


def foremost_dijkstra(n_stops, u, v, dep, dur, s, t_s):
    out = {}
    for i in range(len(u)):
        out.setdefault(int(u[i]), []).append((int(dep[i]), int(dur[i]), int(v[i])))
    best = [INF] * n_stops
    best[s] = t_s
    done = [False] * n_stops
    heap = [(t_s, s)]
    while heap:
        t, x = heapq.heappop(heap)
        if done[x] or t > best[x]:
            continue
        done[x] = True
        for d, lam, y in out.get(x, ()):
            if d >= t and d + lam < best[y]:
                best[y] = d + lam
                heapq.heappush(heap, (d + lam, y))
    return best


def exhaustive_paths(n_stops, u, v, dep, dur, s, t_s, max_conn=20):
    """Depth-first enumeration of all time-respecting paths (use only for a few dozen
    connections)."""
    conns = [(int(u[i]), int(v[i]), int(dep[i]), int(dur[i])) for i in range(len(u))]
    if len(conns) > max_conn:
        raise ValueError("exhaustive enumeration is for tiny inputs only")
    best = [INF] * n_stops
    best[s] = t_s

    def walk(x, t, used):
        for i, (a, b, d, lam) in enumerate(conns):
            if a == x and d >= t and not used[i]:
                arrive = d + lam
                if arrive < best[b]:
                    best[b] = arrive
                used[i] = True
                walk(b, arrive, used)
                used[i] = False

    walk(s, t_s, [False] * len(conns))
    return best
