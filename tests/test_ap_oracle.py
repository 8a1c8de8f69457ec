"""Pins of the oracle's arithmetic-progression cover and cluster split (no GPU).

* the worked examples printed in the paper (tests/golden/ap_worked_examples.txt),
* expansion of the cover == the input set (Section II-C: no extra departures),
* every greedy step takes an AP that, among all APs from the smallest uncovered
  number inside the set, covers the most uncovered numbers (checked by brute
  force enumeration, independent of the oracle's loop),
* getConnection's plain definition against a sorted-list bisection, and the
  cluster split against the hour arithmetic of Section II-D.
"""
import bisect
import os

import numpy as np
import pytest

import oracle
from oracle.ap_greedy import ap_cover, ap_expand

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ap_worked_examples.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        cite, values, aps = [x.strip() for x in line.split("|")]
        if values.startswith("range"):
            a, b, d = map(int, values.split()[1:])
            vals = list(range(a, b + 1, d))
        else:
            vals = [int(x) for x in values.split()]
        want = [tuple(int(y) for y in ap.split(",")) for ap in aps.split(";")]
        rows.append((cite, vals, want))
    return rows


@pytest.mark.parametrize("cite,vals,want", _golden(), ids=lambda x: x if isinstance(x, str) else "")
def test_worked_examples(cite, vals, want):
    assert ap_cover(vals) == want
    assert ap_expand(want) == sorted(vals)


def test_singletons_and_duplicates():
    assert ap_cover([7]) == [(7, 7, 0)]
    assert ap_cover([5, 5, 5]) == [(5, 5, 0)]
    assert ap_cover([]) == []
    assert ap_cover([1, 2]) == [(1, 2, 1)]
    assert ap_cover([3, 100]) == [(3, 100, 97)]


def test_two_interleaved_progressions():
    # Two headways on one edge: 0, 10, 20, 30, 40 and 5, 17, 29 -> the greedy takes 0..40 step 10
    # first (5 uncovered terms), then 5..29 step 12.
    vals = [0, 10, 20, 30, 40, 5, 17, 29]
    assert ap_cover(vals) == [(0, 40, 10), (5, 29, 12)]


def _brute_best_from(a, S, uncovered):
    """All APs from a inside S (every difference, maximal extension), best by
    (uncovered covered, length, -difference)."""
    in_s = set(S)
    best = (1, 1, 0)
    for b in S:
        if b <= a:
            continue
        d = b - a
        n, t, unc = 0, a, 0
        while t in in_s:
            n += 1
            unc += t in uncovered
            t += d
        key = (unc, n, -d)
        if key > best:
            best = key
    return best


@pytest.mark.parametrize("seed", range(40))
def test_greedy_steps_are_optimal_and_cover_exactly(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    base = rng.integers(0, 3600, size=n)
    if seed % 3 == 0:       # add a real AP run so long progressions exist
        h = int(rng.integers(60, 900))
        base = np.concatenate([base, np.arange(int(rng.integers(0, 600)), 3600, h)])
    S = sorted(set(base.tolist()))
    cover = ap_cover(S)
    assert ap_expand(cover) == S
    assert [ap[0] for ap in cover] == sorted(ap[0] for ap in cover)
    # Replay the greedy order (by smallest uncovered first term) and check each step.
    uncovered = set(S)
    for first, last, d in sorted(cover, key=lambda ap: ap[0]):
        assert first == min(uncovered)
        terms = [first] if d == 0 else list(range(first, last + 1, d))
        unc = sum(t in uncovered for t in terms)
        best = _brute_best_from(first, S, uncovered)
        assert (unc, len(terms), -d) == best
        uncovered -= set(terms)
    assert not uncovered


def test_next_departure_definition():
    rng = np.random.default_rng(5)
    deps = sorted(set(rng.integers(0, 90000, size=300).tolist()))
    for e in list(rng.integers(-10, 95000, size=400)) + deps[:5] + [deps[-1], deps[-1] + 1]:
        i = bisect.bisect_left(deps, int(e))
        want = deps[i] if i < len(deps) else oracle.INF
        assert oracle.next_departure(deps, int(e)) == want


def test_cluster_sets_hours():
    deps = [0, 3599, 3600, 7199, 28800, 86399, 86400, 100000]
    got = oracle.cluster_sets(deps)
    assert got == {0: [0, 3599], 1: [3600, 7199], 8: [28800], 23: [86399], 24: [86400], 27: [100000]}
    got = oracle.cluster_sets(deps, width=900, t0=0)
    assert got[0] == [0] and got[3] == [3599] and got[4] == [3600] and got[32] == [28800]
