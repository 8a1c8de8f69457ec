"""Oracle (test infrastructure only): greedy arithmetic-progression cover.

Section I-A ("Arithmetic Progression Technique", after Bast and Storandt) covers a
set S of departure times by APs: repeatedly take the smallest uncovered a in S,
choose the longest AP that starts at a, lies inside S and covers the most
still-uncovered numbers, and mark its terms covered.  An AP is stored as
(first term, last term, difference); Section II-C adds that expanding all APs of
a set gives back exactly S, and that the APs are kept in increasing order of
their first term.

Readings where the text leaves a choice:
  * an AP from a with difference d runs a, a+d, a+2d, ... for as long as the
    terms are in S (so it is the longest one with that difference);
  * "covers the most uncovered numbers" is the primary key and the AP length the
    secondary one; a remaining tie goes to the smallest difference;
  * an AP may contain numbers that an earlier AP already covers;
  * a one-element AP is written with difference 0 and first == last.

Plain loops, meant for the small sets of one cluster; only the tests use it.
"""
from __future__ import annotations


def ap_cover(values):
    """Return the greedy AP cover of the set `values` as a list of (first, last, diff)."""
    S = sorted(set(int(x) for x in values))
    in_s = set(S)
    uncovered = set(S)
    out = []
    while uncovered:
        a = min(uncovered)
        best_terms = [a]
        best_key = (1, 1)          # (uncovered terms covered, length)
        best_d = 0
        for b in S:
            if b <= a:
                continue
            d = b - a
            terms = [a]
            t = a + d
            while t in in_s:
                terms.append(t)
                t += d
            key = (sum(1 for x in terms if x in uncovered), len(terms))
            if key > best_key:     # strict: ties keep the smaller difference seen first
                best_key, best_terms, best_d = key, terms, d
        for x in best_terms:
            uncovered.discard(x)
        out.append((best_terms[0], best_terms[-1], best_d))
    out.sort(key=lambda ap: ap[0])
    return out


def ap_expand(aps):
    """All terms of a list of (first, last, diff) APs, as a sorted list without repeats."""
    terms = set()
    for first, last, d in aps:
        if d == 0:
            terms.add(first)
        else:
            terms.update(range(first, last + 1, d))
    return sorted(terms)
