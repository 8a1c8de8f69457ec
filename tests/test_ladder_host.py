"""Host arrays of the topology-driven variants (built with device=-1, no GPU) against the
oracle: the connection types and their sorted departures (Section II-B), the greedy AP
cover of each type's whole day (Section I-A, Section II-C) and the edges (Section II-E)."""
import numpy as np
import pytest

import oracle
import synth
from oracle.ap_greedy import ap_cover, ap_expand


@pytest.fixture(scope="module")
def eat():
    from paper_1912_00966_gb300 import eat as mod
    return mod


def _check(eat, tt, width, sample=None):
    lad = eat.eat_ladder_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, cluster_width=width,
                               device=-1)
    h = eat.eat_ladder_host_view(lad)
    types = oracle.connection_types(tt)
    uvl = [tuple(int(x) for x in r) for r in h["type_uvl"]]
    assert len(uvl) == len(types) and set(uvl) == set(types)
    assert uvl == sorted(uvl)                       # by tail, then head, then duration
    picks = range(len(uvl)) if sample is None else np.random.default_rng(1).choice(
        len(uvl), size=min(sample, len(uvl)), replace=False)
    for t in picks:
        key = uvl[t]
        dep = h["dep"][h["dep_ptr"][t]:h["dep_ptr"][t + 1]].tolist()
        assert dep == types[key], key
        aps = h["ap"][h["ap_ptr"][t]:h["ap_ptr"][t + 1]]
        got = [(int(f), int(f + (n - 1) * d), int(d)) for f, d, n in aps]
        assert got == ap_cover(types[key]), key
        assert ap_expand(got) == types[key]
    ep = h["edge_ptr"]
    assert ep[0] == 0 and ep[-1] == len(uvl) and (np.diff(ep) > 0).all()
    for e in range(len(ep) - 1):
        uv = {uvl[t][:2] for t in range(ep[e], ep[e + 1])}
        assert len(uv) == 1
        if e:
            assert uvl[ep[e] - 1][:2] != uvl[ep[e]][:2]
    assert len(ep) - 1 == len({k[:2] for k in types})
    lad.close()


def test_small_grid_all_types(eat):
    _check(eat, synth.small_grid(), 3600)


@pytest.mark.parametrize("seed", range(6))
def test_tiny_random_nets(eat, seed):
    tt = synth.tiny_random(3 + seed, 40 + 30 * seed, 900 + seed, t_max=2000 + 500 * seed,
                           dur_max=1 + 7 * seed)
    _check(eat, tt, [3600, 60, 7, 1, 600, 13][seed])


def test_city_sampled_types(eat):
    _check(eat, synth.city(), 1800, sample=300)


def test_query_needs_a_device(eat):
    tt = synth.small_grid()
    lad = eat.eat_ladder_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=-1)
    with pytest.raises(eat.EatError) as ei:
        eat.eat_ladder_query(lad, eat.EAT_VAR_TYPE, 0, 28800, graph=True, n_stops=tt.n_stops)
    assert ei.value.code == eat.EAT_ERR_NO_DEVICE
    with pytest.raises(eat.EatError) as ei:
        eat.eat_ladder_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, device=-1,
                             cluster_width=0, t0=10 ** 6)
    assert ei.value.code == eat.EAT_ERR_INVALID          # departures before t0
