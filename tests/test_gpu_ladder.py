"""Topology-driven variants of Section II (eat_ladder_*): every variant gives the oracle's
arrivals, with the flag read after every round or every few rounds (Section IV-C)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = [1, 2, 3, 4, 5, 6]


@pytest.fixture(scope="module")
def eat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_00966_gb300 import eat as mod
    return mod


def _ladder(eat, tt, width=3600):
    return eat.eat_ladder_build(tt.n_stops, tt.u, tt.v, tt.dep, tt.dur, cluster_width=width,
                                device=0)


@pytest.fixture(scope="module")
def small(eat):
    tt = synth.small_grid()
    return tt, oracle.SortedConnections(tt), _ladder(eat, tt)


@pytest.fixture(scope="module")
def city(eat):
    tt = synth.city()
    return tt, oracle.SortedConnections(tt), _ladder(eat, tt, 1800)


@pytest.mark.parametrize("variant", VARIANTS)
def test_small_grid_all_variants(eat, small, variant):
    tt, sc, lad = small
    q = synth.random_queries(tt, 12, 41)
    srcs = [0] + q.source.tolist()
    tss = [28800] + q.t_s.tolist()
    for s, t_s in zip(srcs, tss):
        want = oracle.csa(sc, s, t_s)
        for every, graph in ((1, False), (3, False), (1, True), (4, True)):
            got, st = eat.eat_ladder_query(lad, variant, s, t_s, flag_every=every, graph=graph,
                                           n_stops=tt.n_stops)
            assert np.array_equal(got, want), (variant, s, t_s, every, graph)
            assert st["rounds"] % every == 0 and st["flag_reads"] == st["rounds"] // every
            assert 1 <= st["rounds"] <= tt.n_stops + every


@pytest.mark.parametrize("seed", range(8))
def test_tiny_random_nets_all_variants(eat, seed):
    tt = synth.tiny_random(2 + seed, 30 + 40 * seed, 700 + seed, t_max=400 + 100 * seed,
                           dur_max=1 + 9 * seed)
    sc = oracle.SortedConnections(tt)
    lad = _ladder(eat, tt, [3600, 60, 7, 1][seed % 4])
    rng = np.random.default_rng(seed)
    for s in range(tt.n_stops):
        t_s = int(rng.integers(-5, int(tt.dep.max()) + 10))
        want = oracle.csa(sc, s, t_s)
        for variant in VARIANTS:
            got, _ = eat.eat_ladder_query(lad, variant, s, t_s, n_stops=tt.n_stops)
            assert np.array_equal(got, want), (variant, s, t_s)
    lad.close()


@pytest.mark.parametrize("variant", VARIANTS)
def test_city_variants(eat, city, variant):
    tt, sc, lad = city
    q = synth.random_queries(tt, 3, 43)
    out = torch.full((tt.n_stops,), -7, dtype=torch.int32, device="cuda")
    for i in range(3):
        want = oracle.csa(sc, int(q.source[i]), int(q.t_s[i]))
        for graph in (False, True):
            out.fill_(-7)
            _, st = eat.eat_ladder_query(lad, variant, int(q.source[i]), int(q.t_s[i]), out=out,
                                         flag_every=8, graph=graph)
            assert np.array_equal(out.cpu().numpy(), want), (variant, i, graph)
            assert st["rounds"] % 8 == 0


def test_invalid_arguments(eat, small):
    tt, _, lad = small
    for variant, s, every in [(0, 0, 1), (7, 0, 1), (4, -1, 1), (4, tt.n_stops, 1), (4, 0, 0)]:
        with pytest.raises(eat.EatError) as ei:
            eat.eat_ladder_query(lad, variant, s, 28800, flag_every=every, n_stops=tt.n_stops)
        assert ei.value.code == eat.EAT_ERR_INVALID
