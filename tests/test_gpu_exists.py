"""GPU tests of existence queries with early termination (pg_count_until):
whether the target is reached equals the oracle's verdict; a run that did
not stop counts exactly; a stopped run reports between target and the true
count."""
import time

import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _cases():
    g1 = sg.chung_lu(3000, 15000, 2.1, 300.0, 401)
    g2 = sg.rmat(10, 8, 0.57, 0.19, 0.19, 402)
    g3 = sg.from_edges(12, [(i, 6 + j) for i in range(6) for j in range(6)])  # K_{6,6}: no triangle
    return [g1, g2, g3]


PATTERNS = [sg.pattern(3, sg.clique_edges(3)), sg.pattern(4, sg.clique_edges(4)), sg.pattern(5, sg.clique_edges(5)),
            sg.pattern(4, sg.cycle_edges(4), vertex_induced=True),
            sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 1), (3, 2)], anti_vertex=[0, 0, 0, 1])]


@pytest.mark.parametrize("gi", range(3))
def test_count_until_verdicts(pg, gi):
    g = _cases()[gi]
    G = pg.Graph.from_synth(g)
    for p in PATTERNS:
        want = oracle.count(g, p)
        plan = pg.Plan.from_dict(p)
        for target in sorted({1, 2, 17, max(1, want // 2), max(1, want), want + 1}):
            got, reached = pg.count_until(G, plan, target)
            assert reached == (want >= target), (p, target, want, got)
            if reached:
                assert target <= got <= want
            else:
                assert got == want
        assert pg.exists(G, plan) == (want > 0)


def test_clustering_coefficient_bound(pg):
    g = sg.chung_lu(3000, 15000, 2.1, 300.0, 403)
    G = pg.Graph.from_synth(g)
    T = oracle.triangles(g)
    W = oracle.stars(g, 2)
    c = 3 * T / W
    ans, tri, w = pg.clustering_coefficient_above(G, c * 0.9)
    assert ans and w == W and tri <= T
    ans, tri, w = pg.clustering_coefficient_above(G, c * 1.1)
    assert not ans and tri == T  # not reached: every triangle was counted


def test_existence_stops_early_on_large_graph(pg):
    """4-cliques exist in the 1M-vertex Chung-Lu workload graph by the
    thousands of millions; the query stops long before a full count."""
    g = sg.workload_graph(2)
    G = pg.Graph.from_synth(g)
    plan = pg.Plan(4, sg.clique_edges(4))
    pg.count_until(G, plan, 1000)  # warm (scratch sizing)
    t = time.perf_counter()
    got, reached = pg.count_until(G, plan, 1000)
    dt = time.perf_counter() - t
    assert reached and got >= 1000
    assert got < pg.count(G, [plan])[0]
    assert dt < 5.0
