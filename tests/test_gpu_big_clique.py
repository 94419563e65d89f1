"""GPU parity of k-cliques above 8 vertices (up to 16) on the k-clique
kernel, bit-exact against the oracle's textbook clique lister and C(n, k),
and the paper's 14-clique existence query (Evaluation, existence table) on
graphs with and without a 14-clique."""
from math import comb

import numpy as np
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def planted(n, m, clique_sizes, seed, max_weight=None):
    """Chung-Lu graph (n, m, gamma 2.1) with cliques of the given sizes
    planted on seeded random vertex sets (overlaps allowed)."""
    g = sg.chung_lu(n, m, 2.1, max_weight or n / 10, seed)
    rng = np.random.default_rng(seed + 1)
    edges = [tuple(e) for e in g.edges().tolist()]
    for s in clique_sizes:
        vs = rng.choice(n, s, replace=False)
        edges += [(int(vs[i]), int(vs[j])) for i in range(s) for j in range(i + 1, s)]
    return sg.from_edges(n, edges)


def _count(pg, G, ks):
    import torch
    plans = [pg.Plan(k, sg.clique_edges(k)) for k in ks]
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    pg.count_async(G, plans, out, kernel=pg.KERNEL_AUTO)
    torch.cuda.synchronize()
    return pg.decode_counts(out)


@pytest.mark.parametrize("heavy_min", [64, 8])
def test_large_cliques_match_oracle(pg, heavy_min):
    """Sizes 9..16 in one launch and alone; heavy_min 8 sends every start
    vertex of out-degree > 8 through the CTA-wide tile."""
    g = planted(3000, 20000, [18, 15, 12], 7101)
    G = pg.Graph.from_synth(g)
    pg.set_tuning(G, clique_heavy_min=heavy_min)
    ks = list(range(9, 17))
    want = [oracle.kcliques(g, k) for k in ks]
    assert want[0] > 0 and want[-1] > 0
    assert _count(pg, G, ks) == want
    assert _count(pg, G, [14]) == [want[5]]
    assert _count(pg, G, [16, 10]) == [want[7], want[1]]
    # sizes on both sides of 8 in one launch (the 16-wide variant)
    assert _count(pg, G, [7, 9]) == [oracle.kcliques(g, 7), want[0]]
    assert pg.count(G, [pg.Plan(12, sg.clique_edges(12))]) == [want[3]]


@pytest.mark.parametrize("n", [20, 24])
def test_large_cliques_complete_graphs(pg, n):
    G = pg.Graph.from_synth(sg.complete_graph(n))
    ks = list(range(9, 17))
    assert _count(pg, G, ks) == [comb(n, k) for k in ks]


def test_fourteen_clique_existence(pg):
    """Existence of a 14-clique stops at the first one found; without one
    the whole graph is explored and the exact count (0) comes back."""
    plan = pg.Plan(14, sg.clique_edges(14))
    g_yes = planted(20000, 150000, [16], 7102, max_weight=100.0)
    G = pg.Graph.from_synth(g_yes)
    got, reached = pg.count_until(G, plan, 1)
    assert reached and 1 <= got <= oracle.kcliques(g_yes, 14)
    assert pg.exists(G, plan)
    g_no = planted(20000, 150000, [13, 13], 7103, max_weight=100.0)
    assert oracle.kcliques(g_no, 14) == 0 and oracle.kcliques(g_no, 13) >= 2
    G2 = pg.Graph.from_synth(g_no)
    got, reached = pg.count_until(G2, plan, 1)
    assert not reached and got == 0
    got, reached = pg.count_until(G2, pg.Plan(13, sg.clique_edges(13)), 2)
    assert reached and got >= 2


def test_large_cliques_refused_elsewhere(pg):
    import torch
    G = pg.Graph.from_synth(sg.complete_graph(12))
    plan = pg.Plan(10, sg.clique_edges(10))
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for kernel in (pg.KERNEL_GENERIC, pg.KERNEL_CLIQUE_PLAIN, pg.KERNEL_BATCHED):
        with pytest.raises(pg.PgError) as e:
            pg.count_async(G, [plan], out, kernel=kernel)
        assert e.value.code == pg.PG_EUNSUPPORTED
    with pytest.raises(pg.PgError) as e:
        pg.match(G, plan)
    assert e.value.code == pg.PG_EUNSUPPORTED
    with pytest.raises(pg.PgError) as e:
        pg.Batch([plan])
    assert e.value.code == pg.PG_EUNSUPPORTED
    assert pg.count(G, [plan]) == [comb(12, 10)]
