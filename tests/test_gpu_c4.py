"""GPU parity of the 4-cycle co-degree kernel (the counted 4-cycle term of
every batch) against the oracle, bit-exact: the oracle's co-degree formula
S(C4) = 1/2 sum over pairs of C(codeg, 2), its backtracking count on small
graphs, and closed forms (K_n: 3 C(n, 4); K_{p,q}: C(p, 2) C(q, 2)).  Graphs
with hubs above 256 neighbours exercise the deferred whole-CTA path (its
x-range tiles of shared-memory counters, 16- and 32-bit)."""
from math import comb

import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


C4 = sg.pattern(4, sg.cycle_edges(4))


def _graphs():
    return {
        "er": sg.erdos_renyi(3000, 0.004, 901),
        "chung_lu_hubs": sg.chung_lu(20000, 150000, 2.1, 3000.0, 902),
        "rmat12": sg.rmat(12, 16, 0.57, 0.19, 0.19, 903),
        "rmat16": sg.workload_graph(3, scale_down=4),
    }


@pytest.mark.parametrize("name", ["er", "chung_lu_hubs", "rmat12", "rmat16"])
def test_c4_kernel_matches_oracle(pg, name):
    g = _graphs()[name]
    G = pg.Graph.from_synth(g)
    want = oracle.motif4_noninduced(g)["cycle"]
    plan = pg.Plan.from_dict(C4)
    assert pg.count(G, [plan]) == [want]
    if name in ("er", "rmat12"):
        assert want == oracle.count(g, C4)
    # the six induced 4-motifs: the 4-cycle term of their expansion goes here
    ind = oracle.motif4_induced(g)
    plans = [pg.Plan.from_dict(p) for p in sg.motif4_patterns()]
    assert pg.count(G, plans) == [ind[p["name"].replace("induced_", "")] for p in sg.motif4_patterns()]


def test_c4_closed_forms(pg):
    plan = pg.Plan.from_dict(C4)
    for n in (4, 5, 40, 700):  # 700: every anchor above 512 neighbours
        assert pg.count(pg.Graph.from_synth(sg.complete_graph(n)), [plan]) == [3 * comb(n, 4)]
    for p_, q_ in ((2, 2), (3, 900), (600, 600)):
        edges = [(i, p_ + j) for i in range(p_) for j in range(q_)]
        G = pg.Graph.from_synth(sg.from_edges(p_ + q_, edges))
        assert pg.count(G, [plan]) == [comb(p_, 2) * comb(q_, 2)]
    star = sg.from_edges(2001, [(0, i) for i in range(1, 2001)])
    assert pg.count(pg.Graph.from_synth(star), [plan]) == [0]


def test_c4_counter_widths_and_tiles(pg):
    """K_{p,q} with the p side as anchors of q neighbours each: q = 65,535
    keeps 16-bit counters at their largest value (the counter of the other
    p vertex reaches q), q = 70,000 takes 32-bit counters; both span several
    x-range tiles of the shared-memory pass."""
    plan = pg.Plan.from_dict(C4)
    for p_, q_ in ((2, 65535), (2, 70000), (3, 66000)):
        edges = [(i, p_ + j) for i in range(p_) for j in range(q_)]
        G = pg.Graph.from_synth(sg.from_edges(p_ + q_, edges))
        assert pg.count(G, [plan]) == [comb(p_, 2) * comb(q_, 2)]


def test_c4_in_mixed_batch_and_interpreter_agree(pg):
    """The same 4-cycle counted by the co-degree kernel inside a batch with
    other patterns, and by the plan interpreter (one intersection per path)."""
    import torch
    g = _graphs()["chung_lu_hubs"]
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan(3, sg.clique_edges(3)), pg.Plan.from_dict(C4), pg.Plan(4, sg.chain_edges(4)),
             pg.Plan(4, sg.cycle_edges(4), labels=None, vertex_induced=True)]
    got = pg.count(G, plans)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    pg.count_async(G, [plans[1]], out, kernel=pg.KERNEL_GENERIC)
    assert pg.decode_counts(out) == [got[1]]
    S = oracle.motif4_noninduced(g)
    I = oracle.motif4_induced(g)
    assert got == [oracle.triangles(g), S["cycle"], S["path"], I["cycle"]]
