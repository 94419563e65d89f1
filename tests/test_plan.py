"""Plan compiler (host) tests: the paper's worked plan, plan facts, compile
latency, and counts from a CPU interpretation of the compiled level program
against the oracle.  CPU only: the library is loaded but no kernel runs."""
import json
import os
import time

import numpy as np
import pytest

import oracle
import synthgraph as sg
import planeval

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pg():
    import paper_2004_02369_b300 as pg
    return pg


def test_diamond_worked_plan():
    """Section 4.1: PO u1<u3, u2<u4; core {u2,u4}; one matching order."""
    f = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))["diamond_plan"]
    pg = _pg()
    plan = pg.Plan(f["pattern"]["k"], f["pattern"]["edges"])
    info = plan.info()
    po = sorted((info.po[2 * i], info.po[2 * i + 1]) for i in range(info.n_po))
    assert po == sorted(tuple(x) for x in f["partial_order_pairs"])
    core = [u for u in range(4) if info.core_mask >> u & 1]
    assert core == f["core"]
    assert info.n_orders == f["n_matching_orders"]
    assert info.automorphisms == f["automorphisms"]
    # the two non-core vertices u1, u3 form one chain counted as C(|S|, 2)
    assert info.counted_group == 2


def test_star_aut_and_chain():
    pg = _pg()
    info = pg.Plan(4, sg.star_edges(4)).info()
    assert info.automorphisms == 6
    assert info.core_mask == 1  # the centre
    assert info.counted_group == 3  # three leaves counted as C(d, 3)


def test_clique_plan_is_oriented():
    pg = _pg()
    for k in range(3, 8):
        info = pg.Plan(k, sg.clique_edges(k)).info()
        assert info.n_orders == 1
        assert bin(info.core_mask).count("1") == k - 1
        # the counted vertex is the PO-smallest one (vertex 0)
        assert not (info.core_mask & 1)


ALL_PATTERNS = ([sg.pattern(k, sg.clique_edges(k)) for k in range(1, 6)]
                + [sg.pattern(k, sg.star_edges(k)) for k in range(3, 7)]
                + [sg.pattern(k, sg.chain_edges(k)) for k in range(2, 6)]
                + [sg.pattern(k, sg.cycle_edges(k)) for k in range(4, 7)]
                + [sg.pattern(4, sg.TAILED_TRIANGLE), sg.pattern(4, sg.DIAMOND)]
                + sg.motif3_patterns() + sg.motif4_patterns()
                + [sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)]),
                   sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1), (3, 2)]),
                   sg.pattern(4, sg.cycle_edges(4), anti_edges=[(0, 2)]),
                   sg.pattern(5, sg.cycle_edges(5), vertex_induced=True),
                   sg.pattern(5, sg.star_edges(5), vertex_induced=True),
                   sg.pattern(5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4)], vertex_induced=True),
                   sg.pattern(6, sg.star_edges(4) + [(3, 4), (3, 5)])])

# Anti-vertex patterns (Section 3.1.2): triangles in no 4-clique, the paper's
# p_e (friend pairs with one mutual friend), edges with no common neighbour,
# wedges whose ends share no other neighbour, a star leaf of degree one, a
# 4-cycle with no vertex adjacent to all four, two anti-vertices on a path,
# a vertex-induced wedge with one, an isolated vertex.
ANTI_VERTEX_PATTERNS = [
    sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 1), (3, 2)], anti_vertex=[0, 0, 0, 1]),
    sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 2)], anti_vertex=[0, 0, 0, 1]),
    sg.pattern(3, [(0, 1)], anti_edges=[(2, 0), (2, 1)], anti_vertex=[0, 0, 1]),
    sg.pattern(4, [(0, 1), (1, 2)], anti_edges=[(3, 0), (3, 2)], anti_vertex=[0, 0, 0, 1]),
    sg.pattern(5, sg.star_edges(4), anti_edges=[(4, 1)], anti_vertex=[0, 0, 0, 0, 1]),
    sg.pattern(5, sg.cycle_edges(4), anti_edges=[(4, 0), (4, 1), (4, 2), (4, 3)], anti_vertex=[0, 0, 0, 0, 1]),
    sg.pattern(5, sg.chain_edges(3), anti_edges=[(3, 0), (3, 1), (4, 1), (4, 2)], anti_vertex=[0, 0, 0, 1, 1]),
    sg.pattern(4, [(0, 1), (1, 2)], anti_edges=[(3, 0), (3, 2)], anti_vertex=[0, 0, 0, 1], vertex_induced=True),
    sg.pattern(2, [], anti_edges=[(0, 1)], anti_vertex=[0, 1]),
    sg.pattern(5, sg.TAILED_TRIANGLE, anti_edges=[(4, 3)], anti_vertex=[0, 0, 0, 0, 1]),
]


def test_compile_latency_under_half_ms():
    """Section 4.1: plans are computed from the pattern alone, typically < 0.5 ms."""
    pg = _pg()
    for p in sg.motif3_patterns() + sg.motif4_patterns() + [sg.pattern(5, sg.clique_edges(5))]:
        plan = pg.Plan.from_dict(p)
        assert plan.info().compile_ms < 0.5, p


def test_plan_aut_matches_oracle():
    pg = _pg()
    for p in ALL_PATTERNS:
        assert pg.Plan.from_dict(p).info().automorphisms == oracle.automorphisms(p)


def _graphs():
    g1 = sg.erdos_renyi(30, 0.25, 101)
    g2 = sg.chung_lu(80, 300, 2.1, 25.0, 102)
    g3 = sg.rmat(6, 6, 0.57, 0.19, 0.19, 103)
    g4 = sg.erdos_renyi(25, 0.3, 104)
    g4.labels = sg.uniform_labels(g4.n, 3, 105)
    return [g1, g2, g3, g4, sg.complete_graph(8)]


@pytest.mark.parametrize("gi", range(5))
def test_plan_interpretation_matches_oracle(gi):
    g = _graphs()[gi]
    for p in ALL_PATTERNS:
        got, _ = planeval.count(g, p)
        assert got == oracle.count(g, p), (p, gi)


@pytest.mark.parametrize("gi", range(5))
def test_listing_program_matches_oracle(gi):
    """The listing program (every vertex on its own level) finds each match once."""
    g = _graphs()[gi]
    for p in ALL_PATTERNS + ANTI_VERTEX_PATTERNS:
        got, _ = planeval.count(g, p, listing=True)
        assert got == oracle.count(g, p), (p, gi)


@pytest.mark.parametrize("gi", range(5))
def test_anti_vertex_plans_match_oracle(gi):
    g = _graphs()[gi]
    for p in ANTI_VERTEX_PATTERNS:
        got, _ = planeval.count(g, p)
        assert got == oracle.count(g, p), (p, gi)


def test_anti_vertex_symmetry_breaking_paper_example():
    """Section 4.3: in p_e the anti-vertex splits the triangle's symmetry; only
    the two vertices it is anti-adjacent to stay interchangeable."""
    pg = _pg()
    info = pg.Plan.from_dict(ANTI_VERTEX_PATTERNS[1]).info()
    assert info.automorphisms == 2
    po = sorted((info.po[2 * i], info.po[2 * i + 1]) for i in range(info.n_po))
    assert po == [(0, 2)]


def test_labeled_plans_match_oracle():
    g = _graphs()[3]
    rng = np.random.default_rng(3)
    for edges, k in [(sg.chain_edges(3), 3), (sg.star_edges(4), 4), (sg.chain_edges(4), 4),
                     (sg.clique_edges(3), 3), (sg.TAILED_TRIANGLE, 4), (sg.cycle_edges(4), 4)]:
        for _ in range(4):
            labels = [int(x) if x < 3 else -1 for x in rng.integers(0, 4, k)]
            for vi in (False, True):
                p = sg.pattern(k, edges, labels=labels, vertex_induced=vi)
                got, _ = planeval.count(g, p)
                assert got == oracle.count(g, p), p


def test_invalid_patterns_rejected():
    pg = _pg()
    with pytest.raises(pg.PgError) as e:
        pg.Plan(3, [(0, 1)])  # vertex 2 disconnected
    assert e.value.code == pg.PG_EINVAL
    with pytest.raises(pg.PgError):  # above 8 vertices only cliques
        pg.Plan(9, [(i, i + 1) for i in range(8)])
    with pytest.raises(pg.PgError):  # cliques up to 16
        pg.Plan(17, sg.clique_edges(17))
    with pytest.raises(pg.PgError):  # a 9-clique without one edge
        pg.Plan(9, sg.clique_edges(9)[1:])
    with pytest.raises(pg.PgError):  # labeled large clique
        pg.Plan(10, sg.clique_edges(10), labels=[0] * 10)
    with pytest.raises(pg.PgError):
        pg.Plan(3, [(0, 1), (1, 2)], anti_edges=[(0, 1)])
    with pytest.raises(pg.PgError):
        pg.Plan(2, [(0, 0)])
    with pytest.raises(pg.PgError):  # anti-vertex with a true edge
        pg.Plan(3, [(0, 1), (1, 2)], anti_vertex=[0, 0, 1])
    with pytest.raises(pg.PgError):  # labeled anti-vertex
        pg.Plan(3, [(0, 1)], anti_edges=[(2, 0)], anti_vertex=[0, 0, 1], labels=[-1, -1, 2])


def test_large_clique_plans():
    """Cliques of 9..16 vertices compile to the clique's total order (no
    level program): |Aut| = k!, k - 1 order pairs, the k-clique kernel."""
    import math
    pg = _pg()
    for k in (9, 12, 14, 16):
        p = pg.Plan(k, sg.clique_edges(k), vertex_induced=(k % 2 == 0))
        info = p.info()
        assert info.k == k and info.n_regular == k
        assert info.automorphisms == math.factorial(k)
        assert info.n_po == k - 1
        assert [(info.po[2 * i], info.po[2 * i + 1]) for i in range(k - 1)] == [(i, i + 1) for i in range(k - 1)]
        assert info.kernel == pg.KERNEL_CLIQUE and info.n_orders == 0
        assert "k-clique kernel" in p.describe()


def test_every_generated_pattern_plans_match_oracle():
    """The counting and listing programs of every connected pattern the
    generators produce (21 induced 5-vertex, 112 induced 6-vertex, and all
    edge-induced ones with up to 5 edges) count what the oracle counts."""
    pg = _pg()
    pats = (pg.generate_all(5) + pg.generate_all(6)
            + [p for e in range(1, 6) for p in pg.generate_all(e, vertex_induced=False)])
    graphs = [sg.erdos_renyi(13, 0.45, 701), sg.chung_lu(24, 70, 2.1, 9.0, 702)]
    for g in graphs:
        for p in pats:
            want = oracle.count(g, p)
            got, _ = planeval.count(g, p)
            assert got == want, (p, g.n)
            got, _ = planeval.count(g, p, listing=True)
            assert got == want, (p, g.n, "listing")


def _ranked_out_degrees(g):
    """Out-degree d+(r) of every degree rank r (rank = position in
    (degree desc, id asc); out-neighbours = neighbours of smaller rank), and
    the rank of every original vertex."""
    deg = np.diff(g.offsets)
    order = sorted(range(g.n), key=lambda v: (-deg[v], v))
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    dout = np.zeros(g.n, dtype=np.int64)
    for v in range(g.n):
        nb = rank[g.adj[g.offsets[v]:g.offsets[v + 1]]]
        dout[rank[v]] = int((nb < rank[v]).sum())
    return dout, rank


@pytest.mark.parametrize("seed", [7, 8])
def test_operand_elements_closed_forms(seed):
    """The operand counter of the plan walk (the numerator of the set-operation
    roofline) against closed forms.  Triangles: level 1 reads N+(v); level 2
    reads N+(v) cut below u and N+(u) for every u in N+(v), so the elements
    are sum d+(v) + sum C(d+(v), 2) + sum_v sum_{u in N+(v)} d+(u), and the
    operations n + m.  The 3-star reads adj(v) once per start vertex."""
    g = sg.chung_lu(300, 1500, 2.2, 40.0, seed)
    dout, rank = _ranked_out_degrees(g)
    second = 0
    for v in range(g.n):
        nb = rank[g.adj[g.offsets[v]:g.offsets[v + 1]]]
        second += int(dout[nb[nb < rank[v]]].sum())
    want = int(dout.sum() + (dout * (dout - 1) // 2).sum()) + second
    assert planeval.operand_elems(g, sg.pattern(3, sg.clique_edges(3))) == (want, g.n + g.m)
    assert planeval.operand_elems(g, sg.pattern(3, sg.star_edges(3))) == (2 * g.m, g.n)
