"""Pins for the CPU oracle against things other than itself: closed forms,
an independent library (networkx subgraph matching), identities the paper
states, and brute force on tiny graphs.  CPU only."""
import itertools
import json
import os
from math import comb, factorial

import networkx as nx
import numpy as np
import pytest
from networkx.algorithms import isomorphism as iso

import oracle
import synthgraph as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_nx(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u, v in g.edges():
        G.add_edge(int(u), int(v))
    if g.labels is not None:
        for v in range(g.n):
            G.nodes[v]["label"] = int(g.labels[v])
    return G


def pat_nx(p):
    P = nx.Graph()
    P.add_nodes_from(range(p["k"]))
    P.add_edges_from(p["edges"])
    if p.get("labels") is not None:
        for u, l in enumerate(p["labels"]):
            P.nodes[u]["label"] = l
    return P


def _node_match(gattr, pattr):
    pl = pattr.get("label", -1)
    return pl < 0 or gattr.get("label") == pl


def nx_maps(G, P, induced):
    """Injective maps P -> G (networkx VF2), induced or not."""
    gm = iso.GraphMatcher(G, P, node_match=_node_match)
    it = gm.subgraph_isomorphisms_iter() if induced else gm.subgraph_monomorphisms_iter()
    return sum(1 for _ in it)


def nx_aut(P):
    gm = iso.GraphMatcher(P, P, node_match=lambda a, b: a.get("label", -1) == b.get("label", -1))
    return sum(1 for _ in gm.isomorphisms_iter())


def small_graphs():
    out = [sg.erdos_renyi(14, 0.35, 11), sg.erdos_renyi(20, 0.2, 12),
           sg.chung_lu(40, 90, 2.1, 12.0, 13), sg.rmat(5, 4, 0.57, 0.19, 0.19, 14),
           sg.complete_graph(7)]
    g = sg.erdos_renyi(18, 0.3, 15)
    g.labels = sg.uniform_labels(g.n, 3, 16)
    out.append(g)
    return out


SHAPES4 = [sg.chain_edges(4), sg.star_edges(4), sg.cycle_edges(4), sg.TAILED_TRIANGLE,
           sg.DIAMOND, sg.clique_edges(4)]
SHAPES = ([sg.chain_edges(2), sg.chain_edges(3), sg.clique_edges(3)] + SHAPES4
          + [sg.cycle_edges(5), sg.clique_edges(5), sg.star_edges(5), sg.chain_edges(5)])


# ---------------------------------------------------------------- |Aut| ----

@pytest.mark.parametrize("edges", SHAPES)
def test_aut_matches_networkx(edges):
    k = max(max(e) for e in edges) + 1
    p = sg.pattern(k, edges)
    assert oracle.automorphisms(p) == nx_aut(pat_nx(p))


def test_aut_closed_forms():
    for k in range(2, 8):
        assert oracle.automorphisms(sg.pattern(k, sg.clique_edges(k))) == factorial(k)
        if k >= 3:
            assert oracle.automorphisms(sg.pattern(k, sg.star_edges(k))) == factorial(k - 1)
    for k in range(3, 9):
        assert oracle.automorphisms(sg.pattern(k, sg.cycle_edges(k))) == 2 * k


def test_aut_labeled_matches_networkx():
    rng = np.random.default_rng(5)
    for edges in SHAPES4:
        for _ in range(4):
            labels = [int(x) for x in rng.integers(0, 2, 4)]
            p = sg.pattern(4, edges, labels=labels)
            assert oracle.automorphisms(p) == nx_aut(pat_nx(p))


def test_star4_aut_paper_fact():
    fact = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))["star4_automorphisms"]
    p = sg.pattern(fact["pattern"]["k"], fact["pattern"]["edges"])
    assert oracle.automorphisms(p) == fact["value"]


def test_pe_anti_vertex_automorphisms_paper_fact():
    f = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))["p_e_anti_vertex_symmetry"]
    pp = f["pattern"]
    p = sg.pattern(pp["k"], pp["edges"], pp["anti_edges"], anti_vertex=pp["anti_vertex"])
    assert oracle.automorphisms(p) == f["automorphisms_regular"]


# ------------------------------------------------------------- counting ----

@pytest.mark.parametrize("gi", range(6))
@pytest.mark.parametrize("edges", SHAPES)
def test_count_matches_networkx(gi, edges):
    g = small_graphs()[gi]
    k = max(max(e) for e in edges) + 1
    G = to_nx(g)
    for induced in (False, True):
        p = sg.pattern(k, edges, vertex_induced=induced)
        maps = oracle.count_maps(g, p, threads=2)
        assert maps == nx_maps(G, pat_nx(p), induced)
        assert oracle.count(g, p) * oracle.automorphisms(p) == maps


def test_count_labeled_matches_networkx():
    g = small_graphs()[5]
    G = to_nx(g)
    rng = np.random.default_rng(7)
    for edges in SHAPES4 + [sg.clique_edges(3)]:
        k = max(max(e) for e in edges) + 1
        for _ in range(3):
            labels = [int(x) if x < 3 else -1 for x in rng.integers(0, 4, k)]
            for induced in (False, True):
                p = sg.pattern(k, edges, labels=labels, vertex_induced=induced)
                assert oracle.count_maps(g, p) == nx_maps(G, pat_nx(p), induced)


def test_complete_graph_closed_forms():
    n = 9
    g = sg.complete_graph(n)
    for edges in SHAPES:
        k = max(max(e) for e in edges) + 1
        p = sg.pattern(k, edges)
        aut = oracle.automorphisms(p)
        assert oracle.count(g, p) == comb(n, k) * factorial(k) // aut
        pi = sg.pattern(k, edges, vertex_induced=True)
        is_clique = len(edges) == k * (k - 1) // 2
        assert oracle.count(g, pi) == (comb(n, k) if is_clique else 0)


def test_triangles_trace_formula():
    for g in small_graphs() + [sg.workload_graph(1)]:
        A = np.zeros((g.n, g.n), dtype=np.int64)
        e = g.edges()
        A[e[:, 0], e[:, 1]] = 1
        A[e[:, 1], e[:, 0]] = 1
        tr = int(np.trace(A @ A @ A)) // 6
        assert oracle.triangles(g) == tr
        assert oracle.count(g, sg.pattern(3, sg.clique_edges(3), vertex_induced=True)) == tr


def test_wedges_and_stars_closed_forms():
    for g in small_graphs() + [sg.workload_graph(1)]:
        d = np.diff(g.offsets)
        T = oracle.triangles(g)
        wedge_ind = sum(comb(int(x), 2) for x in d) - 3 * T
        assert oracle.count(g, sg.pattern(3, sg.chain_edges(3), vertex_induced=True)) == wedge_ind
        for s in (3, 4, 5):
            star = sg.pattern(s, sg.star_edges(s))
            assert oracle.count(g, star) == sum(comb(int(x), s - 1) for x in d)


def test_vertex_induced_theorem():
    """Section 3.1.3: vertex-induced p == p plus anti-edges on all non-adjacent pairs."""
    for g in small_graphs():
        for edges in SHAPES4 + [sg.chain_edges(3)]:
            k = max(max(e) for e in edges) + 1
            es = {tuple(sorted(e)) for e in edges}
            anti = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in es]
            a = oracle.count_maps(g, sg.pattern(k, edges, vertex_induced=True))
            b = oracle.count_maps(g, sg.pattern(k, edges, anti_edges=anti))
            assert a == b


def test_anti_edge_inclusion_exclusion():
    """maps(p with anti-edge ab) = maps(p) - maps(p + edge ab), checked with networkx."""
    cases = [(sg.TAILED_TRIANGLE, [(3, 1)]), (sg.TAILED_TRIANGLE, [(3, 1), (3, 2)]),
             (sg.chain_edges(3), [(0, 2)]), (sg.cycle_edges(4), [(0, 2)]),
             (sg.star_edges(4), [(1, 2)])]
    for g in small_graphs()[:4]:
        G = to_nx(g)
        for edges, anti in cases:
            k = 4 if len(edges) > 2 and max(max(e) for e in edges) == 3 else 3
            p = sg.pattern(k, edges, anti_edges=anti)
            # inclusion-exclusion over the anti-edges, each term by networkx
            expect = 0
            for r in range(len(anti) + 1):
                for sub in itertools.combinations(anti, r):
                    expect += (-1) ** r * nx_maps(G, pat_nx(sg.pattern(k, list(edges) + list(sub))), False)
            assert oracle.count_maps(g, p) == expect


def test_anti_vertex_triangles_not_in_k4():
    """Triangle with an anti-vertex anti-adjacent to all three corners =
    triangles with no common neighbour of all three corners (p7 form)."""
    p = sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 1), (3, 2)],
                   anti_vertex=[0, 0, 0, 1])
    for g in small_graphs():
        G = to_nx(g)
        expect = 0
        for tri in (c for c in nx.enumerate_all_cliques(G) if len(c) == 3):
            a, b, c = tri
            common = set(G[a]) & set(G[b]) & set(G[c])
            expect += not common
        assert oracle.count(g, p) == expect


def test_anti_vertex_p_e():
    """p_e: triangle u1 u2 u3, anti-vertex u4 anti-adjacent to u1 and u3: pairs
    (u1,u3) on a triangle with apex u2 whose only common neighbour is u2."""
    p = sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 2)], anti_vertex=[0, 0, 0, 1])
    for g in small_graphs():
        G = to_nx(g)
        expect = 0
        for a, c in G.edges():
            common = set(G[a]) & set(G[c])
            if len(common) == 1:
                expect += 1  # the single common neighbour is the apex u2
        assert oracle.count(g, p) == expect


# ------------------------------------------------------------- listing -----

LISTING_PATTERNS = [
    sg.pattern(2, [(0, 1)]),
    sg.pattern(3, sg.clique_edges(3)),
    sg.pattern(3, sg.chain_edges(3)),
    sg.pattern(4, sg.cycle_edges(4)),
    sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)]),
    sg.pattern(4, sg.star_edges(4), vertex_induced=True),
    sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 2)], anti_vertex=[0, 0, 0, 1]),
]


def test_automorphism_perms_agree_with_c():
    """The Python permutation list and the C |Aut| are written separately."""
    for p in LISTING_PATTERNS + [sg.pattern(5, sg.star_edges(5)), sg.pattern(5, sg.clique_edges(5)),
                                 sg.pattern(3, sg.chain_edges(3), labels=[1, -1, 1])]:
        perms = oracle.automorphism_perms(p)
        av = p.get("anti_vertex") or [0] * p["k"]
        restricted = {tuple(s[u] if not av[u] else -1 for u in range(p["k"])) for s in perms.tolist()}
        assert len(restricted) == oracle.automorphisms(p), p


def test_match_keys_one_per_match():
    """|distinct matches| = maps / |Aut| for every listed pattern."""
    for g in small_graphs()[:4]:
        for p in LISTING_PATTERNS:
            keys = oracle.match_keys(g, p)
            assert keys.shape[0] == oracle.count(g, p), p
            assert len({tuple(r) for r in keys.tolist()}) == keys.shape[0]


def test_match_keys_brute_force_sets():
    """Edges, triangles, p_e and a labeled edge listed by plain loops."""
    for g in small_graphs()[:4]:
        G = to_nx(g)
        edges = {(min(a, b), max(a, b)) for a, b in G.edges()}
        got = {tuple(r) for r in oracle.match_keys(g, LISTING_PATTERNS[0]).tolist()}
        assert got == edges
        tris = {t for t in itertools.combinations(range(g.n), 3)
                if G.has_edge(t[0], t[1]) and G.has_edge(t[0], t[2]) and G.has_edge(t[1], t[2])}
        got = {tuple(r) for r in oracle.match_keys(g, LISTING_PATTERNS[1]).tolist()}
        assert got == tris
        # p_e: the class of (a, b, c) under the swap of u1, u3 is keyed (min(a,c), b, max(a,c))
        pe = set()
        for a, c in edges:
            common = set(G[a]) & set(G[c])
            if len(common) == 1:
                pe.add((a, common.pop(), c, -1))
        got = {tuple(r) for r in oracle.match_keys(g, LISTING_PATTERNS[6]).tolist()}
        assert got == pe
    g = small_graphs()[0]
    g.labels = sg.uniform_labels(g.n, 3, 77)
    G = to_nx(g)
    p = sg.pattern(2, [(0, 1)], labels=[1, -1])  # no symmetry: one match per (a, b)
    want = {(a, b) for a in range(g.n) for b in G[a] if g.labels[a] == 1}
    assert {tuple(r) for r in oracle.match_keys(g, p).tolist()} == want


# ------------------------------------------------------------- cliques -----

def test_kcliques_complete_graph():
    g = sg.complete_graph(11)
    for k in range(1, 8):
        assert oracle.kcliques(g, k) == comb(11, k)


def test_kcliques_match_networkx_and_bruteforce():
    for g in small_graphs() + [sg.chung_lu(300, 1500, 2.1, 60.0, 21)]:
        G = to_nx(g)
        by_size = {}
        for c in nx.enumerate_all_cliques(G):
            by_size[len(c)] = by_size.get(len(c), 0) + 1
        for k in range(3, 7):
            assert oracle.kcliques(g, k) == by_size.get(k, 0)
        for k in (3, 4):
            assert oracle.count(g, sg.pattern(k, sg.clique_edges(k))) == by_size.get(k, 0)


def test_kcliques_sources_partition():
    g = sg.chung_lu(500, 3000, 2.1, 80.0, 22)
    total = oracle.kcliques(g, 4)
    half = np.arange(0, g.n, 2)
    other = np.arange(1, g.n, 2)
    assert oracle.kcliques(g, 4, sources=half) + oracle.kcliques(g, 4, sources=other) == total


# ------------------------------------------------------------- 4-motifs ----

def test_motif4_linear_system_matches_networkx():
    for g in small_graphs():
        G = to_nx(g)
        ind = oracle.motif4_induced(g)
        non = oracle.motif4_noninduced(g)
        for name, edges in sg.MOTIF4_SHAPES.items():
            P = pat_nx(sg.pattern(4, edges))
            aut = nx_aut(P)
            assert ind[name] == nx_maps(G, P, True) // aut, name
            assert non[name] == nx_maps(G, P, False) // aut, name


def test_motif4_linear_system_matches_bruteforce_rmat():
    g = sg.rmat(9, 8, 0.57, 0.19, 0.19, 23)
    ind = oracle.motif4_induced(g)
    for name, edges in sg.MOTIF4_SHAPES.items():
        assert ind[name] == oracle.count(g, sg.pattern(4, edges, vertex_induced=True)), name


# ------------------------------------------------------------- MNI ---------

def nx_domains(G, P):
    gm = iso.GraphMatcher(G, P, node_match=_node_match)
    dom = {u: set() for u in P.nodes}
    for m in gm.subgraph_monomorphisms_iter():
        for gv, pu in m.items():
            dom[pu].add(gv)
    return [len(dom[u]) for u in sorted(P.nodes)]


def test_mni_hand_example():
    # path 0-1-2-3 plus triangle 3-4-5; wedge pattern (centre 0)
    g = sg.from_edges(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (3, 5)])
    wedge = sg.pattern(3, sg.star_edges(3))
    # centres: every vertex with degree >= 2 -> {1,2,3,4,5}; leaves: all 6
    assert oracle.mni_domains_bruteforce(g, wedge) == [5, 6, 6]
    tri = sg.pattern(3, sg.clique_edges(3))
    assert oracle.mni_domains_bruteforce(g, tri) == [3, 3, 3]


def test_mni_matches_networkx_and_is_antimonotone():
    g = small_graphs()[5]
    G = to_nx(g)
    rng = np.random.default_rng(9)
    for _ in range(6):
        la = [int(x) for x in rng.integers(0, 3, 4)]
        sub = {}
        for name, edges, k in [("edge", [(0, 1)], 2), ("wedge", sg.chain_edges(3), 3),
                               ("path3", sg.chain_edges(4), 4), ("star3", sg.star_edges(4), 4),
                               ("triangle", sg.clique_edges(3), 3)]:
            p = sg.pattern(k, edges, labels=la[:k])
            d = oracle.mni_domains_bruteforce(g, p)
            assert d == nx_domains(G, pat_nx(p))
            sub[name] = min(d)
        # anti-monotone: a pattern's support never exceeds a sub-pattern's
        assert sub["wedge"] <= sub["edge"]
        assert sub["path3"] <= sub["wedge"] and sub["star3"] <= sub["wedge"]
        assert sub["triangle"] <= sub["wedge"]


# ------------------------------------------------------------- FSM ---------

def test_fsm_supports_match_bruteforce_mni():
    """Every labeled pattern with 1..3 edges on small labeled graphs: the
    per-vertex domain search agrees with brute-force MNI (all maps)."""
    for seed, n, p, nl in [(31, 40, 0.12, 3), (32, 30, 0.2, 2), (33, 50, 0.08, 4)]:
        g = sg.erdos_renyi(n, p, seed)
        g.labels = sg.uniform_labels(g.n, nl, seed + 1)
        sup = oracle.fsm_supports(g, nl)
        for (shape, labels), s in sup.items():
            d = oracle.mni_domains_bruteforce(g, oracle.fsm_pattern(shape, labels))
            assert s == min(d), (shape, labels, s, d)


def test_fsm_hub_and_corner_cases():
    # a star centre with exactly one neighbour per label, a triangle and a
    # path whose two ends would have to be the same vertex
    g = sg.from_edges(7, [(0, 1), (0, 2), (0, 3), (1, 2), (3, 4), (4, 5), (5, 3), (5, 6)])
    g.labels = np.array([0, 1, 1, 2, 0, 1, 2], dtype=np.int32)
    sup = oracle.fsm_supports(g, 3)
    for (shape, labels), s in sup.items():
        d = oracle.mni_domains_bruteforce(g, oracle.fsm_pattern(shape, labels))
        assert s == min(d), (shape, labels)
    assert sup[("edge", (0, 1))] == min(2, 3)


def test_fsm_antimonotone():
    g = sg.chung_lu(300, 1200, 2.3, 40.0, 34)
    g.labels = sg.zipf_labels(g.n, 4, 1.2, 35)
    sup = oracle.fsm_supports(g, 4)
    for (shape, labels), s in sup.items():
        if shape == "wedge":
            c, x, y = labels
            assert s <= sup[("edge", tuple(sorted((c, x))))] and s <= sup[("edge", tuple(sorted((c, y))))]
        if shape == "star":
            c, x, y, z = labels
            for a, b in ((x, y), (x, z), (y, z)):
                assert s <= sup[("wedge", (c, min(a, b), max(a, b)))]
        if shape == "triangle":
            x, y, z = labels
            assert s <= sup[("wedge", (x, min(y, z), max(y, z)))]
        if shape == "path":
            a, b, c, d = labels
            assert s <= sup[("wedge", (b, min(a, c), max(a, c)))]
            assert s <= sup[("wedge", (c, min(b, d), max(b, d)))]


# ---------------------------------------- MNI domains, vertex by vertex ----
#
# oracle.domain_sizes decides v in D(u) by backtracking from u -> v until the
# first valid map: the definition of a domain (Section 2.1, MNI over all
# isomorphisms) with no label-count shortcut.  It is pinned by networkx and
# by enumerating every map, and it in turn checks the table-based FSM oracle
# (oracle.fsm_supports), whose leaf positions are decided from label counts.

DOMAIN_PATTERNS = [
    sg.pattern(2, [(0, 1)]),
    sg.pattern(3, sg.chain_edges(3)),
    sg.pattern(3, sg.clique_edges(3)),
    sg.pattern(4, sg.chain_edges(4)),
    sg.pattern(4, sg.star_edges(4)),
    sg.pattern(4, sg.cycle_edges(4)),
    sg.pattern(5, sg.chain_edges(5)),                       # 4 edges
    sg.pattern(5, [(0, 1), (0, 2), (0, 3), (3, 4)]),        # chair, 4 edges
    sg.pattern(4, [(0, 1), (1, 2), (0, 2), (2, 3)]),        # tailed triangle
    sg.pattern(4, sg.chain_edges(4), anti_edges=[(0, 3)]),
    sg.pattern(4, sg.cycle_edges(4), vertex_induced=True),
]


def _labelled_variants(p, rng, nl):
    out = [p]
    for _ in range(2):
        out.append(dict(p, labels=[int(x) for x in rng.integers(-1, nl, p["k"])]))
    return out


def test_domain_sizes_match_networkx_and_enumeration():
    rng = np.random.default_rng(61)
    graphs = [sg.erdos_renyi(16, 0.3, 62), sg.chung_lu(40, 100, 2.1, 14.0, 63), sg.from_edges(
        9, [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (1, 2), (3, 4), (5, 6), (6, 7), (7, 8), (8, 5)])]
    for gi, g in enumerate(graphs):
        g.labels = sg.uniform_labels(g.n, 3, 64 + gi)
        G = to_nx(g)
        for base in DOMAIN_PATTERNS:
            for p in _labelled_variants(base, rng, 3):
                d = oracle.domain_sizes(g, p)
                assert d == oracle.mni_domains_bruteforce(g, p), (gi, p)
                if not p["anti_edges"] and not p["vertex_induced"]:
                    assert d == nx_domains(G, pat_nx(p)), (gi, p)
                for u in range(p["k"]):  # single-vertex form agrees with the sizes
                    assert sum(oracle.domain_member(g, p, u, v) for v in range(g.n)) == d[u]


def _check_tables(g, nl, keys=None):
    sup = oracle.fsm_supports(g, nl)
    for key in (keys if keys is not None else sup):
        shape, labels = key
        want = oracle.mni_support(g, oracle.fsm_pattern(shape, labels))
        assert sup[key] == want, (key, sup[key], want)
    return sup


def test_fsm_tables_match_domain_search_dense_tiny_graphs():
    """Dense tiny graphs with 2-3 labels, every labeled pattern with 1..3
    edges: labels that occur exactly once, twice or three times next to an
    already used vertex (the cases the tables handle by subtraction and by
    coincidence tests) occur throughout."""
    rng = np.random.default_rng(65)
    for i in range(60):
        n = int(rng.integers(5, 12))
        g = sg.erdos_renyi(n, float(rng.uniform(0.35, 0.8)), 660 + i)
        nl = int(rng.integers(2, 4))
        g.labels = sg.uniform_labels(g.n, nl, 760 + i)
        _check_tables(g, nl)


@pytest.mark.parametrize("n,m,gamma,w,seed", [(2000, 12000, 2.1, 400.0, 67), (5000, 30000, 2.3, 700.0, 68)])
def test_fsm_tables_match_domain_search_hub_graphs(n, m, gamma, w, seed):
    """Chung-Lu graphs with hubs and 20 Zipf(1.2) labels (the FSM workload's
    label law): every edge, wedge and triangle, and 400 sampled paths and
    stars (supported ones and unsupported ones), against the domain search."""
    g = sg.chung_lu(n, m, gamma, w, seed)
    g.labels = sg.zipf_labels(g.n, 20, 1.2, seed + 1)
    sup = oracle.fsm_supports(g, 20)
    rng = np.random.default_rng(seed + 2)
    keys = [k for k in sup if k[0] in ("edge", "wedge", "triangle")]
    for shape in ("path", "star"):
        pos = [k for k in sup if k[0] == shape and sup[k] > 0]
        zero = [k for k in sup if k[0] == shape and sup[k] == 0]
        for pool, take in ((pos, 300), (zero, 100)):
            idx = rng.choice(len(pool), min(take, len(pool)), replace=False)
            keys += [pool[i] for i in idx]
    assert max(sup[k] for k in keys) > 50  # hubs make large domains
    _check_tables(g, 20, keys)


def test_fsm_label_count_corner_cases_by_hand():
    """Hand-built cases where a leaf label occurs exactly 1, 2 or 3 times
    next to an already used vertex; expected supports derived by hand."""
    def sup(n, edges, labels, shape, key):
        g = sg.from_edges(n, edges)
        g.labels = np.array(labels, dtype=np.int32)
        tables = _check_tables(g, max(labels) + 1)
        p = oracle.fsm_pattern(shape, key)
        assert oracle.mni_support(g, p) == min(oracle.mni_domains_bruteforce(g, p))
        return tables[(shape, key)]
    # wedge leaf: the only label-1 neighbour of the centre is v itself
    assert sup(3, [(0, 1), (1, 2)], [1, 0, 2], "wedge", (0, 1, 1)) == 0
    assert sup(4, [(0, 1), (1, 2), (1, 3)], [1, 0, 2, 1], "wedge", (0, 1, 1)) == 1
    # star leaf: two label-1 neighbours of the centre (one is v) vs three
    assert sup(4, [(0, 1), (0, 2), (0, 3)], [0, 1, 1, 2], "star", (0, 1, 1, 1)) == 0
    assert sup(5, [(0, 1), (0, 2), (0, 3), (0, 4)], [0, 1, 1, 2, 1], "star", (0, 1, 1, 1)) == 1
    assert sup(4, [(0, 1), (0, 2), (0, 3)], [0, 1, 1, 2], "star", (0, 1, 1, 2)) == 1
    # path end: the only label-1 neighbour of u other than w is v (triangle)
    assert sup(3, [(0, 1), (1, 2), (0, 2)], [1, 0, 0], "path", (0, 0, 1, 1)) == 0
    assert sup(4, [(0, 1), (1, 2), (0, 2), (2, 3)], [1, 0, 0, 1], "path", (1, 0, 0, 1)) == 2
    # path inner: the single a' next to v and the single d' next to w coincide
    assert sup(3, [(0, 1), (0, 2), (1, 2)], [0, 0, 2], "path", (2, 0, 0, 2)) == 0
    assert sup(4, [(0, 1), (0, 2), (1, 2), (1, 3)], [0, 0, 2, 2], "path", (2, 0, 0, 2)) == 2


def test_fsm_full_size_two_oracles_agree():
    """FSM workload at full size (Chung-Lu 500K / 5M, Zipf labels over 20,
    threshold 1000): the stored supports of the per-vertex domain search
    (seeded sample over all five shapes, frequent and infrequent candidates)
    equal the table oracle's stored frequent set: equal supports where
    frequent, below the threshold and absent where not."""
    data = json.load(open(os.path.join(GOLDEN, "workload_counts.json")))
    table = data["fsm"]["counts"]
    search = data["fsm_domains"]["counts"]
    shapes = {}
    for key, v in search.items():
        shape = key.split(":")[0]
        if key in table:
            assert int(table[key]) == int(v), key
            shapes[shape] = shapes.get(shape, 0) + 1
        else:
            assert int(v) < 1000, key
    assert set(shapes) == {"edge", "wedge", "triangle", "path", "star"}
    assert sum(shapes.values()) >= 2000 and len(search) - sum(shapes.values()) >= 1000


def test_labeled_counts_sum_to_unlabeled_closed_forms():
    """Summed over every label combination, labeled triangle and induced
    wedge counts give trace(A^3)/6 and sum C(d,2) - 3T: pins the oracle's
    label filtering, which the labeled 3-motif parity relies on."""
    g = sg.chung_lu(120, 500, 2.1, 25.0, 801)
    g.labels = sg.uniform_labels(g.n, 3, 802)
    tri = sum(oracle.count(g, sg.pattern(3, sg.clique_edges(3), labels=list(t)))
              for t in itertools.combinations_with_replacement(range(3), 3))
    assert tri == oracle.triangles(g)
    wedges = sum(oracle.count(g, sg.pattern(3, [(0, 1), (1, 2)], labels=[x, c, y], vertex_induced=True))
                 for c in range(3) for x, y in itertools.combinations_with_replacement(range(3), 2))
    d = np.diff(g.offsets)
    assert wedges == int(sum(comb(int(x), 2) for x in d)) - 3 * oracle.triangles(g)
