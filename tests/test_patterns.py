"""Pattern generators (Section 3.1 pattern interface: generateAllVertexInduced,
generateAllEdgeInduced, extendByVertex, extendByEdge), host only.  Pinned by
the numbers of connected graphs up to isomorphism (by vertices: 1, 1, 2, 6,
21, 112, 853; by edges: 1, 1, 3, 5, 12, 30, 79) and by networkx isomorphism
tests."""
import itertools

import networkx as nx
import pytest

import synthgraph as sg

BY_VERTICES = [1, 1, 2, 6, 21, 112, 853]
BY_EDGES = [1, 1, 3, 5, 12, 30, 79]


@pytest.fixture(scope="module")
def pg():
    import paper_2004_02369_b300 as pg
    return pg


def _nx(p):
    G = nx.Graph()
    G.add_nodes_from(range(p["k"]))
    G.add_edges_from(p["edges"])
    return G


def _classes(pats):
    """Isomorphism classes as a list of representatives (networkx)."""
    reps = []
    for p in pats:
        G = _nx(p)
        if not any(nx.is_isomorphic(G, R) for R in reps):
            reps.append(G)
    return reps


def test_connected_graph_counts(pg):
    for k, want in enumerate(BY_VERTICES, start=1):
        pats = pg.generate_all(k, vertex_induced=True)
        assert len(pats) == want, k
        assert all(p["k"] == k and p["vertex_induced"] for p in pats)
    for e, want in enumerate(BY_EDGES, start=1):
        pats = pg.generate_all(e, vertex_induced=False)
        assert len(pats) == want, e
        assert all(len(p["edges"]) == e and not p["vertex_induced"] for p in pats)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_generated_patterns_connected_and_distinct(pg, k):
    pats = pg.generate_all(k)
    assert all(nx.is_connected(_nx(p)) for p in pats)
    assert len(_classes(pats)) == len(pats)


def test_extend_by_vertex_and_edge(pg):
    four = pg.generate_all(4)
    five = pg.extend(four, by_vertex=True)
    assert len(five) == 21 and len(_classes(five + pg.generate_all(5))) == 21
    three_edges = pg.generate_all(3, vertex_induced=False)
    assert len(pg.extend(three_edges, by_vertex=False)) == 5
    # a triangle grows only a pendant edge: the tailed triangle
    got = pg.extend([sg.pattern(3, sg.clique_edges(3))], by_vertex=False)
    assert len(got) == 1 and nx.is_isomorphic(_nx(got[0]), _nx(sg.pattern(4, sg.TAILED_TRIANGLE)))
    # extendByVertex of a single edge: wedge and triangle
    got = pg.extend([sg.pattern(2, [(0, 1)])], by_vertex=True)
    assert sorted(len(p["edges"]) for p in got) == [2, 3]
    # isomorphic inputs are merged before extending
    assert len(pg.extend([sg.pattern(3, [(0, 1), (1, 2)]), sg.pattern(3, [(0, 2), (2, 1)])], by_vertex=False)) == \
        len(pg.extend([sg.pattern(3, [(0, 1), (1, 2)])], by_vertex=False))


def test_generator_arguments_checked(pg):
    for bad in [(0, True), (8, True), (0, False), (8, False)]:
        with pytest.raises(pg.PgError):
            pg.generate_all(*bad)
    with pytest.raises(pg.PgError):
        pg.extend([sg.pattern(3, sg.chain_edges(3), labels=[1, 1, 1])], by_vertex=True)


def test_extension_chains_reach_every_size(pg):
    """extendByEdge of all e-edge patterns gives all (e+1)-edge patterns;
    extendByVertex of all k-vertex patterns gives all (k+1)-vertex ones."""
    for e in range(1, 6):
        ext = pg.extend(pg.generate_all(e, vertex_induced=False), by_vertex=False)
        assert len(ext) == BY_EDGES[e]
        assert len(_classes(ext + pg.generate_all(e + 1, vertex_induced=False))) == BY_EDGES[e]
    for k in range(1, 6):
        assert len(pg.extend(pg.generate_all(k), by_vertex=True)) == BY_VERTICES[k]
