"""GPU parity for match listing (pg_match / pg_match_range) and anti-vertex
counting: the CUDA path against the oracle.

Listing output is compared on what is unique: the set of distinct matches.
Each listed row is reduced to its class under Aut(p) (the oracle's
canonical_matches), and the set of classes must equal the oracle's
match_keys exactly, with no class listed twice.  Which member of a class a
row shows is free (it is the one the symmetry-breaking order keeps)."""
import ctypes

import numpy as np
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _graphs():
    g1 = sg.erdos_renyi(40, 0.2, 201)
    g2 = sg.chung_lu(400, 1600, 2.1, 60.0, 202)
    g3 = sg.rmat(8, 6, 0.57, 0.19, 0.19, 203)
    g4 = sg.erdos_renyi(80, 0.1, 204)
    g4.labels = sg.uniform_labels(g4.n, 3, 205)
    return [g1, g2, g3, g4, sg.complete_graph(8)]


LIST_PATTERNS = ([sg.pattern(1, [])]
                 + [sg.pattern(k, sg.clique_edges(k)) for k in range(2, 6)]
                 + [sg.pattern(k, sg.star_edges(k)) for k in range(3, 6)]
                 + [sg.pattern(k, sg.chain_edges(k)) for k in range(3, 6)]
                 + [sg.pattern(4, sg.cycle_edges(4)), sg.pattern(4, sg.TAILED_TRIANGLE),
                    sg.pattern(4, sg.DIAMOND)]
                 + sg.motif4_patterns()
                 + [sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)]),
                    sg.pattern(5, sg.cycle_edges(5), vertex_induced=True)])

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


def _classes(rows, p):
    keys = oracle.canonical_matches(rows, p)
    return {tuple(r) for r in keys.tolist()}, keys.shape[0]


# Above this many oracle maps the per-class comparison (every map as a row,
# times |Aut| permutations) takes minutes; such cases compare the listed
# total with the oracle's count only.  Every pattern is still compared class
# by class on the smaller graphs.
MAX_ORACLE_MAPS = 400_000


def _check_listing(pg, g, G, p):
    plan = pg.Plan.from_dict(p)
    rows, n_total = pg.match(G, plan)
    maps = oracle.count_maps(g, p, threads=8)
    if maps > MAX_ORACLE_MAPS:
        assert maps % oracle.automorphisms(p) == 0
        assert n_total == rows.shape[0] == maps // oracle.automorphisms(p), p
        return
    rows = rows.cpu().numpy()
    want = oracle.match_keys(g, p)
    assert n_total == want.shape[0] == rows.shape[0], p
    got, n = _classes(rows, p)
    assert len(got) == n, ("a match listed twice", p)
    assert got == {tuple(r) for r in want.tolist()}, p


@pytest.mark.parametrize("gi", range(5))
def test_listing_equals_oracle(pg, gi):
    g = _graphs()[gi]
    G = pg.Graph.from_synth(g)
    pats = list(LIST_PATTERNS)
    if g.labels is not None:
        pats += [sg.pattern(3, sg.chain_edges(3), labels=[0, 1, -1]),
                 sg.pattern(3, sg.clique_edges(3), labels=[2, 2, -1]),
                 sg.pattern(2, [(0, 1)], labels=[1, -1])]
    for p in pats:
        _check_listing(pg, g, G, p)


@pytest.mark.parametrize("gi", range(5))
def test_anti_vertex_listing_equals_oracle(pg, gi):
    g = _graphs()[gi]
    G = pg.Graph.from_synth(g)
    for p in ANTI_VERTEX_PATTERNS:
        _check_listing(pg, g, G, p)


@pytest.mark.parametrize("gi", range(5))
def test_anti_vertex_counts_equal_oracle(pg, gi):
    g = _graphs()[gi]
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in ANTI_VERTEX_PATTERNS]
    got = pg.count(G, plans)
    want = [oracle.count(g, p) for p in ANTI_VERTEX_PATTERNS]
    assert got == want


def test_anti_vertex_counts_mid_size(pg):
    """Triangles in no 4-clique and p_e on a 20K-vertex power-law graph (many
    work tiles, hub lists through the hub bitmaps)."""
    g = sg.chung_lu(20000, 120000, 2.1, 1500.0, 206)
    G = pg.Graph.from_synth(g)
    for p in ANTI_VERTEX_PATTERNS[:3]:
        assert pg.count(G, [pg.Plan.from_dict(p)]) == [oracle.count(g, p, threads=8)], p


def test_anti_vertex_refused_by_batch(pg):
    plan = pg.Plan.from_dict(ANTI_VERTEX_PATTERNS[0])
    with pytest.raises(pg.PgError) as e:
        pg.Batch([plan])
    assert e.value.code == pg.PG_EUNSUPPORTED


def test_truncated_listing(pg):
    """capacity < total: PG_ETRUNC semantics (total exact, rows valid and distinct)."""
    import torch
    g = _graphs()[1]
    G = pg.Graph.from_synth(g)
    p = sg.pattern(4, sg.TAILED_TRIANGLE)
    plan = pg.Plan.from_dict(p)
    want = {tuple(r) for r in oracle.match_keys(g, p).tolist()}
    cap = len(want) // 3
    out = torch.full((cap, 4), -7, dtype=torch.int32, device="cuda")
    rows, n_total = pg.match(G, plan, out=out)
    assert n_total == len(want)
    assert rows.shape[0] == cap
    got, n = _classes(rows.cpu().numpy(), p)
    assert len(got) == n == cap and got <= want
    # capacity 0 only counts
    total = ctypes.c_uint64()
    rc = pg.lib().pg_match(G.handle, plan.handle, None, 0, ctypes.byref(total), None)
    assert rc == pg.PG_ETRUNC and total.value == len(want)


def test_paged_listing_partitions_matches(pg):
    """pg_match_range over a partition of the start ranks lists every match
    exactly once."""
    g = _graphs()[2]
    G = pg.Graph.from_synth(g)
    for p in [sg.pattern(4, sg.cycle_edges(4)), sg.pattern(4, sg.star_edges(4), vertex_induced=True)]:
        plan = pg.Plan.from_dict(p)
        cuts = [0, 1, 7, g.n // 3, g.n // 2, g.n]
        seen = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            rows, n = pg.match(G, plan, rank_range=(a, b))
            seen += [tuple(r) for r in oracle.canonical_matches(rows.cpu().numpy(), p).tolist()]
        want = {tuple(r) for r in oracle.match_keys(g, p).tolist()}
        assert len(seen) == len(set(seen)) == len(want)
        assert set(seen) == want


def test_listing_edge_cases(pg):
    # no match: triangles of a tree (a path), and a graph without edges
    g = sg.from_edges(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)])
    G = pg.Graph.from_synth(g)
    rows, n = pg.match(G, pg.Plan(3, sg.clique_edges(3)))
    assert n == 0 and rows.shape == (0, 3)
    g0 = sg.from_edges(5, [])
    G0 = pg.Graph.from_synth(g0)
    rows, n = pg.match(G0, pg.Plan(1, []))
    assert n == 5 and sorted(rows.cpu().numpy()[:, 0].tolist()) == list(range(5))
    rows, n = pg.match(G0, pg.Plan(2, [(0, 1)]))
    assert n == 0
    # isolated vertices = single vertex with an anti-vertex
    rows, n = pg.match(G0, pg.Plan(2, [], anti_edges=[(0, 1)], anti_vertex=[0, 1]))
    assert n == 5 and (rows.cpu().numpy()[:, 1] == -1).all()
    with pytest.raises(pg.PgError):
        pg.match(G, pg.Plan(3, sg.clique_edges(3)), rank_range=(0, g.n + 1))


def test_listing_at_scale_properties(pg):
    """4-cliques on a 100K-vertex power-law graph (about 6.2M of them):
    n_total equals the count, every row is a 4-clique of distinct vertices,
    and no clique repeats."""
    g = sg.chung_lu(100000, 600000, 2.1, 2500.0, 207)
    G = pg.Graph.from_synth(g)
    plan = pg.Plan(4, sg.clique_edges(4))
    want = pg.count(G, [plan])[0]
    assert want == oracle.kcliques(g, 4, threads=8)
    rows, n = pg.match(G, plan)
    assert n == want
    r = np.sort(rows.cpu().numpy().astype(np.int64), axis=1)
    assert (np.diff(r, axis=1) > 0).all()
    # adjacency of every pair via a sorted edge-key table
    deg = np.diff(g.offsets)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    ekeys = src * g.n + g.adj.astype(np.int64)
    for i in range(4):
        for j in range(i + 1, 4):
            q = r[:, i] * g.n + r[:, j]
            pos = np.searchsorted(ekeys, q)
            assert (ekeys[np.minimum(pos, ekeys.size - 1)] == q).all()
    srt = r[np.lexsort(r.T[::-1])]
    assert not (np.diff(srt, axis=0) == 0).all(axis=1).any()
