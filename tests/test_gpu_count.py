"""GPU parity: counts from the CUDA path (through the C-ABI) against the
oracle, bit-exact, plus graph-residency checks and edge cases."""
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


def _graphs():
    g1 = sg.erdos_renyi(30, 0.25, 101)
    g2 = sg.chung_lu(300, 1500, 2.1, 60.0, 102)
    g3 = sg.rmat(8, 8, 0.57, 0.19, 0.19, 103)
    g4 = sg.erdos_renyi(60, 0.15, 104)
    g4.labels = sg.uniform_labels(g4.n, 3, 105)
    return [g1, g2, g3, g4, sg.complete_graph(9)]


PATTERNS = ([sg.pattern(k, sg.clique_edges(k)) for k in range(1, 6)]
            + [sg.pattern(k, sg.star_edges(k)) for k in range(3, 7)]
            + [sg.pattern(k, sg.chain_edges(k)) for k in range(2, 6)]
            + [sg.pattern(k, sg.cycle_edges(k)) for k in range(4, 6)]
            + [sg.pattern(4, sg.TAILED_TRIANGLE), sg.pattern(4, sg.DIAMOND)]
            + sg.motif3_patterns() + sg.motif4_patterns()
            + [sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)]),
               sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1), (3, 2)]),
               sg.pattern(5, sg.cycle_edges(5), vertex_induced=True),
               sg.pattern(5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4)], vertex_induced=True)])


def _is(p, edges):
    return sorted(tuple(sorted(e)) for e in p["edges"]) == sorted(tuple(sorted(e)) for e in edges)


def expected(g, p, brute_k_max):
    """Oracle count through the cheapest pinned route."""
    k = p["k"]
    plain = not p.get("anti_edges") and p.get("labels") is None
    if plain and k >= 3 and _is(p, sg.star_edges(k)) and not p["vertex_induced"]:
        return oracle.stars(g, k - 1)
    if plain and k >= 2 and _is(p, sg.clique_edges(k)):
        return oracle.kcliques(g, k)
    if plain and k == 4 and p["vertex_induced"]:
        for name, e in sg.MOTIF4_SHAPES.items():
            if _is(p, e):
                return oracle.motif4_induced(g)[name]
    if k > brute_k_max:
        return None
    return oracle.count(g, p)


@pytest.mark.parametrize("gi", range(5))
def test_counts_match_oracle(pg, gi):
    g = _graphs()[gi]
    brute_k_max = 4 if gi in (1, 2) else 8
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in PATTERNS]
    got = pg.count(G, plans)
    checked = 0
    for p, c in zip(PATTERNS, got):
        e = expected(g, p, brute_k_max)
        if e is not None:
            assert c == e, p
            checked += 1
    assert checked >= len(PATTERNS) - 6


def test_labeled_counts_match_oracle(pg):
    g = _graphs()[3]
    G = pg.Graph.from_synth(g)
    rng = np.random.default_rng(3)
    pats = []
    for edges, k in [(sg.chain_edges(3), 3), (sg.star_edges(4), 4), (sg.chain_edges(4), 4),
                     (sg.clique_edges(3), 3), (sg.TAILED_TRIANGLE, 4), (sg.cycle_edges(4), 4)]:
        for _ in range(3):
            labels = [int(x) if x < 3 else -1 for x in rng.integers(0, 4, k)]
            for vi in (False, True):
                pats.append(sg.pattern(k, edges, labels=labels, vertex_induced=vi))
    got = pg.count(G, [pg.Plan.from_dict(p) for p in pats])
    for p, c in zip(pats, got):
        assert c == oracle.count(g, p), p


def test_motif3_er2000_full(pg):
    """ER G(2000, 0.005): induced triangles and wedges, full size."""
    g = sg.workload_graph(1)
    G = pg.Graph.from_synth(g)
    tri, wedge = pg.count(G, [pg.Plan.from_dict(p) for p in sg.motif3_patterns()])
    assert tri == oracle.triangles(g)
    assert wedge == oracle.wedges_induced(g)
    assert tri == oracle.count(g, sg.motif3_patterns()[0])
    assert wedge == oracle.count(g, sg.motif3_patterns()[1])


def test_graph_residency(pg):
    g = sg.chung_lu(2000, 12000, 2.1, 300.0, 7)
    G = pg.Graph.from_synth(g)
    info = G.info()
    deg = np.diff(g.offsets)
    assert info.n == g.n and info.m == g.m and info.max_degree == deg.max()
    rank = G.rank()
    assert sorted(rank.tolist()) == list(range(g.n))
    # rank order = (degree desc, id asc)
    order = np.empty(g.n, dtype=np.int64)
    order[rank] = np.arange(g.n)
    key = [(-int(deg[v]), int(v)) for v in order]
    assert key == sorted(key)


def test_device_inputs_and_determinism(pg):
    import torch
    g = sg.rmat(10, 8, 0.57, 0.19, 0.19, 9)
    off = torch.from_numpy(g.offsets).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    G = pg.Graph(off, adj)
    plans = [pg.Plan.from_dict(p) for p in sg.motif4_patterns()]
    a = pg.count(G, plans)
    b = pg.count(G, plans)
    assert a == b
    assert a == [oracle.motif4_induced(g)[n] for n in sg.MOTIF4_SHAPES]


def test_count_async_into_torch(pg):
    import torch
    g = sg.erdos_renyi(200, 0.1, 11)
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan(3, sg.clique_edges(3)), pg.Plan(4, sg.clique_edges(4))]
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    pg.count_async(G, plans, out)
    torch.cuda.synchronize()
    assert pg.decode_counts(out) == [oracle.kcliques(g, 3), oracle.kcliques(g, 4)]


def test_128bit_counts(pg):
    """A 3000-leaf star holds C(3000, 7) > 2^64 seven-leaf stars."""
    n = 3001
    g = sg.from_edges(n, [(0, i) for i in range(1, n)])
    G = pg.Graph.from_synth(g)
    got = pg.count(G, [pg.Plan(8, sg.star_edges(8)), pg.Plan(3, sg.star_edges(3))])
    assert got == [comb(3000, 7), comb(3000, 2)]
    assert got[0] > 2 ** 64


def test_edge_cases(pg):
    # no edges
    g = sg.from_edges(5, [])
    G = pg.Graph.from_synth(g)
    assert pg.count(G, [pg.Plan(1, []), pg.Plan(2, [(0, 1)]), pg.Plan(3, sg.clique_edges(3))]) == [5, 0, 0]
    # empty graph
    g0 = sg.from_edges(0, [])
    G0 = pg.Graph.from_synth(g0)
    assert pg.count(G0, [pg.Plan(3, sg.clique_edges(3))]) == [0]
    # single edge
    G1 = pg.Graph.from_synth(sg.from_edges(2, [(0, 1)]))
    assert pg.count(G1, [pg.Plan(2, [(0, 1)]), pg.Plan(3, sg.chain_edges(3))]) == [1, 0]


def test_invalid_csr_rejected(pg):
    off = np.array([0, 1, 1], dtype=np.int64)
    adj = np.array([1], dtype=np.int32)  # 0->1 without 1->0
    with pytest.raises(pg.PgError) as e:
        pg.Graph(off, adj)
    assert e.value.code == pg.PG_EINVAL
    off = np.array([0, 0, 1], dtype=np.int64)
    adj = np.array([0], dtype=np.int32)  # 1->0 without 0->1 (a downward entry alone)
    with pytest.raises(pg.PgError) as e:
        pg.Graph(off, adj)
    assert e.value.code == pg.PG_EINVAL
    # a triangle with one direction of one edge missing, and one with a
    # reversed extra entry: the symmetric part is fine, one entry is not
    for off, adj in ((np.array([0, 2, 4, 5]), np.array([1, 2, 0, 2, 1])),
                     (np.array([0, 1, 3, 5]), np.array([1, 0, 2, 0, 1]))):
        with pytest.raises(pg.PgError) as e:
            pg.Graph(off.astype(np.int64), adj.astype(np.int32))
        assert e.value.code == pg.PG_EINVAL
    ok = pg.Graph(np.array([0, 2, 4, 6], dtype=np.int64), np.array([1, 2, 0, 2, 0, 1], dtype=np.int32))
    assert pg.count(ok, [pg.Plan(3, sg.clique_edges(3))]) == [1]
    off = np.array([0, 2, 3, 4], dtype=np.int64)
    adj = np.array([2, 1, 0, 0], dtype=np.int32)  # unsorted list of 0
    with pytest.raises(pg.PgError):
        pg.Graph(off, adj)
    off = np.array([0, 1, 2], dtype=np.int64)
    adj = np.array([0, 1], dtype=np.int32)  # self loops
    with pytest.raises(pg.PgError):
        pg.Graph(off, adj)
    with pytest.raises(pg.PgError):
        pg.count(pg.Graph.from_synth(sg.erdos_renyi(10, 0.5, 1)), [pg.Plan(2, [(0, 1)], labels=[0, 1])])


def test_batched_matches_generic_and_oracle(pg):
    import torch
    g = sg.rmat(9, 8, 0.57, 0.19, 0.19, 77)
    G = pg.Graph.from_synth(g)
    pats = sg.motif4_patterns() + sg.motif3_patterns() + [sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)]),
                                                          sg.pattern(4, sg.DIAMOND), sg.pattern(5, sg.cycle_edges(5))]
    plans = [pg.Plan.from_dict(p) for p in pats]
    batch = pg.Batch(plans)
    info = batch.info()
    assert info["nodes"] < info["levels_total"]  # prefixes are shared within a pattern
    shared = pg.Batch(plans, share_prefixes=True)
    assert shared.info()["nodes"] < info["nodes"]  # and across patterns in one tree
    out_s = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    pg.count_batch(G, shared, out_s)
    direct_info = pg.Batch(plans, expand_anti_edges=False).info()
    # unlabeled k-cliques are counted by the clique kernel, outside the tree
    is_clique = [p["k"] >= 3 and len(p["edges"]) == p["k"] * (p["k"] - 1) // 2 for p in pats]
    assert direct_info["programs"] == sum(pl.info().n_orders for pl, c in zip(plans, is_clique) if not c)
    assert direct_info["nodes"] < direct_info["levels_total"]
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    pg.count_batch(G, batch, out)
    torch.cuda.synchronize()
    got = pg.decode_counts(out)
    assert pg.decode_counts(out_s) == got
    out2 = torch.zeros_like(out)
    pg.count_async(G, plans, out2, kernel=pg.KERNEL_GENERIC)
    torch.cuda.synchronize()
    assert got == pg.decode_counts(out2)
    # anti-edges as set differences inside the batch (no pattern expansion)
    direct = pg.Batch(plans, expand_anti_edges=False)
    out3 = torch.zeros_like(out)
    pg.count_batch(G, direct, out3)
    torch.cuda.synchronize()
    assert got == pg.decode_counts(out3)
    for p, c in zip(pats, got):
        assert c == expected(g, p, 5), p


def test_batched_labeled_mix(pg):
    g = _graphs()[3]
    G = pg.Graph.from_synth(g)
    pats = [sg.pattern(3, sg.clique_edges(3), labels=[0, 1, -1]),
            sg.pattern(4, sg.star_edges(4), labels=[2, -1, -1, 0]),
            sg.pattern(4, sg.chain_edges(4), labels=[1, 0, -1, 2], vertex_induced=True),
            sg.pattern(1, [], labels=[1]), sg.pattern(2, [(0, 1)])]
    got = pg.count(G, [pg.Plan.from_dict(p) for p in pats])
    assert got == [oracle.count(g, p) for p in pats]
