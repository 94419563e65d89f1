"""GPU parity for labeled 3-motifs with label discovery (pg_labeled_motif3):
every nonzero (shape, labels) count equals the oracle's count of that
labeled vertex-induced pattern; at full size the sums over labels equal the
unlabeled closed forms (triangles, induced wedges) and sampled entries equal
the oracle."""
import itertools

import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _tri(a, b, c):
    return sg.pattern(3, sg.clique_edges(3), labels=[a, b, c])


def _wedge(c, x, y):
    return sg.pattern(3, [(0, 1), (1, 2)], labels=[x, c, y], vertex_induced=True)


def _expected(g, L):
    want = {}
    for a, b, c in itertools.combinations_with_replacement(range(L), 3):
        n = oracle.count(g, _tri(a, b, c))
        if n:
            want[("triangle", (a, b, c))] = n
    for c in range(L):
        for x, y in itertools.combinations_with_replacement(range(L), 2):
            n = oracle.count(g, _wedge(c, x, y))
            if n:
                want[("wedge", (c, x, y))] = n
    return want


@pytest.mark.parametrize("case", range(4))
def test_labeled_motif3_equals_oracle(pg, case):
    g, L = [(sg.erdos_renyi(60, 0.15, 601), 3), (sg.chung_lu(300, 1200, 2.1, 50.0, 602), 5),
            (sg.rmat(8, 8, 0.57, 0.19, 0.19, 603), 4), (sg.complete_graph(7), 2)][case]
    g.labels = sg.uniform_labels(g.n, L, 610 + case)
    G = pg.Graph.from_synth(g)
    assert pg.labeled_motif3(G) == _expected(g, int(g.labels.max()) + 1)


def test_labeled_motif3_full_size_sums(pg):
    """Chung-Lu 500K / 5M with Zipf labels over 20 (the FSM workload graph)."""
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    got = pg.labeled_motif3(G)
    assert sum(v for (s, _), v in got.items() if s == "triangle") == oracle.triangles(g, threads=8)
    assert sum(v for (s, _), v in got.items() if s == "wedge") == oracle.wedges_induced(g, threads=8)
    for key in sorted(got)[::97][:6]:
        shape, lab = key
        p = _tri(*lab) if shape == "triangle" else _wedge(*lab)
        if shape == "triangle" or lab[0] > 2:  # keep the oracle's wedge enumeration cheap
            assert got[key] == oracle.count(g, p, threads=8), key


def test_labeled_motif3_errors(pg):
    g = sg.erdos_renyi(50, 0.1, 620)
    with pytest.raises(pg.PgError) as e:
        pg.labeled_motif3(pg.Graph.from_synth(g))
    assert e.value.code == pg.PG_EINVAL
    g.labels = sg.uniform_labels(g.n, 3, 621)
    g.labels[0] = 40
    with pytest.raises(pg.PgError) as e:
        pg.labeled_motif3(pg.Graph.from_synth(g))
    assert e.value.code == pg.PG_EUNSUPPORTED


@pytest.mark.parametrize("case", range(2))
def test_labeled_motif4_discovery(pg, case):
    """Labeled 4-motifs with label discovery: every labeling of every shape is
    checked against the oracle's vertex-induced labeled count (absent =
    zero), and per shape the labeled counts sum to the unlabeled induced
    count of the motif linear system."""
    import itertools
    g = [sg.erdos_renyi(120, 0.08, 1401), sg.chung_lu(300, 1200, 2.1, 40.0, 1402)][case]
    nl = 3
    g.labels = sg.uniform_labels(g.n, nl, 1410 + case)
    G = pg.Graph.from_synth(g)
    got = pg.labeled_motif4(G)
    assert all(v > 0 for v in got.values())
    ind = oracle.motif4_induced(g)
    for shape, edges in sg.MOTIF4_SHAPES.items():
        assert sum(v for (sh, _), v in got.items() if sh == shape) == ind[shape], shape
        seen = set()
        for lab in itertools.product(range(nl), repeat=4):
            want = oracle.count(g, sg.pattern(4, edges, labels=list(lab), vertex_induced=True))
            key = (shape, lab)
            if key in got:
                assert got[key] == want, key
                seen.add(key)
        assert seen == {k for k in got if k[0] == shape}
