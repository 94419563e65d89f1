"""GPU parity of frequent subgraph mining (MNI support, 1..3 edges) against
the oracle: every frequent labeled pattern and its support, exactly."""
import json
import os

import numpy as np
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _labeled(g, nl, seed, zipf=False):
    g.labels = sg.zipf_labels(g.n, nl, 1.2, seed) if zipf else sg.uniform_labels(g.n, nl, seed)
    return g


@pytest.mark.parametrize("case", range(4))
def test_fsm_small_graphs_all_patterns(pg, case):
    g = [_labeled(sg.erdos_renyi(40, 0.12, 31), 3, 32),
         _labeled(sg.erdos_renyi(30, 0.2, 33), 2, 34),
         _labeled(sg.chung_lu(400, 1600, 2.3, 60.0, 35), 5, 36, zipf=True),
         _labeled(sg.rmat(8, 8, 0.57, 0.19, 0.19, 37), 4, 38)][case]
    nl = int(g.labels.max()) + 1
    G = pg.Graph.from_synth(g)
    got = pg.fsm(G, threshold=1)
    want = oracle.fsm(g, nl, 1)
    assert got == want


def test_fsm_corner_cases(pg):
    g = sg.from_edges(7, [(0, 1), (0, 2), (0, 3), (1, 2), (3, 4), (4, 5), (5, 3), (5, 6)])
    g.labels = np.array([0, 1, 1, 2, 0, 1, 2], dtype=np.int32)
    G = pg.Graph.from_synth(g)
    assert pg.fsm(G, threshold=1) == oracle.fsm(g, 3, 1)


def test_fsm_levels_and_threshold(pg):
    g = _labeled(sg.chung_lu(3000, 20000, 2.3, 300.0, 39), 20, 40, zipf=True)
    G = pg.Graph.from_synth(g)
    full = oracle.fsm(g, 20, 20)
    assert pg.fsm(G, threshold=20) == full
    assert pg.fsm(G, threshold=20, max_edges=1) == {k: v for k, v in full.items() if k[0] == "edge"}
    assert pg.fsm(G, threshold=20, max_edges=2) == {k: v for k, v in full.items() if k[0] in ("edge", "wedge")}


def test_fsm_needs_labels(pg):
    G = pg.Graph.from_synth(sg.erdos_renyi(20, 0.2, 1))
    with pytest.raises(pg.PgError):
        pg.fsm(G, threshold=1)


def test_fsm_chunglu_500k_full(pg):
    """Chung-Lu 500K / 5M, gamma 2.3, Zipf(1.2) labels over 20, support >= 1000."""
    gold = json.load(open(GOLDEN))["fsm"]["counts"]
    want = {}
    for key, v in gold.items():
        shape, labels = key.split(":")
        want[(shape, tuple(int(x) for x in labels.split(",")))] = int(v)
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    assert pg.fsm(G, threshold=1000) == want


def test_fsm_full_size_against_domain_search(pg):
    """Full FSM workload: pg_fsm's supports against the per-vertex domain
    search oracle (oracle.domain_sizes, first-hit backtracking from u -> v,
    no label-count shortcut) on its stored seeded sample: every sampled
    frequent pattern over the five shapes has that support, and every sampled
    infrequent candidate is absent from the result."""
    search = json.load(open(GOLDEN))["fsm_domains"]["counts"]
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    got = {f"{shape}:{','.join(map(str, labels))}": v for (shape, labels), v in pg.fsm(G, threshold=1000).items()}
    n_freq = 0
    for key, v in search.items():
        if int(v) >= 1000:
            assert got.get(key) == int(v), key
            n_freq += 1
        else:
            assert key not in got, key
    assert n_freq >= 2000
