"""GPU parity of FSM for any number of edges (pg_fsm_general) against the
oracle: every connected labeled pattern with up to 4 (or 5) edges is
enumerated here, its MNI support computed by the oracle's per-vertex domain
search, and the frequent set with its supports must come back exactly.  At
full FSM-workload size (<= 3 edges) the general path must return the
oracle's stored frequent set: a second GPU path independent of pg_fsm."""
import itertools
import json
import os

import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "workload_counts.json")


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def canon(k, edges, labels):
    """Canonical form of a labeled pattern: the smallest (labels, edges)
    over all vertex permutations (brute force, k <= 6)."""
    best = None
    for perm in itertools.permutations(range(k)):
        inv = {perm[i]: i for i in range(k)}
        lab = tuple(labels[perm[i]] for i in range(k))
        es = tuple(sorted(tuple(sorted((inv[u], inv[v]))) for u, v in edges))
        c = (lab, es)
        if best is None or c < best:
            best = c
    return (k,) + best


def connected_shapes(max_edges):
    """Every connected graph with 1..max_edges edges (up to max_edges + 1
    vertices), one per isomorphism class."""
    seen, out = set(), []
    for k in range(2, max_edges + 2):
        pairs = list(itertools.combinations(range(k), 2))
        for m in range(k - 1, max_edges + 1):
            for es in itertools.combinations(pairs, m):
                adj = {u: set() for u in range(k)}
                for u, v in es:
                    adj[u].add(v)
                    adj[v].add(u)
                stack, comp = [0], {0}
                while stack:
                    for w in adj[stack.pop()]:
                        if w not in comp:
                            comp.add(w)
                            stack.append(w)
                if len(comp) != k:
                    continue
                c = canon(k, es, [0] * k)
                if c not in seen:
                    seen.add(c)
                    out.append((k, list(es)))
    return out


def oracle_frequent(g, nl, threshold, max_edges):
    want = {}
    for k, es in connected_shapes(max_edges):
        done = set()
        for labels in itertools.product(range(nl), repeat=k):
            c = canon(k, es, labels)
            if c in done:
                continue
            done.add(c)
            s = oracle.mni_support(g, sg.pattern(k, es, labels=list(labels)))
            if s >= threshold:
                want[c] = s
    return want


def got_frequent(res):
    return {canon(r["k"], r["edges"], r["labels"]): r["support"] for r in res}


@pytest.mark.parametrize("case", range(3))
def test_fsm_general_small_graphs(pg, case):
    g, nl, tau, me = [(sg.erdos_renyi(40, 0.12, 1201), 3, 3, 4),
                      (sg.chung_lu(300, 900, 2.3, 40.0, 1202), 3, 8, 4),
                      (sg.erdos_renyi(16, 0.35, 1203), 2, 2, 5)][case]
    g.labels = sg.zipf_labels(g.n, nl, 1.2, 1210 + case) if case == 1 else sg.uniform_labels(g.n, nl, 1210 + case)
    G = pg.Graph.from_synth(g)
    got = got_frequent(pg.fsm_general(G, threshold=tau, max_edges=me))
    want = oracle_frequent(g, nl, tau, me)
    assert got == want
    # a larger threshold keeps exactly the patterns at or above it
    hi = sorted(want.values())[len(want) // 2] if want else 1
    assert got_frequent(pg.fsm_general(G, threshold=hi, max_edges=me)) == {c: s for c, s in want.items() if s >= hi}


def test_fsm_general_full_size_equals_stored_frequent_set(pg):
    """FSM workload (Chung-Lu 500K / 5M, Zipf labels over 20, threshold 1000,
    <= 3 edges): the general path returns the oracle's stored frequent set."""
    want = {}
    for key, v in json.load(open(GOLDEN))["fsm"]["counts"].items():
        shape, labels = key.split(":")
        p = oracle.fsm_pattern(shape, tuple(int(x) for x in labels.split(",")))
        want[canon(p["k"], p["edges"], p["labels"])] = int(v)
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    assert got_frequent(pg.fsm_general(G, threshold=1000, max_edges=3)) == want
