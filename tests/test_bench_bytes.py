"""The roofline numerators of bench.py against brute force on small graphs
(CPU): the clique kernel's level-1 operand bytes and the 4-cycle kernel's
suffix elements, each recounted by plain loops over the degree-ranked
lists."""
import numpy as np
import pytest

import bench
import synthgraph as sg


def _ranked(g):
    deg = np.diff(g.offsets)
    order = sorted(range(g.n), key=lambda v: (-deg[v], v))
    rank = np.empty(g.n, dtype=np.int64)
    rank[order] = np.arange(g.n)
    adj = {int(rank[v]): sorted(int(rank[x]) for x in g.adj[g.offsets[v]:g.offsets[v + 1]]) for v in range(g.n)}
    return rank, adj


GRAPHS = [lambda: sg.chung_lu(400, 2400, 2.1, 60.0, 71), lambda: sg.rmat(8, 8, 0.57, 0.19, 0.19, 72),
          lambda: sg.erdos_renyi(120, 0.08, 73)]


@pytest.mark.parametrize("gi", range(3))
@pytest.mark.parametrize("kmin", [3, 4, 5])
def test_clique_level1_bytes(gi, kmin):
    g = GRAPHS[gi]()
    rank, adj = _ranked(g)
    total = 0
    for r in range(g.n):
        out = [x for x in adj[r] if x < r]           # N+(r), ascending ranks
        if len(out) < kmin - 1:
            continue
        total += len(out)                            # the start vertex's out-list
        for u in out[1:]:                            # every out-neighbour but the first
            total += sum(1 for x in adj[u] if x < u)
    assert bench.algorithmic_bytes(g, rank, kmin) == 4 * total + 16 * g.n


@pytest.mark.parametrize("gi", range(3))
def test_c4_suffix_elements(gi):
    g = GRAPHS[gi]()
    rank, adj = _ranked(g)
    total = 0
    for w in range(g.n):
        above = [a for a in adj[w] if a > w]
        total += len(above)                          # the anchor's own suffix
        for a in above:
            total += sum(1 for x in adj[a] if x > w)  # suffix of adj(a) above w
    assert bench.c4_increments(g, rank) == total
