"""The multi-GPU split of counting (pg_set_partition): on one GPU, the counts
of parts 0..N-1 (tasks t with t mod N == part) sum to the whole count for
every counting kernel, equal to the oracle.  Each part is an ordinary
launch; no kernel waits on another.  Also the non-persistent form of the
k-clique kernel (the plain one-pattern-per-launch comparison arm)."""
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _parts(pg, G, plans, n_parts, kernel=None):
    import torch
    tot = [0] * len(plans)
    for part in range(n_parts):
        pg.set_partition(G, part, n_parts)
        if kernel is None:
            got = pg.count(G, plans)
        else:
            out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
            pg.count_async(G, plans, out, kernel=kernel)
            torch.cuda.synchronize()
            got = pg.decode_counts(out)
        tot = [a + b for a, b in zip(tot, got)]
    pg.set_partition(G, 0, 1)
    return tot


@pytest.mark.parametrize("n_parts", [2, 3, 8])
def test_partitions_sum_to_whole(pg, n_parts):
    g = sg.chung_lu(20000, 150000, 2.1, 2000.0, 1101)
    G = pg.Graph.from_synth(g)
    cliques = [pg.Plan(k, sg.clique_edges(k)) for k in (3, 4, 5)]
    want_cl = [oracle.kcliques(g, k) for k in (3, 4, 5)]
    assert _parts(pg, G, cliques, n_parts) == want_cl
    motifs = [pg.Plan.from_dict(p) for p in sg.motif4_patterns()]  # batched kernel + 4-cycle + clique kernels
    ind = oracle.motif4_induced(g)
    assert _parts(pg, G, motifs, n_parts) == [ind[p["name"].replace("induced_", "")] for p in sg.motif4_patterns()]
    tt = sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)])
    assert _parts(pg, G, [pg.Plan.from_dict(tt)], n_parts, kernel=pg.KERNEL_GENERIC) == [oracle.count(g, tt)]
    assert _parts(pg, G, cliques[1:], n_parts, kernel=pg.KERNEL_CLIQUE_NONPERSISTENT) == want_cl[1:]


def test_partition_validation(pg):
    G = pg.Graph.from_synth(sg.complete_graph(10))
    for part, n in ((1, 1), (-1, 2), (2, 2), (0, 0)):
        with pytest.raises(pg.PgError) as e:
            pg.set_partition(G, part, n)
        assert e.value.code == pg.PG_EINVAL


@pytest.mark.parametrize("seed", [1, 2])
def test_nonpersistent_clique_kernel(pg, seed):
    import torch
    g = sg.chung_lu(30000, 250000, 2.1, 3000.0, 1110 + seed)
    G = pg.Graph.from_synth(g)
    ks = [3, 4, 5, 6, 9]
    plans = [pg.Plan(k, sg.clique_edges(k)) for k in ks]
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    pg.count_async(G, plans, out, kernel=pg.KERNEL_CLIQUE_NONPERSISTENT)
    torch.cuda.synchronize()
    assert pg.decode_counts(out) == [oracle.kcliques(g, k) for k in ks]
