"""GPU parity of the fused batched launch for the six induced 4-vertex
motifs (R-MAT scale 20, edge factor 16) against oracle-written counts, and
of its evaluation strategies (anti-edges expanded or as set differences;
one task group per pattern or one shared prefix tree) at a smaller scale."""
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


def _batch_counts(pg, G, plans, expand, share=False):
    import torch
    b = pg.Batch(plans, expand_anti_edges=expand, share_prefixes=share)
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    pg.count_batch(G, b, out)
    torch.cuda.synchronize()
    return pg.decode_counts(out)


def test_motif4_small_rmat_both_strategies(pg):
    g = sg.workload_graph(3, scale_down=9)  # R-MAT scale 11, same generator
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in sg.motif4_patterns()]
    want = oracle.motif4_induced(g)
    want = [want[name] for name in sg.MOTIF4_SHAPES]
    assert _batch_counts(pg, G, plans, True) == want
    assert _batch_counts(pg, G, plans, False) == want
    # one tree for all patterns instead of one task group per pattern
    assert _batch_counts(pg, G, plans, True, share=True) == want
    assert _batch_counts(pg, G, plans, False, share=True) == want
    # brute-force definition on the induced patterns themselves
    for p, w in zip(sg.motif4_patterns(), want):
        if p["name"] in ("induced_clique", "induced_diamond", "induced_cycle"):
            assert oracle.count(g, p) == w


def test_motif4_rmat20_full(pg):
    """All six induced 4-motifs of R-MAT scale 20 in one fused launch."""
    gold = json.load(open(GOLDEN))["motif4"]["counts"]
    g = sg.workload_graph(3)
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in sg.motif4_patterns()]
    got = _batch_counts(pg, G, plans, True)
    assert got == [int(gold[p["name"]]) for p in sg.motif4_patterns()]
