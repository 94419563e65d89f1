"""GPU parity for the 21 induced 5-vertex motifs (generateAllVertexInduced(5))
counted together: one batched launch (anti-edges expanded where the batch's
slots allow), the unexpanded batch, and the plan interpreter, all equal to
the oracle's per-pattern counts."""
import pytest
import torch

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _graphs():
    g1 = sg.erdos_renyi(40, 0.2, 501)
    g2 = sg.chung_lu(150, 450, 2.1, 25.0, 502)
    g3 = sg.rmat(6, 6, 0.57, 0.19, 0.19, 503)
    return [g1, g2, g3]


@pytest.mark.parametrize("gi", range(3))
def test_all_induced_5_motifs(pg, gi):
    g = _graphs()[gi]
    G = pg.Graph.from_synth(g)
    pats = pg.generate_all(5, vertex_induced=True)
    assert len(pats) == 21
    want = [oracle.count(g, p) for p in pats]
    plans = [pg.Plan.from_dict(p) for p in pats]
    assert pg.count(G, plans) == want
    for expand in (True, False):
        for share in (False, True):
            b = pg.Batch(plans, expand_anti_edges=expand, share_prefixes=share)
            out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
            pg.count_batch(G, b, out)
            assert pg.decode_counts(out) == want, (expand, share)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for pl, w in zip(plans[::4], want[::4]):
        pg.count_async(G, [pl], out, kernel=pg.KERNEL_GENERIC)
        assert pg.decode_counts(out) == [w]
