"""A batched count captured in a CUDA graph and replayed (the launch-bound
3-motif workload uses this): after one warm-up call has sized the graph's
scratch, pg_count_batch only enqueues memsets and launches, so the captured
graph replays to the oracle's counts, replay after replay."""
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def test_captured_batch_replays_to_oracle_counts(pg):
    import torch
    g = sg.rmat(12, 16, 0.57, 0.19, 0.19, 1301)
    G = pg.Graph.from_synth(g)
    pats = sg.motif4_patterns() + [sg.pattern(3, sg.clique_edges(3)), sg.pattern(5, sg.clique_edges(5))]
    plans = [pg.Plan.from_dict(p) for p in pats]
    batch = pg.Batch(plans)  # prefix-tree kernel, 4-cycle kernel and clique kernel
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        pg.count_batch(G, batch, out, stream=side)  # sizes the scratch arena
        side.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            pg.count_batch(G, batch, out, stream=side)
    ind = oracle.motif4_induced(g)
    want = [ind[p["name"].replace("induced_", "")] for p in sg.motif4_patterns()]
    want += [oracle.kcliques(g, 3), oracle.kcliques(g, 5)]
    for _ in range(3):
        out.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert pg.decode_counts(out) == want
