"""GPU check of pg_plan_operand_bytes (the numerator of the set-operation
roofline): the device walk's bytes and operation counts equal those of the
CPU walk of the same compiled plan (tests/planeval), which is pinned to
closed forms on CPU, for cliques, cycles, induced and anti-edge patterns,
labels, anti-vertices and a 5-vertex pattern; the parts of a task partition
sum to the whole."""
import pytest

import planeval
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


PATTERNS = [
    sg.pattern(3, sg.clique_edges(3)),
    sg.pattern(3, sg.star_edges(3)),
    sg.pattern(4, sg.clique_edges(4)),
    sg.pattern(4, sg.cycle_edges(4)),
    sg.pattern(4, sg.chain_edges(4), vertex_induced=True),
    sg.pattern(4, [(0, 1), (1, 2), (0, 2), (0, 3)], anti_edges=[(1, 3)]),
    sg.pattern(5, sg.cycle_edges(5)),
    sg.pattern(4, [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3)]),
]


@pytest.mark.parametrize("gi", range(2))
def test_operand_bytes_equal_cpu_walk(pg, gi):
    g = [sg.chung_lu(2000, 12000, 2.1, 150.0, 3101), sg.rmat(10, 8, 0.57, 0.19, 0.19, 3102)][gi]
    G = pg.Graph.from_synth(g)
    for p in PATTERNS:
        elems, ops = planeval.operand_elems(g, p)
        assert pg.plan_operand_bytes(G, pg.Plan.from_dict(p)) == (4 * elems, ops), p


def test_operand_bytes_labels_and_anti_vertices(pg):
    g = sg.chung_lu(1500, 9000, 2.2, 120.0, 3103)
    g.labels = sg.uniform_labels(g.n, 3, 3104)
    G = pg.Graph.from_synth(g)
    ps = [sg.pattern(3, sg.clique_edges(3), labels=[0, 1, 1]),
          sg.pattern(4, sg.cycle_edges(4), labels=[0, 1, 0, 2]),
          sg.pattern(4, [(0, 1), (1, 2), (0, 2)], anti_edges=[(0, 3), (1, 3), (2, 3)],
                     anti_vertex=[0, 0, 0, 1])]
    for p in ps:
        elems, ops = planeval.operand_elems(g, p)
        assert pg.plan_operand_bytes(G, pg.Plan.from_dict(p)) == (4 * elems, ops), p


def test_operand_bytes_partition_sums_to_whole(pg):
    g = sg.rmat(11, 8, 0.57, 0.19, 0.19, 3105)
    G = pg.Graph.from_synth(g)
    plan = pg.Plan(4, sg.clique_edges(4))
    whole = pg.plan_operand_bytes(G, plan)
    parts = []
    for part in range(3):
        pg.set_partition(G, part, 3)
        parts.append(pg.plan_operand_bytes(G, plan))
    pg.set_partition(G, 0, 1)
    assert (sum(b for b, _ in parts), sum(o for _, o in parts)) == whole
    assert pg.plan_operand_bytes(G, plan) == whole
