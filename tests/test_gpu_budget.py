"""Device work budget (PG_ETIMEOUT): a synchronous call whose kernels run
out of their budget stops at the next poll and reports PG_ETIMEOUT; the
context stays usable and the same call without a budget is exact against
the oracle.  The failure is a budget that nothing can meet, never a device
fault.  The server's per-query time limit uses the same mechanism."""
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


@pytest.fixture(scope="module")
def graph():
    return sg.chung_lu(200_000, 2_000_000, 2.1, 4000.0, 7201)


PATTERNS = {
    "5-clique (k-clique kernel)": sg.pattern(5, sg.clique_edges(5)),
    "4-cycle (batched kernel)": sg.pattern(4, sg.cycle_edges(4)),
    "triangle in no 4-clique (interpreter, anti-vertex)":
        sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 1), (3, 2)], anti_vertex=[0, 0, 0, 1]),
}


@pytest.mark.parametrize("name", sorted(PATTERNS))
def test_budget_exhausted_then_exact(pg, graph, name):
    p = PATTERNS[name]
    G = pg.Graph.from_synth(graph)
    plan = pg.Plan.from_dict(p)
    pg.set_time_budget(G, 0.001)  # 1 microsecond
    assert pg.get_time_budget(G) == pytest.approx(0.001)
    with pytest.raises(pg.PgError) as e:
        pg.count(G, [plan])
    assert e.value.code == pg.PG_ETIMEOUT
    with pytest.raises(pg.PgError) as e:
        pg.count_until(G, plan, 1 << 62)
    assert e.value.code == pg.PG_ETIMEOUT
    pg.set_time_budget(G, 600_000.0)  # ample: the call completes
    want = pg.count(G, [plan])
    pg.set_time_budget(G, 0)
    assert pg.count(G, [plan]) == want
    small = sg.chung_lu(3000, 15000, 2.1, 300.0, 7202)
    Gs = pg.Graph.from_synth(small)
    assert pg.count(Gs, [plan]) == [oracle.count(small, p)]


def test_budget_on_listing(pg, graph):
    G = pg.Graph.from_synth(graph)
    plan = pg.Plan(3, sg.clique_edges(3))
    pg.set_time_budget(G, 0.001)
    with pytest.raises(pg.PgError) as e:
        pg.match(G, plan)
    assert e.value.code == pg.PG_ETIMEOUT
    pg.set_time_budget(G, 0)
    rows, total = pg.match(G, plan)
    assert total == pg.count(G, [plan])[0]


def test_server_query_timeout(pg, graph):
    """Queries whose launch cannot finish within the limit come back with
    PG_ETIMEOUT; a server without the limit answers the same queries."""
    G = pg.Graph.from_synth(graph)
    qs = [sg.pattern(4, sg.cycle_edges(4)), sg.pattern(5, sg.clique_edges(5))]
    srv = pg.Server(G, n_streams=2, max_batch=1, query_timeout_s=1e-6)
    for q in qs:
        srv.submit(q)
    srv.drain(120)
    res = srv.poll()
    srv.close()
    assert len(res) == 2 and all(r["status"] == pg.PG_ETIMEOUT for r in res)
    srv = pg.Server(G, n_streams=2, max_batch=1)
    tickets = [srv.submit(q) for q in qs]
    srv.drain(600)
    res = {r["ticket"]: r for r in srv.poll()}
    srv.close()
    assert [res[t]["status"] for t in tickets] == [pg.PG_OK, pg.PG_OK]
    assert [res[t]["count"] for t in tickets] == [pg.count(G, [pg.Plan.from_dict(q)])[0] for q in qs]
