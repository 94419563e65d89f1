"""GPU tests of the serving loop: every query's count in a concurrent,
batched mix equals its count alone (bit-exact), in batched and serial
modes, and memory admission splits or rejects what does not fit."""
import time

import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


@pytest.fixture(scope="module")
def graph(pg):
    g = sg.rmat(11, 16, 0.57, 0.19, 0.19, 0x5EED0005)
    g.labels = sg.uniform_labels(g.n, 8, 0x5EED0105)
    return g, pg.Graph.from_synth(g)


def _alone(pg, G, qs):
    return [pg.count(G, [pg.Plan.from_dict(q)])[0] for q in qs]


def _serve(pg, G, qs, **kw):
    srv = pg.Server(G, **kw)
    tickets = []
    for i, q in enumerate(qs):
        tickets.append(srv.submit(q))
        if i % 7 == 0:
            time.sleep(0.001)  # arrivals while earlier batches run
    srv.drain(300)
    res = {r["ticket"]: r for r in srv.poll(100000)}
    stats = srv.stats()
    srv.close()
    return [res[t] for t in tickets], stats


def test_mix_equals_alone(pg, graph):
    g, G = graph
    qs = sg.serving_queries(80, seed=7, labeled_fraction=0.2)
    alone = _alone(pg, G, qs)
    got, stats = _serve(pg, G, qs, n_streams=4, max_batch=16)
    assert all(r["status"] == 0 for r in got)
    assert [r["count"] for r in got] == alone
    assert stats["batches"] < len(qs)  # queries were batched
    assert max(r["batch_size"] for r in got) > 1
    for r in got:
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]


def test_anti_vertex_queries_in_mix(pg, graph):
    """Anti-vertex queries (run alone on the plan interpreter) interleaved
    with batched ones: every count equals the oracle's / its count alone."""
    g, G = graph
    av = [sg.pattern(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 1), (3, 2)], anti_vertex=[0, 0, 0, 1]),
          sg.pattern(3, [(0, 1)], anti_edges=[(2, 0), (2, 1)], anti_vertex=[0, 0, 1])]
    qs = sg.serving_queries(30, seed=11, labeled_fraction=0.2)
    mix = []
    for i, q in enumerate(qs):
        mix.append(q)
        if i % 5 == 0:
            mix.append(av[(i // 5) % 2])
    got, _ = _serve(pg, G, mix, n_streams=4, max_batch=16)
    assert all(r["status"] == 0 for r in got)
    want = {0: oracle.count(g, av[0], threads=8), 1: oracle.count(g, av[1], threads=8)}
    alone = _alone(pg, G, [q for q in mix if not q.get("anti_vertex")])
    it = iter(alone)
    for q, r in zip(mix, got):
        if q.get("anti_vertex"):
            assert r["count"] == want[av.index(q)]
        else:
            assert r["count"] == next(it)


def test_serial_mode_equals_alone(pg, graph):
    g, G = graph
    qs = sg.serving_queries(20, seed=8, labeled_fraction=0.3)
    got, stats = _serve(pg, G, qs, serial=True)
    assert [r["count"] for r in got] == _alone(pg, G, qs)
    assert stats["batches"] == len(qs) and all(r["batch_size"] == 1 for r in got)


def test_mix_matches_oracle_sample(pg, graph):
    g, G = graph
    qs = [sg.pattern(3, sg.clique_edges(3)), sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)]),
          sg.pattern(4, sg.chain_edges(4), labels=[0, 1, 2, 3]), sg.pattern(5, sg.star_edges(5))]
    got, _ = _serve(pg, G, qs, n_streams=2, max_batch=8)
    assert got[0]["count"] == oracle.triangles(g)
    assert got[1]["count"] == oracle.count(g, qs[1])
    assert got[2]["count"] == oracle.count(g, qs[2])
    assert got[3]["count"] == oracle.stars(g, 4)


def test_memory_admission(pg, graph):
    g, G = graph
    qs = sg.serving_queries(12, seed=9, labeled_fraction=0.0)
    # a budget far below one query's scratch: every query is rejected, none hangs
    got, _ = _serve(pg, G, qs, n_streams=2, max_batch=8, memory_budget=4096)
    assert all(r["status"] == pg.PG_ENOMEM for r in got if r["status"] != 0)
    assert any(r["status"] == pg.PG_ENOMEM for r in got)


def test_cancel_waiting_and_running_queries(pg):
    """A running query (unlabeled 5-cycles on R-MAT 16: far longer than the
    test allows) is cancelled mid-launch and a waiting one before it starts;
    both report PG_ECANCELED, and the queries around them come back with
    their counts alone.  No device fault is involved: the launch sees its
    stop word and returns."""
    import time
    g = sg.workload_graph(5, scale_down=6)
    G = pg.Graph.from_synth(g)
    fast = [sg.pattern(3, sg.clique_edges(3)), sg.pattern(3, sg.star_edges(3)), sg.pattern(4, sg.clique_edges(4))]
    want = [pg.count(G, [pg.Plan.from_dict(q)])[0] for q in fast]
    srv = pg.Server(G, n_streams=1, max_batch=1)
    slow = srv.submit(sg.pattern(5, sg.cycle_edges(5)))
    time.sleep(0.5)
    waiting = srv.submit(sg.pattern(4, sg.chain_edges(4)))
    tickets = [srv.submit(q) for q in fast]
    srv.cancel(waiting)
    srv.cancel(slow)
    t = time.perf_counter()
    srv.drain(120)
    took = time.perf_counter() - t
    res = {r["ticket"]: r for r in srv.poll()}
    srv.close()
    assert res[slow]["status"] == pg.PG_ECANCELED and res[waiting]["status"] == pg.PG_ECANCELED
    assert [res[x]["status"] for x in tickets] == [pg.PG_OK] * 3
    assert [res[x]["count"] for x in tickets] == want
    assert took < 30
    srv = pg.Server(G, n_streams=1, memory_budget=1 << 28)
    with pytest.raises(pg.PgError):
        srv.cancel(10 ** 9)
    srv.close()


def _straggler_run(pg, G, fast, **kw):
    import time
    srv = pg.Server(G, query_timeout_s=4.0, **kw)
    t = time.perf_counter()
    tickets = [srv.submit(q) for q in fast]
    slow = srv.submit(sg.pattern(5, sg.cycle_edges(5)))
    more = [srv.submit(q) for q in fast]
    srv.drain(120)
    took = time.perf_counter() - t
    res = {r["ticket"]: r for r in srv.poll()}
    srv.close()
    return res, tickets + more, slow, took


@pytest.mark.parametrize("mode", ["measured", "batch_everything"])
def test_query_time_limit_fails_only_the_slow_query(pg, mode):
    """A query time limit with one slow query (unlabeled 5-cycles on R-MAT
    16, far longer than the limit) among short ones: only the slow one
    reports PG_ETIMEOUT; the short ones return their counts alone.
    measured: one stream; each pattern's first query runs alone with a
    quarter of the limit, so the slow one goes to the back of the queue and
    the short ones behind it run first.  batch_everything: no measuring, two
    streams; the batch holding the slow query runs out of its budget (half
    the time left) and its queries are launched again one by one."""
    g = sg.workload_graph(5, scale_down=6)
    G = pg.Graph.from_synth(g)
    fast = [sg.pattern(3, sg.clique_edges(3)), sg.pattern(3, sg.star_edges(3)),
            sg.pattern(4, sg.clique_edges(4)), sg.pattern(4, sg.cycle_edges(4))]
    want = [pg.count(G, [pg.Plan.from_dict(q)])[0] for q in fast]
    kw = dict(n_streams=1, max_batch=8) if mode == "measured" else dict(n_streams=2, max_batch=8, batch_limit_ms=-1)
    res, ok, slow, took = _straggler_run(pg, G, fast, **kw)
    assert res[slow]["status"] == pg.PG_ETIMEOUT
    assert [res[x]["status"] for x in ok] == [pg.PG_OK] * len(ok)
    assert [res[x]["count"] for x in ok] == want + want
    assert took < 30
    # no query outlives its limit by more than a poll interval and a launch tail
    assert max(r["t_done"] - r["t_submit"] for r in res.values()) < 4.0 + 1.0
    if mode == "measured":
        # the second round of short queries was fused into one launch
        assert max(res[x]["batch_size"] for x in ok[len(fast):]) > 1
