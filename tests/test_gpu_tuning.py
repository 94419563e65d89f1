"""GPU tests of the launch-parameter knobs and the autotuner: counts are
bit-exact under every knob value (checked against the oracle), the tuner
keeps one of the offered values and never reports a slower choice than the
parameters it started from."""
import pytest

import oracle
import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


@pytest.fixture(scope="module")
def clique_case(pg):
    g = sg.chung_lu(20000, 200000, 2.1, 2000.0, 301)
    want = [oracle.kcliques(g, k, threads=8) for k in (3, 4, 5, 6)]
    return g, want


@pytest.fixture(scope="module")
def motif_case(pg):
    g = sg.rmat(12, 8, 0.57, 0.19, 0.19, 302)
    g.labels = sg.uniform_labels(g.n, 4, 303)
    extra = [sg.pattern(4, sg.clique_edges(4)), sg.pattern(3, sg.chain_edges(3), labels=[0, 1, 2]),
             sg.pattern(4, sg.TAILED_TRIANGLE, anti_edges=[(3, 1)])]
    pats = sg.motif4_patterns() + extra
    m4 = oracle.motif4_induced(g, threads=8)
    want = [m4[p["name"].replace("induced_", "")] for p in sg.motif4_patterns()]
    want += [oracle.count(g, p, threads=8) for p in extra]
    return g, pats, want


CLIQUE_VALUES = {"clique_heavy_min": [8, 16, 33, 64], "clique_chunk": [1, 3, 16, 64],
                 "clique_blocks_per_sm": [1, 2, 0], "clique_min_blocks": [4, 3]}
BATCHED_VALUES = {"batched_split_grain": [16, 100, 0, 512], "batched_regcap": [1, 2, 0], "batched_warps": [2, 8, 4],
                  "batched_chunk": [1, 5, 64], "batched_blocks_per_sm": [1, 3, 0],
                  "hub_min_degree": [1, 300, 1 << 30, 1024], "hub_max": [0, 7, 2048, 512]}


def test_clique_counts_under_every_knob(pg, clique_case):
    g, want = clique_case
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan(k, sg.clique_edges(k)) for k in (3, 4, 5, 6)]
    default = pg.get_tuning(G)
    for knob, values in CLIQUE_VALUES.items():
        for v in values:
            pg.set_tuning(G, **{knob: v})
            assert pg.count(G, plans) == want, (knob, v)
        pg.set_tuning(G, **{knob: default[knob]})
    assert pg.get_tuning(G) == default


def test_batched_counts_under_every_knob(pg, motif_case):
    g, pats, want = motif_case
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in pats]
    for knob, values in BATCHED_VALUES.items():
        for v in values:
            pg.set_tuning(G, **{knob: v})
            assert pg.count(G, plans) == want, (knob, v)


def test_autotune_clique(pg, clique_case):
    g, want = clique_case
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan(k, sg.clique_edges(k)) for k in (4, 5)]
    rep = pg.autotune(G, plans)
    assert rep["kernel"] == pg.KERNEL_CLIQUE
    assert rep["tuned_ms"] <= rep["default_ms"]
    assert rep["trials"] >= 1 + sum(len(v) for v in ([16, 32, 48], [1, 2, 8, 16], [1, 2], [4]))
    assert pg.get_tuning(G) == rep["chosen"]
    assert rep["chosen"]["clique_heavy_min"] in (16, 32, 48, 64)
    assert pg.count(G, plans) == want[1:3]


def test_autotune_batched_sampled(pg, motif_case):
    g, pats, want = motif_case
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in pats]
    default = pg.get_tuning(G)
    rep = pg.autotune(G, plans, sample_stride=7)
    assert rep["kernel"] == pg.KERNEL_BATCHED and rep["sample_stride"] == 7
    assert rep["tuned_ms"] <= rep["default_ms"]
    assert rep["chosen"]["batched_warps"] in (2, 4, 8)
    assert pg.get_tuning(G) == rep["chosen"]
    if rep["full_tuned_ms"] >= 0:  # a sampled choice is kept only if the full launch is faster
        assert rep["full_tuned_ms"] < rep["full_default_ms"] or rep["chosen"] == default
    assert pg.count(G, plans) == want  # full counts after a sampled search


def test_tuning_validation(pg):
    g = sg.erdos_renyi(100, 0.05, 304)
    G = pg.Graph.from_synth(g)
    for bad in [dict(batched_warps=3), dict(clique_chunk=0), dict(clique_heavy_min=65), dict(hub_max=-1),
                dict(batched_split_grain=8), dict(batched_regcap=3), dict(clique_min_blocks=2)]:
        with pytest.raises(pg.PgError) as e:
            pg.set_tuning(G, **bad)
        assert e.value.code == pg.PG_EINVAL
    anti = pg.Plan(4, sg.clique_edges(3), anti_edges=[(3, 0), (3, 1), (3, 2)], anti_vertex=[0, 0, 0, 1])
    with pytest.raises(pg.PgError) as e:
        pg.autotune(G, [anti])
    assert e.value.code == pg.PG_EUNSUPPORTED
    srv = pg.Server(G, n_streams=1)
    with pytest.raises(pg.PgError):
        pg.set_tuning(G, batched_chunk=2)
    srv.close()
    pg.set_tuning(G, batched_chunk=2)
