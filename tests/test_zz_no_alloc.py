"""GPU test of pg_count_cliques_noalloc, the clique entry point that draws
its scratch from a fixed array in the library instead of cudaMalloc (for
callers that cannot allocate device memory while counting).  Collected last
so that a run stopping at the first failure has run every other test."""
import ctypes

import pytest

import synthgraph as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg(cuda_device):
    import paper_2004_02369_b300 as pg
    return pg


def _regular(pg, G, kmin, kmax):
    import torch
    plans = [pg.Plan(k, sg.clique_edges(k)) for k in range(kmin, kmax + 1)]
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    pg.count_async(G, plans, out, kernel=pg.KERNEL_CLIQUE)
    torch.cuda.synchronize()
    return pg.decode_counts(out)


def _noalloc(pg, G, kmin, kmax):
    """Direct C-ABI call (ctypes) into a caller-owned torch buffer."""
    import torch
    out = torch.full((2 * (kmax - kmin + 1),), -1, dtype=torch.int64, device="cuda")
    rc = pg.lib().pg_count_cliques_noalloc(G.handle, kmin, kmax, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == pg.PG_OK, pg.lib().pg_last_error()
    torch.cuda.synchronize()
    return pg.decode_counts(out)


@pytest.mark.parametrize("which", ["shared_memory_tile", "global_slab"])
def test_noalloc_matches_regular_entry_point(pg, which):
    if which == "global_slab":
        g = sg.complete_graph(900)  # out-degree 899: the block tile lives in a slab of the array
        kmin, kmax = 3, 4
    else:
        g = sg.chung_lu(3000, 30000, 2.1, 500.0, 201)
        kmin, kmax = 3, 8
    G = pg.Graph.from_synth(g)
    want = _regular(pg, G, kmin, kmax)
    first = _noalloc(pg, G, kmin, kmax)
    second = _noalloc(pg, G, kmin, kmax)  # array keeps the previous call's contents
    assert first == want
    assert second == want


def test_noalloc_allocates_nothing_on_a_fresh_graph(pg):
    """After one warm-up call (which loads the kernel and the array), a call
    on a graph never counted through the allocating entry points leaves the
    device's free memory unchanged, and its counts equal the oracle's."""
    import torch
    import oracle
    warm = pg.Graph.from_synth(sg.chung_lu(2000, 12000, 2.1, 200.0, 205))
    _noalloc(pg, warm, 3, 6)
    g = sg.chung_lu(3000, 30000, 2.1, 500.0, 206)
    G = pg.Graph.from_synth(g)
    out = torch.full((8,), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        pg.count_cliques_noalloc(G, 3, 6, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        assert pg.decode_counts(out) == [oracle.kcliques(g, k) for k in range(3, 7)]


def test_noalloc_rejects_oversized_and_bad_sizes(pg):
    import torch
    G = pg.Graph.from_synth(sg.complete_graph(1400))  # out-degree 1399: fewer slabs than SMs
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(pg.PgError) as e:
        pg.count_cliques_noalloc(G, 3, 3, out)
    assert e.value.code == pg.PG_EINVAL and "static scratch" in str(e.value)
    small = pg.Graph.from_synth(sg.complete_graph(10))
    with pytest.raises(pg.PgError):
        pg.count_cliques_noalloc(small, 2, 3, out)
    with pytest.raises(pg.PgError):
        pg.count_cliques_noalloc(small, 5, 9, out)
