"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds input generation only: random graphs, vertex labels and
plain pattern descriptions written as edge lists.  It holds none of the
matching method's arithmetic (no symmetry breaking, no vertex covers, no
counting), so that both the oracle and the GPU path can draw identical
inputs from it without sharing any of the code that is being checked.

Graphs come back as an undirected simple graph in CSR form with every
adjacency list sorted ascending: ``offsets`` int64[n+1], ``adj`` int32[2m].

Workload recipes (all seeded with numpy's PCG64):

* Erdos-Renyi G(n, p): every pair i<j kept independently with probability p.
* Chung-Lu power law: expected degree w_i = C (i + i0)^(-1/(gamma-1)), with C
  and i0 solved so that w_0 = max_weight and sum w = 2m; endpoint pairs are
  drawn independently with probability proportional to w; loops and duplicate
  pairs are dropped and sampling continues until m distinct edges exist; ids
  are then shuffled by a seeded permutation.
* R-MAT (a, b, c, d): edge_factor * 2^scale samples, each choosing one of the
  four quadrants per level; the result is symmetrised, loops and duplicates
  removed, ids shuffled by a seeded permutation.
* Labels: i.i.d. Zipf(s) over L labels (P(l) proportional to l^-s, l = 1..L,
  returned 0-based), or uniform over L labels.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 0x5EED0000


@dataclasses.dataclass
class Graph:
    n: int
    offsets: np.ndarray  # int64[n+1]
    adj: np.ndarray  # int32[2m], each list sorted ascending
    labels: np.ndarray | None = None  # int32[n] or None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.adj.shape[0] // 2)

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)

    def neighbors(self, v: int) -> np.ndarray:
        return self.adj[self.offsets[v]:self.offsets[v + 1]]

    def edges(self) -> np.ndarray:
        """Undirected edges (u < v) as an int64[m, 2] array."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.adj.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)


def _unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + neighbour compare)."""
    s = np.sort(x)
    if s.shape[0] == 0:
        return s
    keep = np.empty(s.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def _first_occurrences(x: np.ndarray) -> np.ndarray:
    """Distinct values of x in the order of their first occurrence."""
    order = np.argsort(x, kind="stable")
    s = x[order]
    keep = np.empty(s.shape[0], dtype=bool)
    if s.shape[0]:
        keep[0] = True
        np.not_equal(s[1:], s[:-1], out=keep[1:])
    first = np.sort(order[keep])
    return x[first]


def csr_from_pairs(n: int, pairs: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Undirected simple CSR from an int64[k, 2] array of endpoint pairs.

    Loops are dropped, duplicates (in either direction) merged, and every
    adjacency list sorted ascending.
    """
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    u, v = pairs[:, 0], pairs[:, 1]
    keep = u != v
    u, v = u[keep], v[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = _unique(lo * n + hi)
    lo, hi = key // n, key % n
    both = np.sort(np.concatenate([lo * n + hi, hi * n + lo]))
    src, dst = both // n, both % n
    counts = np.bincount(src, minlength=n).astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return offsets, dst.astype(np.int32)


def _relabel_pairs(pairs: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    perm = rng.permutation(n).astype(np.int64)
    return perm[pairs]


def _finish(n: int, pairs: np.ndarray, meta: dict) -> Graph:
    offsets, adj = csr_from_pairs(n, pairs)
    deg = np.diff(offsets)
    meta = dict(meta)
    meta.update(n=int(n), m=int(adj.shape[0] // 2),
                max_degree=int(deg.max()) if n else 0)
    return Graph(n=n, offsets=offsets, adj=adj, meta=meta)


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    """G(n, p): each pair i < j is an edge independently with probability p."""
    rng = np.random.default_rng(seed)
    chunks = []
    # Row blocks keep the dense uniform draws small.
    block = max(1, int(4_000_000 // max(n, 1)))
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        x = rng.random((r1 - r0, n))
        ii, jj = np.nonzero(x < p)
        ii = ii + r0
        keep = ii < jj
        chunks.append(np.stack([ii[keep], jj[keep]], axis=1))
    pairs = np.concatenate(chunks) if chunks else np.zeros((0, 2), np.int64)
    return _finish(n, pairs, dict(kind="erdos_renyi", p=p, seed=seed))


def chung_lu_weights(n: int, m: int, gamma: float, max_weight: float) -> np.ndarray:
    """Expected degrees w_i = C (i + i0)^(-1/(gamma-1)) with w_0 = max_weight
    and sum(w) = 2m (i0 found by bisection)."""
    alpha = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def total(i0: float) -> float:
        return float(max_weight * np.sum((i0 / (idx + i0)) ** alpha))

    lo, hi = 1e-9, 1e12
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if total(mid) < 2.0 * m:
            lo = mid
        else:
            hi = mid
    i0 = math.sqrt(lo * hi)
    return max_weight * (i0 / (idx + i0)) ** alpha


def chung_lu(n: int, m: int, gamma: float, max_weight: float, seed: int) -> Graph:
    """Chung-Lu power-law graph with exactly m distinct undirected edges."""
    rng = np.random.default_rng(seed)
    w = chung_lu_weights(n, m, gamma, max_weight)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    have = np.zeros(0, dtype=np.int64)
    rounds = 0
    while have.shape[0] < m:
        need = m - have.shape[0]
        draw = int(need * 1.15) + 1024
        a = np.searchsorted(cdf, rng.random(draw), side="right")
        b = np.searchsorted(cdf, rng.random(draw), side="right")
        a = np.minimum(a, n - 1).astype(np.int64)
        b = np.minimum(b, n - 1).astype(np.int64)
        keep = a != b
        a, b = a[keep], b[keep]
        key = np.minimum(a, b) * n + np.maximum(a, b)
        # Keep first occurrences in draw order so that the realised edge set
        # does not depend on how many extra samples were drawn.
        have = _first_occurrences(np.concatenate([have, key]))
        rounds += 1
    have = have[:m]
    pairs = np.stack([have // n, have % n], axis=1)
    pairs = _relabel_pairs(pairs, n, rng)
    return _finish(n, pairs, dict(kind="chung_lu", gamma=gamma,
                                  max_weight=max_weight, seed=seed,
                                  sampling_rounds=rounds))


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float,
         seed: int, chunk: int = 1 << 22) -> Graph:
    """R-MAT graph, symmetrised, loops and duplicates removed, ids shuffled."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    total = edge_factor * n
    keys = []
    ab, abc = a + b, a + b + c
    for s0 in range(0, total, chunk):
        k = min(chunk, total - s0)
        src = np.zeros(k, dtype=np.int64)
        dst = np.zeros(k, dtype=np.int64)
        for _level in range(scale):
            r = rng.random(k)
            sbit = (r >= ab).astype(np.int64)
            dbit = (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int64)
            src = (src << 1) | sbit
            dst = (dst << 1) | dbit
        keep = src != dst
        src, dst = src[keep], dst[keep]
        keys.append(_unique(np.minimum(src, dst) * n + np.maximum(src, dst)))
    key = _unique(np.concatenate(keys))
    pairs = np.stack([key // n, key % n], axis=1)
    pairs = _relabel_pairs(pairs, n, rng)
    return _finish(n, pairs, dict(kind="rmat", scale=scale,
                                  edge_factor=edge_factor,
                                  abcd=(a, b, c, 1.0 - a - b - c), seed=seed,
                                  samples=total))


def zipf_labels(n: int, n_labels: int, s: float, seed: int) -> np.ndarray:
    """i.i.d. labels with P(l) proportional to l^-s, l = 1..n_labels (0-based out)."""
    rng = np.random.default_rng(seed)
    p = np.arange(1, n_labels + 1, dtype=np.float64) ** (-s)
    p /= p.sum()
    return rng.choice(n_labels, size=n, p=p).astype(np.int32)


def uniform_labels(n: int, n_labels: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_labels, size=n).astype(np.int32)


def complete_graph(n: int) -> Graph:
    ii, jj = np.triu_indices(n, 1)
    pairs = np.stack([ii, jj], axis=1).astype(np.int64)
    return _finish(n, pairs, dict(kind="complete"))


def from_edges(n: int, edges) -> Graph:
    pairs = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return _finish(n, pairs, dict(kind="explicit"))


# ---------------------------------------------------------------------------
# The five benchmark workloads (graph part).  Sizes follow the workload table:
# (1) ER n=2000 p=0.005; (2) Chung-Lu 1M / 10M, gamma 2.1, max weight 20K;
# (3) R-MAT scale 20, edge factor 16, (.57,.19,.19,.05);
# (4) Chung-Lu 500K / 5M, gamma 2.3, max weight 10K, Zipf(1.2) over 20 labels;
# (5) R-MAT scale 22, edge factor 16, uniform labels over 8.
# ---------------------------------------------------------------------------

def workload_graph(config_id: int, scale_down: int = 0) -> Graph:
    """Graph of workload ``config_id`` (1..5).

    ``scale_down`` > 0 shrinks the vertex and edge counts by 2**scale_down,
    keeping the generator, its shape parameters and the seed recipe, for
    parity cases that the oracle finishes in seconds.
    """
    seed = SEED_BASE + config_id
    f = 1 << scale_down
    if config_id == 1:
        g = erdos_renyi(2000 // f, 0.005 * f, seed)
    elif config_id == 2:
        g = chung_lu(1_000_000 // f, 10_000_000 // f, 2.1, 20_000.0 / f, seed)
    elif config_id == 3:
        g = rmat(20 - scale_down, 16, 0.57, 0.19, 0.19, seed)
    elif config_id == 4:
        g = chung_lu(500_000 // f, 5_000_000 // f, 2.3, 10_000.0 / f, seed)
        g.labels = zipf_labels(g.n, 20, 1.2, seed + 0x100)
    elif config_id == 5:
        g = rmat(22 - scale_down, 16, 0.57, 0.19, 0.19, seed)
        g.labels = uniform_labels(g.n, 8, seed + 0x100)
    else:
        raise ValueError(f"unknown workload {config_id}")
    g.meta["config_id"] = config_id
    g.meta["scale_down"] = scale_down
    return g


# ---------------------------------------------------------------------------
# Plain pattern descriptions (edge lists only; no analysis).
# A pattern is a dict: k, edges [(u,v)], anti_edges [(u,v)], labels (list of
# k ints, -1 = any) or None, anti_vertex (list of k 0/1) or None,
# vertex_induced (bool).
# ---------------------------------------------------------------------------

def pattern(k, edges, anti_edges=(), labels=None, anti_vertex=None,
            vertex_induced=False, name=None) -> dict:
    return dict(k=int(k), edges=[tuple(e) for e in edges],
                anti_edges=[tuple(e) for e in anti_edges],
                labels=None if labels is None else [int(x) for x in labels],
                anti_vertex=None if anti_vertex is None else [int(x) for x in anti_vertex],
                vertex_induced=bool(vertex_induced), name=name)


def clique_edges(k):
    return [(i, j) for i in range(k) for j in range(i + 1, k)]


def star_edges(k):
    """Star on k vertices: vertex 0 is the centre, 1..k-1 the leaves."""
    return [(0, i) for i in range(1, k)]


def chain_edges(k):
    return [(i, i + 1) for i in range(k - 1)]


def cycle_edges(k):
    return [(i, (i + 1) % k) for i in range(k)]


TAILED_TRIANGLE = [(0, 1), (0, 2), (1, 2), (0, 3)]  # tail 3 hangs off 0
DIAMOND = [(0, 1), (1, 2), (2, 3), (3, 0), (1, 3)]  # 4-cycle + chord 1-3

MOTIF4_SHAPES = {
    "path": chain_edges(4),
    "star": star_edges(4),
    "cycle": cycle_edges(4),
    "tailed_triangle": TAILED_TRIANGLE,
    "diamond": DIAMOND,
    "clique": clique_edges(4),
}


def motif4_patterns() -> list[dict]:
    return [pattern(4, e, vertex_induced=True, name=f"induced_{k}")
            for k, e in MOTIF4_SHAPES.items()]


def motif3_patterns() -> list[dict]:
    return [pattern(3, clique_edges(3), vertex_induced=True, name="induced_triangle"),
            pattern(3, chain_edges(3), vertex_induced=True, name="induced_wedge")]


# ---------------------------------------------------------------------------
# Serving query stream: count queries mixing 3-6 cliques, 4-5 cycles, the
# 4-vertex chain, 3-5 vertex stars, tailed triangles (plain, with the tail
# anti-adjacent to both other triangle vertices, and to one of them), with a
# fraction of labeled variants (every pattern vertex labeled uniformly).
# ---------------------------------------------------------------------------

SERVING_TYPES = {
    "K3": (3, clique_edges(3), []), "K4": (4, clique_edges(4), []),
    "K5": (5, clique_edges(5), []), "K6": (6, clique_edges(6), []),
    "C4": (4, cycle_edges(4), []), "C5": (5, cycle_edges(5), []),
    "P4": (4, chain_edges(4), []),
    "S3": (3, star_edges(3), []), "S4": (4, star_edges(4), []), "S5": (5, star_edges(5), []),
    "TT": (4, TAILED_TRIANGLE, []), "TT_anti2": (4, TAILED_TRIANGLE, [(3, 1), (3, 2)]),
    "TT_anti1": (4, TAILED_TRIANGLE, [(3, 1)]),
}


def serving_queries(n: int, seed: int, n_labels: int = 8, labeled_fraction: float = 0.1,
                    types=None, labeled_only=()) -> list[dict]:
    """n query patterns drawn uniformly over the types, a seeded fraction of
    them (all of those whose type is in labeled_only) with every vertex
    labeled uniformly over n_labels."""
    rng = np.random.default_rng(seed)
    names = list(types or SERVING_TYPES)
    out = []
    for _ in range(n):
        name = names[int(rng.integers(len(names)))]
        k, edges, anti = SERVING_TYPES[name]
        labels = None
        if rng.random() < labeled_fraction or name in labeled_only:
            labels = [int(x) for x in rng.integers(0, n_labels, k)]
        out.append(pattern(k, edges, anti_edges=anti, labels=labels,
                           name=name + ("_lab" if labels else "")))
    return out


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))
