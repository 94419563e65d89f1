"""Plain CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does, and this
package never imports the product.  The arithmetic lives in ``oracle.c``
(plain C, OpenMP over start vertices); this module marshals arguments and
adds the few closed forms that are easier to read in Python:

* ``count``            distinct matches = valid injective maps / |Aut|
                       (Section 2.1 definitions; Section 3.1.1 anti-edges;
                       Section 3.1.2 anti-vertices).
* ``motif4_induced``   the six induced 4-vertex motifs from non-induced
                       counts through the spanning-subgraph linear system.
* ``fsm_mni``          labeled frequent subgraphs up to three edges with MNI
                       support (Section 2.1 FSM / MNI; Section 3.2.1 label
                       discovery), by per-vertex existence of a match.
* ``domain_sizes``     MNI domains by their definition, vertex by vertex
                       (backtracking from u -> v, first hit); checks the
                       table-based FSM oracle above.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAXK = 8

OR_ERRORS = {1: "invalid argument", 2: "out of memory", 3: "uint64 overflow"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("off", ctypes.c_void_p),
                ("adj", ctypes.c_void_p), ("label", ctypes.c_void_p)]


class _Pattern(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("rel", ctypes.c_uint8 * (MAXK * MAXK)),
                ("label", ctypes.c_int32 * MAXK), ("anti_vertex", ctypes.c_uint8 * MAXK),
                ("vertex_induced", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.or_pattern_aut.argtypes = [ctypes.POINTER(_Pattern), u64p]
        L.or_count_maps.argtypes = [ctypes.POINTER(_Graph), ctypes.POINTER(_Pattern), ctypes.c_int, u64p]
        L.or_list_maps.argtypes = [ctypes.POINTER(_Graph), ctypes.POINTER(_Pattern), ctypes.c_void_p,
                                   ctypes.c_uint64, u64p]
        L.or_mni_bruteforce.argtypes = [ctypes.POINTER(_Graph), ctypes.POINTER(_Pattern), u64p]
        L.or_triangles.argtypes = [ctypes.POINTER(_Graph), ctypes.c_int]
        L.or_triangles.restype = ctypes.c_uint64
        L.or_triangles_per_vertex.argtypes = [ctypes.POINTER(_Graph), ctypes.c_int, ctypes.c_void_p]
        L.or_kcliques.argtypes = [ctypes.POINTER(_Graph), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_void_p, ctypes.c_int64, u64p]
        L.or_motif4_noninduced.argtypes = [ctypes.POINTER(_Graph), ctypes.c_int, u64p]
        L.or_domain_sizes.argtypes = [ctypes.POINTER(_Graph), ctypes.POINTER(_Pattern), ctypes.c_int, u64p]
        L.or_domain_member.argtypes = [ctypes.POINTER(_Graph), ctypes.POINTER(_Pattern), ctypes.c_int,
                                       ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
        L.or_fsm_domains.argtypes = [ctypes.POINTER(_Graph), ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 8
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"oracle error {rc}: {OR_ERRORS.get(rc, '?')}")


class _GraphRef:
    """Keeps the numpy arrays alive while C holds raw pointers to them."""

    def __init__(self, g):
        self.off = np.ascontiguousarray(g.offsets, dtype=np.int64)
        self.adj = np.ascontiguousarray(g.adj, dtype=np.int32)
        self.lab = None if g.labels is None else np.ascontiguousarray(g.labels, dtype=np.int32)
        self.s = _Graph(g.n, self.off.ctypes.data, self.adj.ctypes.data if self.adj.size else 0,
                        None if self.lab is None else self.lab.ctypes.data)


def _pattern_struct(p: dict) -> _Pattern:
    k = p["k"]
    if not 1 <= k <= MAXK:
        raise ValueError("pattern size out of range")
    s = _Pattern()
    s.k = k
    for (u, w) in p["edges"]:
        s.rel[u * MAXK + w] = 1
        s.rel[w * MAXK + u] = 1
    for (u, w) in p.get("anti_edges", ()):
        s.rel[u * MAXK + w] = 2
        s.rel[w * MAXK + u] = 2
    labels = p.get("labels")
    for u in range(MAXK):
        s.label[u] = -1 if labels is None or u >= k else int(labels[u])
    av = p.get("anti_vertex")
    for u in range(MAXK):
        s.anti_vertex[u] = 0 if av is None or u >= k else int(av[u])
    s.vertex_induced = 1 if p.get("vertex_induced") else 0
    return s


def automorphisms(p: dict) -> int:
    out = ctypes.c_uint64()
    _check(lib().or_pattern_aut(ctypes.byref(_pattern_struct(p)), ctypes.byref(out)))
    return int(out.value)


def count_maps(g, p: dict, threads: int = 0) -> int:
    """Number of valid injective maps (no symmetry breaking)."""
    gr = _GraphRef(g)
    out = ctypes.c_uint64()
    _check(lib().or_count_maps(ctypes.byref(gr.s), ctypes.byref(_pattern_struct(p)),
                               threads, ctypes.byref(out)))
    return int(out.value)


def count(g, p: dict, threads: int = 0) -> int:
    """Distinct matches of p in g: valid maps / |Aut(p)| (exact division)."""
    maps = count_maps(g, p, threads)
    aut = automorphisms(p)
    if maps % aut:
        raise AssertionError(f"maps {maps} not divisible by |Aut| {aut}")
    return maps // aut


def automorphism_perms(p: dict) -> np.ndarray:
    """Every permutation s of the pattern vertices (row: s[u] for u = 0..k-1)
    that keeps edges, anti-edges, labels and anti-vertex status: brute force
    over all k! permutations (Section 2.1)."""
    k = p["k"]
    rel = [[0] * k for _ in range(k)]
    for (u, w) in p["edges"]:
        rel[u][w] = rel[w][u] = 1
    for (u, w) in p.get("anti_edges", ()):
        rel[u][w] = rel[w][u] = 2
    lab = p.get("labels") or [-1] * k
    av = p.get("anti_vertex") or [0] * k
    out = [s for s in itertools.permutations(range(k))
           if all(lab[u] == lab[s[u]] and av[u] == av[s[u]] for u in range(k))
           and all(rel[u][w] == rel[s[u]][s[w]] for u in range(k) for w in range(k))]
    return np.array(out, dtype=np.int64)


def list_maps(g, p: dict) -> np.ndarray:
    """Every valid map as a row (column u = data vertex of pattern vertex u,
    -1 at anti-vertices); rows = count_maps(g, p)."""
    n = count_maps(g, p)
    out = np.zeros((max(n, 1), p["k"]), dtype=np.int32)
    gr = _GraphRef(g)
    got = ctypes.c_uint64()
    _check(lib().or_list_maps(ctypes.byref(gr.s), ctypes.byref(_pattern_struct(p)), out.ctypes.data,
                              n, ctypes.byref(got)))
    assert int(got.value) == n
    return out[:n]


def canonical_matches(rows: np.ndarray, p: dict) -> np.ndarray:
    """The class of map m under Aut(p) is {m o s}; its representative here is
    the lexicographically smallest row m[s] over s in Aut(p)."""
    rows = np.asarray(rows, dtype=np.int64)
    best = rows.copy()
    if rows.shape[0] == 0:
        return best
    for s in automorphism_perms(p):
        cand = rows[:, s]
        diff = cand != best
        first = np.argmax(diff, axis=1)
        r = np.arange(rows.shape[0])
        less = diff.any(axis=1) & (cand[r, first] < best[r, first])
        best[less] = cand[less]
    return best


def match_keys(g, p: dict) -> np.ndarray:
    """The distinct matches of p in g (Section 2.1): one canonical row per
    class of valid maps under Aut(p), sorted; len = count(g, p)."""
    keys = canonical_matches(list_maps(g, p), p)
    return np.unique(keys, axis=0) if keys.shape[0] else keys


def mni_domains_bruteforce(g, p: dict) -> list[int]:
    gr = _GraphRef(g)
    out = (ctypes.c_uint64 * MAXK)()
    _check(lib().or_mni_bruteforce(ctypes.byref(gr.s), ctypes.byref(_pattern_struct(p)), out))
    return [int(out[i]) for i in range(p["k"])]


def domain_sizes(g, p: dict, threads: int = 0) -> list[int]:
    """|D(u)| per pattern vertex by per-vertex existence of a map u -> v
    (first hit ends the search); MNI support = min over regular vertices."""
    gr = _GraphRef(g)
    out = (ctypes.c_uint64 * MAXK)()
    _check(lib().or_domain_sizes(ctypes.byref(gr.s), ctypes.byref(_pattern_struct(p)), threads, out))
    return [int(out[i]) for i in range(p["k"])]


def domain_member(g, p: dict, u: int, v: int) -> bool:
    gr = _GraphRef(g)
    m = ctypes.c_int()
    _check(lib().or_domain_member(ctypes.byref(gr.s), ctypes.byref(_pattern_struct(p)), u, v, ctypes.byref(m)))
    return bool(m.value)


def mni_support(g, p: dict, threads: int = 0) -> int:
    """MNI support (Section 2.1): the smallest domain over pattern vertices."""
    d = domain_sizes(g, p, threads)
    return min(d[u] for u in range(p["k"]) if not (p.get("anti_vertex") or [0] * p["k"])[u])


def triangles(g, threads: int = 0) -> int:
    gr = _GraphRef(g)
    return int(lib().or_triangles(ctypes.byref(gr.s), threads))


def triangles_per_vertex(g, threads: int = 0) -> np.ndarray:
    gr = _GraphRef(g)
    t = np.zeros(max(g.n, 1), dtype=np.uint64)
    _check(lib().or_triangles_per_vertex(ctypes.byref(gr.s), threads, t.ctypes.data))
    return t[:g.n]


def kcliques(g, k: int, threads: int = 0, sources=None) -> int:
    gr = _GraphRef(g)
    out = ctypes.c_uint64()
    if sources is None:
        _check(lib().or_kcliques(ctypes.byref(gr.s), k, threads, None, 0, ctypes.byref(out)))
    else:
        src = np.ascontiguousarray(sources, dtype=np.int32)
        _check(lib().or_kcliques(ctypes.byref(gr.s), k, threads, src.ctypes.data,
                                 src.shape[0], ctypes.byref(out)))
    return int(out.value)


MOTIF4_ORDER = ("star", "path", "tailed_triangle", "cycle", "diamond", "clique")


def motif4_noninduced(g, threads: int = 0) -> dict:
    gr = _GraphRef(g)
    out = (ctypes.c_uint64 * 6)()
    _check(lib().or_motif4_noninduced(ctypes.byref(gr.s), threads, out))
    return {name: int(out[i]) for i, name in enumerate(MOTIF4_ORDER)}


def motif4_induced(g, threads: int = 0) -> dict:
    """Induced counts I from non-induced counts S of the connected 4-vertex
    graphs.  S(H) = sum over induced shapes H' of (number of spanning copies
    of H inside H') * I(H'):

        S(K4)      = I(K4)
        S(diamond) = I(diamond) + 6 I(K4)
        S(C4)      = I(C4) + I(diamond) + 3 I(K4)
        S(tailed)  = I(tailed) + 4 I(diamond) + 12 I(K4)
        S(star)    = I(star) + I(tailed) + 2 I(diamond) + 4 I(K4)
        S(path)    = I(path) + 4 I(C4) + 2 I(tailed) + 6 I(diamond) + 12 I(K4)
    """
    S = motif4_noninduced(g, threads)
    I = {}
    I["clique"] = S["clique"]
    I["diamond"] = S["diamond"] - 6 * I["clique"]
    I["cycle"] = S["cycle"] - I["diamond"] - 3 * I["clique"]
    I["tailed_triangle"] = S["tailed_triangle"] - 4 * I["diamond"] - 12 * I["clique"]
    I["star"] = S["star"] - I["tailed_triangle"] - 2 * I["diamond"] - 4 * I["clique"]
    I["path"] = (S["path"] - 4 * I["cycle"] - 2 * I["tailed_triangle"]
                 - 6 * I["diamond"] - 12 * I["clique"])
    for k, v in I.items():
        if v < 0:
            raise AssertionError(f"negative induced count for {k}")
    return I


def wedges_induced(g, threads: int = 0) -> int:
    """Induced wedges (open triplets) = sum_v C(d_v, 2) - 3 T."""
    d = np.diff(g.offsets).astype(object)
    return int(sum(comb(int(x), 2) for x in d)) - 3 * triangles(g, threads)


def stars(g, leaves: int) -> int:
    """Edge-induced stars with the given number of leaves = sum_v C(d_v, leaves)."""
    d = np.diff(g.offsets)
    return int(sum(comb(int(x), leaves) for x in d))


FSM_SHAPES = ("edge", "wedge", "triangle", "path", "star")


def fsm_domain_tables(g, n_labels: int, threads: int = 0) -> dict:
    """Per-vertex-label domain counts of every labeled position (oracle.c)."""
    gr = _GraphRef(g)
    L = n_labels
    t = {"E": np.zeros((L, L), np.uint64), "WC": np.zeros((L, L, L), np.uint64),
         "WL": np.zeros((L, L, L), np.uint64), "T": np.zeros((L, L, L), np.uint64),
         "SC": np.zeros((L, L, L, L), np.uint64), "SL": np.zeros((L, L, L, L), np.uint64),
         "PE": np.zeros((L, L, L, L), np.uint64), "PI": np.zeros((L, L, L, L), np.uint64)}
    _check(lib().or_fsm_domains(ctypes.byref(gr.s), L, threads,
                                *[t[k].ctypes.data for k in ("E", "WC", "WL", "T", "SC", "SL", "PE", "PI")]))
    return t


def fsm_supports(g, n_labels: int, threads: int = 0) -> dict:
    """MNI support of every labeled connected pattern with 1..3 edges, keyed
    by (shape, canonical label tuple):
      edge (x, y) x<=y; wedge (c, x, y) x<=y; triangle (x, y, z) sorted;
      path (a, b, c, d) = min of the tuple and its reverse; star (c, x, y, z).
    Support = min over pattern positions of the domain size (MNI)."""
    t = fsm_domain_tables(g, n_labels, threads)
    E, WC, WL, T, SC, SL, PE, PI = (t[k] for k in ("E", "WC", "WL", "T", "SC", "SL", "PE", "PI"))
    L = n_labels
    out = {}
    R = range(L)
    for x in R:
        for y in R:
            if x <= y:
                out[("edge", (x, y))] = int(min(E[x, y], E[y, x]))
    for c in R:
        for x in R:
            for y in R:
                if x <= y:
                    out[("wedge", (c, x, y))] = int(min(WC[c, x, y], WL[x, c, y], WL[y, c, x]))
    for x in R:
        for y in R:
            for z in R:
                if x <= y <= z:
                    out[("triangle", (x, y, z))] = int(min(T[x, y, z], T[y, x, z], T[z, x, y]))
                for c in R:
                    if x <= y <= z:
                        out[("star", (c, x, y, z))] = int(min(SC[c, x, y, z], SL[x, c, y, z],
                                                              SL[y, c, x, z], SL[z, c, x, y]))
    for a in R:
        for b in R:
            for c in R:
                for d in R:
                    key = min((a, b, c, d), (d, c, b, a))
                    if key != (a, b, c, d):
                        continue
                    out[("path", key)] = int(min(PE[a, b, c, d], PE[d, c, b, a], PI[b, a, c, d], PI[c, d, b, a]))
    return out


def fsm(g, n_labels: int, threshold: int, threads: int = 0) -> dict:
    """Frequent labeled patterns (support >= threshold) with 1..3 edges."""
    return {k: v for k, v in fsm_supports(g, n_labels, threads).items() if v >= threshold}


def fsm_pattern(shape: str, labels) -> dict:
    """Pattern description of an FSM key (vertex 0 first in the tuple order)."""
    edges = {"edge": [(0, 1)], "wedge": [(0, 1), (0, 2)], "triangle": [(0, 1), (1, 2), (0, 2)],
             "path": [(0, 1), (1, 2), (2, 3)], "star": [(0, 1), (0, 2), (0, 3)]}[shape]
    k = 1 + max(max(e) for e in edges)
    return dict(k=k, edges=edges, anti_edges=[], labels=list(labels), anti_vertex=None,
                vertex_induced=False)
