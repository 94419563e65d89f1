"""Python binding of libpg (pattern-aware subgraph matching on one CUDA device).

Argument marshalling only: every step of matching runs in the library's CUDA
kernels.  The shared library must have been built in-tree
(``python paper_2004_02369_b300/build.py``); importing this package without it
raises ImportError instead of falling back to anything else.

PyTorch supplies device memory and streams: graph inputs may be torch CUDA
tensors (read in place), ``count_async`` writes into a caller-owned torch
CUDA tensor on the caller's stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpg.so")

PG_OK, PG_EINVAL, PG_ENOMEM, PG_ETRUNC, PG_ETIMEOUT, PG_EDEVICE, PG_EUNSUPPORTED, PG_ECANCELED = range(8)
KERNEL_AUTO, KERNEL_GENERIC, KERNEL_CLIQUE_PLAIN, KERNEL_CLIQUE, KERNEL_BATCHED, KERNEL_CLIQUE_NONPERSISTENT = range(6)
MAX_PATTERN = 8
MAX_CLIQUE = 16

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2004_02369_b300/build.py`")


class PgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libpg error {code}: {msg}")
        self.code = code


class _PatternDesc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("edges", ctypes.c_void_p),
                ("n_anti", ctypes.c_int32), ("anti_edges", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("anti_vertex", ctypes.c_void_p),
                ("vertex_induced", ctypes.c_int32)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("max_degree", ctypes.c_int64),
                ("max_out_degree", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("labeled", ctypes.c_int32), ("n_labels", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_regular", ctypes.c_int32),
                ("automorphisms", ctypes.c_uint64), ("n_po", ctypes.c_int32),
                ("po", ctypes.c_int32 * 56), ("core_mask", ctypes.c_uint32),
                ("n_orders", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("counted_group", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("compile_ms", ctypes.c_double)]


_lib = ctypes.CDLL(LIB_PATH)
_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_lib.pg_load_graph.argtypes = [_vp, _i64, _vp, _i64, _vp, _i32, _vp, ctypes.POINTER(_vp)]
_lib.pg_graph_get_info.argtypes = [_vp, ctypes.POINTER(GraphInfo)]
_lib.pg_graph_rank.argtypes = [_vp, _vp]
_lib.pg_free_graph.argtypes = [_vp]
_lib.pg_free_graph.restype = None
_lib.pg_compile_pattern.argtypes = [ctypes.POINTER(_PatternDesc), ctypes.POINTER(_vp)]
_lib.pg_plan_get_info.argtypes = [_vp, ctypes.POINTER(PlanInfo)]
_lib.pg_plan_describe.argtypes = [_vp, ctypes.c_char_p, _i64]
_lib.pg_free_plan.argtypes = [_vp]
_lib.pg_free_plan.restype = None
_lib.pg_count.argtypes = [_vp, _vp, _i32, _vp, _vp]
_lib.pg_count_ex.argtypes = [_vp, _vp, _i32, _vp, _i32, _vp]
_lib.pg_fsm.argtypes = [_vp, _i32, ctypes.c_uint64, _vp, _i64, ctypes.POINTER(_i64), _vp]
_lib.pg_server_create.argtypes = [_vp, _vp, ctypes.POINTER(_vp)]
_lib.pg_server_submit.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)]
_lib.pg_server_poll.argtypes = [_vp, _vp, _i32, ctypes.POINTER(_i32)]
_lib.pg_server_drain.argtypes = [_vp, ctypes.c_double]
_lib.pg_server_cancel.argtypes = [_vp, ctypes.c_uint64]
_lib.pg_server_get_stats.argtypes = [_vp, _vp]
_lib.pg_server_free.argtypes = [_vp]
_lib.pg_server_free.restype = None
_lib.pg_count_cliques_noalloc.argtypes = [_vp, _i32, _i32, _vp, _vp]
_lib.pg_compile_batch.argtypes = [_vp, _i32, _i32, ctypes.POINTER(_vp)]
_lib.pg_batch_get_info.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
_lib.pg_count_batch.argtypes = [_vp, _vp, _vp, _vp]
_lib.pg_free_batch.argtypes = [_vp]
_lib.pg_free_batch.restype = None
_lib.pg_patterns_all.argtypes = [_i32, _i32, ctypes.POINTER(_vp)]
_lib.pg_patterns_from.argtypes = [_vp, _i64, ctypes.POINTER(_vp)]
_lib.pg_patterns_extend.argtypes = [_vp, _i32, ctypes.POINTER(_vp)]
_lib.pg_patterns_size.argtypes = [_vp, ctypes.POINTER(_i64)]
_lib.pg_patterns_get.argtypes = [_vp, _i64, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _vp, ctypes.POINTER(_i32)]
_lib.pg_free_patterns.argtypes = [_vp]
_lib.pg_free_patterns.restype = None
_lib.pg_labeled_motif4.argtypes = [_vp, _vp, _i64, ctypes.POINTER(_i64), _vp]
_lib.pg_fsm_general.argtypes = [_vp, _i32, ctypes.c_uint64, _vp, _i64, ctypes.POINTER(_i64), _vp]
_lib.pg_labeled_motif3.argtypes = [_vp, _vp, _i64, ctypes.POINTER(_i64), _vp]
_lib.pg_count_until.argtypes = [_vp, _vp, ctypes.c_uint64, _vp, ctypes.POINTER(_i32), _vp]
_lib.pg_plan_operand_bytes.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _vp]
_lib.pg_match.argtypes = [_vp, _vp, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _vp]
_lib.pg_match_range.argtypes = [_vp, _vp, _i64, _i64, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), _vp]
_lib.pg_get_tuning.argtypes = [_vp, _vp]
_lib.pg_set_tuning.argtypes = [_vp, _vp, _vp]
_lib.pg_autotune.argtypes = [_vp, _vp, _i32, _i32, _vp, _vp]
_lib.pg_set_time_budget.argtypes = [_vp, ctypes.c_double]
_lib.pg_set_partition.argtypes = [_vp, _i32, _i32]
_lib.pg_clustering_coefficient_above.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(_i32), _vp, _vp, _vp]
_lib.pg_get_time_budget.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
_lib.pg_last_error.restype = ctypes.c_char_p


def lib():
    return _lib


def _check(rc: int):
    if rc != PG_OK:
        raise PgError(rc, _lib.pg_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


class Graph:
    """A data graph resident on the current CUDA device.

    ``offsets`` int64[n+1] and ``adj`` int32[2m]: undirected simple CSR with
    sorted lists (numpy arrays, or torch CUDA tensors read in place);
    ``labels`` optional int32[n].
    """

    def __init__(self, offsets, adj, labels=None, stream=None):
        on_dev = _is_torch_cuda(offsets)
        if on_dev:
            import torch
            offsets = offsets.to(torch.int64).contiguous()
            adj = adj.to(torch.int32).contiguous()
            labels = None if labels is None else labels.to(torch.int32).contiguous()
            p_off, p_adj = offsets.data_ptr(), adj.data_ptr()
            p_lab = None if labels is None else labels.data_ptr()
            n, nnz = offsets.numel() - 1, adj.numel()
        else:
            offsets = np.ascontiguousarray(offsets, dtype=np.int64)
            adj = np.ascontiguousarray(adj, dtype=np.int32)
            labels = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
            p_off = offsets.ctypes.data
            p_adj = adj.ctypes.data if adj.size else None
            p_lab = None if labels is None else labels.ctypes.data
            n, nnz = offsets.shape[0] - 1, adj.shape[0]
        h = _vp()
        _check(_lib.pg_load_graph(p_off, n, p_adj, nnz, p_lab, 1 if on_dev else 0,
                                  _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_synth(cls, g, stream=None):
        return cls(g.offsets, g.adj, g.labels, stream=stream)

    @property
    def handle(self):
        return self._h

    def info(self) -> GraphInfo:
        out = GraphInfo()
        _check(_lib.pg_graph_get_info(self._h, ctypes.byref(out)))
        return out

    def rank(self) -> np.ndarray:
        n = self.info().n
        out = np.zeros(max(n, 1), dtype=np.int32)
        _check(_lib.pg_graph_rank(self._h, out.ctypes.data))
        return out[:n]

    def close(self):
        if getattr(self, "_h", None):
            _lib.pg_free_graph(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Plan:
    """Compiled exploration plan of one pattern (host object)."""

    def __init__(self, k, edges, anti_edges=(), labels=None, anti_vertex=None,
                 vertex_induced=False, name=None):
        self.name = name
        self.pattern = dict(k=int(k), edges=[tuple(e) for e in edges],
                            anti_edges=[tuple(e) for e in anti_edges],
                            labels=None if labels is None else list(labels),
                            anti_vertex=None if anti_vertex is None else list(anti_vertex),
                            vertex_induced=bool(vertex_induced))
        e = np.ascontiguousarray(np.asarray(list(edges), dtype=np.int32).reshape(-1))
        a = np.ascontiguousarray(np.asarray(list(anti_edges), dtype=np.int32).reshape(-1))
        lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
        av = None if anti_vertex is None else np.ascontiguousarray(anti_vertex, dtype=np.uint8)
        d = _PatternDesc(int(k), e.size // 2, e.ctypes.data if e.size else None,
                         a.size // 2, a.ctypes.data if a.size else None,
                         None if lab is None else lab.ctypes.data,
                         None if av is None else av.ctypes.data, 1 if vertex_induced else 0)
        h = _vp()
        _check(_lib.pg_compile_pattern(ctypes.byref(d), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_dict(cls, p: dict):
        return cls(p["k"], p["edges"], p.get("anti_edges", ()), p.get("labels"),
                   p.get("anti_vertex"), p.get("vertex_induced", False), p.get("name"))

    @property
    def handle(self):
        return self._h

    def info(self) -> PlanInfo:
        out = PlanInfo()
        _check(_lib.pg_plan_get_info(self._h, ctypes.byref(out)))
        return out

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(1 << 16)
        _check(_lib.pg_plan_describe(self._h, buf, len(buf)))
        return buf.value.decode()

    def close(self):
        if getattr(self, "_h", None):
            _lib.pg_free_plan(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Batch:
    """Several plans counted in one launch (pg_compile_batch)."""

    EXPAND_ANTI = 1
    SHARE_PREFIXES = 2

    def __init__(self, plans, expand_anti_edges: bool = True, share_prefixes: bool = False):
        self.plans = list(plans)
        h = _vp()
        flags = (self.EXPAND_ANTI if expand_anti_edges else 0) | (self.SHARE_PREFIXES if share_prefixes else 0)
        _check(_lib.pg_compile_batch(_plan_array(self.plans), len(self.plans), flags, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        a, b, c = _i32(), _i32(), _i32()
        _check(_lib.pg_batch_get_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"nodes": a.value, "programs": b.value, "levels_total": c.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.pg_free_batch(self._h)
            self._h = None

    def __del__(self):
        self.close()


def count_batch(graph: Graph, batch: Batch, out, stream=None):
    """Enqueue the counts of every plan of ``batch`` into ``out`` (torch CUDA
    int64, 2*len(plans) words) in one launch; no host sync."""
    if out.numel() < 2 * len(batch.plans) or not out.is_cuda:
        raise ValueError("out must be a CUDA tensor with 2*len(plans) 64-bit elements")
    _check(_lib.pg_count_batch(graph.handle, batch.handle, out.data_ptr(), _stream_ptr(stream)))


def _plan_array(plans):
    arr = (_vp * len(plans))(*[p.handle.value for p in plans])
    return arr


def _u128(lo: int, hi: int) -> int:
    return (int(hi) << 64) | int(lo)


def count(graph: Graph, plans, stream=None) -> list[int]:
    """Exact match counts of each plan's pattern (synchronous)."""
    plans = list(plans)
    out = np.zeros(2 * max(len(plans), 1), dtype=np.uint64)
    _check(_lib.pg_count(graph.handle, _plan_array(plans), len(plans), out.ctypes.data,
                         _stream_ptr(stream)))
    return [_u128(out[2 * i], out[2 * i + 1]) for i in range(len(plans))]


def count_async(graph: Graph, plans, out, kernel: int = KERNEL_AUTO, stream=None):
    """Enqueue counting into ``out`` (torch CUDA int64 tensor with 2*len(plans)
    elements, (low, high) words per count) on ``stream``; no host sync."""
    plans = list(plans)
    if out.numel() < 2 * len(plans) or not out.is_cuda:
        raise ValueError("out must be a CUDA tensor with 2*len(plans) 64-bit elements")
    _check(_lib.pg_count_ex(graph.handle, _plan_array(plans), len(plans), out.data_ptr(),
                            kernel, _stream_ptr(stream)))


def _pattern_list(h) -> list[dict]:
    try:
        n = _i64()
        _check(_lib.pg_patterns_size(h, ctypes.byref(n)))
        out = []
        edges = (ctypes.c_int32 * 56)()
        for i in range(n.value):
            k, ne, vi = _i32(), _i32(), _i32()
            _check(_lib.pg_patterns_get(h, i, ctypes.byref(k), ctypes.byref(ne), edges, ctypes.byref(vi)))
            out.append(dict(k=k.value, edges=[(edges[2 * j], edges[2 * j + 1]) for j in range(ne.value)],
                            anti_edges=[], labels=None, anti_vertex=None, vertex_induced=bool(vi.value)))
        return out
    finally:
        _lib.pg_free_patterns(h)


def generate_all(size: int, vertex_induced: bool = True) -> list[dict]:
    """Every connected pattern with ``size`` vertices (vertex-induced) or
    ``size`` edges (edge-induced), one per isomorphism class."""
    h = _vp()
    _check(_lib.pg_patterns_all(int(size), 1 if vertex_induced else 0, ctypes.byref(h)))
    return _pattern_list(h)


def extend(patterns, by_vertex: bool) -> list[dict]:
    """extendByVertex / extendByEdge of a list of unlabeled pattern dicts."""
    patterns = list(patterns)
    keep = []
    descs = (_PatternDesc * max(len(patterns), 1))()
    for i, p in enumerate(patterns):
        e = np.ascontiguousarray(np.asarray(p["edges"], dtype=np.int32).reshape(-1))
        a = np.ascontiguousarray(np.asarray(p.get("anti_edges", []), dtype=np.int32).reshape(-1))
        lab = None if p.get("labels") is None else np.ascontiguousarray(p["labels"], dtype=np.int32)
        av = None if p.get("anti_vertex") is None else np.ascontiguousarray(p["anti_vertex"], dtype=np.uint8)
        keep += [e, a, lab, av]
        descs[i] = _PatternDesc(int(p["k"]), e.size // 2, e.ctypes.data if e.size else None, a.size // 2,
                                a.ctypes.data if a.size else None, None if lab is None else lab.ctypes.data,
                                None if av is None else av.ctypes.data, 1 if p.get("vertex_induced") else 0)
    src = _vp()
    _check(_lib.pg_patterns_from(descs, len(patterns), ctypes.byref(src)))
    try:
        h = _vp()
        _check(_lib.pg_patterns_extend(src, 1 if by_vertex else 0, ctypes.byref(h)))
    finally:
        _lib.pg_free_patterns(src)
    return _pattern_list(h)


def count_until(graph: Graph, plan: Plan, target: int, stream=None):
    """(count, reached): count matches until ``target`` are found.  The count
    is exact when reached is False, else a partial count >= target."""
    out = np.zeros(2, dtype=np.uint64)
    reached = _i32()
    _check(_lib.pg_count_until(graph.handle, plan.handle, int(target), out.ctypes.data, ctypes.byref(reached),
                               _stream_ptr(stream)))
    return _u128(out[0], out[1]), bool(reached.value)


def plan_operand_bytes(graph: Graph, plan: Plan, stream=None):
    """pg_plan_operand_bytes: (algorithmic bytes, set operations) of the
    plan's level program on the graph (4 B per element of every
    partial-order-bounded operand slice of every set operation)."""
    b = ctypes.c_uint64()
    n = ctypes.c_uint64()
    _check(_lib.pg_plan_operand_bytes(graph.handle, plan.handle, ctypes.byref(b), ctypes.byref(n),
                                      _stream_ptr(stream)))
    return int(b.value), int(n.value)


def exists(graph: Graph, plan: Plan, stream=None) -> bool:
    """Whether the graph has at least one match (stops at the first)."""
    return count_until(graph, plan, 1, stream)[1]


def clustering_coefficient_above(graph: Graph, bound: float, stream=None):
    """pg_clustering_coefficient_above: whether 3T / W exceeds ``bound``.
    Returns (answer, triangles counted, W)."""
    ans = _i32()
    t = np.zeros(2, dtype=np.uint64)
    w = np.zeros(2, dtype=np.uint64)
    _check(_lib.pg_clustering_coefficient_above(graph.handle, float(bound), ctypes.byref(ans), t.ctypes.data,
                                                w.ctypes.data, _stream_ptr(stream)))
    return bool(ans.value), _u128(t[0], t[1]), _u128(w[0], w[1])


def set_partition(graph: Graph, part: int, n_parts: int):
    """Count only the tasks t with t mod n_parts == part (pg_set_partition)."""
    _check(_lib.pg_set_partition(graph.handle, int(part), int(n_parts)))


def set_time_budget(graph: Graph, budget_ms: float):
    """Device work budget of the synchronous calls on ``graph`` (0 = none);
    a call that runs out raises PgError with code PG_ETIMEOUT."""
    _check(_lib.pg_set_time_budget(graph.handle, float(budget_ms)))


def get_time_budget(graph: Graph) -> float:
    out = ctypes.c_double()
    _check(_lib.pg_get_time_budget(graph.handle, ctypes.byref(out)))
    return out.value


def match(graph: Graph, plan: Plan, out=None, rank_range=None, stream=None):
    """List the distinct matches of ``plan``'s pattern.

    Returns ``(rows, n_total)``: ``rows`` is a torch CUDA int32 tensor of
    shape (min(n_total, capacity), k), column u the original id of the data
    vertex matched to pattern vertex u (-1 at anti-vertices).  ``out`` is an
    optional caller-owned int32 CUDA tensor of shape (capacity, k); without
    it the matches are counted first (pg_match with capacity 0) and a tensor
    of exactly that size is allocated.  ``rank_range`` = (begin, end) lists
    only the matches whose start vertex has degree rank in [begin, end).
    A result larger than ``out`` keeps the first rows and raises nothing;
    compare ``n_total`` with the capacity.
    """
    import torch
    k = plan.pattern["k"]
    n = graph.info().n
    lo, hi = (0, n) if rank_range is None else (int(rank_range[0]), int(rank_range[1]))
    total = ctypes.c_uint64()
    sp = _stream_ptr(stream)

    def call(ptr, cap):
        return _lib.pg_match_range(graph.handle, plan.handle, lo, hi, ptr, cap, ctypes.byref(total), sp)

    if out is None:
        rc = call(None, 0)
        if rc not in (PG_OK, PG_ETRUNC):
            _check(rc)
        out = torch.empty((max(int(total.value), 1), k), dtype=torch.int32, device="cuda")
        if int(total.value) == 0:
            return out[:0], 0
    if not out.is_cuda or out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != k or not out.is_contiguous():
        raise ValueError("out must be a contiguous int32 CUDA tensor of shape (capacity, k)")
    cap = out.shape[0]
    rc = call(out.data_ptr(), cap)
    if rc not in (PG_OK, PG_ETRUNC):
        _check(rc)
    n_total = int(total.value)
    return out[:min(n_total, cap)], n_total


def count_cliques_noalloc(graph: Graph, kmin: int, kmax: int, out, stream=None):
    """k-clique counts for k = kmin..kmax into ``out`` (torch CUDA int64,
    2*(kmax-kmin+1) elements) using the library's fixed scratch array: no
    device allocation.  Calls that overlap on the GPU race (shared array)."""
    if out.numel() < 2 * (kmax - kmin + 1) or not out.is_cuda:
        raise ValueError("out must be a CUDA tensor with 2*(kmax-kmin+1) 64-bit elements")
    _check(_lib.pg_count_cliques_noalloc(graph.handle, kmin, kmax, out.data_ptr(), _stream_ptr(stream)))


class Tuning(ctypes.Structure):
    """Launch parameters of the persistent kernels (pg_tuning in pg.h)."""
    _fields_ = [("clique_chunk", ctypes.c_int32), ("clique_blocks_per_sm", ctypes.c_int32),
                ("clique_heavy_min", ctypes.c_int32), ("batched_warps", ctypes.c_int32),
                ("batched_chunk", ctypes.c_int32), ("batched_blocks_per_sm", ctypes.c_int32),
                ("hub_min_degree", ctypes.c_int32), ("hub_max", ctypes.c_int32),
                ("batched_split_grain", ctypes.c_int32), ("batched_regcap", ctypes.c_int32),
                ("clique_min_blocks", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "pad"}


class TuneReport(ctypes.Structure):
    _fields_ = [("chosen", Tuning), ("default_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double),
                ("full_default_ms", ctypes.c_double), ("full_tuned_ms", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("trials", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("sample_stride", ctypes.c_int32), ("pad", ctypes.c_int32)]


def get_tuning(graph: Graph) -> dict:
    t = Tuning()
    _check(_lib.pg_get_tuning(graph.handle, ctypes.byref(t)))
    return t.as_dict()


def set_tuning(graph: Graph, stream=None, **values):
    """Change some launch parameters of ``graph`` (others keep their value)."""
    t = Tuning()
    _check(_lib.pg_get_tuning(graph.handle, ctypes.byref(t)))
    for k, v in values.items():
        if k not in dict(Tuning._fields_):
            raise KeyError(k)
        setattr(t, k, int(v))
    _check(_lib.pg_set_tuning(graph.handle, ctypes.byref(t), _stream_ptr(stream)))


def autotune(graph: Graph, plans, sample_stride: int = 1, stream=None) -> dict:
    """Measure and keep the best launch parameters for counting ``plans``."""
    plans = list(plans)
    r = TuneReport()
    _check(_lib.pg_autotune(graph.handle, _plan_array(plans), len(plans), sample_stride, ctypes.byref(r),
                            _stream_ptr(stream)))
    return {"chosen": r.chosen.as_dict(), "default_ms": r.default_ms, "tuned_ms": r.tuned_ms,
            "full_default_ms": r.full_default_ms, "full_tuned_ms": r.full_tuned_ms,
            "wall_ms": r.wall_ms, "trials": int(r.trials), "kernel": int(r.kernel),
            "sample_stride": int(r.sample_stride)}


class FsmPattern(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("labels", ctypes.c_int32 * 4), ("pad", ctypes.c_int32),
                ("support", ctypes.c_uint64)]


FSM_SHAPE_NAMES = {1: "edge", 2: "wedge", 3: "triangle", 4: "path", 5: "star"}


def fsm(graph: Graph, threshold: int, max_edges: int = 3, stream=None) -> dict:
    """Frequent labeled patterns with 1..max_edges edges and their MNI
    supports: {(shape_name, label tuple): support}."""
    cap = 1 << 16
    while True:
        arr = (FsmPattern * cap)()
        n = _i64()
        rc = _lib.pg_fsm(graph.handle, max_edges, threshold, arr, cap, ctypes.byref(n), _stream_ptr(stream))
        if rc == PG_ETRUNC:
            cap = int(n.value) + 1
            continue
        _check(rc)
        break
    out = {}
    width = {1: 2, 2: 3, 3: 3, 4: 4, 5: 4}
    for i in range(n.value):
        r = arr[i]
        out[(FSM_SHAPE_NAMES[r.shape], tuple(r.labels[j] for j in range(width[r.shape])))] = int(r.support)
    return out


class FsmGeneralPattern(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("edges", ctypes.c_int32 * 14),
                ("labels", ctypes.c_int32 * 8), ("support", ctypes.c_uint64)]


class LabeledCount4(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("labels", ctypes.c_int32 * 4), ("pad", ctypes.c_int32),
                ("count_lo", ctypes.c_uint64), ("count_hi", ctypes.c_uint64)]


MOTIF4_SHAPE_NAMES = {1: "path", 2: "star", 3: "cycle", 4: "tailed_triangle", 5: "diamond", 6: "clique"}


def labeled_motif4(graph: Graph, stream=None) -> dict:
    """pg_labeled_motif4: {(shape name, (l0, l1, l2, l3)): vertex-induced count}
    for every labeled connected 4-vertex pattern present."""
    cap = 1 << 16  # a second call only when more labeled patterns are present
    while True:
        arr = (LabeledCount4 * cap)()
        n = _i64()
        rc = _lib.pg_labeled_motif4(graph.handle, arr, cap, ctypes.byref(n), _stream_ptr(stream))
        if rc == PG_ETRUNC:
            cap = int(n.value) + 1
            continue
        _check(rc)
        break
    return {(MOTIF4_SHAPE_NAMES[r.shape], tuple(int(x) for x in r.labels)): _u128(r.count_lo, r.count_hi)
            for r in arr[:n.value]}


def fsm_general(graph: Graph, threshold: int, max_edges: int = 4, stream=None) -> list[dict]:
    """pg_fsm_general: every frequent labeled pattern with 1..max_edges
    edges as dicts (k, edges, labels, support), sorted by edge count."""
    n = _i64()
    rc = _lib.pg_fsm_general(graph.handle, max_edges, threshold, None, 0, ctypes.byref(n), _stream_ptr(stream))
    if rc not in (PG_OK, PG_ETRUNC):
        _check(rc)
    arr = (FsmGeneralPattern * max(1, n.value))()
    _check(_lib.pg_fsm_general(graph.handle, max_edges, threshold, arr, n.value, ctypes.byref(n),
                               _stream_ptr(stream)))
    out = []
    for r in arr[:n.value]:
        out.append(dict(k=int(r.k), edges=[(int(r.edges[2 * i]), int(r.edges[2 * i + 1])) for i in range(r.n_edges)],
                        labels=[int(r.labels[i]) for i in range(r.k)], support=int(r.support)))
    return out


class LabeledCount(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("labels", ctypes.c_int32 * 3),
                ("count_lo", ctypes.c_uint64), ("count_hi", ctypes.c_uint64)]


def labeled_motif3(graph: Graph, stream=None) -> dict:
    """Vertex-induced labeled 3-motif counts with label discovery:
    {("triangle", (a, b, c)): n, ("wedge", (centre, x, y)): n}, nonzero only."""
    cap = 1 << 16  # a second call only when more labeled patterns are present
    while True:
        arr = (LabeledCount * cap)()
        n = _i64()
        rc = _lib.pg_labeled_motif3(graph.handle, arr, cap, ctypes.byref(n), _stream_ptr(stream))
        if rc == PG_ETRUNC:
            cap = int(n.value) + 1
            continue
        _check(rc)
        break
    return {(FSM_SHAPE_NAMES[r.shape], tuple(r.labels)): _u128(r.count_lo, r.count_hi) for r in arr[:n.value]}


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("serial", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("query_timeout_s", ctypes.c_double), ("batch_limit_ms", ctypes.c_double),
                ("alone_sm_fraction", ctypes.c_double)]


class QueryResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("count_lo", ctypes.c_uint64), ("count_hi", ctypes.c_uint64),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("pad", ctypes.c_int32), ("batches", ctypes.c_int64),
                ("launched_queries", ctypes.c_int64), ("outstanding", ctypes.c_int64),
                ("cached_plans", ctypes.c_int64), ("scratch_bytes_per_stream", ctypes.c_int64),
                ("now", ctypes.c_double)]


class Server:
    """Request loop over a resident graph (native worker thread, see pg.h)."""

    def __init__(self, graph: Graph, n_streams: int = 4, max_batch: int = 32, memory_budget: int = 0,
                 serial: bool = False, query_timeout_s: float = 0.0, batch_limit_ms: float = 0.0,
                 alone_sm_fraction: float = 0.0):
        self.graph = graph  # keep the graph alive
        cfg = ServerConfig(n_streams, max_batch, memory_budget, 1 if serial else 0, 0, float(query_timeout_s),
                           float(batch_limit_ms), float(alone_sm_fraction))
        h = _vp()
        _check(_lib.pg_server_create(graph.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = []

    def submit(self, p: dict) -> int:
        """Enqueue a count query (pattern dict as in Plan.from_dict); returns its ticket."""
        e = np.ascontiguousarray(np.asarray(p["edges"], dtype=np.int32).reshape(-1))
        a = np.ascontiguousarray(np.asarray(p.get("anti_edges", []), dtype=np.int32).reshape(-1))
        lab = None if p.get("labels") is None else np.ascontiguousarray(p["labels"], dtype=np.int32)
        av = None if p.get("anti_vertex") is None else np.ascontiguousarray(p["anti_vertex"], dtype=np.uint8)
        d = _PatternDesc(int(p["k"]), e.size // 2, e.ctypes.data if e.size else None, a.size // 2,
                         a.ctypes.data if a.size else None, None if lab is None else lab.ctypes.data,
                         None if av is None else av.ctypes.data, 1 if p.get("vertex_induced") else 0)
        t = ctypes.c_uint64()
        _check(_lib.pg_server_submit(self._h, ctypes.byref(d), ctypes.byref(t)))
        return int(t.value)

    def poll(self, max_results: int = 4096) -> list[dict]:
        arr = (QueryResult * max_results)()
        n = _i32()
        _check(_lib.pg_server_poll(self._h, arr, max_results, ctypes.byref(n)))
        return [dict(ticket=int(r.ticket), status=int(r.status), count=_u128(r.count_lo, r.count_hi),
                     t_submit=r.t_submit, t_start=r.t_start, t_done=r.t_done, batch_size=int(r.batch_size))
                for r in arr[:n.value]]

    def cancel(self, ticket: int):
        """Withdraw a query (pg_server_cancel); its result reports PG_ECANCELED."""
        _check(_lib.pg_server_cancel(self._h, ticket))

    def drain(self, timeout_s: float = 600.0):
        _check(_lib.pg_server_drain(self._h, timeout_s))

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.pg_server_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_ if k != "pad"}

    def close(self):
        if getattr(self, "_h", None):
            _lib.pg_server_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


def decode_counts(words) -> list[int]:
    """(low, high) 64-bit words (numpy or torch int64) -> Python ints."""
    w = np.asarray(words.cpu() if hasattr(words, "cpu") else words).view(np.uint64)
    return [_u128(w[2 * i], w[2 * i + 1]) for i in range(w.shape[0] // 2)]
