"""Builds and loads the CPU interpreter of compiled plans (test aid only)."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SRC = [os.path.join(HERE, "hosteval.cpp"),
       os.path.join(ROOT, "paper_2004_02369_b300", "csrc", "plan.cpp")]
DEPS = SRC + [os.path.join(ROOT, "paper_2004_02369_b300", "csrc", "plan.h"),
              os.path.join(ROOT, "include", "pg.h")]
LIB = os.path.join(HERE, "libplaneval.so")

_lib = None


class _Desc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("edges", ctypes.c_void_p),
                ("n_anti", ctypes.c_int32), ("anti_edges", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("anti_vertex", ctypes.c_void_p),
                ("vertex_induced", ctypes.c_int32)]


def build():
    stale = not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, *SRC])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.pe_count.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(_Desc), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
        _lib.pe_operand_elems.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(_Desc), ctypes.c_void_p]
    return _lib


def _desc(p: dict):
    e = np.ascontiguousarray(np.asarray(p["edges"], dtype=np.int32).reshape(-1))
    a = np.ascontiguousarray(np.asarray(p.get("anti_edges", []), dtype=np.int32).reshape(-1))
    pl = None if p.get("labels") is None else np.ascontiguousarray(p["labels"], dtype=np.int32)
    av = None if p.get("anti_vertex") is None else np.ascontiguousarray(p["anti_vertex"], dtype=np.uint8)
    d = _Desc(p["k"], e.size // 2, e.ctypes.data if e.size else None, a.size // 2,
              a.ctypes.data if a.size else None, None if pl is None else pl.ctypes.data,
              None if av is None else av.ctypes.data, 1 if p.get("vertex_induced") else 0)
    return d, (e, a, pl, av)


def operand_elems(g, p: dict):
    """(operand elements, set operations) of p's counting program on g:
    the length of every partial-order-bounded operand list of every set
    operation, summed over every task, prefix and level."""
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32)
    lab = None if g.labels is None else np.ascontiguousarray(g.labels, dtype=np.int32)
    d, keep = _desc(p)
    out = np.zeros(2, dtype=np.uint64)
    rc = lib().pe_operand_elems(off.ctypes.data, g.n, adj.ctypes.data if adj.size else None,
                                None if lab is None else lab.ctypes.data, ctypes.byref(d), out.ctypes.data)
    if rc:
        raise RuntimeError(f"plan compile error {rc}")
    return int(out[0]), int(out[1])


def count(g, p: dict, listing: bool = False):
    """(count, info) of pattern p on synthgraph graph g by interpreting the
    plan's counting program (or, with listing=True, its listing program)."""
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    adj = np.ascontiguousarray(g.adj, dtype=np.int32)
    lab = None if g.labels is None else np.ascontiguousarray(g.labels, dtype=np.int32)
    e = np.ascontiguousarray(np.asarray(p["edges"], dtype=np.int32).reshape(-1))
    a = np.ascontiguousarray(np.asarray(p.get("anti_edges", []), dtype=np.int32).reshape(-1))
    pl = None if p.get("labels") is None else np.ascontiguousarray(p["labels"], dtype=np.int32)
    av = None if p.get("anti_vertex") is None else np.ascontiguousarray(p["anti_vertex"], dtype=np.uint8)
    d = _Desc(p["k"], e.size // 2, e.ctypes.data if e.size else None, a.size // 2,
              a.ctypes.data if a.size else None, None if pl is None else pl.ctypes.data,
              None if av is None else av.ctypes.data, 1 if p.get("vertex_induced") else 0)
    out = np.zeros(2, dtype=np.uint64)
    info = np.zeros(4, dtype=np.int32)
    rc = lib().pe_count(off.ctypes.data, g.n, adj.ctypes.data if adj.size else None,
                        None if lab is None else lab.ctypes.data, ctypes.byref(d),
                        1 if listing else 0, out.ctypes.data, info.ctypes.data)
    if rc:
        raise RuntimeError(f"plan compile error {rc}")
    return (int(out[1]) << 64) | int(out[0]), info
