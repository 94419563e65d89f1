"""The C-ABI library loads and exports every function include/pg.h declares
(no compute calls, CPU only)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(pg_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    import paper_2004_02369_b300 as pg
    names = declared_functions()
    assert "pg_load_graph" in names and "pg_count" in names and len(names) >= 12
    lib = ctypes.CDLL(pg.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string():
    import paper_2004_02369_b300 as pg
    assert pg.lib().pg_version() >= 100
    assert isinstance(pg.lib().pg_last_error(), bytes)


def test_null_arguments_rejected_without_a_device():
    """Every entry point that takes a graph, plan or output pointer answers
    PG_EINVAL (never a crash) to NULL, before touching the device."""
    import paper_2004_02369_b300 as pg
    L = pg.lib()
    v = ctypes.c_void_p()
    u64 = ctypes.c_uint64()
    i64 = ctypes.c_int64()
    i32 = ctypes.c_int32()
    calls = [
        lambda: L.pg_count(None, None, 1, None, None),
        lambda: L.pg_count_ex(None, None, 1, None, 0, None),
        lambda: L.pg_count_until(None, None, 1, None, ctypes.byref(i32), None),
        lambda: L.pg_plan_operand_bytes(None, None, ctypes.byref(u64), ctypes.byref(u64), None),
        lambda: L.pg_match(None, None, None, 0, ctypes.byref(u64), None),
        lambda: L.pg_match_range(None, None, 0, 0, None, 0, ctypes.byref(u64), None),
        lambda: L.pg_fsm(None, 3, 1, None, 0, ctypes.byref(i64), None),
        lambda: L.pg_labeled_motif3(None, None, 0, ctypes.byref(i64), None),
        lambda: L.pg_get_tuning(None, None),
        lambda: L.pg_set_tuning(None, None, None),
        lambda: L.pg_autotune(None, None, 1, 1, None, None),
        lambda: L.pg_graph_get_info(None, None),
        lambda: L.pg_plan_get_info(None, None),
        lambda: L.pg_compile_pattern(None, ctypes.byref(v)),
        lambda: L.pg_compile_batch(None, 1, 0, ctypes.byref(v)),
        lambda: L.pg_patterns_all(3, 1, None),
        lambda: L.pg_patterns_size(None, ctypes.byref(i64)),
        lambda: L.pg_server_create(None, None, ctypes.byref(v)),
    ]
    for i, call in enumerate(calls):
        assert call() == pg.PG_EINVAL, i
        assert L.pg_last_error()


def test_pattern_errors_on_host():
    """Pattern compilation is host-only: bad patterns fail with PG_EINVAL."""
    import paper_2004_02369_b300 as pg
    bad = [dict(k=0, edges=[]), dict(k=3, edges=[(0, 1)]), dict(k=2, edges=[(0, 5)]),
           dict(k=3, edges=[(0, 1), (1, 2)], anti_edges=[(0, 1)])]
    for p in bad:
        try:
            pg.Plan(p["k"], p["edges"], p.get("anti_edges", ()))
        except pg.PgError as e:
            assert e.code == pg.PG_EINVAL
        else:
            raise AssertionError(p)
