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
