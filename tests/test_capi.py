"""The C-ABI library builds, loads and exports every function include/*.h declares (CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_library_exports_every_declared_symbol():
    import paper_2605_04335_gb300 as pkg
    path = pkg.library_path()
    if not os.path.exists(path):
        import __graft_entry__
        __graft_entry__.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "poisson_solve" in names and "ibm_classify" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_status_strings():
    import paper_2605_04335_gb300 as pkg
    lib = pkg.load_library()
    assert lib.ibm_status_str(0) == b"ok"
    assert lib.ibm_status_str(5) == b"not converged"


def test_ctx_create_rejects_bad_device_without_gpu():
    import paper_2605_04335_gb300 as pkg
    lib = pkg.load_library()
    h = ctypes.c_void_p()
    s = lib.ibm_ctx_create(ctypes.byref(h), -1)
    assert s != 0
