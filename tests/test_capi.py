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
    s = lib.ibm_ctx_create(ctypes.byref(h), -1, None)
    assert s != 0


def test_null_handles_are_rejected_before_any_device_call():
    """Every entry point that takes tables or a context returns IBM_ERR_INVALID_ARG for a NULL
    handle, on the host, without touching a device."""
    import paper_2605_04335_gb300 as pkg
    lib = pkg.load_library()
    INVALID = 1
    assert lib.ibm_surface_forces(None, None, 0, None, None, None, None, None, None, None) == INVALID
    assert lib.ibm_boundary_velocity_rigid(None, None, 0, None, None) == INVALID
    assert lib.ibm_tables_export_self_weight(None, None, None) == INVALID
    assert lib.ibm_helmholtz_solve(None, None, 0.1, None, None, 1e-10, None, None, None, None) == INVALID
    ms = ctypes.c_double()
    assert lib.ibm_helmholtz_sweeps_timed(None, None, 0.1, 2, 1, None, None, None, ctypes.byref(ms)) == INVALID
    assert lib.ibm_set_neumann(None, None, None) == INVALID
    assert lib.ibm_neumann_rigid(None, None, 0, None) == INVALID


def test_helmholtz_option_defaults():
    import paper_2605_04335_gb300 as pkg
    from paper_2605_04335_gb300.ibm import ibm_helmholtz_opts
    o = ibm_helmholtz_opts()
    pkg.load_library().ibm_helmholtz_opts_default(ctypes.byref(o))
    assert (o.precision, o.srj_steps, o.max_cycles) == (2, 8, 100)
    d = pkg.HelmholtzOpts()
    assert (d.precision, d.srj_steps, d.max_cycles) == (2, 8, 100)


def _struct_fields(name):
    """Field names of a typedef'd struct in include/ibm_poisson.h, in declaration order."""
    src = open(os.path.join(ROOT, "include", "ibm_poisson.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct(?: %s)? \{([^{}]*)\} %s;" % (name, name), src, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        words = decl.split(None, 1)   # type, then one or more comma-separated names
        if len(words) == 2:
            names += [w.strip(" *\n") for w in words[1].split(",")]
    return names


def test_solve_options_binding_matches_the_header():
    """The ctypes mirror of ibm_solve_opts has the header's fields in the header's order, and
    the C defaults are the binding's defaults."""
    import dataclasses
    import paper_2605_04335_gb300 as pkg
    from paper_2605_04335_gb300.ibm import ibm_solve_opts
    assert [f[0] for f in ibm_solve_opts._fields_] == _struct_fields("ibm_solve_opts")
    o = ibm_solve_opts()
    pkg.load_library().ibm_solve_opts_default(ctypes.byref(o))
    d = pkg.SolveOpts()
    for f in dataclasses.fields(d):
        assert getattr(o, f.name) == pytest.approx(getattr(d, f.name)), f.name
    assert o.batch_schedule == 0
