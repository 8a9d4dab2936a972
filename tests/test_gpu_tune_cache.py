"""ibm_autotune with a tune cache file (ibm_ctx_create's tune_cache_path): the first tuning
writes the schedule, a second context on the same file gets it back without launching
anything, and a different grid or precision gets an entry of its own."""
import json

import pytest

import synth
from tests.gpu_util import require_gpu, torch

pytestmark = pytest.mark.gpu


def _problem(n):
    f = synth.faces_tanh(n, 2.0)
    return f, f, f, [synth.octa_sphere(3, (0.5, 0.5, 0.5), 0.2)], synth.rhs_divergence(f, f, f, 3)


def test_tune_cache_round_trip(tmp_path):
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    path = str(tmp_path / "tune.json")
    xf, yf, zf, meshes, b = _problem(24)
    rhs = torch.from_numpy(b).cuda()
    p = torch.zeros_like(rhs)
    with pkg.Context(0, tune_cache=path) as c1:
        T = pkg.Tables(c1, xf, yf, zf, meshes)
        o1, ms1 = pkg.ibm_autotune(c1.h, T.h, 2, rhs, p, 1e-10)
        T.close()
    doc = json.load(open(path))
    assert len(doc["entries"]) == 1
    e = doc["entries"][0]
    assert "precision=2" in e["key"] and "grid=24x24x24" in e["key"]
    assert (e["omega"], e["nu1"], e["nu2"], e["inner_cycles"], e["krylov"], e["sweep_chunk"]) == \
        (o1.omega, o1.nu1, o1.nu2, o1.inner_cycles, o1.krylov, o1.sweep_chunk)
    assert o1.sweep_chunk in (0, 128, 64, 32)
    # a new context on the same file: the entry comes back, no kernel is launched
    with pkg.Context(0, tune_cache=path) as c2:
        T = pkg.Tables(c2, xf, yf, zf, meshes)
        l0 = pkg.ibm_ctx_launch_count(c2.h)
        o2, ms2 = pkg.ibm_autotune(c2.h, T.h, 2, rhs, p, 1e-10)
        assert pkg.ibm_ctx_launch_count(c2.h) == l0
        assert (o2.omega, o2.nu1, o2.nu2, o2.inner_cycles, o2.krylov, o2.sweep_chunk, o2.precision) == \
            (o1.omega, o1.nu1, o1.nu2, o1.inner_cycles, o1.krylov, o1.sweep_chunk, 2)
        assert abs(ms2 - ms1) <= 1e-5 * ms1
        # the cached schedule solves the problem
        rep = T.solve(rhs, p, 1e-10, o2)
        assert rep["status"] == "IBM_OK"
        # another precision, then another grid: new entries, the old one kept
        pkg.ibm_autotune(c2.h, T.h, 1, rhs, p, 1e-10)
        T.close()
        xf2, yf2, zf2, m2, b2 = _problem(20)
        T2 = pkg.Tables(c2, xf2, yf2, zf2, m2)
        r2 = torch.from_numpy(b2).cuda()
        pkg.ibm_autotune(c2.h, T2.h, 2, r2, torch.zeros_like(r2), 1e-10)
        T2.close()
    keys = [x["key"] for x in json.load(open(path))["entries"]]
    assert len(keys) == 3 and len(set(keys)) == 3 and keys[0] == e["key"]
