"""Reclassification of existing tables (moving bodies on a fixed grid).

The tables after ibm_reclassify must equal fresh ibm_classify tables of the same meshes bit
for bit, and the oracle's classification of those meshes; a solve after reclassifying (whose
solver work arrays were built for the previous bodies, with a captured cycle) must give the
same bits as a solve on fresh tables, and the oracle's pressure within 1e-8."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import solve as OS
from oracle.grid import Grid
from tests.gpu_util import require_gpu, torch

pytestmark = pytest.mark.gpu
TOL = 1e-10
PARITY = 1e-8


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _faces():
    return synth.faces_tanh(40, 2.0), synth.faces_uniform(36), synth.faces_tanh(44, 1.5)


def _bodies(tag):
    if tag == "none":
        return []
    if tag == "small":
        return [synth.octa_sphere(3, (0.45, 0.5, 0.52), 0.1)]
    if tag == "ellipsoid":
        return [synth.ellipsoid(4, (0.22, 0.1, 0.09), 25.0, (0.5, 0.47, 0.5))]
    if tag == "moved":
        return [synth.ellipsoid(4, (0.22, 0.1, 0.09), 40.0, (0.53, 0.5, 0.48))]
    if tag == "big":
        return [synth.octa_sphere(4, (0.5, 0.5, 0.5), 0.3), synth.octa_sphere(3, (0.15, 0.2, 0.8), 0.08)]
    raise ValueError(tag)


def _export_np(T):
    return {k: v.cpu().numpy() for k, v in T.export().items()}


def _same_tables(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_reclassify_equals_fresh_classify_and_oracle(ctx):
    pkg, c = ctx
    xf, yf, zf = _faces()
    T = pkg.Tables(c, xf, yf, zf, _bodies("small"))
    g = Grid(xf, yf, zf)
    for tag in ("ellipsoid", "big", "none", "moved", "small"):
        T.reclassify(_bodies(tag))
        F = pkg.Tables(c, xf, yf, zf, _bodies(tag))
        assert (T.nfluid, T.nghost, T.nsolid) == (F.nfluid, F.nghost, F.nsolid), tag
        ex = _export_np(T)
        _same_tables(ex, _export_np(F))
        ib, G = OC.classify(g, _bodies(tag))
        assert np.array_equal(ex["iblank"], ib), tag
        assert np.array_equal(ex["cell"], G.cell), tag
        assert np.array_equal(ex["w"], G.w), tag
        F.close()
    T.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_after_reclassify_matches_fresh_tables(ctx, prec):
    """The reused hierarchy (refreshed geometry, captured cycle replayed or recaptured when
    the ghost capacity grew) gives the bits of a fresh hierarchy, body after body."""
    pkg, c = ctx
    xf, yf, zf = _faces()
    b = synth.rhs_divergence(xf, yf, zf, 9)
    rhs = torch.from_numpy(b).cuda()
    T = pkg.Tables(c, xf, yf, zf, _bodies("small"))
    p = torch.zeros_like(rhs)
    T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))          # builds the hierarchy and its graph
    for tag in ("moved", "big", "none", "ellipsoid", "small"):
        T.reclassify(_bodies(tag))
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))
        F = pkg.Tables(c, xf, yf, zf, _bodies(tag))
        q = torch.zeros_like(rhs)
        rep_f = F.solve(rhs, q, TOL, pkg.SolveOpts(precision=prec))
        F.close()
        assert rep["status"] == "IBM_OK" and rep["cycles"] == rep_f["cycles"], (tag, rep, rep_f)
        assert torch.equal(p, q), tag
        assert np.array_equal(rep["history"], rep_f["history"]), tag
    T.close()


def test_reclassified_solve_matches_oracle(ctx):
    pkg, c = ctx
    xf, yf, zf = _faces()
    g = Grid(xf, yf, zf)
    b = synth.rhs_divergence(xf, yf, zf, 4)
    rhs = torch.from_numpy(b).cuda()
    T = pkg.Tables(c, xf, yf, zf, _bodies("ellipsoid"))
    p = torch.zeros_like(rhs)
    T.solve(rhs, p, TOL, pkg.SolveOpts(precision=2))
    T.reclassify(_bodies("moved"))
    ib, G = OC.classify(g, _bodies("moved"))
    p_o, _ = OS.solve_gmres(g, ib, G, b)
    fl = ib == 0
    for prec in (0, 1, 2):
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))
        assert rep["status"] == "IBM_OK"
        pg = p.cpu().numpy()
        err = np.linalg.norm((pg - p_o)[fl]) / np.linalg.norm(p_o[fl])
        assert err <= PARITY, (prec, err)
    T.close()
