"""Failure paths through the C ABI, made on the host (no GPU fault): a closed mesh with a hole
(IBM_ERR_MESH_NOT_CLOSED, the same rule as the oracle's), and a right-hand side or initial
guess holding NaN or Inf (IBM_ERR_DIVERGED before any cycle, in every precision mode and
batched).  After each failure the context keeps working."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle.grid import Grid
from tests.gpu_util import assert_tables_equal, require_gpu, torch

pytestmark = pytest.mark.gpu
MESH_NOT_CLOSED = 10
DIVERGED = "IBM_ERR_DIVERGED"


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _leaky():
    f = synth.faces_tanh(24, 1.5)
    xf, yf, zf = f, synth.faces_uniform(22), f
    whole = synth.octa_sphere(2, (0.5, 0.5, 0.5), 0.36)
    g = Grid(xf, yf, zf)
    cz = whole.verts[whole.tris].mean(axis=1)[:, 2]
    for t in np.argsort(-cz):
        leaky = synth.Mesh(whole.verts, np.delete(whole.tris, t, axis=0), 1)
        if OC.odd_columns(g, leaky.verts, leaky.tris).shape[0] > 0:
            return xf, yf, zf, whole, leaky
    raise AssertionError("no triangle of the upper half lies over a column")


def test_leaky_mesh_is_refused_like_the_oracle(ctx):
    pkg, c = ctx
    xf, yf, zf, whole, leaky = _leaky()
    g = Grid(xf, yf, zf)
    with pytest.raises(OC.MeshNotClosed):
        OC.iblank_closed(g, [leaky])
    with pytest.raises(pkg.IbmError) as e:
        pkg.Tables(c, xf, yf, zf, [leaky])
    assert e.value.status == MESH_NOT_CLOSED
    # reclassification of existing tables refuses it too; the same tables then take the
    # watertight mesh again, bit-exact against the oracle
    T = pkg.Tables(c, xf, yf, zf, [whole])
    with pytest.raises(pkg.IbmError) as e:
        T.reclassify([leaky])
    assert e.value.status == MESH_NOT_CLOSED
    T.reclassify([whole])
    ib, G = OC.classify(g, [whole])
    ex = {k: v.cpu().numpy() for k, v in T.export().items()}
    assert_tables_equal(ex, ib, G)
    T.close()


def test_body_above_the_top_centre_is_watertight(ctx):
    """Crossings above the last cell centre count: a sphere poking through the top of the
    grid is classified, bit-exact against the oracle."""
    pkg, c = ctx
    f = synth.faces_tanh(24, 1.5)
    m = synth.octa_sphere(3, (0.47, 0.52, 0.93), 0.2)
    g = Grid(f, synth.faces_uniform(22), f)
    ib, G = OC.classify(g, [m])
    T = pkg.Tables(c, f, synth.faces_uniform(22), f, [m])
    ex = {k: v.cpu().numpy() for k, v in T.export().items()}
    assert_tables_equal(ex, ib, G)
    T.close()


@pytest.mark.parametrize("bad", ["nan_rhs", "inf_rhs", "nan_guess"])
def test_non_finite_input_diverges_before_any_cycle(ctx, bad):
    pkg, c = ctx
    f = synth.faces_tanh(20, 2.0)
    m = [synth.octa_sphere(3, (0.5, 0.5, 0.5), 0.2)]
    T = pkg.Tables(c, f, f, f, m)
    b = synth.rhs_divergence(f, f, f, 9)
    ib = T.export()["iblank"].cpu().numpy()
    fl = np.flatnonzero(ib.ravel() == 0)
    cell = fl[fl.size // 3]
    rhs = torch.from_numpy(b).cuda()
    good = rhs.clone()
    p0 = torch.zeros_like(rhs)
    if bad == "nan_rhs":
        rhs.view(-1)[cell] = float("nan")
    elif bad == "inf_rhs":
        rhs.view(-1)[cell] = float("inf")
    else:
        p0.view(-1)[cell] = float("nan")
    for prec in (0, 1, 2):
        p = p0.clone()
        rep = T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=prec), raise_on_error=False)
        assert rep["status"] == DIVERGED and rep["cycles"] == 0, (prec, rep)
    status, reps = pkg.poisson_solve_batched(c.h, [T.h], [rhs], 1e-10, [p0.clone()], pkg.SolveOpts(precision=1),
                                             raise_on_error=False)
    assert status == DIVERGED and reps[0]["cycles"] == 0
    # the context and tables keep working
    p = torch.zeros_like(rhs)
    rep = T.solve(good, p, 1e-10, pkg.SolveOpts(precision=1))
    assert rep["status"] == "IBM_OK" and torch.isfinite(p).all()
    T.close()


def test_sweep_wait_that_runs_out_reports_timeout(ctx):
    """The fused sweep's first bounded wait given zero tries: every item gives up at once,
    drains its copies in flight and returns; the solve reports IBM_ERR_TIMEOUT and the context
    then solves normally again (graph and direct launches)."""
    pkg, c = ctx
    f = synth.faces_tanh(72, 2.0)
    m = [synth.octa_sphere(3, (0.5, 0.5, 0.5), 0.2)]
    T = pkg.Tables(c, f, f, f, m)
    rhs = torch.from_numpy(synth.rhs_divergence(f, f, f, 19)).cuda()
    for graph in (0, 1):
        pkg.ibm_ctx_set_sweep_wait_limit(c.h, 0)
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=2, max_cycles=2, use_graph=graph), raise_on_error=False)
        assert rep["status"] == "IBM_ERR_TIMEOUT", rep
        pkg.ibm_ctx_set_sweep_wait_limit(c.h, -1)
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=2, use_graph=graph))
        assert rep["status"] == "IBM_OK" and rep["rel_resid"] <= 1e-10
    T.close()
