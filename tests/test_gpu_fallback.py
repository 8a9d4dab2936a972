"""Fallback ghost rows on the GPU: two closed bodies whose surfaces cut through each other
give ghosts whose image points land deep in solid; those rows take the fluid face-neighbour
nearest to the image point.  Tables bit-exact against the oracle; solves within 1e-8 of the
oracle's in every precision mode, without and with a moving-boundary datum."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import solve as OS
from oracle.grid import Grid
from tests.gpu_util import assert_tables_equal, require_gpu, torch

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


@pytest.mark.parametrize("n,zc", [(24, 0.47), (32, 0.5)])
def test_fallback_rows_bit_exact_and_solved(ctx, n, zc):
    pkg, c = ctx
    f = synth.faces_uniform(n)
    meshes = synth.overlapping_bodies(zc)
    g = Grid(f, f, f)
    ib, G = OC.classify(g, meshes)
    assert np.sum((G.flags & OC.FLAG_FALLBACK) != 0) >= 8
    T = pkg.Tables(c, f, f, f, meshes)
    ex = {k: v.cpu().numpy() for k, v in T.export().items()}
    assert_tables_equal(ex, ib, G)
    b = synth.rhs_divergence(f, f, f, 13)
    rhs = torch.from_numpy(b).cuda()
    fl = ib == 0
    for with_datum in (False, True):
        if with_datum:
            q = np.random.default_rng(17).standard_normal(len(G))
            OC.set_neumann(G, q)
            T.set_neumann(torch.from_numpy(q).cuda())
            assert np.array_equal(T.export()["d"].cpu().numpy(), G.kappa * q)
        p_o, lam_o = OS.solve_sparse(g, ib, G, b)
        for prec in (0, 1, 2):
            p = torch.zeros_like(rhs)
            rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))
            pg = p.cpu().numpy()
            err = np.linalg.norm((pg - p_o)[fl]) / np.linalg.norm(p_o[fl])
            assert rep["status"] == "IBM_OK" and err <= PARITY, (with_datum, prec, err, rep)
            gerr = np.max(np.abs(pg.ravel()[G.cell] - p_o.ravel()[G.cell])) / np.max(np.abs(p_o[fl]))
            assert gerr <= 10 * PARITY
    T.close()
