"""Moving-boundary Neumann datum on the GPU against the oracle: ghost-row data kappa q in
every precision mode, single and batched, closed bodies and membranes; the rigid-body data
against the kinematics written out; classification clears the data."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import membrane as OM
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


def _closed():
    xf, yf, zf = synth.faces_tanh(26, 2.0), synth.faces_uniform(22), synth.faces_tanh(24, 1.5)
    return xf, yf, zf, [synth.ellipsoid(4, (0.21, 0.13, 0.12), 23.0, (0.49, 0.51, 0.5))]


def _membrane():
    f = synth.faces_tanh(26, 2.0)
    return f, f, f, [synth.plate(0.3, nq_x=10, nq_y=6)]


def test_closed_body_datum_matches_oracle(ctx):
    pkg, c = ctx
    xf, yf, zf, meshes = _closed()
    grid = Grid(xf, yf, zf)
    ib, G = OC.classify(grid, meshes)
    b = synth.rhs_divergence(xf, yf, zf, 3)
    q = np.random.default_rng(11).standard_normal(len(G))
    OC.set_neumann(G, q)
    p_o, lam_o = OS.solve_sparse(grid, ib, G, b)
    fl = ib == 0
    T = pkg.Tables(c, xf, yf, zf, meshes)
    T.set_neumann(torch.from_numpy(q).cuda())
    assert np.array_equal(T.export()["d"].cpu().numpy(), G.kappa * q)
    rhs = torch.from_numpy(b).cuda()
    for prec in (0, 1, 2):
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))
        pg = p.cpu().numpy()
        err = np.linalg.norm((pg - p_o)[fl]) / np.linalg.norm(p_o[fl])
        assert rep["status"] == "IBM_OK" and err <= PARITY, (prec, err)
        assert abs(rep["lambda"] - lam_o) <= 1e-6 * max(1.0, abs(lam_o))
    # the same problem batched with a datum-free copy of itself
    F = pkg.Tables(c, xf, yf, zf, meshes)
    ps = [torch.zeros_like(rhs), torch.zeros_like(rhs)]
    status, _ = pkg.poisson_solve_batched(c.h, [T.h, F.h], [rhs, rhs], TOL, ps, pkg.SolveOpts(precision=2))
    assert status == "IBM_OK"
    assert np.linalg.norm((ps[0].cpu().numpy() - p_o)[fl]) / np.linalg.norm(p_o[fl]) <= PARITY
    OC.set_neumann(G, np.zeros(len(G)))
    p_z, _ = OS.solve_sparse(grid, ib, G, b)
    assert np.linalg.norm((ps[1].cpu().numpy() - p_z)[fl]) / np.linalg.norm(p_z[fl]) <= PARITY
    F.close()
    T.close()


def test_membrane_datum_matches_oracle(ctx):
    pkg, c = ctx
    xf, yf, zf, meshes = _membrane()
    grid = Grid(xf, yf, zf)
    _, G = OM.classify(grid, meshes)
    b = synth.rhs_divergence(xf, yf, zf, 4)
    q = np.random.default_rng(12).standard_normal(len(G))
    OC.set_neumann(G, q)
    p_o, g_o, lam_o = OM.solve_sparse(grid, G, b)
    T = pkg.Tables(c, xf, yf, zf, meshes)
    T.set_neumann(torch.from_numpy(q).cuda())
    rhs = torch.from_numpy(b).cuda()
    for prec in (0, 1, 2):
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))
        err = np.linalg.norm(p.cpu().numpy() - p_o) / np.linalg.norm(p_o)
        assert rep["status"] == "IBM_OK" and err <= PARITY, (prec, err, rep["cycles"])
    T.close()


def _rigid_oracle(grid, G, tri_off, motions):
    """d = kappa q, q = -a(BI).n for rigid kinematics (written out with numpy)."""
    nz, ny, nx = grid.shape
    m = np.searchsorted(np.asarray(tri_off), G.tri, side="right") - 1
    M = np.asarray(motions, dtype=np.float64).reshape(-1, 12)[m]
    a0, al, om, cen = M[:, 0:3], M[:, 3:6], M[:, 6:9], M[:, 9:12]
    r = G.bi - cen
    a = a0 + np.cross(al, r) + np.cross(om, np.cross(om, r))
    GC = grid.centre(G.cell)
    t = G.ip - GC
    fb = (G.flags & OC.FLAG_FALLBACK) != 0
    if fb.any():
        nb = G.ref[fb, 0]
        t[fb] = np.stack([grid.xc[nb % nx], grid.yc[(nb // nx) % ny], grid.zc[nb // (nx * ny)]], -1) - GC[fb]
    q = -np.sum(a * t, axis=1) / np.linalg.norm(t, axis=1)
    return G.kappa * q


def test_rigid_datum_matches_kinematics(ctx):
    pkg, c = ctx
    f = synth.faces_tanh(28, 2.0)
    grid = Grid(f, f, f)
    meshes = [synth.octa_sphere(3, (0.35, 0.5, 0.5), 0.12), synth.ellipsoid(3, (0.15, 0.08, 0.08), 30.0, (0.68, 0.5, 0.5))]
    ib, G = OC.classify(grid, meshes)
    motions = np.array([[0.3, -0.2, 1.1, 0.5, -0.7, 0.2, 1.3, 0.4, -0.9, 0.35, 0.5, 0.5],
                        [-1.0, 0.6, 0.0, 0.0, 2.0, -1.0, 0.2, -1.5, 0.7, 0.68, 0.5, 0.5]])
    tri_off = [0, meshes[0].tris.shape[0], meshes[0].tris.shape[0] + meshes[1].tris.shape[0]]
    d_o = _rigid_oracle(grid, G, tri_off, motions)
    T = pkg.Tables(c, f, f, f, meshes)
    T.neumann_rigid(motions)
    d = T.export()["d"].cpu().numpy()
    assert np.abs(d_o).max() > 1e-3
    assert np.allclose(d, d_o, rtol=1e-12, atol=1e-14 * np.abs(d_o).max())
    with pytest.raises(pkg.IbmError):
        T.neumann_rigid(motions[:1])               # one motion per mesh
    T.close()


def test_classification_clears_the_datum(ctx):
    pkg, c = ctx
    xf, yf, zf, meshes = _closed()
    b = synth.rhs_divergence(xf, yf, zf, 5)
    rhs = torch.from_numpy(b).cuda()
    T = pkg.Tables(c, xf, yf, zf, meshes)
    p0 = torch.zeros_like(rhs)
    T.solve(rhs, p0, TOL, pkg.SolveOpts(precision=2))
    T.set_neumann(torch.ones(T.nghost, dtype=torch.float64, device="cuda"))
    p1 = torch.zeros_like(rhs)
    T.solve(rhs, p1, TOL, pkg.SolveOpts(precision=2))
    assert float((p1 - p0).norm()) > 1e-6 * float(p0.norm())
    T.reclassify(meshes)
    assert float(T.export()["d"].abs().max()) == 0.0
    p2 = torch.zeros_like(rhs)
    T.solve(rhs, p2, TOL, pkg.SolveOpts(precision=2))
    assert torch.equal(p2, p0)
    T.set_neumann(None)
    T.close()
