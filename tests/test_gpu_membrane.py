"""GPU membrane classification vs the oracle: cut links, sides, ghost entries and their
interpolation rows bit for bit (same lattice predicates, same FP64 evaluation order)."""
import numpy as np
import pytest

import synth
from oracle import membrane as OM
from oracle.grid import Grid
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _square_plate(x0, x1, y0, y1, z):
    V = np.array([[x0, y0, z], [x1, y0, z], [x1, y1, z], [x0, y1, z]])
    return synth.Mesh(V, np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32), 0)


def _tilted_plate(nq=6):
    m = synth.plate(0.13, chord=0.5, span=0.35, nq_x=nq, nq_y=nq, heave=0.05, pitch_deg=25.0,
                    center=(0.503, 0.491, 0.517))
    c, s = np.cos(0.11), np.sin(0.11)
    R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    return synth.Mesh((m.verts - 0.5) @ R.T + 0.5, m.tris, 0)


def _check(pkg, T, grid, meshes):
    ib_o, G = OM.classify(grid, meshes)
    ex = {k: v.cpu().numpy() for k, v in T.export().items()}
    assert T.membrane and T.nsolid == 0 and T.nfluid == grid.shape[0] * grid.shape[1] * grid.shape[2]
    assert np.array_equal(ex["iblank"], ib_o)
    assert np.array_equal(ex["cut"], G.cut)
    assert np.array_equal(ex["cside"] & ex["cut"], G.cside & G.cut)
    assert T.nghost == len(G) and len(G) > 0
    assert np.array_equal(ex["cell"], G.cell)
    assert np.array_equal(ex["side"], G.side)
    for k, o in (("bi", G.bi), ("ip", G.ip), ("base", G.base), ("flags", G.flags), ("ref", G.ref), ("w", G.w),
                 ("scale", G.scale), ("kappa", G.kappa)):
        assert np.array_equal(ex[k], o), k
    assert np.array_equal(ex["tri"].astype(np.int64), G.tri)


def test_tilted_plate_ragged_stretched(ctx):
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(23, 2.0), synth.faces_uniform(19), synth.faces_tanh(27, 1.5)
    m = [_tilted_plate()]
    T = pkg.Tables(c, xf, yf, zf, m)
    _check(pkg, T, Grid(xf, yf, zf), m)
    T.close()


def test_flat_plate_with_lattice_ties(ctx):
    pkg, c = ctx
    f = synth.faces_uniform(32)
    m = [_square_plate(0.25, 0.75, 0.25, 0.75, 0.5)]
    T = pkg.Tables(c, f, f, f, m)
    _check(pkg, T, Grid(f, f, f), m)
    T.close()


def test_flapping_plate_phases_and_reclassify(ctx):
    pkg, c = ctx
    f = synth.faces_tanh(40, 2.0)
    grid = Grid(f, f, f)
    phases = [[synth.plate(q / 8, nq_x=12, nq_y=8)] for q in (0, 3)]
    T = pkg.Tables(c, f, f, f, phases[0])
    _check(pkg, T, grid, phases[0])
    T.reclassify(phases[1])
    _check(pkg, T, grid, phases[1])
    T.close()


def test_membranes_are_not_mixed_with_closed_bodies(ctx):
    pkg, c = ctx
    f = synth.faces_uniform(16)
    with pytest.raises(pkg.IbmError):
        pkg.Tables(c, f, f, f, [_tilted_plate(), synth.octa_sphere(3, (0.5, 0.5, 0.2), 0.1)])


# ----------------------------------------------------------------------------- solves

TOL = 1e-10
PARITY = 1e-8


def _solve_parity(pkg, c, xf, yf, zf, meshes, seed, T=None):
    grid = Grid(xf, yf, zf)
    _, G = OM.classify(grid, meshes)
    b = synth.rhs_divergence(xf, yf, zf, seed)
    p_o, g_o, lam_o = OM.solve_sparse(grid, G, b)
    import torch
    own = T is None
    if own:
        T = pkg.Tables(c, xf, yf, zf, meshes)
    rhs = torch.from_numpy(b).cuda()
    for prec in (0, 1, 2):
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec))
        assert rep["status"] == "IBM_OK" and rep["rel_resid"] <= TOL, (prec, rep)
        pg = p.cpu().numpy()
        err = np.linalg.norm(pg - p_o) / np.linalg.norm(p_o)
        assert err <= PARITY, (prec, err, rep["cycles"])
        assert abs(rep["lambda"] - lam_o) <= 1e-6 * max(1.0, abs(lam_o))
    if own:
        T.close()


def test_membrane_solve_matches_oracle(ctx):
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(24, 2.0), synth.faces_uniform(20), synth.faces_tanh(28, 1.5)
    _solve_parity(pkg, c, xf, yf, zf, [_tilted_plate()], 6)


def test_membrane_reclassified_solves(ctx):
    pkg, c = ctx
    f = synth.faces_tanh(32, 2.0)
    phases = [[synth.plate(q / 8, nq_x=12, nq_y=8)] for q in (1, 5)]
    T = pkg.Tables(c, f, f, f, phases[0])
    _solve_parity(pkg, c, f, f, f, phases[0], 8, T)
    T.reclassify(phases[1])
    _solve_parity(pkg, c, f, f, f, phases[1], 8, T)
    T.close()


def test_krylov_acceleration_on_and_off(ctx):
    """GCR acceleration (automatic for membranes) and plain refinement reach the same
    solution; GCR on a closed body too."""
    pkg, c = ctx
    import torch
    xf, yf, zf = synth.faces_tanh(24, 2.0), synth.faces_uniform(20), synth.faces_tanh(28, 1.5)
    grid = Grid(xf, yf, zf)
    m = [_tilted_plate()]
    _, G = OM.classify(grid, m)
    b = synth.rhs_divergence(xf, yf, zf, 6)
    p_o, _, _ = OM.solve_sparse(grid, G, b)
    T = pkg.Tables(c, xf, yf, zf, m)
    rhs = torch.from_numpy(b).cuda()
    for prec in (0, 1, 2):
        for kr in (0, 3, 8):
            p = torch.zeros_like(rhs)
            rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec, krylov=kr))
            err = np.linalg.norm(p.cpu().numpy() - p_o) / np.linalg.norm(p_o)
            assert rep["status"] == "IBM_OK" and err <= PARITY, (prec, kr, err, rep["cycles"])
    T.close()
    from oracle import classify as OC
    from oracle import solve as OS
    f = synth.faces_tanh(30, 2.0)
    grid = Grid(f, f, f)
    mb = [synth.ellipsoid(4, (0.25, 0.12, 0.1), 33.0, (0.45, 0.5, 0.5))]
    ib, Gc = OC.classify(grid, mb)
    b = synth.rhs_divergence(f, f, f, 7)
    p_o, _ = OS.solve_gmres(grid, ib, Gc, b)
    fl = ib == 0
    T = pkg.Tables(c, f, f, f, mb)
    rhs = torch.from_numpy(b).cuda()
    for prec in (0, 1, 2):
        p = torch.zeros_like(rhs)
        rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec, krylov=4))
        err = np.linalg.norm((p.cpu().numpy() - p_o)[fl]) / np.linalg.norm(p_o[fl])
        assert rep["status"] == "IBM_OK" and err <= PARITY, (prec, err)
    T.close()
