"""Surface pressure and nodal pressure forces on the GPU against the oracle (bit for bit on
the same cell pressures): closed bodies and membranes, with a per-triangle datum and with
rigid kinematics; forces of a solved pressure field; the flapping plate at 512^3; argument
errors."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import forces as OF
from oracle import membrane as OM
from oracle.grid import Grid
from tests.gpu_util import require_gpu, torch
from tests.test_gpu_neumann import _rigid_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _compare(out, ps, flags, F):
    assert np.array_equal(out["flags"].cpu().numpy().astype(np.int32), flags)
    assert np.array_equal(out["p_side"].cpu().numpy(), ps)
    assert np.array_equal(out["f_node"].cpu().numpy(), F)


def _tilted_plate(t=0.13, nq_x=9, nq_y=6):
    m = synth.plate(t, chord=0.45, span=0.3, nq_x=nq_x, nq_y=nq_y, heave=0.04, pitch_deg=25.0,
                    center=(0.503, 0.491, 0.517))
    c, s = np.cos(0.3), np.sin(0.3)
    R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    return synth.Mesh((m.verts - 0.5) @ R.T + 0.5, m.tris, 0)


def test_closed_bodies_bit_exact(ctx):
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(40, 2.0), synth.faces_uniform(36), synth.faces_tanh(38, 1.5)
    grid = Grid(xf, yf, zf)
    meshes = [synth.octa_sphere(3, (0.3, 0.5, 0.5), 0.12), synth.ellipsoid(3, (0.14, 0.08, 0.08), 30.0, (0.7, 0.5, 0.5)),
              synth.box_mesh((0.42, 0.2, 0.2), (0.58, 0.3, 0.33))]
    ib = OC.iblank_closed(grid, meshes)
    p = synth.smooth_field(xf, yf, zf, 7) + synth.counter_normal(8, 0, np.arange(grid.nx * grid.ny * grid.nz)).reshape(grid.shape)
    T = pkg.Tables(c, xf, yf, zf, meshes)
    assert np.array_equal(T.export()["iblank"].cpu().numpy() & 1, ib & 1)
    pd = torch.from_numpy(p).cuda()
    ntri = sum(m.ntris for m in meshes)
    q = synth.counter_normal(9, 0, np.arange(ntri))
    motions = np.array([[0.3, -0.2, 1.1, 0.5, -0.7, 0.2, 1.3, 0.4, -0.9, 0.3, 0.5, 0.5],
                        [-1.0, 0.6, 0.0, 0.0, 2.0, -1.0, 0.2, -1.5, 0.7, 0.7, 0.5, 0.5],
                        [0.0, 0.0, 0.5, 1.0, 0.0, 0.0, 0.0, 0.0, 0.3, 0.5, 0.25, 0.26]])
    for kw_o, kw_g in (({}, {}), ({"q": q}, {"q": torch.from_numpy(q).cuda()}),
                       ({"motions": motions}, {"motions": motions})):
        ps, flags, F = OF.surface_forces(grid, ib, meshes, p, **kw_o)
        _compare(T.surface_forces(meshes, pd, **kw_g), ps, flags, F)
    T.close()


def test_membrane_bit_exact(ctx):
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(44, 2.0), synth.faces_uniform(40), synth.faces_tanh(42, 1.5)
    grid = Grid(xf, yf, zf)
    meshes = [_tilted_plate()]
    p = synth.smooth_field(xf, yf, zf, 11)
    T = pkg.Tables(c, xf, yf, zf, meshes)
    pd = torch.from_numpy(p).cuda()
    motions = synth.plate_motion(0.13)[None]
    for kw in ({}, {"motions": motions}):
        ps, flags, F = OF.surface_forces(grid, None, meshes, p, **kw)
        _compare(T.surface_forces(meshes, pd, **kw), ps, flags, F)
    # moved vertices, same topology (the forces follow the mesh, not the classification)
    moved = [_tilted_plate(0.2)]
    ps, flags, F = OF.surface_forces(grid, None, moved, p)
    _compare(T.surface_forces(moved, pd), ps, flags, F)
    T.close()


def test_forces_of_a_solved_membrane_pressure(ctx):
    """The oracle's solution through both force paths (bit for bit), and the GPU solve's
    forces against the oracle's (the solve's parity bar carries over)."""
    pkg, c = ctx
    f = synth.faces_tanh(30, 2.0)
    grid = Grid(f, f, f)
    meshes = [synth.plate(0.3, nq_x=10, nq_y=6)]
    _, G = OM.classify(grid, meshes)
    b = synth.rhs_divergence(f, f, f, 4)
    motions = synth.plate_motion(0.3)[None]
    G.d = _rigid_oracle(grid, G, [0, meshes[0].ntris], motions)
    p_o, _, _ = OM.solve_sparse(grid, G, b)
    T = pkg.Tables(c, f, f, f, meshes)
    T.neumann_rigid(motions)
    ps, flags, F = OF.surface_forces(grid, None, meshes, p_o.reshape(grid.shape), motions=motions)
    _compare(T.surface_forces(meshes, torch.from_numpy(p_o).cuda(), motions=motions), ps, flags, F)
    rhs = torch.from_numpy(b).cuda()
    p = torch.zeros_like(rhs)
    rep = T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=2))
    assert rep["status"] == "IBM_OK"
    out = T.surface_forces(meshes, p, motions=motions)
    Fg = out["f_node"].cpu().numpy()
    assert np.linalg.norm(Fg - F) <= 1e-6 * np.linalg.norm(F)
    T.close()


def test_flapping_plate_512(ctx):
    """The benchmark's membrane workload: 512^3 stretched grid, 20 000-triangle plate."""
    pkg, c = ctx
    n = 512
    f = synth.faces_tanh(n, 2.0)
    grid = Grid(f, f, f)
    meshes = [synth.plate(0.375)]
    p = synth.smooth_field(f, f, f, 5)
    T = pkg.Tables(c, f, f, f, meshes)
    motions = synth.plate_motion(0.375)[None]
    ps, flags, F = OF.surface_forces(grid, None, meshes, p, motions=motions)
    _compare(T.surface_forces(meshes, torch.from_numpy(p).cuda(), motions=motions), ps, flags, F)
    T.close()


def test_argument_errors(ctx):
    pkg, c = ctx
    f = synth.faces_uniform(20)
    meshes = [synth.octa_sphere(2, (0.5, 0.5, 0.5), 0.2)]
    T = pkg.Tables(c, f, f, f, meshes)
    pd = torch.zeros((20, 20, 20), dtype=torch.float64, device="cuda")
    ntri = meshes[0].ntris
    with pytest.raises(pkg.IbmError):           # a datum and kinematics together
        T.surface_forces(meshes, pd, q=torch.zeros(ntri, dtype=torch.float64, device="cuda"),
                         motions=np.zeros((1, 12)))
    with pytest.raises(pkg.IbmError):           # not the classified meshes
        T.surface_forces([synth.octa_sphere(1, (0.5, 0.5, 0.5), 0.2)], pd)
    with pytest.raises(pkg.IbmError):           # a membrane against closed-body tables
        T.surface_forces([synth.Mesh(meshes[0].verts, meshes[0].tris, 0)], pd)
    out = T.surface_forces(meshes, pd)
    assert float(out["f_node"].abs().max()) == 0.0
    T.close()
