"""Pins of the surface-pressure and nodal-force oracle (Sec. "Force Formulations", pressure
part).

* A linear field p = a + g.x on a convex closed body, with the datum q = g.n: the side
  pressure equals the field at every centroid, and the total force equals Archimedes' closed
  form -g x volume (volume of the polyhedron from signed tetrahedra).
* A grid-aligned membrane with a different linear field on each side (common normal
  derivative): both side pressures exact, total force in closed form.
* A tilted plate with a constant pressure on each side: dp on every triangle, total
  force -dp n A; reversing the triangles' orientation swaps the sides and leaves every nodal
  force unchanged.
* The nodal shares: total force and moment about the origin of the nodal forces equal those
  of the triangle forces applied at the centroids.
* The rigid-body datum: q = -a(c).n against second differences of the moving plate's own
  centroids.
* Planted mistakes (the datum term dropped or with the wrong sign) fail the first pin.
"""
import numpy as np

import synth
from oracle import classify as OC
from oracle import forces as OF
from oracle import membrane as OM
from oracle.grid import Grid

A0 = 0.37
G = np.array([0.7, -1.3, 2.1])


def _cells(grid):
    nz, ny, nx = grid.shape
    return grid.centre(np.arange(nz * ny * nx))


def _volume(V, T):
    v0, v1, v2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", v0, np.cross(v1, v2)))) / 6.0


def _convex_case():
    grid = Grid(synth.faces_tanh(30, 2.0), synth.faces_uniform(26), synth.faces_tanh(28, 1.5))
    mesh = synth.ellipsoid(3, (0.22, 0.15, 0.13), 23.0, (0.49, 0.51, 0.5))
    V, T = mesh.verts, mesh.tris.astype(np.int64)
    # convex: every vertex on the inner side of every triangle's plane
    N, a2, n, c = OF.triangle_geometry(V, T)
    assert np.max(np.einsum("tvk,tk->tv", V[None] - c[:, None], n)) < 1e-12
    ib = OC.iblank_closed(grid, [mesh])
    return grid, ib, mesh, n, c


def test_linear_field_on_convex_body_and_archimedes():
    grid, ib, mesh, n, c = _convex_case()
    p = (A0 + _cells(grid) @ G).reshape(grid.shape)
    q = n @ G
    ps, flags, F = OF.surface_forces(grid, ib, [mesh], p, q=q)
    assert np.all(flags == 0)
    exact = A0 + c @ G
    assert np.max(np.abs(ps[:, 0] - exact)) < 1e-12 * np.max(np.abs(exact))
    assert np.all(ps[:, 1] == 0.0)
    vol = _volume(mesh.verts, mesh.tris.astype(np.int64))
    assert vol > 0.0
    assert np.allclose(F.sum(axis=0), -G * vol, rtol=1e-12, atol=1e-13 * np.abs(G).max() * vol)
    # constant pressure: no net force on a closed surface
    ps0, _, F0 = OF.surface_forces(grid, ib, [mesh], np.full(grid.shape, 3.0))
    area = 0.5 * float(np.sum(np.linalg.norm(OF.triangle_geometry(mesh.verts, mesh.tris)[0], axis=1)))
    assert np.max(np.abs(F0.sum(axis=0))) < 1e-14 * 3.0 * area * 100


def test_planted_datum_mistakes_fail():
    grid, ib, mesh, n, c = _convex_case()
    p = (A0 + _cells(grid) @ G).reshape(grid.shape)
    exact = A0 + c @ G
    q = n @ G
    for wrong in (None, -q):                      # datum term dropped / sign flipped
        ps, _, _ = OF.surface_forces(grid, ib, [mesh], p, q=wrong)
        assert np.max(np.abs(ps[:, 0] - exact)) > 1e-3


def test_grid_aligned_membrane_linear_fields():
    n = 24
    f = synth.faces_uniform(n)
    grid = Grid(f, f, f)
    z0 = 0.5 + 0.2 / n                            # between two centre planes
    mesh = synth.plate(0.0, chord=0.4, span=0.3, nq_x=8, nq_y=6, heave=0.0, pitch_deg=0.0,
                       center=(0.5, 0.5, z0))
    q0 = 0.9
    g1, g2 = np.array([0.3, -0.7, q0]), np.array([-1.1, 0.4, q0])
    a1, a2 = 1.25, -0.5
    X = _cells(grid)
    above = X[:, 2] > z0
    p = np.where(above, a1 + X @ g1, a2 + X @ g2).reshape(grid.shape)
    V, T = mesh.verts, mesh.tris.astype(np.int64)
    N, a2n, nn, c = OF.triangle_geometry(V, T)
    assert np.allclose(nn, [0.0, 0.0, 1.0])
    ps, flags, F = OF.surface_forces(grid, None, [mesh], p, q=np.full(T.shape[0], q0))
    assert np.all(flags == 0)
    assert np.max(np.abs(ps[:, 0] - (a1 + c @ g1))) < 1e-12
    assert np.max(np.abs(ps[:, 1] - (a2 + c @ g2))) < 1e-12
    area = 0.4 * 0.3
    xbar = np.array([0.5, 0.5, z0])
    Fz = -((a1 - a2) + (g1 - g2) @ xbar) * area
    assert np.allclose(F.sum(axis=0), [0.0, 0.0, Fz], rtol=1e-12, atol=1e-13)


def _tilted_plate():
    m = synth.plate(0.13, chord=0.45, span=0.3, nq_x=7, nq_y=5, heave=0.04, pitch_deg=25.0,
                    center=(0.503, 0.491, 0.517))
    c, s = np.cos(0.3), np.sin(0.3)
    R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    return synth.Mesh((m.verts - 0.5) @ R.T + 0.5, m.tris, 0)


def test_tilted_plate_constant_jump_and_orientation():
    grid = Grid(synth.faces_tanh(28, 2.0), synth.faces_uniform(25), synth.faces_tanh(27, 1.5))
    mesh = _tilted_plate()
    V, T = mesh.verts, mesh.tris.astype(np.int64)
    N, a2, n, c = OF.triangle_geometry(V, T)
    nhat = n[0]
    assert np.allclose(n, nhat, atol=1e-14)       # flat
    P0 = V.mean(axis=0)
    a1, a2c = 2.5, -0.75
    X = _cells(grid)
    p = np.where((X - P0) @ nhat > 0.0, a1, a2c).reshape(grid.shape)
    ps, flags, F = OF.surface_forces(grid, None, [mesh], p)
    assert np.all(flags == 0)
    assert np.max(np.abs(ps - [a1, a2c])) < 1e-14        # (sum w a) / (sum w) = a up to rounding
    area = 0.45 * 0.3
    assert np.allclose(F.sum(axis=0), -(a1 - a2c) * area * nhat, rtol=1e-12, atol=1e-14)
    flipped = synth.Mesh(V, T[:, [0, 2, 1]].astype(np.int32), 0)
    ps2, _, F2 = OF.surface_forces(grid, None, [flipped], p)
    # the centroid's sum order changes with the vertex order: equal up to rounding
    assert np.max(np.abs(ps2[:, [1, 0]] - ps)) < 1e-14
    assert np.max(np.abs(F2 - F)) < 1e-14 * np.abs(F).max()


def test_nodal_shares_keep_force_and_moment():
    grid = Grid(synth.faces_tanh(24, 2.0), synth.faces_uniform(22), synth.faces_uniform(23))
    rng = np.random.default_rng(3)
    meshes = [synth.octa_sphere(2, (0.3, 0.5, 0.5), 0.12), synth.ellipsoid(2, (0.14, 0.08, 0.08), 30.0, (0.7, 0.5, 0.5))]
    ib = OC.iblank_closed(grid, meshes)
    p = rng.standard_normal(grid.shape)
    ps, flags, F = OF.surface_forces(grid, ib, meshes, p)
    V, T, _ = OF.concat_meshes(meshes)
    N, a2, n, c = OF.triangle_geometry(V, T)
    f = -((ps[:, 0] - ps[:, 1])[:, None] * (0.5 * N))
    scale = np.abs(f).sum()
    assert np.allclose(F.sum(axis=0), f.sum(axis=0), rtol=0, atol=1e-14 * scale)
    assert np.allclose(np.cross(V, F).sum(axis=0), np.cross(c, f).sum(axis=0), rtol=0, atol=1e-14 * scale)
    # a node index mistake (shares sent to the wrong corner) breaks the moment identity
    Fw = np.zeros_like(F)
    for t in range(T.shape[0]):
        for k in range(3):
            Fw[T[t, (k + 1) % 3] if k == 0 else T[t, k]] += f[t] / 3.0
    assert np.abs(np.cross(V, Fw).sum(axis=0) - np.cross(c, f).sum(axis=0)).max() > 1e-6 * scale


def test_rigid_datum_against_second_differences():
    t, dt = 0.3, 1e-4
    m0, mp, mm = synth.plate(t, nq_x=4, nq_y=3), synth.plate(t + dt, nq_x=4, nq_y=3), synth.plate(t - dt, nq_x=4, nq_y=3)
    T = m0.tris.astype(np.int64)
    _, _, n, c0 = OF.triangle_geometry(m0.verts, T)
    cp = OF.triangle_geometry(mp.verts, T)[3]
    cm = OF.triangle_geometry(mm.verts, T)[3]
    acc = (cp - 2.0 * c0 + cm) / (dt * dt)
    q = OF.rigid_q(c0, n, [0, T.shape[0]], synth.plate_motion(t))
    assert np.allclose(q, -np.einsum("ij,ij->i", acc, n), rtol=1e-5, atol=1e-5 * np.abs(acc).max())


def test_zero_area_triangle_is_flagged_and_carries_no_force():
    """A degenerate (zero-area) triangle appended to a membrane: flag bit 2, side pressures 0,
    and every nodal force equal to the mesh without it."""
    grid = Grid(synth.faces_tanh(24, 2.0), synth.faces_uniform(22), synth.faces_uniform(23))
    mesh = _tilted_plate()
    V = np.concatenate([mesh.verts, mesh.verts[:1] + 0.01])
    T = np.concatenate([mesh.tris, [[0, 0, V.shape[0] - 1]]]).astype(np.int32)
    deg = synth.Mesh(V, T, 0)
    p = synth.smooth_field(grid.xf, grid.yf, grid.zf, 4)
    ps, flags, F = OF.surface_forces(grid, None, [mesh], p)
    ps2, flags2, F2 = OF.surface_forces(grid, None, [deg], p)
    assert flags2[-1] == OF.FLAG_ZERO_AREA and np.all(ps2[-1] == 0.0)
    assert np.array_equal(flags2[:-1], flags) and np.array_equal(ps2[:-1], ps)
    assert np.array_equal(F2[:-1], F) and np.all(F2[-1] == 0.0)


def test_tilted_plate_linear_fields_each_side():
    """A tilted plate with p = a1 + g1.x above and a2 + g2.x below its plane (common normal
    derivative q = g.n): every probe box lies on its own side, so both side pressures equal the
    fields at the centroids (the plane test, the probe offset and the datum together)."""
    grid = Grid(synth.faces_tanh(30, 2.0), synth.faces_uniform(27), synth.faces_tanh(29, 1.5))
    mesh = _tilted_plate()
    V, T = mesh.verts, mesh.tris.astype(np.int64)
    N, a2, n, c = OF.triangle_geometry(V, T)
    nhat = n[0]
    P0 = V.mean(axis=0)
    q0 = 0.6
    t1, t2 = np.cross(nhat, [1.0, 0.0, 0.0]), np.cross(nhat, [0.0, 1.0, 0.0])
    g1 = q0 * nhat + 0.8 * t1 - 0.3 * t2
    g2 = q0 * nhat - 0.5 * t1 + 1.1 * t2
    X = _cells(grid)
    above = (X - P0) @ nhat > 0.0
    p = np.where(above, 1.5 + X @ g1, -0.25 + X @ g2).reshape(grid.shape)
    ps, flags, F = OF.surface_forces(grid, None, [mesh], p, q=n @ g1)
    assert np.all(flags == 0)
    assert np.allclose(n @ g1, n @ g2, atol=1e-14)
    assert np.max(np.abs(ps[:, 0] - (1.5 + c @ g1))) < 1e-12
    assert np.max(np.abs(ps[:, 1] - (-0.25 + c @ g2))) < 1e-12
