"""Pins of the oracle's iblanking, ghost cells, image points and weights.

Each check is independent of the code under test: an exact winding number by
a different ray, analytic inside/outside sets, the optimality condition of a
projection onto a convex set, a closed-form plane reflection and exact
reproduction of linear fields.
"""
import math

import numpy as np
import pytest

import synth
from oracle import classify as C
from oracle.grid import Grid


# ----------------------------------------------------------------------------- helpers

def _rot(ax, ay, az):
    cx, sx, cy, sy, cz, sz = math.cos(ax), math.sin(ax), math.cos(ay), math.sin(ay), math.cos(az), math.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _winding_inside(grid, mesh, rng, skip=None):
    """Exact winding number by a generic integer ray (signed crossings), int64 exact.

    Returns a boolean [k][j][i] (winding != 0), or None if a point lies on the
    surface along every ray tried (not expected for the inputs used here).
    """
    Xc, Yc, Zc = C.snap(grid.xc), C.snap(grid.yc), C.snap(grid.zc)
    Q = np.stack(np.meshgrid(Xc, Yc, Zc, indexing="ij"), -1).transpose(2, 1, 0, 3).reshape(-1, 3)
    V = C.snap(mesh.verts)
    A, B, Cc = V[mesh.tris[:, 0]], V[mesh.tris[:, 1]], V[mesh.tris[:, 2]]
    e1, e2 = B - A, Cc - A
    keep = np.ones(Q.shape[0], dtype=bool) if skip is None else ~skip.ravel()
    Q = Q[keep]
    for _ in range(8):
        d = rng.integers(-31, 32, size=3)
        d[2] = d[2] if d[2] != 0 else 17
        e2xd = np.cross(e2, d)                               # |.| <= 2^33
        det = -np.einsum("ij,ij->i", e1, e2xd)               # |.| <= 2^62
        wind = np.zeros(Q.shape[0], dtype=np.int64)
        degenerate = False
        for s0 in range(0, Q.shape[0], 512):
            s = Q[s0:s0 + 512, None, :] - A[None]            # (P, T, 3)
            # Cramer: M [u v t]^T = s with M = [e1 e2 -d]
            du = -np.einsum("ptk,tk->pt", s, e2xd)
            e1xs = np.cross(e1[None], s)
            dv = np.einsum("ptk,k->pt", e1xs, -d)
            sg = np.sign(det)[None]
            u, v, D = du * sg, dv * sg, np.abs(det)[None]
            valid = D > 0
            inproj = valid & (u >= 0) & (v >= 0) & (u + v <= D)
            # t = [e1, e2, s] / det is cubic in the coordinates: exact Python integers,
            # only for the few (point, triangle) pairs whose projection test passes
            pp, tt = np.nonzero(inproj)
            tsign = np.zeros(pp.size, dtype=np.int64)
            for a, (p_, t_) in enumerate(zip(pp.tolist(), tt.tolist())):
                nrm = [int(x) for x in np.cross(e1[t_], e2[t_])]
                sv = [int(x) for x in s[p_, t_]]
                val = (nrm[0] * sv[0] + nrm[1] * sv[1] + nrm[2] * sv[2]) * int(sg[0, t_])
                tsign[a] = (val > 0) - (val < 0)
            strict = (u[pp, tt] > 0) & (v[pp, tt] > 0) & (u[pp, tt] + v[pp, tt] < D[0, tt])
            if np.any(tsign == 0) or np.any(~strict & (tsign >= 0)):
                degenerate = True
                break
            hit = np.zeros(inproj.shape, dtype=bool)
            hit[pp[tsign > 0], tt[tsign > 0]] = True
            wind[s0:s0 + 512] = np.sum(np.where(hit, np.sign(det)[None], 0), axis=1)
        if not degenerate:
            out = np.zeros(keep.size, dtype=bool)
            out[keep] = wind != 0
            return out.reshape(grid.shape)
    return None


def _rotated_mesh(mesh, R, centre):
    c = mesh.verts.mean(axis=0)
    return synth.Mesh((mesh.verts - c) @ R.T + np.asarray(centre), mesh.tris.copy(), 1)


# ----------------------------------------------------------------------------- inside test

@pytest.mark.parametrize("n,ratio,seed", [(16, 1.0, 0), (18, 2.0, 1), (20, 1.0, 2)])
def test_inside_matches_exact_winding_sphere(n, ratio, seed):
    rng = np.random.default_rng(seed)
    f = synth.faces_tanh(n, ratio)
    g = Grid(f, f[:n - 1] * 0 + synth.faces_tanh(n - 2, ratio), f)
    s = synth.octa_sphere(3, (0, 0, 0), rng.uniform(0.2, 0.35))
    m = _rotated_mesh(s, _rot(*rng.uniform(0, 2 * np.pi, 3)), rng.uniform(0.4, 0.6, 3))
    got = C.inside_mesh(g, m.verts, m.tris)
    ref = _winding_inside(g, m, rng)
    assert ref is not None
    assert np.array_equal(got, ref)
    assert got.sum() > 50


def test_inside_matches_exact_winding_rotated_cube_vertex_on_columns():
    # cube rotated 45 deg about z: vertices and edges pass through column lines
    n = 16
    f = synth.faces_uniform(n)
    g = Grid(f, f, f)
    h = 1.0 / n
    c = 0.5 + h / 2                  # a cell centre
    r = 4 * h                        # half-diagonal, so vertices land on centre columns
    V = np.array([[c - r, c, 0.23], [c, c - r, 0.23], [c + r, c, 0.23], [c, c + r, 0.23],
                  [c - r, c, 0.71], [c, c - r, 0.71], [c + r, c, 0.71], [c, c + r, 0.71]])
    T = synth.box_mesh((0, 0, 0), (1, 1, 1)).tris
    m = synth.Mesh(V, T, 1)
    # centres on the vertical faces |x-c| + |y-c| = r (lattice-exact) are on the surface
    Xs, Ys, Zs = C.snap(g.xc), C.snap(g.yc), C.snap(g.zc)
    cs, rs = int(C.snap(c)), int(C.snap(r))
    Z3, Y3, X3 = np.meshgrid(Zs, Ys, Xs, indexing="ij")
    on = (np.abs(X3 - cs) + np.abs(Y3 - cs) == rs) & (Z3 >= C.snap(0.23)) & (Z3 <= C.snap(0.71))
    assert on.sum() > 0
    rng = np.random.default_rng(5)
    got = C.inside_mesh(g, m.verts, m.tris)
    ref = _winding_inside(g, m, rng, skip=on)
    assert ref is not None
    assert not np.any(got[on])
    assert np.array_equal(got[~on], ref[~on])
    assert got.sum() > 100


def test_inside_grid_aligned_box_faces_through_centres():
    """Faces, edges and vertices on cell centres and column lines: strictly inside
    cells are solid, cells on the surface are fluid (closed-form expectation)."""
    n = 12
    f = synth.faces_uniform(n)
    g = Grid(f, f, f)
    lo_i, hi_i = (2, 3, 1), (8, 9, 10)          # box corners at centres of these cells
    lo = [g.xc[lo_i[0]], g.yc[lo_i[1]], g.zc[lo_i[2]]]
    hi = [g.xc[hi_i[0]], g.yc[hi_i[1]], g.zc[hi_i[2]]]
    m = synth.box_mesh(lo, hi)
    got = C.inside_mesh(g, m.verts, m.tris)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ref = (i > lo_i[0]) & (i < hi_i[0]) & (j > lo_i[1]) & (j < hi_i[1]) & (k > lo_i[2]) & (k < hi_i[2])
    assert np.array_equal(got, ref)


def test_inside_sphere_analytic_bounds_and_union():
    n = 40
    f = synth.faces_tanh(n, 2.0)
    g = Grid(f, f, f)
    L = 4
    spheres = [((0.3, 0.35, 0.4), 0.12), ((0.68, 0.62, 0.6), 0.15)]
    ms = [synth.octa_sphere(L, c, r) for c, r in spheres]
    ib = C.iblank_closed(g, ms)
    Z, Y, X = np.meshgrid(g.zc, g.yc, g.xc, indexing="ij")
    for c, r in spheres:
        d = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        # the geodesic polyhedron lies between the inscribed radius and r
        rin = r * math.cos(math.pi / 2 ** (L + 1))
        assert np.all(ib[d < 0.98 * rin] == 1)
    dmin = np.min([np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - r for c, r in spheres], axis=0)
    assert np.all(ib[dmin > 0] == 0)


def test_ghosts_brute_force():
    n = 14
    f = synth.faces_uniform(n)
    g = Grid(f, f, f)
    ib = C.iblank_closed(g, [synth.octa_sphere(3, (0.5, 0.47, 0.52), 0.27)])
    ghosts = C.mark_ghosts(ib)
    ref = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                if not ib[k, j, i] & 1:
                    continue
                nbs = [(k, j, i - 1), (k, j, i + 1), (k, j - 1, i), (k, j + 1, i), (k - 1, j, i), (k + 1, j, i)]
                if any(0 <= a < n and 0 <= b < n and 0 <= c < n and not ib[a, b, c] & 1 for a, b, c in nbs):
                    ref.append((k * n + j) * n + i)
    assert ghosts.tolist() == ref
    assert np.all((ib.ravel()[ghosts] & 3) == 3)


# ----------------------------------------------------------------------------- closest point

def test_closest_point_is_the_projection_onto_the_triangle():
    """Q solves min |P-X|^2 over the triangle iff Q is in it and (P-Q).(V-Q) <= 0 at all vertices."""
    rng = np.random.default_rng(3)
    T = rng.normal(size=(4000, 3, 3))
    T[:50, 2] = T[:50, 0] + 1e-3 * rng.normal(size=(50, 3))        # slivers
    T[50:60, 1] = T[50:60, 0]                                     # degenerate edges
    P = rng.normal(size=(4000, 3)) * 2.0
    Q, d2 = C.closest_point_on_triangles(P, T[:, 0], T[:, 1], T[:, 2])
    scale = np.max(np.abs(T)) ** 2
    for vtx in range(3):
        assert np.all(np.einsum("ij,ij->i", P - Q, T[:, vtx] - Q) <= 1e-11 * scale)
    # Q in the triangle: minimal-norm barycentrics via least squares
    for s in range(0, 4000, 97):
        M = np.stack([T[s, 1] - T[s, 0], T[s, 2] - T[s, 0]], 1)
        uv, *_ = np.linalg.lstsq(M, Q[s] - T[s, 0], rcond=None)
        if s >= 60:
            assert uv.min() > -1e-9 and uv.sum() < 1 + 1e-9
    assert np.allclose(d2, np.sum((P - Q) ** 2, axis=1), rtol=1e-12, atol=0)


def test_image_point_plane_reflection_closed_form():
    # tilted plane as two huge triangles; IP = GC - 2 ((GC - P0).n) n
    nrm = np.array([0.3, -0.2, 1.0]); nrm /= np.linalg.norm(nrm)
    P0 = np.array([0.5, 0.5, 0.5])
    u = np.cross(nrm, [1.0, 0, 0]); u /= np.linalg.norm(u)
    v = np.cross(nrm, u)
    V = np.array([P0 + 3 * (-u - v), P0 + 3 * (u - v), P0 + 3 * (u + v), P0 + 3 * (-u + v)])
    m = synth.Mesh(V, np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32), 1)
    rng = np.random.default_rng(1)
    GC = P0 + rng.uniform(-0.1, 0.1, size=(500, 3))
    BI, _ = C.closest_points(GC, [m])
    IP = (BI + BI) - GC
    ref = GC - 2.0 * ((GC - P0) @ nrm)[:, None] * nrm[None]
    assert np.allclose(IP, ref, rtol=0, atol=1e-14)
    assert np.allclose(0.5 * (GC + IP), BI, rtol=0, atol=1e-15)
    assert np.allclose(np.linalg.norm(IP - BI, axis=1), np.linalg.norm(GC - BI, axis=1), rtol=1e-13)


# ----------------------------------------------------------------------------- tables

@pytest.mark.parametrize("ratio", [1.0, 2.0])
def test_ghost_tables_weights(ratio):
    n = 24
    f = synth.faces_tanh(n, ratio)
    g = Grid(f, f, f)
    m = synth.ellipsoid(4, (0.3, 0.18, 0.15), 25.0)
    ib, G = C.classify(g, [m])
    assert len(G) > 100
    # exact reflection and equal distances
    GC = g.centre(G.cell)
    assert np.allclose(0.5 * (GC + G.ip), G.bi, rtol=0, atol=4e-16)
    # face-interior hits: GC - BI parallel to the face normal of the nearest triangle
    BI, tri = C.closest_points(GC, [m])
    Tv = m.verts[m.tris[tri]]
    nrm = np.cross(Tv[:, 1] - Tv[:, 0], Tv[:, 2] - Tv[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    dvec = GC - BI
    cosang = np.abs(np.einsum("ij,ij->i", dvec, nrm)) / np.linalg.norm(dvec, axis=1)
    assert np.mean(cosang > 1 - 1e-12) > 0.5
    # weights: nonnegative, sum to one, refs are active cells, base corner brackets IP
    assert np.all(G.w >= 0)
    assert np.allclose(G.w.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    assert np.all(ib.ravel()[G.ref[G.ref >= 0]] != 1)
    assert np.all(G.ref[G.w == 0] == -1) and np.all(G.ref[G.w > 0] >= 0)
    assert np.all(G.scale > 0)
    # full-support rows reproduce any linear field at IP exactly
    full = ((G.flags >> 8) & 0xFF) == 0xFF
    n = g.nx
    gi, gj, gk = G.cell % n, (G.cell // n) % n, G.cell // (n * n)
    self_in = np.all([(G.base[:, 0] <= gi) & (gi <= G.base[:, 0] + 1), (G.base[:, 1] <= gj) & (gj <= G.base[:, 1] + 1),
                      (G.base[:, 2] <= gk) & (gk <= G.base[:, 2] + 1)], axis=0)
    lin = full & ~self_in & ((G.flags & C.FLAG_FALLBACK) == 0)
    assert lin.sum() > 10
    coef = np.array([0.3, -1.7, 2.2, 0.9])
    cc = g.centre(np.where(G.ref >= 0, G.ref, 0))
    fv = coef[0] + cc @ coef[1:]
    val = np.sum(np.where(G.ref >= 0, G.w * fv, 0.0), axis=1)
    ip = np.clip(G.ip, [g.xc[0], g.yc[0], g.zc[0]], [g.xc[-1], g.yc[-1], g.zc[-1]])
    assert np.allclose(val[lin], (coef[0] + ip @ coef[1:])[lin], rtol=0, atol=1e-13)


def test_grid_aligned_wall_ghost_is_mirror():
    n = 16
    f = synth.faces_uniform(n)
    g = Grid(f, f, f)
    m = synth.box_mesh((0.5, -1.0, -1.0), (2.0, 2.0, 2.0))
    ib, G = C.classify(g, [m])
    assert len(G) == n * n
    i = G.cell % n
    assert np.all(i == n // 2)
    # one weight of exactly 1, on the mirror fluid cell (clamped base corners at the
    # last row/plane put it in another slot)
    assert np.all(np.sum(G.w == 1.0, axis=1) == 1) and np.all(np.sum(G.w != 0.0, axis=1) == 1)
    assert np.array_equal(G.ref[G.w == 1.0], G.cell - 1)


def test_closest_points_mesh_pruning_equals_full_scan():
    """The mesh-level pruning of the closest-point search changes nothing: same points, same
    triangle indices as a scan of every triangle of every mesh (ties included)."""
    rng = np.random.default_rng(8)
    meshes = [synth.octa_sphere(2, tuple(c), r) for c, r in
              (((0.3, 0.3, 0.3), 0.1), ((0.7, 0.35, 0.4), 0.12), ((0.5, 0.7, 0.6), 0.15))]
    meshes.append(synth.box_mesh((0.2, 0.6, 0.1), (0.35, 0.9, 0.3)))
    P = rng.uniform(0.0, 1.0, size=(700, 3))
    P[:40] = meshes[3].verts[rng.integers(0, 8, 40)] + np.array([0.0, 0.0, -0.05])   # ties on box faces
    q, t = C.closest_points(P, meshes, chunk=32)
    T = np.concatenate([np.asarray(m.verts)[np.asarray(m.tris)] for m in meshes])
    Q, d2 = C.closest_point_on_triangles(np.broadcast_to(P[:, None], (P.shape[0], T.shape[0], 3)),
                                         T[None, :, 0], T[None, :, 1], T[None, :, 2])
    tf = np.argmin(d2, axis=1)
    assert np.array_equal(t, tf)
    assert np.array_equal(q, Q[np.arange(P.shape[0]), tf])


# ----------------------------------------------------------------------------- watertightness

def _centres_strictly_inside_projection(grid, a, b, c, margin):
    """Columns (j, i) whose centre lies inside the xy-projection of triangle abc by more than
    `margin` from every edge (floats; the caller checks that no centre lies within the
    margin, so the answer is not a tie)."""
    X, Y = np.meshgrid(grid.xc, grid.yc, indexing="xy")
    out, near = set(), False
    area = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    sgn = 1.0 if area > 0 else -1.0
    for p, q in ((a, b), (b, c), (c, a)):
        L = math.hypot(q[0] - p[0], q[1] - p[1])
        d = sgn * ((q[0] - p[0]) * (Y - p[1]) - (q[1] - p[1]) * (X - p[0])) / L
        near |= bool(np.any(np.abs(d) <= margin))
        if p is a:
            ok = d > margin
        else:
            ok &= d > margin
    for j, i in zip(*np.nonzero(ok)):
        out.add((int(j), int(i)))
    return out, near


def test_watertight_meshes_have_no_odd_column_and_a_hole_gives_exactly_its_columns():
    """Jordan: a watertight surface crosses every vertical line an even number of times, so
    no column is odd -- also for a body poking above the top cell centre (its crossings
    above the last centre count).  Deleting one triangle of the upper half leaves a hole:
    exactly the columns through the inside of its xy-projection become odd, and the inside
    test refuses the mesh."""
    f = synth.faces_tanh(24, 1.5)
    g = Grid(f, synth.faces_uniform(22), f)
    whole = synth.octa_sphere(2, (0.5, 0.5, 0.5), 0.36)
    top = synth.octa_sphere(3, (0.47, 0.52, 0.93), 0.2)        # reaches z = 1.13 > the top centre
    for m in (whole, top):
        assert C.odd_columns(g, m.verts, m.tris).shape[0] == 0
        C.iblank_closed(g, [m])
    V = whole.verts
    cz = V[whole.tris].mean(axis=1)[:, 2]
    tested = 0
    for t in np.argsort(-cz):
        a, b, c = (V[whole.tris[t, q]] for q in range(3))
        expect, near = _centres_strictly_inside_projection(g, a, b, c, 1e-7)
        if near or len(expect) < 2:
            continue
        leaky = synth.Mesh(V, np.delete(whole.tris, t, axis=0), 1)
        got = {(int(j), int(i)) for j, i in C.odd_columns(g, leaky.verts, leaky.tris)}
        assert got == expect, (t, sorted(got ^ expect))
        with pytest.raises(C.MeshNotClosed):
            C.iblank_closed(g, [leaky])
        tested += 1
        if tested == 3:
            break
    assert tested == 3
