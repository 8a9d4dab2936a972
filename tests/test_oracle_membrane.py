"""Pins of the membrane oracle (oracle/membrane.py) against definitions it does not share code with."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import membrane as OM
from oracle.classify import snap
from oracle.grid import Grid


def _square_plate(x0, x1, y0, y1, z):
    """Two triangles, counter-clockwise seen from +z (normal +z)."""
    V = np.array([[x0, y0, z], [x1, y0, z], [x1, y1, z], [x0, y1, z]])
    return synth.Mesh(V, np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32), 0)


def _tilted_plate(nq=4, seed_angle=0.37):
    m = synth.plate(0.13, chord=0.5, span=0.35, nq_x=nq, nq_y=nq, heave=0.05, pitch_deg=25.0,
                    center=(0.503, 0.491, 0.517))
    # a small rotation about x keeps every triangle generic w.r.t. the lattice lines
    c, s = np.cos(seed_angle * 0.3), np.sin(seed_angle * 0.3)
    R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    V = (m.verts - 0.5) @ R.T + 0.5
    return synth.Mesh(V, m.tris, 0)


def _brute_cut(grid, mesh):
    """Every (link, triangle) pair in exact rationals: segment-plane crossing strictly inside
    the triangle and strictly between the centres; the lowest crossing triangle decides;
    side = sign of n . (P - X*)."""
    nz, ny, nx = grid.shape
    C = [snap(grid.xc), snap(grid.yc), snap(grid.zc)]
    V = snap(mesh.verts)
    tris = [[[Fraction(int(v)) for v in V[q]] for q in t] for t in mesh.tris]
    cut = np.zeros(grid.shape, dtype=np.uint8)
    side = np.zeros(grid.shape, dtype=np.uint8)
    best = {}
    for a in range(3):
        for k in range(nz - (a == 2)):
            for j in range(ny - (a == 1)):
                for i in range(nx - (a == 0)):
                    lo = [i, j, k]
                    hi = [i + (a == 0), j + (a == 1), k + (a == 2)]
                    P = [Fraction(int(C[q][lo[q]])) for q in range(3)]
                    Q = [Fraction(int(C[q][hi[q]])) for q in range(3)]
                    for t, (A, B, Cc) in enumerate(tris):
                        ab = [B[q] - A[q] for q in range(3)]
                        ac = [Cc[q] - A[q] for q in range(3)]
                        n = [ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0]]
                        den = n[a]
                        if den == 0:
                            continue
                        d = sum(n[q] * (A[q] - P[q]) for q in range(3))
                        tt = d / den                               # X* = P + tt (Q - P)/|Q - P|, along axis a
                        if not (0 < tt < Q[a] - P[a]):
                            continue
                        X = list(P)
                        X[a] = P[a] + tt
                        # barycentric inside test (strict; generic position has no ties)
                        def tri_area(p1, p2, p3):
                            u = [p2[q] - p1[q] for q in range(3)]
                            v = [p3[q] - p1[q] for q in range(3)]
                            cr = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
                            return sum(cr[q] * n[q] for q in range(3))
                        s1, s2, s3 = tri_area(A, B, X), tri_area(B, Cc, X), tri_area(Cc, A, X)
                        assert s1 != 0 and s2 != 0 and s3 != 0, "tie: choose a more generic plate"
                        if not ((s1 > 0 and s2 > 0 and s3 > 0) or (s1 < 0 and s2 < 0 and s3 < 0)):
                            continue
                        for end, cell in ((0, tuple(lo)), (1, tuple(hi))):
                            E = P if end == 0 else Q
                            sg = sum(n[q] * (E[q] - X[q]) for q in range(3))
                            key = (a, tuple(lo), end)
                            if key not in best or t < best[key][0]:
                                best[key] = (t, 1 if sg > 0 else 0, cell)
    for (a, _lo, end), (_t, s, cell) in best.items():
        dbit = 2 * a + (1 if end == 0 else 0)
        i, j, k = cell
        cut[k, j, i] |= 1 << dbit
        if s:
            side[k, j, i] |= 1 << dbit
    return cut, side


def test_cut_links_match_exact_brute_force():
    grid = Grid(synth.faces_tanh(11, 2.0), synth.faces_uniform(10), synth.faces_tanh(12, 1.5))
    m = _tilted_plate()
    cut, side = OM.cut_links(grid, [m])
    cb, sb = _brute_cut(grid, m)
    assert cut.sum() > 0
    assert np.array_equal(cut, cb)
    assert np.array_equal(side & cut, sb & cb)


def test_flat_plate_cuts_exactly_the_links_through_it():
    n = 16
    f = synth.faces_uniform(n)
    grid = Grid(f, f, f)
    cut, side = OM.cut_links(grid, [_square_plate(0.25, 0.75, 0.25, 0.75, 0.5)])
    xc = grid.xc
    inside = (xc > 0.25) & (xc < 0.75)
    expect_up = np.zeros(grid.shape, dtype=bool)                 # +z links from plane n/2 - 1
    expect_up[n // 2 - 1] = inside[None, :, None] & inside[None, None, :]
    assert np.array_equal(((cut >> 5) & 1).astype(bool), expect_up)
    expect_dn = np.roll(expect_up, 1, axis=0)
    assert np.array_equal(((cut >> 4) & 1).astype(bool), expect_dn)
    assert np.all(cut & 0b001111 == 0)
    # normal +z: cells below are on the negative side, cells above on the positive side
    assert np.all(((side >> 5) & 1)[expect_up] == 0)
    assert np.all(((side >> 4) & 1)[expect_dn] == 1)


def _half_box_solution(grid, b, k_split):
    """Exact Neumann solutions of the two half boxes (DCT-II), each with its own mean removed."""
    from scipy.fft import dctn, idctn
    out = np.zeros(grid.shape)
    for sl in (slice(0, k_split), slice(k_split, grid.shape[0])):
        bb = b[sl] - b[sl].mean()
        nz, ny, nx = bb.shape
        h = 1.0 / nx
        lam = lambda m: -4.0 * np.sin(np.pi * np.arange(m) / (2 * m)) ** 2 / h ** 2
        L = lam(nz)[:, None, None] + lam(ny)[None, :, None] + lam(nx)[None, None, :]
        B = dctn(bb, type=2, norm="ortho")
        L[0, 0, 0] = 1.0
        X = B / L
        X[0, 0, 0] = 0.0
        out[sl] = idctn(X, type=2, norm="ortho")
    return out


def test_spanning_plate_is_two_neumann_boxes():
    """A plate through a face plane over the whole cross-section: the two half boxes'
    exact Neumann solutions, with ghost values from their rows, satisfy every row."""
    n = 16
    f = synth.faces_uniform(n)
    grid = Grid(f, f, f)
    _, G = OM.classify(grid, [_square_plate(-0.1, 1.1, -0.1, 1.1, 0.5)])
    b = synth.rhs_divergence(f, f, f, 3)
    p = _half_box_solution(grid, b, n // 2)
    ncell = n ** 3
    g = np.zeros(len(G))
    for e in range(len(G)):                       # ghost values from the ghost rows
        vals = [p.ravel()[r] if r < ncell else 0.0 for r in G.ref[e] if r >= 0]
        g[e] = sum(w * v for w, v in zip(G.w[e][G.ref[e] >= 0], vals))
    assert np.all(G.ref[G.ref >= 0] < ncell)      # mirrors land on the own side's cells
    rf, rg = OM.residual(grid, G, b, p, g)
    means = np.where(np.arange(n)[:, None, None] < n // 2, b[: n // 2].mean(), b[n // 2:].mean())
    assert np.max(np.abs(rf - means)) < 1e-9 * np.max(np.abs(b))
    assert np.max(np.abs(rg)) == 0.0


def test_constant_is_in_the_kernel():
    grid = Grid(synth.faces_tanh(12, 2.0), synth.faces_uniform(11), synth.faces_uniform(13))
    _, G = OM.classify(grid, [_tilted_plate()])
    A, _ = OM.assemble(grid, G)
    one = np.ones(A.shape[0])
    assert len(G) > 0
    assert np.max(np.abs(A @ one)) < 1e-9 * abs(A).max()


def _mms_error(n, flip=False):
    f = synth.faces_uniform(n)
    grid = Grid(f, f, f)
    mesh = _square_plate(0.25, 0.75, 0.25, 0.75, 0.5)
    cut, side = OM.cut_links(grid, [mesh])
    if flip:
        side = side ^ cut
    G = OM.ghost_tables(grid, cut, side, [mesh])
    X, Y = np.meshgrid(grid.xc, grid.yc, indexing="xy")
    fexact = np.broadcast_to(np.cos(np.pi * X) * np.cos(np.pi * Y), grid.shape)
    b = -2.0 * np.pi ** 2 * fexact
    p, g, lam = OM.solve_sparse(grid, G, b)
    e = p - (fexact - fexact.mean())
    return float(np.sqrt(np.mean(e * e)))


def test_finite_plate_keeps_second_order():
    """cos(pi x) cos(pi y) has zero normal derivative on a plate z = 0.5 and on the walls, so
    the plate must not disturb it: the error falls at second order."""
    e1, e2 = _mms_error(16), _mms_error(32)
    assert e2 < 0.3 * e1 and e2 < 2e-3


def _sealing_plate():
    """A tilted planar plate reaching past the box: it splits the box into two chambers."""
    m = synth.plate(0.0, chord=2.4, span=2.4, nq_x=6, nq_y=6, heave=0.0, pitch_deg=0.0, center=(0.5, 0.5, 0.5))
    a, b = np.radians(17.0), np.radians(11.0)
    Ry = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    V = (m.verts - 0.5) @ (Rx @ Ry).T + np.array([0.5, 0.5, 0.47])
    return synth.Mesh(V, m.tris, 0), (Rx @ Ry) @ np.array([0.0, 0.0, 1.0])


def _chamber_residual(flip):
    grid = Grid(synth.faces_tanh(14, 2.0), synth.faces_uniform(13), synth.faces_uniform(15))
    mesh, normal = _sealing_plate()
    cut, side = OM.cut_links(grid, [mesh])
    if flip:
        side = side ^ cut
    G = OM.ghost_tables(grid, cut, side, [mesh])
    # chamber of every cell centre by the plane's own equation (no centre lies on it)
    X, Y, Z = np.meshgrid(grid.xc, grid.yc, grid.zc, indexing="ij")
    h = ((X - 0.5) * normal[0] + (Y - 0.5) * normal[1] + (Z - 0.47) * normal[2]).transpose(2, 1, 0)
    assert np.min(np.abs(h)) > 1e-6
    alpha = {1: 3.0, 0: -5.0}                  # positive side of the normal: alpha[1]
    p = np.where(h > 0, alpha[1], alpha[0])
    g = np.array([alpha[int(s_)] for s_ in G.side])
    A, _ = OM.assemble(grid, G)
    r = A @ np.concatenate([p.ravel(), g])
    assert len(G) > 100
    return float(np.max(np.abs(r)) / abs(A).max())


def test_sealing_plate_isolates_the_chambers():
    """Constant values per chamber (ghost entries take their side's value) satisfy every
    fluid and ghost row: no row mixes values from both sides of the membrane."""
    assert _chamber_residual(False) < 1e-12


def test_planted_wrong_side_fails():
    assert _chamber_residual(True) > 1e-3
