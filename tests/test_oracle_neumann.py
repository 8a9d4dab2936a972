"""Pins of the moving-boundary Neumann datum in the oracle's ghost rows.

A linear pressure field p(x) = a + c.x has the normal derivative c.n on any surface.  The
image-point rows reproduce it exactly: trilinear weights interpolate linear fields exactly
when all eight corners are used. With the datum q = c.n along each row's own direction, the
ghost row g - sum w v = kappa q then holds with g = p(GC). Checked on every such row of a
closed body and of a membrane; planted mistakes in kappa must fail."""
import numpy as np

import synth
from oracle import classify as OC
from oracle import membrane as OM
from oracle.grid import Grid

C = np.array([0.7, -1.3, 2.1])
A0 = 0.37


def _plin(X):
    return A0 + X @ C


def _row_dirs(grid, G, GC):
    """Unit direction of each row: towards IP, or towards the fallback neighbour."""
    nz, ny, nx = grid.shape
    d = G.ip - GC
    fb = (G.flags & OC.FLAG_FALLBACK) != 0
    nb = np.where(fb, G.ref[:, 0], 0)
    cen = np.stack([grid.xc[nb % nx], grid.yc[(nb // nx) % ny], grid.zc[nb // (nx * ny)]], -1)
    d = np.where(fb[:, None], cen - GC, d)
    return d / np.linalg.norm(d, axis=1)[:, None], fb


def _ghost_row_residuals(grid, G, GC, values_of_ref, kappa):
    """r_G = sum w v - g + kappa q for the linear field (v and g exact)."""
    n, fb = _row_dirs(grid, G, GC)
    q = n @ C
    vals = np.where(G.ref >= 0, values_of_ref(np.where(G.ref >= 0, G.ref, 0)), 0.0)
    interp = np.sum(np.where(G.ref >= 0, G.w * vals, 0.0), axis=1)
    return interp - _plin(GC) + kappa * q, fb


def _full_corner_rows(G):
    """Rows whose eight corners were all used (bits 8-15 of the flags), and fallbacks."""
    return ((G.flags >> 8) & 0xFF) == 0xFF


def _closed_case():
    xf, yf, zf = synth.faces_tanh(26, 2.0), synth.faces_uniform(22), synth.faces_tanh(24, 1.5)
    grid = Grid(xf, yf, zf)
    mesh = synth.ellipsoid(4, (0.21, 0.17, 0.15), 23.0, (0.49, 0.51, 0.5))
    ib, G = OC.classify(grid, [mesh])
    GC = grid.centre(G.cell)
    nz, ny, nx = grid.shape
    lin = np.arange(nz * ny * nx)
    X = grid.centre(lin)
    pfull = _plin(X)
    return grid, G, GC, lambda ref: pfull[ref]


def test_linear_field_satisfies_closed_body_rows():
    grid, G, GC, vals = _closed_case()
    r, fb = _ghost_row_residuals(grid, G, GC, vals, G.kappa)
    full = _full_corner_rows(G) | fb
    assert full.sum() > 50
    assert np.max(np.abs(r[full])) < 1e-12 * np.max(np.abs(_plin(GC)))
    # rows whose own weight was moved to the left-hand side are among them: kappa differs
    # from -|IP - GC| exactly there
    length = np.linalg.norm(G.ip - GC, axis=1)
    moved = ~fb & (np.abs(G.kappa + length) > 1e-15 * length)
    assert (moved & full).sum() > 0


def test_planted_kappa_mistakes_fail():
    grid, G, GC, vals = _closed_case()
    full = _full_corner_rows(G)
    r_flip, _ = _ghost_row_residuals(grid, G, GC, vals, -G.kappa)
    assert np.max(np.abs(r_flip[full])) > 1e-3
    length = np.linalg.norm(G.ip - GC, axis=1)
    r_noself, _ = _ghost_row_residuals(grid, G, GC, vals, -length)   # self factor dropped
    moved = full & (np.abs(G.kappa + length) > 1e-15 * length)
    assert np.max(np.abs(r_noself[moved])) > 1e-6


def test_linear_field_satisfies_membrane_rows():
    grid = Grid(synth.faces_tanh(22, 2.0), synth.faces_uniform(20), synth.faces_uniform(23))
    m = synth.plate(0.13, chord=0.5, span=0.35, nq_x=5, nq_y=5, heave=0.05, pitch_deg=25.0,
                    center=(0.503, 0.491, 0.517))
    c, s = np.cos(0.1), np.sin(0.1)
    R = np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    mesh = synth.Mesh((m.verts - 0.5) @ R.T + 0.5, m.tris, 0)
    _, G = OM.classify(grid, [mesh])
    nz, ny, nx = grid.shape
    ncell = nz * ny * nx
    GC = grid.centre(G.cell)
    pcell = _plin(grid.centre(np.arange(ncell)))
    pent = _plin(GC)                                   # entry values: the field at their cells

    def vals(ref):
        return np.where(ref < ncell, pcell[np.minimum(ref, ncell - 1)], pent[np.maximum(ref - ncell, 0)])

    r, fb = _ghost_row_residuals(grid, G, GC, vals, G.kappa)
    full = _full_corner_rows(G) | fb
    assert full.sum() > 20
    assert np.max(np.abs(r[full])) < 1e-12 * np.max(np.abs(pent))
    r_flip, _ = _ghost_row_residuals(grid, G, GC, vals, -G.kappa)
    assert np.max(np.abs(r_flip[full & ~fb])) > 1e-3


def test_datum_moves_the_solution_consistently():
    """The system with ghost-row data: the oracle's residual of its own solution is at the
    FP64 floor, and scaling the data scales the response (linearity in d)."""
    from oracle import solve as OS
    from oracle import system as SYS
    f = synth.faces_uniform(14)
    grid = Grid(f, f, f)
    ib, G = OC.classify(grid, [synth.octa_sphere(3, (0.5, 0.5, 0.5), 0.25)])
    b = synth.rhs_divergence(f, f, f, 2)
    rng = np.random.default_rng(5)
    q = rng.standard_normal(len(G))
    p0, _ = OS.solve_sparse(grid, ib, G, b)
    OC.set_neumann(G, q)
    p1, _ = OS.solve_sparse(grid, ib, G, b)
    assert SYS.relative_residual(grid, ib, G, b, p1) < 1e-11
    OC.set_neumann(G, 2.0 * q)
    p2, _ = OS.solve_sparse(grid, ib, G, b)
    fl = ib == 0
    assert np.linalg.norm((p1 - p0)[fl]) > 1e-3 * np.linalg.norm(p0[fl])
    assert np.allclose((p2 - p0)[fl], 2.0 * (p1 - p0)[fl], rtol=1e-8, atol=1e-10)
