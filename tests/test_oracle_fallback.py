"""Pins of the oracle's fallback ghost rows (the reading for image points whose interpolation
box holds almost no usable corner).

Geometry: a box and a sphere that overlap (solid = inside either).  A ghost of the union near
the rim where the sphere dives into the box can have its closest surface point on the buried
part of the sphere; its image point then lands deep in solid, every corner of its box is a
plain solid cell, and the row falls back to the ghost's fluid face-neighbour nearest to the
image point, with weight 1 and kappa = -|centre(nb) - GC|.

Each check recomputes the rule from its statement, cell by cell in plain Python: which rows
qualify (valid corner weight below 1e-3, or an own weight of at least 1 - 1e-12), which
neighbour they take, and their kappa.  A linear field with the datum along each row's
direction satisfies the fallback rows exactly, and planted mistakes (the neighbour nearest
to the ghost instead of the image point, kappa from the image point's distance) fail.
"""
import math

import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import solve as OS
from oracle import system as OSys
from oracle.grid import Grid

DIRS = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def _case(n=24, zc=0.47):
    f = synth.faces_uniform(n)
    g = Grid(f, f, f)
    meshes = synth.overlapping_bodies(zc)
    ib, G = OC.classify(g, meshes)
    return g, meshes, ib, G


def _centre(g, l):
    nz, ny, nx = g.shape
    return (float(g.xc[l % nx]), float(g.yc[(l // nx) % ny]), float(g.zc[l // (nx * ny)]))


def _expected_row(g, ib, gcell, ip):
    """(qualifies as a fallback, nearest fluid face-neighbour to IP) by the rule's statement."""
    nz, ny, nx = g.shape
    flat = ib.ravel()

    def locate(c, v):
        i0 = int(np.searchsorted(c, v, "right")) - 1
        i0 = min(max(i0, 0), c.size - 2)
        t = (v - c[i0]) / (c[i0 + 1] - c[i0])
        return i0, min(max(t, 0.0), 1.0)

    (i0, tx), (j0, ty), (k0, tz) = locate(g.xc, ip[0]), locate(g.yc, ip[1]), locate(g.zc, ip[2])
    s, wself = 0.0, 0.0
    for c in range(8):
        bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        w = (tx if bx else 1 - tx) * (ty if by else 1 - ty) * (tz if bz else 1 - tz)
        l = ((k0 + bz) * ny + (j0 + by)) * nx + (i0 + bx)
        if flat[l] != OC.IBLANK_SOLID:
            s += w
            if l == gcell:
                wself = w
    qualifies = s < 1e-3 or (s > 0 and wself / s >= 1.0 - 1e-12)
    gk, gj, gi = gcell // (nx * ny), (gcell // nx) % ny, gcell % nx
    best, bestd = -1, math.inf
    for di, dj, dk in DIRS:
        i, j, k = gi + di, gj + dj, gk + dk
        if not (0 <= i < nx and 0 <= j < ny and 0 <= k < nz):
            continue
        l = (k * ny + j) * nx + i
        if flat[l] != OC.IBLANK_FLUID:
            continue
        d = math.dist(ip, _centre(g, l))
        if d < bestd:
            best, bestd = l, d
    return qualifies, best


@pytest.mark.parametrize("n,zc", [(16, 0.5), (24, 0.47), (32, 0.5)])
def test_fallback_rows_follow_the_rule(n, zc):
    g, _, ib, G = _case(n, zc)
    fb = (G.flags & OC.FLAG_FALLBACK) != 0
    assert fb.sum() >= 8
    for q in range(len(G)):
        qual, nb = _expected_row(g, ib, int(G.cell[q]), tuple(G.ip[q]))
        assert bool(fb[q]) == qual, q
        if not qual:
            continue
        assert nb >= 0
        assert G.ref[q, 0] == nb and np.all(G.ref[q, 1:] == -1), (q, G.ref[q], nb)
        assert G.w[q, 0] == 1.0 and np.all(G.w[q, 1:] == 0.0)
        ell = math.dist(_centre(g, nb), _centre(g, int(G.cell[q])))
        assert abs(G.kappa[q] + ell) <= 1e-15 * ell
        assert G.wself[q] == 0.0


def test_planted_nearest_to_the_ghost_differs():
    """The neighbour nearest to IP is not simply the first fluid neighbour of the ghost (all
    face-neighbours of a uniform grid are equally near the ghost centre), so a fallback that
    measured from GC would take a different cell on some rows."""
    g, _, ib, G = _case(24, 0.47)
    nz, ny, nx = g.shape
    flat = ib.ravel()
    fb = np.flatnonzero((G.flags & OC.FLAG_FALLBACK) != 0)
    differ = 0
    for q in fb:
        gc = int(G.cell[q])
        gk, gj, gi = gc // (nx * ny), (gc // nx) % ny, gc % nx
        first = -1
        for di, dj, dk in DIRS:
            i, j, k = gi + di, gj + dj, gk + dk
            l = (k * ny + j) * nx + i
            if 0 <= i < nx and 0 <= j < ny and 0 <= k < nz and flat[l] == OC.IBLANK_FLUID:
                first = l
                break
        differ += first != G.ref[q, 0]
    assert differ > 0


def test_linear_field_satisfies_fallback_rows():
    """p = a + c.x: a fallback row g - v_nb = kappa q holds exactly with q = c.e, e the unit
    vector from the ghost centre to the neighbour's; kappa from |IP - GC| (a planted mistake)
    does not."""
    g, _, _, G = _case(24, 0.47)
    c = np.array([0.7, -1.3, 2.1])
    fb = np.flatnonzero((G.flags & OC.FLAG_FALLBACK) != 0)
    GC = g.centre(G.cell[fb])
    NB = g.centre(G.ref[fb, 0])
    e = (NB - GC) / np.linalg.norm(NB - GC, axis=1)[:, None]
    q = e @ c
    r = (0.37 + NB @ c) - (0.37 + GC @ c) + G.kappa[fb] * q
    assert np.max(np.abs(r)) < 1e-13
    wrong = -np.linalg.norm(G.ip[fb] - GC, axis=1)
    r_bad = (0.37 + NB @ c) - (0.37 + GC @ c) + wrong * q
    assert np.max(np.abs(r_bad)) > 1e-3


def test_system_with_fallback_rows():
    """A 1 = 0 on every row (fallback rows included); the dense bordered solve and the sparse
    solve agree; the solution meets its own rows, and each fallback ghost equals its
    neighbour's pressure (homogeneous datum)."""
    g, _, ib, G = _case(16, 0.5)
    fb = np.flatnonzero((G.flags & OC.FLAG_FALLBACK) != 0)
    assert fb.size > 0
    A, cells, _ = OSys.assemble(g, ib, G)
    assert np.max(np.abs(A @ np.ones(cells.size))) < 1e-9 * np.max(np.abs(A.diagonal()))
    b = synth.rhs_divergence(g.xf, g.yf, g.zf, 8)
    pd, ld = OS.solve_dense(g, ib, G, b)
    ps, ls = OS.solve_sparse(g, ib, G, b)
    fl = ib == 0
    assert np.linalg.norm((pd - ps)[fl]) <= 1e-11 * np.linalg.norm(pd[fl])
    assert abs(ld - ls) <= 1e-9 * max(1.0, abs(ld))
    assert OSys.relative_residual(g, ib, G, b, ps) < 1e-11
    flat = ps.ravel()
    assert np.allclose(flat[G.cell[fb]], flat[G.ref[fb, 0]], rtol=0, atol=1e-10 * np.max(np.abs(flat)))
