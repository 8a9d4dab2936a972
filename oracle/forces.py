"""Surface pressure on the body's triangles and the nodal pressure forces (oracle).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs use
this module; the GPU library never calls it.

Paper: Sec. "Force Formulations" -- the external force on a structure node is the sum,
over the triangles that share the node, of one third of the triangle's fluid traction
times its area; its pressure part is -dp n A with dp the pressure difference across the
membrane.  The paper does not say how dp is taken from the cell-centred pressure.
Readings (the probe rule of ghost-cell methods, with the image-point interpolation):

* Triangle t with vertices v0, v1, v2: N = (v1 - v0) x (v2 - v0), |N| = 2 A, unit normal
  n = N / |N| (the side n points to is "+"), centroid c = ((v0 + v1) + v2) / 3.
* Probe distance d = 1.5 sqrt(hx^2 + hy^2 + hz^2), h the widths of the cell that holds c
  (the last cell whose lower face is <= c, clamped to the grid).  At 1.5 cell diagonals the
  probe's interpolation box lies on its own side of a surface that is flat at the cell scale.
* Side s (+1: slot 0, -1: slot 1): probe X = c + (s d) n.  Trilinear weights of X on the
  cell-centre lattice exactly as for image points (base corner by binary search, clamped to
  [0, n - 2], t clamped to [0, 1]; corner slot bx + 2 by + 4 bz).  A corner is used when it
  holds fluid on side s: closed bodies, the cell is fluid (iblank 0); membranes, the corner
  centre lies strictly on side s of the triangle's plane, s ((x_k - c) . n) > 0.  With
  s_w = the sum of the used weights and v = the sum of weight x p over them (slot order),
  p_s = v / s_w - (s d) q, where q is the pressure's normal derivative dp/dn at c (zero for a
  fixed body; -a(c) . n for a body with acceleration a, rho = 1): p(X) = p(c) + s d q to first
  order, so a linear field is recovered exactly.  If s_w < 1e-3 the side has no data:
  p_s = 0 and bit s of the triangle's flags is set.  A zero-area triangle has flags bit 2,
  p_s = 0 and no force.
* Closed bodies have fluid on the + side only (outward normals): p_- = 0, not flagged.
* dp = p_+ - p_-; the triangle's force f = -(dp (N / 2)); each of its three nodes receives
  f / 3.  Nodal sums run over the triangles in ascending order.
* Several meshes: vertices are numbered mesh after mesh, triangles likewise.
* The shear part of the traction (the velocity gradients) is not computed.

Floating-point order: every expression is evaluated as written, left to right, with
separately rounded operations and IEEE division and square root.

Parity status: pinned by exact recovery of linear fields on a convex closed body and on a
grid-aligned membrane, Archimedes' closed form (total force of a linear field = -grad p x
the polyhedron's volume), a constant jump across a tilted plate (-dp n x plate area),
orientation independence and the nodal moment identity (tests/test_oracle_forces.py).
"""
from __future__ import annotations

import numpy as np

from .classify import IBLANK_FLUID, WEIGHT_SUM_MIN, _base_and_t
from .grid import Grid

PROBE_FACTOR = 1.5
FLAG_ZERO_AREA = 4


def concat_meshes(meshes):
    """All meshes' vertices (V, 3) and triangles (T, 3) with global vertex indices, and the
    first triangle of each mesh (plus the total)."""
    V, T, off, vo = [], [], [0], 0
    for m in meshes:
        v = np.asarray(m.verts, dtype=np.float64).reshape(-1, 3)
        t = np.asarray(m.tris, dtype=np.int64).reshape(-1, 3)
        V.append(v)
        T.append(t + vo)
        vo += v.shape[0]
        off.append(off[-1] + t.shape[0])
    return np.concatenate(V), np.concatenate(T), np.asarray(off)


def triangle_geometry(V: np.ndarray, T: np.ndarray):
    """N = (v1 - v0) x (v2 - v0), |N|, the unit normal (0 for a zero-area triangle) and the
    centroid of every triangle."""
    v0, v1, v2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    e1, e2 = v1 - v0, v2 - v0
    N = np.stack([e1[:, 1] * e2[:, 2] - e1[:, 2] * e2[:, 1],
                  e1[:, 2] * e2[:, 0] - e1[:, 0] * e2[:, 2],
                  e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]], -1)
    a2 = np.sqrt((N[:, 0] * N[:, 0] + N[:, 1] * N[:, 1]) + N[:, 2] * N[:, 2])
    with np.errstate(divide="ignore", invalid="ignore"):
        n = np.where(a2[:, None] > 0.0, N / a2[:, None], 0.0)
    c = ((v0 + v1) + v2) / 3.0
    return N, a2, n, c


def rigid_q(c: np.ndarray, n: np.ndarray, tri_off, motions) -> np.ndarray:
    """q = -a(c) . n per triangle for rigid kinematics per mesh (a0, angular acceleration,
    angular velocity, centre): a = a0 + alpha x r + omega x (omega x r), r = c - centre."""
    M = np.asarray(motions, dtype=np.float64).reshape(-1, 12)
    m = np.searchsorted(np.asarray(tri_off), np.arange(c.shape[0]), side="right") - 1
    mm = M[m]
    r = c - mm[:, 9:12]
    al, om = mm[:, 3:6], mm[:, 6:9]
    wr = np.stack([om[:, 1] * r[:, 2] - om[:, 2] * r[:, 1], om[:, 2] * r[:, 0] - om[:, 0] * r[:, 2],
                   om[:, 0] * r[:, 1] - om[:, 1] * r[:, 0]], -1)
    a0 = (mm[:, 0] + (al[:, 1] * r[:, 2] - al[:, 2] * r[:, 1])) + (om[:, 1] * wr[:, 2] - om[:, 2] * wr[:, 1])
    a1 = (mm[:, 1] + (al[:, 2] * r[:, 0] - al[:, 0] * r[:, 2])) + (om[:, 2] * wr[:, 0] - om[:, 0] * wr[:, 2])
    a2 = (mm[:, 2] + (al[:, 0] * r[:, 1] - al[:, 1] * r[:, 0])) + (om[:, 0] * wr[:, 1] - om[:, 1] * wr[:, 0])
    return -((a0 * n[:, 0] + a1 * n[:, 1]) + a2 * n[:, 2])


def _cell_of(f: np.ndarray, v: np.ndarray) -> np.ndarray:
    return np.clip(np.searchsorted(f, v, "right") - 1, 0, f.size - 2)


def surface_pressure(grid: Grid, iblank, membrane: bool, V: np.ndarray, T: np.ndarray, p: np.ndarray,
                     q=None):
    """Pressure on the + and - side of every triangle ((T, 2)) and the flags (see module doc).

    iblank: [nz][ny][nx] (closed bodies; ignored for membranes); p: cell pressures
    [nz][ny][nx]; q: per-triangle dp/dn (None: 0)."""
    nz, ny, nx = grid.shape
    nt = T.shape[0]
    N, a2, n, c = triangle_geometry(V, T)
    qq = np.zeros(nt) if q is None else np.asarray(q, dtype=np.float64)
    i, j, k = _cell_of(grid.xf, c[:, 0]), _cell_of(grid.yf, c[:, 1]), _cell_of(grid.zf, c[:, 2])
    hx, hy, hz = grid.dx[i], grid.dy[j], grid.dz[k]
    d = PROBE_FACTOR * np.sqrt((hx * hx + hy * hy) + hz * hz)
    pf = np.asarray(p, dtype=np.float64).ravel()
    ibf = None if membrane else np.asarray(iblank).ravel()
    out = np.zeros((nt, 2))
    flags = np.where(a2 > 0.0, 0, FLAG_ZERO_AREA).astype(np.int32)
    live = a2 > 0.0
    for slot, sgn in ((0, 1.0), (1, -1.0)):
        if slot == 1 and not membrane:
            break
        sd = sgn * d
        X = c + sd[:, None] * n
        i0, tx = _base_and_t(grid.xc, X[:, 0])
        j0, ty = _base_and_t(grid.yc, X[:, 1])
        k0, tz = _base_and_t(grid.zc, X[:, 2])
        wx = np.stack([1.0 - tx, tx], -1)
        wy = np.stack([1.0 - ty, ty], -1)
        wz = np.stack([1.0 - tz, tz], -1)
        sw = np.zeros(nt)
        v = np.zeros(nt)
        for cc in range(8):
            bx, by, bz = cc & 1, (cc >> 1) & 1, (cc >> 2) & 1
            lin = ((k0 + bz) * ny + (j0 + by)) * nx + (i0 + bx)
            w = (wx[:, bx] * wy[:, by]) * wz[:, bz]
            if membrane:
                dot = (((grid.xc[i0 + bx] - c[:, 0]) * n[:, 0] + (grid.yc[j0 + by] - c[:, 1]) * n[:, 1])
                       + (grid.zc[k0 + bz] - c[:, 2]) * n[:, 2])
                use = dot > 0.0 if slot == 0 else dot < 0.0
            else:
                use = ibf[lin] == IBLANK_FLUID
            sw = sw + np.where(use, w, 0.0)
            v = v + np.where(use, w * pf[lin], 0.0)
        ok = live & (sw >= WEIGHT_SUM_MIN)
        with np.errstate(divide="ignore", invalid="ignore"):
            val = v / sw - sd * qq
        out[:, slot] = np.where(ok, val, 0.0)
        flags |= np.where(live & ~ok, 1 << slot, 0).astype(np.int32)
    return out, flags


def nodal_forces(V: np.ndarray, T: np.ndarray, p_side: np.ndarray) -> np.ndarray:
    """F_i = sum over the triangles t holding node i of f_t / 3, f_t = -(dp_t (N_t / 2)),
    accumulated in ascending triangle order."""
    N, a2, n, c = triangle_geometry(V, T)
    dp = p_side[:, 0] - p_side[:, 1]
    f = -(dp[:, None] * (0.5 * N))
    f = np.where(a2[:, None] > 0.0, f, 0.0)
    share = f / 3.0
    F = np.zeros((V.shape[0], 3))
    for t in range(T.shape[0]):
        for corner in range(3):
            F[T[t, corner]] = F[T[t, corner]] + share[t]
    return F


def surface_forces(grid: Grid, iblank, meshes, p: np.ndarray, q=None, motions=None):
    """(p_side (T, 2), flags (T,), nodal forces (V, 3)) for the meshes' triangles; q per
    triangle or motions per mesh (rigid kinematics), not both."""
    V, T, off = concat_meshes(meshes)
    membrane = len(meshes) > 0 and not int(meshes[0].closed)
    if motions is not None:
        assert q is None
        _, _, n, c = triangle_geometry(V, T)
        q = rigid_q(c, n, off, motions)
    ps, flags = surface_pressure(grid, iblank, membrane, V, T, p, q)
    return ps, flags, nodal_forces(V, T, ps)
