"""Iblanking, ghost cells, image points and interpolation weights (oracle).

Paper: Sec. "GPU Porting", item 1 (voxel segmentation / rasterisation of the
grid against a triangulated body, "iblanking") and item 2 (ghost-cell method
modules applying the internal boundary condition); the image-point
interpolation is the ghost-cell method of the reference the paper cites for
it.  Readings where the paper is silent:

* Exact inside test.  Cell centres and mesh vertices are snapped to the
  lattice 2^-24 (``snap``; coordinates must lie in [-4, 4]).  A cell centre q
  is inside a closed mesh when the number of triangles crossed by the
  vertical line through q strictly below q is odd.  A triangle "covers" the
  column of q by the half-open (top-left) rule on its xy-projection, so a
  column through a shared edge or vertex is counted once.  A centre lying
  exactly on the surface is fluid.  Several closed meshes: solid = inside any.
* Ghost cell: a solid cell with at least one fluid face-neighbour.
* Boundary intercept BI: closest point of the (faceted) surface to the ghost
  centre GC, minimum over all triangles, lowest triangle index on ties.
  Closest point on one triangle: the stationary point of the squared distance
  in the triangle's plane when it lies inside, else the best of the three
  edge projections (``closest_point_on_triangles``).
* Image point IP = 2 BI - GC (reflection of GC through BI).
* Trilinear weights in physical coordinates on the cell-centre lattice, base
  corner i0 with x_{i0} <= IP_x < x_{i0+1} (clamped to [0, n-2], t clamped to
  [0, 1]).  Corners that are plain solid (not ghost) get weight 0; the rest are
  renormalised by their sum s.  If s < 1e-3, or the ghost's own weight is
  >= 1 - 1e-12, the ghost takes the value of its fluid face-neighbour nearest
  to IP (weight 1).  A ghost's own weight is moved to the left-hand side and
  the other weights divided by (1 - w_self).

Floating-point order: every expression is evaluated left to right with
separately rounded operations (no fused multiply-add) and IEEE division, so
results are reproducible bit for bit by any implementation that keeps this
order.

Parity status: the inside test is pinned by exact rational winding numbers and
analytic sphere bounds; closest points by brute force and closed forms (plane
reflection); weights by linear-field reproduction (tests/test_oracle_classify.py).
"""
from __future__ import annotations

import numpy as np

from .grid import Grid

SNAP_BITS = 24
SNAP_SCALE = float(2 ** SNAP_BITS)
COORD_LIMIT = 4.0
WEIGHT_SUM_MIN = 1e-3
SELF_WEIGHT_MAX = 1.0 - 1e-12

IBLANK_FLUID = 0
IBLANK_SOLID = 1
IBLANK_GHOST_BIT = 2

FLAG_FALLBACK = 1


def snap(x) -> np.ndarray:
    """Round coordinates to the integer lattice 2^-24 (round half to even)."""
    x = np.asarray(x, dtype=np.float64)
    if x.size and np.max(np.abs(x)) > COORD_LIMIT:
        raise ValueError("coordinates must lie in [-4, 4]")
    return np.rint(x * SNAP_SCALE).astype(np.int64)


def _top_left(px, py, qx, qy) -> bool:
    """Does the directed edge P->Q of a counter-clockwise triangle own points on it?"""
    return (qx > px) or (qx == px and py > qy)


def _orient2d(ax, ay, bx, by, qx, qy):
    """Twice the signed area of (a, b, q); exact in int64 for lattice coordinates."""
    return (bx - ax) * (qy - ay) - (by - ay) * (qx - ax)


def _closed_range(sorted_vals: np.ndarray, lo, hi):
    return int(np.searchsorted(sorted_vals, lo, "left")), int(np.searchsorted(sorted_vals, hi, "right"))


def inside_mesh(grid: Grid, verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Boolean [k][j][i]: cell centre strictly inside the closed mesh (exact test)."""
    Xc, Yc, Zc = snap(grid.xc), snap(grid.yc), snap(grid.zc)
    V = snap(verts)
    nz, ny, nx = grid.shape
    toggles = np.zeros((nz + 1, ny, nx), dtype=np.uint8)
    onsurf = np.zeros((nz, ny, nx), dtype=bool)
    for t in range(tris.shape[0]):
        A = [int(v) for v in V[tris[t, 0]]]
        B = [int(v) for v in V[tris[t, 1]]]
        C = [int(v) for v in V[tris[t, 2]]]
        area = _orient2d(A[0], A[1], B[0], B[1], C[0], C[1])
        xs = (min(A[0], B[0], C[0]), max(A[0], B[0], C[0]))
        ys = (min(A[1], B[1], C[1]), max(A[1], B[1], C[1]))
        i0, i1 = _closed_range(Xc, *xs)
        j0, j1 = _closed_range(Yc, *ys)
        if i0 >= i1 or j0 >= j1:
            continue
        QX, QY = np.meshgrid(Xc[i0:i1], Yc[j0:j1], indexing="xy")   # [j][i]
        if area == 0:
            _mark_vertical(A, B, C, QX, QY, Zc, onsurf, i0, j0)
            continue
        if area < 0:
            B, C = C, B
            area = -area
        wa = _orient2d(B[0], B[1], C[0], C[1], QX, QY)
        wb = _orient2d(C[0], C[1], A[0], A[1], QX, QY)
        wc = _orient2d(A[0], A[1], B[0], B[1], QX, QY)
        cov = ((wa > 0) | ((wa == 0) & _top_left(B[0], B[1], C[0], C[1]))) \
            & ((wb > 0) | ((wb == 0) & _top_left(C[0], C[1], A[0], A[1]))) \
            & ((wc > 0) | ((wc == 0) & _top_left(A[0], A[1], B[0], B[1])))
        jj, ii = np.nonzero(cov)
        for a, b in zip(jj.tolist(), ii.tolist()):
            # height of the crossing: N / D with D = 2*area > 0 (exact rationals)
            N = int(wa[a, b]) * A[2] + int(wb[a, b]) * B[2] + int(wc[a, b]) * C[2]
            q, rem = divmod(N, area)
            ks = int(np.searchsorted(Zc, q, "right"))   # first centre strictly above the crossing
            toggles[ks, j0 + a, i0 + b] ^= 1
            if rem == 0 and ks >= 1 and int(Zc[ks - 1]) == q:
                onsurf[ks - 1, j0 + a, i0 + b] = True
    parity = np.bitwise_xor.accumulate(toggles[:nz], axis=0).astype(bool)
    return parity & ~onsurf


def _mark_vertical(A, B, C, QX, QY, Zc, onsurf, i0, j0):
    """Cells lying on a triangle whose xy-projection is a segment."""
    ab = (B[0] - A[0], B[1] - A[1], B[2] - A[2])
    ac = (C[0] - A[0], C[1] - A[1], C[2] - A[2])
    n = (ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0])
    if n == (0, 0, 0):
        return
    # a projected segment P0-P1 carrying all three vertices
    pts = [A, B, C]
    P0 = min(pts, key=lambda v: (v[0], v[1]))
    P1 = max(pts, key=lambda v: (v[0], v[1]))
    online = _orient2d(P0[0], P0[1], P1[0], P1[1], QX, QY) == 0
    use_x = n[1] != 0                    # project onto (x, z) unless the plane is x = const
    zlo, zhi = min(A[2], B[2], C[2]), max(A[2], B[2], C[2])
    k0, k1 = _closed_range(Zc, zlo, zhi)
    for a, b in zip(*np.nonzero(online)):
        qu = int(QX[a, b]) if use_x else int(QY[a, b])
        for k in range(k0, k1):
            qz = int(Zc[k])
            e = []
            for P, Q in ((A, B), (B, C), (C, A)):
                pu, qqu = (P[0], Q[0]) if use_x else (P[1], Q[1])
                e.append(_orient2d(pu, P[2], qqu, Q[2], qu, qz))
            if (e[0] >= 0 and e[1] >= 0 and e[2] >= 0) or (e[0] <= 0 and e[1] <= 0 and e[2] <= 0):
                onsurf[k, j0 + a, i0 + b] = True


def iblank_closed(grid: Grid, meshes) -> np.ndarray:
    """uint8 [k][j][i]: 0 fluid, 1 solid (inside any closed mesh); ghost bit added by ``mark_ghosts``."""
    solid = np.zeros(grid.shape, dtype=bool)
    for m in meshes:
        if int(m.closed):
            solid |= inside_mesh(grid, m.verts, m.tris)
    return solid.astype(np.uint8)


def mark_ghosts(iblank: np.ndarray) -> np.ndarray:
    """Ghost cells: solid with >= 1 fluid face-neighbour.  Returns sorted linear indices
    and sets bit 1 of iblank for them (in place)."""
    solid = (iblank & IBLANK_SOLID).astype(bool)
    fluid = ~solid
    nb = np.zeros_like(solid)
    nb[1:] |= fluid[:-1]; nb[:-1] |= fluid[1:]
    nb[:, 1:] |= fluid[:, :-1]; nb[:, :-1] |= fluid[:, 1:]
    nb[:, :, 1:] |= fluid[:, :, :-1]; nb[:, :, :-1] |= fluid[:, :, 1:]
    ghost = solid & nb
    iblank[ghost] |= IBLANK_GHOST_BIT
    return np.flatnonzero(ghost.ravel()).astype(np.int64)


# ----------------------------------------------------------------------------- closest point

def _dot(ax, ay, az, bx, by, bz):
    return (ax * bx + ay * by) + az * bz


def closest_point_on_triangles(P: np.ndarray, A: np.ndarray, B: np.ndarray, C: np.ndarray):
    """Closest points Q and squared distances for points P (..., 3) to triangles (..., 3).

    Interior case: minimise |P - (A + u ab + v ac)|^2; the normal equations
    [a b; b c][u; v] = [d; e] give det*u = c d - b e, det*v = a e - b d, and
    the minimiser is inside when both are >= 0 and their sum <= det.
    Otherwise the closest point lies on the boundary: the best of the three
    segment projections AB, BC, CA (first one wins ties).
    """
    with np.errstate(divide="ignore", invalid="ignore"):
        Px, Py, Pz = P[..., 0], P[..., 1], P[..., 2]
        Ax, Ay, Az = A[..., 0], A[..., 1], A[..., 2]
        abx, aby, abz = B[..., 0] - Ax, B[..., 1] - Ay, B[..., 2] - Az
        acx, acy, acz = C[..., 0] - Ax, C[..., 1] - Ay, C[..., 2] - Az
        apx, apy, apz = Px - Ax, Py - Ay, Pz - Az
        a = _dot(abx, aby, abz, abx, aby, abz)
        b = _dot(abx, aby, abz, acx, acy, acz)
        c = _dot(acx, acy, acz, acx, acy, acz)
        d = _dot(abx, aby, abz, apx, apy, apz)
        e = _dot(acx, acy, acz, apx, apy, apz)
        det = a * c - b * b
        su = c * d - b * e
        sv = a * e - b * d
        inner = (det > 0) & (su >= 0) & (sv >= 0) & (su + sv <= det)
        u = su / det
        v = sv / det
        Qi = np.stack([(Ax + u * abx) + v * acx, (Ay + u * aby) + v * acy, (Az + u * abz) + v * acz], -1)
        best_q = None
        best_d = None
        for P0, P1 in ((A, B), (B, C), (C, A)):
            ex, ey, ez = P1[..., 0] - P0[..., 0], P1[..., 1] - P0[..., 1], P1[..., 2] - P0[..., 2]
            px, py, pz = Px - P0[..., 0], Py - P0[..., 1], Pz - P0[..., 2]
            num = _dot(ex, ey, ez, px, py, pz)
            den = _dot(ex, ey, ez, ex, ey, ez)
            t = num / den
            Qe = np.stack([P0[..., 0] + t * ex, P0[..., 1] + t * ey, P0[..., 2] + t * ez], -1)
            lo = (num <= 0) | (den <= 0)
            hi = (~lo) & (num >= den)
            Qe = np.where(lo[..., None], P0, np.where(hi[..., None], P1, Qe))
            dx, dy, dz = Px - Qe[..., 0], Py - Qe[..., 1], Pz - Qe[..., 2]
            de = _dot(dx, dy, dz, dx, dy, dz)
            if best_q is None:
                best_q, best_d = Qe, de
            else:
                take = de < best_d
                best_q = np.where(take[..., None], Qe, best_q)
                best_d = np.where(take, de, best_d)
        Q = np.where(inner[..., None], Qi, best_q)
        dx, dy, dz = Px - Q[..., 0], Py - Q[..., 1], Pz - Q[..., 2]
        d2 = _dot(dx, dy, dz, dx, dy, dz)
    return Q, d2


def closest_points(P: np.ndarray, meshes, chunk: int = 64):
    """Boundary intercepts: for each point, the closest surface point over all triangles
    of all given meshes (global index order, lowest index wins exact ties)."""
    Vs = [np.asarray(m.verts, dtype=np.float64)[np.asarray(m.tris)] for m in meshes]
    T = np.concatenate(Vs, axis=0)                    # (ntri, 3 vertices, 3)
    A, B, C = T[:, 0], T[:, 1], T[:, 2]
    out_q = np.empty((P.shape[0], 3))
    out_t = np.empty(P.shape[0], dtype=np.int64)
    for s in range(0, P.shape[0], chunk):
        Pc = P[s:s + chunk, None, :]
        Q, d2 = closest_point_on_triangles(np.broadcast_to(Pc, (Pc.shape[0], A.shape[0], 3)),
                                           A[None], B[None], C[None])
        t = np.argmin(d2, axis=1)                     # first minimum = lowest index
        out_t[s:s + chunk] = t
        out_q[s:s + chunk] = Q[np.arange(Q.shape[0]), t]
    return out_q, out_t


# ----------------------------------------------------------------------------- ghost tables

class GhostTable:
    """Per ghost entry: cell, BI, IP, base corner, flags, 8 (ref, weight) pairs, row scale."""

    def __init__(self, n):
        self.cell = np.zeros(n, dtype=np.int64)
        self.bi = np.zeros((n, 3))
        self.ip = np.zeros((n, 3))
        self.base = np.zeros((n, 3), dtype=np.int32)
        self.flags = np.zeros(n, dtype=np.int32)
        self.ref = np.full((n, 8), -1, dtype=np.int64)
        self.w = np.zeros((n, 8))
        self.scale = np.zeros(n)

    def __len__(self):
        return self.cell.size


def _base_and_t(c: np.ndarray, v: np.ndarray):
    n = c.size
    i0 = np.searchsorted(c, v, "right") - 1
    i0 = np.clip(i0, 0, n - 2)
    t = (v - c[i0]) / (c[i0 + 1] - c[i0])
    t = np.where(t < 0.0, 0.0, np.where(t > 1.0, 1.0, t))
    return i0.astype(np.int64), t


def ghost_tables(grid: Grid, iblank: np.ndarray, ghosts: np.ndarray, meshes) -> GhostTable:
    """Image points and interpolation rows of closed-body ghost cells (see module doc)."""
    nz, ny, nx = grid.shape
    G = GhostTable(ghosts.size)
    G.cell[:] = ghosts
    if ghosts.size == 0:
        return G
    closed = [m for m in meshes if int(m.closed)]
    GC = grid.centre(ghosts)
    BI, _ = closest_points(GC, closed)
    IP = (BI + BI) - GC
    G.bi[:] = BI
    G.ip[:] = IP
    i0, tx = _base_and_t(grid.xc, IP[:, 0])
    j0, ty = _base_and_t(grid.yc, IP[:, 1])
    k0, tz = _base_and_t(grid.zc, IP[:, 2])
    G.base[:] = np.stack([i0, j0, k0], -1)
    wx = np.stack([1.0 - tx, tx], -1)
    wy = np.stack([1.0 - ty, ty], -1)
    wz = np.stack([1.0 - tz, tz], -1)
    flat = iblank.ravel()
    gk, gj, gi = ghosts // (nx * ny), (ghosts // nx) % ny, ghosts % nx
    for g in range(ghosts.size):
        w = np.zeros(8)
        ref = np.full(8, -1, dtype=np.int64)
        valid = np.zeros(8, dtype=bool)
        for c in range(8):
            bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
            lin = ((k0[g] + bz) * ny + (j0[g] + by)) * nx + (i0[g] + bx)
            ref[c] = lin
            w[c] = (wx[g, bx] * wy[g, by]) * wz[g, bz]
            valid[c] = flat[lin] != IBLANK_SOLID
        s = 0.0
        for c in range(8):
            if valid[c]:
                s = s + w[c]
        fallback = s < WEIGHT_SUM_MIN
        if not fallback:
            wn = np.where(valid, w / s, 0.0)
            selfc = np.flatnonzero(valid & (ref == ghosts[g]))
            if selfc.size:
                ws = wn[selfc[0]]
                if ws >= SELF_WEIGHT_MAX:
                    fallback = True
                else:
                    wn = wn / (1.0 - ws)
                    wn[selfc[0]] = 0.0
        if fallback:
            G.flags[g] |= FLAG_FALLBACK
            G.ref[g] = -1
            G.w[g] = 0.0
            best, bestd = -1, None
            for (di, dj, dk) in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                ii, jj, kk = gi[g] + di, gj[g] + dj, gk[g] + dk
                if not (0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz):
                    continue
                lin = (kk * ny + jj) * nx + ii
                if flat[lin] != IBLANK_FLUID:
                    continue
                ex = IP[g, 0] - grid.xc[ii]; ey = IP[g, 1] - grid.yc[jj]; ez = IP[g, 2] - grid.zc[kk]
                d2 = (ex * ex + ey * ey) + ez * ez
                if bestd is None or d2 < bestd:
                    best, bestd = lin, d2
            G.ref[g, 0] = best
            G.w[g, 0] = 1.0
        else:
            G.ref[g] = np.where(wn != 0.0, ref, -1)
            G.w[g] = wn
            G.flags[g] |= int(np.sum(valid.astype(np.int32) << np.arange(8))) << 8
        # row scale: coefficients of the fluid rows that reference this ghost
        sc = 0.0
        for (di, dj, dk, cf) in ((-1, 0, 0, grid.cxp), (1, 0, 0, grid.cxm), (0, -1, 0, grid.cyp),
                                 (0, 1, 0, grid.cym), (0, 0, -1, grid.czp), (0, 0, 1, grid.czm)):
            ii, jj, kk = gi[g] + di, gj[g] + dj, gk[g] + dk
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz and flat[(kk * ny + jj) * nx + ii] == IBLANK_FLUID:
                sc = sc + cf[ii if di else (jj if dj else kk)]
        G.scale[g] = sc
    return G


def classify(grid: Grid, meshes):
    """Closed bodies: (iblank uint8 [k][j][i], ghost table)."""
    ib = iblank_closed(grid, meshes)
    ghosts = mark_ghosts(ib)
    return ib, ghost_tables(grid, ib, ghosts, meshes)
