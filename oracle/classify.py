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

* Watertightness: a closed surface crosses every vertical line an even number
  of times; a grid column with an odd count (crossings above the top centre
  included) marks a hole and the mesh is refused (``MeshNotClosed``).

Parity status: the inside test is pinned by exact rational winding numbers and
analytic sphere bounds; closest points by brute force and closed forms (plane
reflection); weights by linear-field reproduction; the watertightness rule by a
sphere with one triangle deleted (tests/test_oracle_classify.py); the fallback
rows by the rule recomputed cell by cell on two overlapping bodies
(tests/test_oracle_fallback.py).
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
    nz, ny, nx = grid.shape
    out = np.zeros((nz, ny, nx), dtype=bool)
    box, sub = inside_mesh_box(grid, verts, tris)
    if box is not None:
        (k0, j0, i0) = box
        out[k0:, j0:j0 + sub.shape[1], i0:i0 + sub.shape[2]] = sub
    return out


class MeshNotClosed(ValueError):
    """A closed mesh is crossed an odd number of times by some grid column."""


def inside_mesh_box(grid: Grid, verts: np.ndarray, tris: np.ndarray):
    """(box, inside) of ``column_parity``: the inside test of the cells that can be inside."""
    box, inside, _ = column_parity(grid, verts, tris)
    return box, inside


def odd_columns(grid: Grid, verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """(j, i) pairs of the grid columns (vertical lines through the cell centres) that the
    surface crosses an odd number of times.  A watertight surface separates space into an
    inside and an outside, so every line enters and leaves it alike: the count is even on
    every column.  An odd count means a hole in the surface on that line."""
    box, _, odd = column_parity(grid, verts, tris)
    if box is None:
        return np.zeros((0, 2), dtype=np.int64)
    _, j0, i0 = box
    jj, ii = np.nonzero(odd)
    return np.stack([jj + j0, ii + i0], axis=1).astype(np.int64)


def column_parity(grid: Grid, verts: np.ndarray, tris: np.ndarray):
    """The inside test on the cells that can be inside: columns whose centre lies in the
    mesh's xy box, planes from the mesh's lowest centre up to the top of the grid (cells
    outside that region have no crossing below them, so their parity is even).

    Every (triangle, column) pair of a triangle's xy box is tested at once: integer edge
    functions (exact in int64), the top-left rule, then the crossing height N / D.  N needs
    up to 82 bits, so its floor is taken from a float64 estimate whose error is far below
    one lattice unit, and pairs whose estimate lies within 1e-6 of an integer are redone
    in exact Python integers.

    Returns ((k0, j0, i0), boolean inside [nz-k0][nj][ni], boolean odd [nj][ni]) or
    (None, None, None); odd marks the columns with an odd total number of crossings (the
    slot above the top centre included).  A mesh above every centre gives k0 = nz (no
    inside cell), its columns still counted.
    """
    Xc, Yc, Zc = snap(grid.xc), snap(grid.yc), snap(grid.zc)
    V = snap(verts)
    nz, ny, nx = grid.shape
    if V.size == 0:
        return None, None, None
    bi0, bi1 = _closed_range(Xc, int(V[:, 0].min()), int(V[:, 0].max()))
    bj0, bj1 = _closed_range(Yc, int(V[:, 1].min()), int(V[:, 1].max()))
    bk0 = int(np.searchsorted(Zc, int(V[:, 2].min()), "left"))
    if bi0 >= bi1 or bj0 >= bj1:
        return None, None, None
    # local sub-box: columns [bj0, bj1) x [bi0, bi1), planes [bk0, nz)
    Xc, Yc, Zc = Xc[bi0:bi1], Yc[bj0:bj1], Zc[bk0:]
    nz, ny, nx = Zc.size, Yc.size, Xc.size
    toggles = np.zeros((nz + 1, ny, nx), dtype=np.uint8)
    onsurf = np.zeros((nz, ny, nx), dtype=bool)
    T = np.asarray(tris, dtype=np.int64)
    A, B, Cv = V[T[:, 0]].copy(), V[T[:, 1]].copy(), V[T[:, 2]].copy()
    area = _orient2d(A[:, 0], A[:, 1], B[:, 0], B[:, 1], Cv[:, 0], Cv[:, 1])
    for t in np.flatnonzero(area == 0):                  # vertical (or degenerate) triangles
        a, b, c = [[int(v) for v in X[t]] for X in (A, B, Cv)]
        xs = (min(a[0], b[0], c[0]), max(a[0], b[0], c[0]))
        ys = (min(a[1], b[1], c[1]), max(a[1], b[1], c[1]))
        i0, i1 = _closed_range(Xc, *xs)
        j0, j1 = _closed_range(Yc, *ys)
        if i0 < i1 and j0 < j1:
            QX, QY = np.meshgrid(Xc[i0:i1], Yc[j0:j1], indexing="xy")
            _mark_vertical(a, b, c, QX, QY, Zc, onsurf, i0, j0)
    sel = np.flatnonzero(area != 0)
    A, B, Cv, area = A[sel], B[sel], Cv[sel], area[sel]
    neg = area < 0                                       # make every projection counter-clockwise
    B[neg], Cv[neg] = Cv[neg].copy(), B[neg].copy()
    area = np.abs(area)
    lo = np.minimum(np.minimum(A, B), Cv)
    hi = np.maximum(np.maximum(A, B), Cv)
    i0 = np.searchsorted(Xc, lo[:, 0], "left"); i1 = np.searchsorted(Xc, hi[:, 0], "right")
    j0 = np.searchsorted(Yc, lo[:, 1], "left"); j1 = np.searchsorted(Yc, hi[:, 1], "right")
    ni, nj = np.maximum(i1 - i0, 0), np.maximum(j1 - j0, 0)
    cnt = ni * nj
    tri = np.repeat(np.arange(cnt.size), cnt)
    loc = np.arange(tri.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    ii = i0[tri] + loc % np.maximum(ni[tri], 1)
    jj = j0[tri] + loc // np.maximum(ni[tri], 1)
    qx, qy = Xc[ii], Yc[jj]
    a, b, c = A[tri], B[tri], Cv[tri]
    wa = _orient2d(b[:, 0], b[:, 1], c[:, 0], c[:, 1], qx, qy)
    wb = _orient2d(c[:, 0], c[:, 1], a[:, 0], a[:, 1], qx, qy)
    wc = _orient2d(a[:, 0], a[:, 1], b[:, 0], b[:, 1], qx, qy)
    tl = lambda p, q: (q[:, 0] > p[:, 0]) | ((q[:, 0] == p[:, 0]) & (p[:, 1] > q[:, 1]))
    cov = ((wa > 0) | ((wa == 0) & tl(b, c))) & ((wb > 0) | ((wb == 0) & tl(c, a))) \
        & ((wc > 0) | ((wc == 0) & tl(a, b)))
    k = np.flatnonzero(cov)
    wa, wb, wc, a, b, c, ar, ii, jj = wa[k], wb[k], wc[k], a[k], b[k], c[k], area[tri[k]], ii[k], jj[k]
    zf = (wa.astype(np.float64) * a[:, 2] + wb.astype(np.float64) * b[:, 2] + wc.astype(np.float64) * c[:, 2]) \
        / ar.astype(np.float64)
    q = np.floor(zf).astype(np.int64)
    exact_hit = np.zeros(zf.size, dtype=bool)
    for e in np.flatnonzero(np.abs(zf - np.rint(zf)) < 1e-6):   # near-integer: exact integers
        N = int(wa[e]) * int(a[e, 2]) + int(wb[e]) * int(b[e, 2]) + int(wc[e]) * int(c[e, 2])
        qq, rem = divmod(N, int(ar[e]))
        q[e] = qq
        exact_hit[e] = rem == 0
    ks = np.searchsorted(Zc, q, "right")                 # first centre strictly above the crossing
    np.bitwise_xor.at(toggles, (ks, jj, ii), 1)
    on = exact_hit & (ks >= 1)
    on &= Zc[np.maximum(ks - 1, 0)] == q
    onsurf[ks[on] - 1, jj[on], ii[on]] = True
    parity = np.bitwise_xor.accumulate(toggles[:nz], axis=0).astype(bool)
    odd = np.bitwise_xor.reduce(toggles, axis=0).astype(bool)
    return (bk0, bj0, bi0), parity & ~onsurf, odd


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
    """uint8 [k][j][i]: 0 fluid, 1 solid (inside any closed mesh); ghost bit added by ``mark_ghosts``.
    Raises MeshNotClosed when a closed mesh has an odd crossing count on some column."""
    solid = np.zeros(grid.shape, dtype=bool)
    for m in meshes:
        if int(m.closed):
            box, sub, odd = column_parity(grid, m.verts, m.tris)
            if odd is not None and np.any(odd):
                raise MeshNotClosed("closed mesh crossed an odd number of times by %d grid column(s)"
                                    % int(np.count_nonzero(odd)))
            if box is not None and sub.shape[0] > 0:
                k0, j0, i0 = box
                solid[k0:, j0:j0 + sub.shape[1], i0:i0 + sub.shape[2]] |= sub
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
    of all given meshes (global index order, lowest index wins exact ties).

    Whole meshes are skipped for a chunk of points when the distance from every point of
    the chunk to the mesh's bounding box exceeds an upper bound of that point's answer (the
    exact distance to the mesh whose box is nearest): a box distance is a lower bound of
    the distance to any triangle inside it, so no skipped triangle could be the minimum or
    tie with it.  The remaining meshes are scanned in index order with strict improvement,
    which keeps the lowest-index rule.
    """
    Ts = [np.asarray(m.verts, dtype=np.float64)[np.asarray(m.tris)] for m in meshes]
    lo = np.array([T.reshape(-1, 3).min(axis=0) for T in Ts])
    hi = np.array([T.reshape(-1, 3).max(axis=0) for T in Ts])
    base = np.cumsum([0] + [T.shape[0] for T in Ts])
    out_q = np.empty((P.shape[0], 3))
    out_t = np.empty(P.shape[0], dtype=np.int64)

    tlo = [T.min(axis=1) for T in Ts]
    thi = [T.max(axis=1) for T in Ts]
    cents = [T.mean(axis=1) for T in Ts]

    def box_gap(plo, phi, qlo, qhi):
        g = np.maximum(np.maximum(qlo - phi, 0.0), plo - qhi)
        return np.sqrt(np.sum(g * g, axis=-1))

    def scan(Pc, m, ub):
        """Closest triangle of mesh m for each point, evaluating only triangles whose box
        distance to the point is <= ub (no other triangle can be as close)."""
        T = Ts[m]
        # triangles out of reach of the whole chunk, then of each point
        near = np.flatnonzero(box_gap(Pc.min(axis=0), Pc.max(axis=0), tlo[m], thi[m]) <= ub.max())
        lbt = box_gap(Pc[:, None], Pc[:, None], tlo[m][near][None], thi[m][near][None])
        pp, kk = np.nonzero(lbt <= ub[:, None])
        tt = near[kk]
        Q, d2 = closest_point_on_triangles(Pc[pp], T[tt, 0], T[tt, 1], T[tt, 2])
        order = np.lexsort((tt, d2, pp))                 # per point: smallest d2, then lowest index
        pp, tt, Q, d2 = pp[order], tt[order], Q[order], d2[order]
        first = np.ones(pp.size, dtype=bool)
        first[1:] = pp[1:] != pp[:-1]
        bq = np.zeros((Pc.shape[0], 3))
        bd = np.full(Pc.shape[0], np.inf)
        bt = np.zeros(Pc.shape[0], dtype=np.int64)
        bq[pp[first]], bd[pp[first]], bt[pp[first]] = Q[first], d2[first], tt[first] + base[m]
        return bq, bd, bt

    for s in range(0, P.shape[0], chunk):
        Pc = P[s:s + chunk]
        lb = box_gap(Pc[:, None], Pc[:, None], lo[None], hi[None])      # (points, meshes)
        m0 = int(np.argmin(lb.sum(axis=0)))
        # an upper bound per point: exact distance to a nearby triangle of mesh m0 (the
        # nearest centroid among the triangles closest to the chunk's box)
        dc = box_gap(Pc.min(axis=0), Pc.max(axis=0), tlo[m0], thi[m0])
        pool = np.argsort(dc, kind="stable")[:256]
        cd = np.sum((cents[m0][pool][None] - Pc[:, None]) ** 2, axis=2)
        tn = pool[np.argmin(cd, axis=1)]
        _, d2n = closest_point_on_triangles(Pc, Ts[m0][tn, 0], Ts[m0][tn, 1], Ts[m0][tn, 2])
        ub = np.sqrt(d2n) * (1 + 1e-12) + 1e-300
        cand = [m for m in range(len(Ts)) if np.any(lb[:, m] <= ub)]
        bq = np.zeros((Pc.shape[0], 3))
        bd = np.full(Pc.shape[0], np.inf)
        bt = np.zeros(Pc.shape[0], dtype=np.int64)
        for m in cand:                                   # index order, strict improvement
            q, d2, t = scan(Pc, m, ub)
            take = d2 < bd
            bq[take], bd[take], bt[take] = q[take], d2[take], t[take]
        out_q[s:s + chunk] = bq
        out_t[s:s + chunk] = bt
    return out_q, out_t


# ----------------------------------------------------------------------------- ghost tables

class GhostTable:
    """Per ghost entry: cell, BI, IP, base corner, flags, 8 (ref, weight) pairs, row scale;
    the closest triangle (global index), the Neumann coefficient kappa and the row's
    right-hand side d (see set_neumann); the row's own interpolation weight wself where it
    was moved to the left-hand side (0 otherwise), which Dirichlet rows need."""

    def __init__(self, n):
        self.cell = np.zeros(n, dtype=np.int64)
        self.bi = np.zeros((n, 3))
        self.ip = np.zeros((n, 3))
        self.base = np.zeros((n, 3), dtype=np.int32)
        self.flags = np.zeros(n, dtype=np.int32)
        self.ref = np.full((n, 8), -1, dtype=np.int64)
        self.w = np.zeros((n, 8))
        self.scale = np.zeros(n)
        self.tri = np.full(n, -1, dtype=np.int64)
        self.kappa = np.zeros(n)
        self.d = np.zeros(n)
        self.wself = np.zeros(n)

    def __len__(self):
        return self.cell.size


def row_kappa(grid: Grid, G: GhostTable, GC: np.ndarray, fallback: np.ndarray, moved: np.ndarray,
              ws: np.ndarray, best: np.ndarray) -> np.ndarray:
    """Neumann coefficient of each ghost row (dp/dn = q at the boundary, Sec. "Governing
    Equations and Numerical Methods": the moving-boundary pressure condition).

    The ghost value is the image-point value less the normal derivative times the distance
    along the row: g = p(IP) - l q with l = |IP - GC|, q the derivative along (IP - GC)/l.
    A row whose own weight w_self was moved to the left-hand side divides by 1 - w_self like
    its weights; a nearest-neighbour fallback row takes l = |centre(nb) - GC|.  The row reads
    g - sum w v = kappa q with kappa = -l (or -l / (1 - w_self))."""
    nz, ny, nx = grid.shape
    ex, ey, ez = G.ip[:, 0] - GC[:, 0], G.ip[:, 1] - GC[:, 1], G.ip[:, 2] - GC[:, 2]
    length = np.sqrt((ex * ex + ey * ey) + ez * ez)
    with np.errstate(divide="ignore", invalid="ignore"):
        kap = np.where(moved, -length / (1.0 - ws), -length)
    bb = np.where(best >= 0, best, 0)
    bi, bj, bk = bb % nx, (bb // nx) % ny, bb // (nx * ny)
    fx, fy, fz = grid.xc[bi] - GC[:, 0], grid.yc[bj] - GC[:, 1], grid.zc[bk] - GC[:, 2]
    lf = np.sqrt((fx * fx + fy * fy) + fz * fz)
    kap = np.where(fallback, np.where(best >= 0, -lf, 0.0), kap)
    return kap


def set_neumann(G: GhostTable, q: np.ndarray) -> None:
    """Ghost-row right-hand sides d = kappa q for the normal derivatives q along each row's
    direction (q = 0: the homogeneous condition of a fixed body)."""
    G.d = G.kappa * np.asarray(q, dtype=np.float64)


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
    BI, TRI = closest_points(GC, closed)
    IP = (BI + BI) - GC
    G.tri[:] = TRI
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
    ng = ghosts.size
    gk, gj, gi = ghosts // (nx * ny), (ghosts // nx) % ny, ghosts % nx
    rows = np.arange(ng)
    # the 8 corners: slot c = bx + 2 by + 4 bz
    lin = np.zeros((ng, 8), dtype=np.int64)
    w = np.zeros((ng, 8))
    for c in range(8):
        bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        lin[:, c] = ((k0 + bz) * ny + (j0 + by)) * nx + (i0 + bx)
        w[:, c] = (wx[:, bx] * wy[:, by]) * wz[:, bz]
    valid = flat[lin] != IBLANK_SOLID
    s = np.zeros(ng)
    for c in range(8):                                   # valid weights, summed in slot order
        s = s + np.where(valid[:, c], w[:, c], 0.0)
    fallback = s < WEIGHT_SUM_MIN
    with np.errstate(divide="ignore", invalid="ignore"):
        wn = np.where(valid, w / s[:, None], 0.0)
    is_self = valid & (lin == ghosts[:, None])
    has_self = is_self.any(axis=1)
    selfc = np.argmax(is_self, axis=1)
    ws = wn[rows, selfc]
    fallback |= has_self & (ws >= SELF_WEIGHT_MAX)
    move = has_self & ~fallback
    with np.errstate(divide="ignore", invalid="ignore"):
        wn = np.where(move[:, None], wn / (1.0 - ws)[:, None], wn)
    wn[rows[move], selfc[move]] = 0.0
    # nearest fluid face-neighbour of the ghost (to IP), for the fallback rows
    best = np.full(ng, -1, dtype=np.int64)
    bestd = np.full(ng, np.inf)
    for (di, dj, dk) in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        ii, jj, kk = gi + di, gj + dj, gk + dk
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
        l2 = np.where(ok, (kk * ny + jj) * nx + ii, 0)
        ok &= flat[l2] == IBLANK_FLUID
        ex = IP[:, 0] - grid.xc[np.clip(ii, 0, nx - 1)]
        ey = IP[:, 1] - grid.yc[np.clip(jj, 0, ny - 1)]
        ez = IP[:, 2] - grid.zc[np.clip(kk, 0, nz - 1)]
        d2 = (ex * ex + ey * ey) + ez * ez
        take = ok & (d2 < bestd)
        best[take], bestd[take] = l2[take], d2[take]
    G.flags[:] = np.where(fallback, FLAG_FALLBACK,
                          np.sum(valid.astype(np.int32) << np.arange(8), axis=1) << 8).astype(np.int32)
    G.w[:] = np.where(fallback[:, None], 0.0, wn)
    G.ref[:] = np.where(fallback[:, None], -1, np.where(wn != 0.0, lin, -1))
    G.w[fallback, 0] = 1.0
    G.ref[fallback, 0] = best[fallback]
    G.kappa[:] = row_kappa(grid, G, GC, fallback, move, ws, best)
    G.wself[:] = np.where(move, ws, 0.0)
    # row scale: coefficients of the fluid rows that reference this ghost, in direction order
    sc = np.zeros(ng)
    for (di, dj, dk, cf, idx) in ((-1, 0, 0, grid.cxp, gi - 1), (1, 0, 0, grid.cxm, gi + 1),
                                  (0, -1, 0, grid.cyp, gj - 1), (0, 1, 0, grid.cym, gj + 1),
                                  (0, 0, -1, grid.czp, gk - 1), (0, 0, 1, grid.czm, gk + 1)):
        ii, jj, kk = gi + di, gj + dj, gk + dk
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
        l2 = np.where(ok, (kk * ny + jj) * nx + ii, 0)
        ok &= flat[l2] == IBLANK_FLUID
        n_ax = cf.size
        sc = sc + np.where(ok, cf[np.clip(idx, 0, n_ax - 1)], 0.0)
    G.scale[:] = sc
    return G


def classify(grid: Grid, meshes):
    """Closed bodies: (iblank uint8 [k][j][i], ghost table)."""
    ib = iblank_closed(grid, meshes)
    ghosts = mark_ghosts(ib)
    return ib, ghost_tables(grid, ib, ghosts, meshes)
