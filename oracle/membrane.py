"""Zero-thickness membranes: cut links, sided ghost entries, image points and the system (oracle).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

Paper: Sec. "GPU Porting" items 1 and 2 (iblanking and the ghost-cell modules) and the
membrane wings of Sec. "Fluid-Structure Interaction in Bat" (a thin membrane moving
through the fluid).  The paper gives no formulas for ghost cells of a zero-thickness
surface; the readings taken here:

* Membranes and closed bodies are not mixed in one classification; with membranes only,
  every cell is a fluid row (iblank 0).
* Cut link.  The segment between the centres of face-neighbours i and j (snapped to the
  lattice 2^-24 like the closed-body test) is cut when a membrane triangle covers the
  segment's line in the projection along the segment's axis (edge functions with the
  top-left rule, as for the closed-body column test) and the crossing coordinate lies
  strictly between the two centres (exact rational comparison).  A triangle parallel to
  the axis cuts nothing.
* Side.  side(i) of a cut link is the sign of orient3d(A, B, C, centre i) of the crossing
  triangle (vertex order as given): 1 when positive, 0 otherwise.  When several triangles
  cross one link, the one with the lowest index decides both ends' sides.
* Ghost entries.  Every cut link i -> j gives the entry (j, side(i)): the value of cell j
  as seen from i's side.  Entries are unique, ordered by cell, then side.  Fluid row i uses
  g_(j, side(i)) in place of p_j across a cut link.
* Boundary intercept and image point: BI = closest point of the membrane triangles to the
  centre GC of j (lowest triangle index on ties), IP = 2 BI - GC; base corner and
  trilinear weights as for closed bodies.
* Corners.  A corner cell k is used with its own value p_k when the segment
  snap(IP) -> snap(centre k) is not cut (``segments_cut``); otherwise with the value of the
  entry (k, s) of the same side s if that entry exists (this covers GC itself, whose
  weight then moves to the left-hand side); otherwise its weight is dropped.  The rest
  is renormalised.  If the sum is below 1e-3, or the own weight reaches 1 - 1e-12, the
  entry takes the value of the nearest (to IP) cell among the face-neighbours of j that
  cut to j from side s (weight 1); such a neighbour exists, since it created the entry.
* Ghost row scale: the sum of the face coefficients of the fluid rows that use the entry.
* A reference to a ghost entry is stored as ncell + entry index.

Segment-triangle test (``segments_cut``): the endpoints lie strictly on opposite sides of
the triangle's plane and the segment's line passes through the closed triangle (the
three orientations of the line against the edges share a sign or vanish).

Parity status: cut links and sides are pinned by an independent brute force over
(link, triangle) pairs in exact rational arithmetic; the system by the grid-aligned plate
spanning the box (two independent Neumann sub-boxes, solved by DCT), a finite plate whose
normal derivative of a manufactured field vanishes (second order), invariants (A 1 = 0)
and a planted wrong side (tests/test_oracle_membrane.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .classify import (FLAG_FALLBACK, SELF_WEIGHT_MAX, WEIGHT_SUM_MIN, GhostTable, _base_and_t, closest_points, row_kappa,
                       snap)
from .grid import Grid

# direction d of a link from cell i: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z (bit d of cut / side)
DIRS = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def _orient3d_exact(a, b, c, d) -> int:
    """(d - a) . ((b - a) x (c - a)) in exact integers."""
    ab = [int(b[q]) - int(a[q]) for q in range(3)]
    ac = [int(c[q]) - int(a[q]) for q in range(3)]
    ad = [int(d[q]) - int(a[q]) for q in range(3)]
    n = (ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2], ab[0] * ac[1] - ab[1] * ac[0])
    return ad[0] * n[0] + ad[1] * n[1] + ad[2] * n[2]


def _sgn(v: int) -> int:
    return (v > 0) - (v < 0)


def membrane_triangles(meshes):
    """Snapped vertices (T, 3, 3) int64 of every membrane triangle, in global index order."""
    out = [snap(np.asarray(m.verts, dtype=np.float64))[np.asarray(m.tris, dtype=np.int64)]
           for m in meshes if not int(m.closed)]
    return np.concatenate(out) if out else np.zeros((0, 3, 3), dtype=np.int64)


def cut_links(grid: Grid, meshes):
    """(cut, side): uint8 [k][j][i] arrays; bit d of cut: the link from the cell in direction d
    is cut; bit d of side: the cell's side of that link."""
    nz, ny, nx = grid.shape
    C = [snap(grid.xc), snap(grid.yc), snap(grid.zc)]
    T = membrane_triangles(meshes)
    cut = np.zeros((nz, ny, nx), dtype=np.uint8)
    side = np.zeros((nz, ny, nx), dtype=np.uint8)
    # crossing triangle of each link: key (axis, lower cell linear index) -> lowest triangle index
    best = {}
    for a in range(3):
        u_ax, v_ax = (a + 1) % 3, (a + 2) % 3
        Cu, Cv, Ca = C[u_ax], C[v_ax], C[a]
        for t in range(T.shape[0]):
            P = [T[t, q] for q in range(3)]
            A2 = [(int(p[u_ax]), int(p[v_ax])) for p in P]
            D = (A2[1][0] - A2[0][0]) * (A2[2][1] - A2[0][1]) - (A2[1][1] - A2[0][1]) * (A2[2][0] - A2[0][0])
            if D == 0:
                continue
            idx = [0, 1, 2] if D > 0 else [0, 2, 1]          # counter-clockwise in (u, v)
            D = abs(D)
            pa, pb, pc = [A2[q] for q in idx]
            za, zb, zc = [int(P[q][a]) for q in idx]
            ulo, uhi = min(pa[0], pb[0], pc[0]), max(pa[0], pb[0], pc[0])
            vlo, vhi = min(pa[1], pb[1], pc[1]), max(pa[1], pb[1], pc[1])
            iu0, iu1 = np.searchsorted(Cu, ulo, "left"), np.searchsorted(Cu, uhi, "right")
            iv0, iv1 = np.searchsorted(Cv, vlo, "left"), np.searchsorted(Cv, vhi, "right")

            def tl(p, q):
                return (q[0] > p[0]) or (q[0] == p[0] and p[1] > q[1])

            for iu in range(iu0, iu1):
                for iv in range(iv0, iv1):
                    qu, qv = int(Cu[iu]), int(Cv[iv])
                    wa = (pc[0] - pb[0]) * (qv - pb[1]) - (pc[1] - pb[1]) * (qu - pb[0])
                    wb = (pa[0] - pc[0]) * (qv - pc[1]) - (pa[1] - pc[1]) * (qu - pc[0])
                    wc = (pb[0] - pa[0]) * (qv - pa[1]) - (pb[1] - pa[1]) * (qu - pa[0])
                    if not ((wa > 0 or (wa == 0 and tl(pb, pc))) and (wb > 0 or (wb == 0 and tl(pc, pa)))
                            and (wc > 0 or (wc == 0 and tl(pa, pb)))):
                        continue
                    N = wa * za + wb * zb + wc * zc              # crossing coordinate N / D
                    q, r = divmod(N, D)
                    m = int(np.searchsorted(Ca, q, "right" if r > 0 else "left"))   # centres < N/D
                    lo = m - 1
                    if lo < 0 or lo + 1 >= Ca.size or not int(Ca[lo + 1]) > q:
                        continue
                    ijk = [0, 0, 0]
                    ijk[a], ijk[u_ax], ijk[v_ax] = lo, iu, iv
                    key = (a, (ijk[2] * ny + ijk[1]) * nx + ijk[0])
                    if key not in best or t < best[key]:
                        best[key] = t
    flat_cut, flat_side = cut.reshape(-1), side.reshape(-1)
    step = (1, nx, nx * ny)
    for (a, lin_lo), t in best.items():
        P = [T[t, q] for q in range(3)]
        for end, lin in ((0, lin_lo), (1, lin_lo + step[a])):
            cc = [int(C[0][lin % nx]), int(C[1][(lin // nx) % ny]), int(C[2][lin // (nx * ny)])]
            d = 2 * a + (1 if end == 0 else 0)    # the lower end looks in +a, the upper in -a
            flat_cut[lin] |= np.uint8(1 << d)
            if _orient3d_exact(P[0], P[1], P[2], cc) > 0:
                flat_side[lin] |= np.uint8(1 << d)
    return cut, side


def ghost_entries(grid: Grid, cut: np.ndarray, side: np.ndarray):
    """Unique (cell, side) pairs of the cut links, ordered by cell then side."""
    nz, ny, nx = grid.shape
    keys = []
    for d, (di, dj, dk) in enumerate(DIRS):
        kk, jj, ii = np.nonzero((cut >> d) & 1)
        nb = ((kk + dk) * ny + (jj + dj)) * nx + (ii + di)
        s = (side[kk, jj, ii] >> d) & 1
        keys.append(nb.astype(np.int64) * 2 + s.astype(np.int64))
    keys = np.unique(np.concatenate(keys)) if keys else np.zeros(0, dtype=np.int64)
    return keys // 2, (keys % 2).astype(np.uint8)


def segments_cut(P: np.ndarray, Q: np.ndarray, T: np.ndarray) -> np.ndarray:
    """For snapped points P[n], Q[n] (int64 (n, 3)): is the segment P-Q cut by any triangle of T?"""
    out = np.zeros(P.shape[0], dtype=bool)
    if T.shape[0] == 0:
        return out
    tlo, thi = T.min(axis=1), T.max(axis=1)
    for e in range(P.shape[0]):
        p, q = P[e], Q[e]
        lo, hi = np.minimum(p, q), np.maximum(p, q)
        near = np.flatnonzero(np.all(thi >= lo, axis=1) & np.all(tlo <= hi, axis=1))
        for t in near:
            a, b, c = T[t, 0], T[t, 1], T[t, 2]
            sp_, sq = _sgn(_orient3d_exact(a, b, c, p)), _sgn(_orient3d_exact(a, b, c, q))
            if sp_ == 0 or sq == 0 or sp_ == sq:
                continue
            e1 = _sgn(_orient3d_exact(p, q, a, b))
            e2 = _sgn(_orient3d_exact(p, q, b, c))
            e3 = _sgn(_orient3d_exact(p, q, c, a))
            if (e1 >= 0 and e2 >= 0 and e3 >= 0) or (e1 <= 0 and e2 <= 0 and e3 <= 0):
                out[e] = True
                break
    return out


class MembraneTables(GhostTable):
    """GhostTable of membrane entries, plus the entry side and the cut/side arrays."""

    def __init__(self, n):
        super().__init__(n)
        self.side = np.zeros(n, dtype=np.uint8)
        self.cut = None
        self.cside = None


def ghost_tables(grid: Grid, cut: np.ndarray, side: np.ndarray, meshes) -> MembraneTables:
    """Image points and interpolation rows of the membrane ghost entries (see module doc)."""
    nz, ny, nx = grid.shape
    ncell = nz * ny * nx
    gcell, gside = ghost_entries(grid, cut, side)
    ng = gcell.size
    G = MembraneTables(ng)
    G.cut, G.cside = cut, side
    G.cell[:] = gcell
    G.side[:] = gside
    if ng == 0:
        return G
    mem = [m for m in meshes if not int(m.closed)]
    T = membrane_triangles(mem)
    GC = grid.centre(gcell)
    BI, TRI = closest_points(GC, mem)
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
    rows = np.arange(ng)
    lin = np.zeros((ng, 8), dtype=np.int64)
    w = np.zeros((ng, 8))
    for c in range(8):
        bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        lin[:, c] = ((k0 + bz) * ny + (j0 + by)) * nx + (i0 + bx)
        w[:, c] = (wx[:, bx] * wy[:, by]) * wz[:, bz]
    # corner values: own value if IP -> corner is not cut, else the same-side entry if any
    key_of = {(int(c), int(s)): e for e, (c, s) in enumerate(zip(gcell, gside))}
    sIP = snap(IP)
    Csn = np.stack([snap(grid.xc)[lin % nx], snap(grid.yc)[(lin // nx) % ny], snap(grid.zc)[lin // (nx * ny)]], -1)
    blocked = segments_cut(np.repeat(sIP, 8, axis=0), Csn.reshape(-1, 3), T).reshape(ng, 8)
    ref = np.full((ng, 8), -1, dtype=np.int64)
    valid = np.zeros((ng, 8), dtype=bool)
    for g in range(ng):
        for c in range(8):
            if not blocked[g, c]:
                ref[g, c], valid[g, c] = lin[g, c], True
            else:
                e = key_of.get((int(lin[g, c]), int(gside[g])))
                if e is not None:
                    ref[g, c], valid[g, c] = ncell + e, True
    s = np.zeros(ng)
    for c in range(8):
        s = s + np.where(valid[:, c], w[:, c], 0.0)
    fallback = s < WEIGHT_SUM_MIN
    with np.errstate(divide="ignore", invalid="ignore"):
        wn = np.where(valid, w / s[:, None], 0.0)
    is_self = valid & (ref == (ncell + rows)[:, None])
    has_self = is_self.any(axis=1)
    selfc = np.argmax(is_self, axis=1)
    ws = wn[rows, selfc]
    fallback |= has_self & (ws >= SELF_WEIGHT_MAX)
    move = has_self & ~fallback
    with np.errstate(divide="ignore", invalid="ignore"):
        wn = np.where(move[:, None], wn / (1.0 - ws)[:, None], wn)
    wn[rows[move], selfc[move]] = 0.0
    # the cells that use the entry: face-neighbours n of j whose link n -> j is cut from side s
    gk, gj, gi = gcell // (nx * ny), (gcell // nx) % ny, gcell % nx
    best = np.full(ng, -1, dtype=np.int64)
    bestd = np.full(ng, np.inf)
    sc = np.zeros(ng)
    coef = (grid.cxp, grid.cxm, grid.cyp, grid.cym, grid.czp, grid.czm)
    for d, (di, dj, dk) in enumerate(DIRS):
        ii, jj, kk = gi + di, gj + dj, gk + dk
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
        iic, jjc, kkc = np.clip(ii, 0, nx - 1), np.clip(jj, 0, ny - 1), np.clip(kk, 0, nz - 1)
        back = d ^ 1                                       # direction from n back to j
        ok &= ((cut[kkc, jjc, iic] >> back) & 1).astype(bool)
        ok &= ((side[kkc, jjc, iic] >> back) & 1) == gside
        l2 = (kkc * ny + jjc) * nx + iic
        ex = IP[:, 0] - grid.xc[iic]
        ey = IP[:, 1] - grid.yc[jjc]
        ez = IP[:, 2] - grid.zc[kkc]
        d2 = (ex * ex + ey * ey) + ez * ez
        take = ok & (d2 < bestd)
        best[take], bestd[take] = l2[take], d2[take]
        axis_idx = (iic, iic, jjc, jjc, kkc, kkc)[d]
        sc = sc + np.where(ok, coef[d][axis_idx], 0.0)
    G.flags[:] = np.where(fallback, FLAG_FALLBACK,
                          np.sum(valid.astype(np.int32) << np.arange(8), axis=1) << 8).astype(np.int32)
    G.w[:] = np.where(fallback[:, None], 0.0, wn)
    G.ref[:] = np.where(fallback[:, None], -1, np.where(wn != 0.0, ref, -1))
    G.w[fallback, 0] = 1.0
    G.ref[fallback, 0] = best[fallback]
    G.scale[:] = sc
    G.tri[:] = TRI
    G.kappa[:] = row_kappa(grid, G, GC, fallback, move, ws, best)
    G.wself[:] = np.where(move, ws, 0.0)
    return G


def classify(grid: Grid, meshes):
    """Membranes only: (iblank zeros uint8 [k][j][i], MembraneTables)."""
    if any(int(m.closed) for m in meshes):
        raise ValueError("membranes and closed bodies are not mixed")
    cut, side = cut_links(grid, meshes)
    return np.zeros(grid.shape, dtype=np.uint8), ghost_tables(grid, cut, side, meshes)


# ----------------------------------------------------------------------------- system

def _entry_index(grid: Grid, G: MembraneTables):
    return {(int(c), int(s)): e for e, (c, s) in enumerate(zip(G.cell, G.side))}


def assemble(grid: Grid, G: MembraneTables):
    """Sparse A over [cells (all fluid rows), ghost entries] (CSR)."""
    nz, ny, nx = grid.shape
    ncell = nz * ny * nx
    ng = len(G)
    key = _entry_index(grid, G)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kk, jj, ii = kk.ravel(), jj.ravel(), ii.ravel()
    lin = np.arange(ncell)
    cutf, sidef = G.cut.reshape(-1), G.cside.reshape(-1)
    rows, cols, vals = [], [], []
    diag = np.zeros(ncell)
    coefs = (grid.cxm[ii], grid.cxp[ii], grid.cym[jj], grid.cyp[jj], grid.czm[kk], grid.czp[kk])
    for d, (di, dj, dk) in enumerate(DIRS):
        c = coefs[d]
        ok = c != 0.0
        nb = ((kk + dk) * ny + (jj + dj)) * nx + (ii + di)
        iscut = ((cutf >> d) & 1).astype(bool) & ok
        col = np.where(ok, nb, 0)
        for q in np.flatnonzero(iscut):
            col[q] = ncell + key[(int(nb[q]), int((sidef[q] >> d) & 1))]
        rows.append(lin[ok]); cols.append(col[ok]); vals.append(c[ok])
        diag -= c
    rows.append(lin); cols.append(lin); vals.append(diag)
    if ng:
        grow = ncell + np.arange(ng)
        rows.append(grow); cols.append(grow); vals.append(np.ones(ng))
        m = G.ref >= 0
        rows.append(np.repeat(grow, 8)[m.ravel()]); cols.append(G.ref[m]); vals.append(-G.w[m])
    R = np.concatenate(rows); Cc = np.concatenate(cols); Vv = np.concatenate(vals)
    A = sp.csr_matrix((Vv, (R, Cc)), shape=(ncell + ng, ncell + ng))
    is_fluid = np.concatenate([np.ones(ncell, dtype=bool), np.zeros(ng, dtype=bool)])
    return A, is_fluid


def solve_sparse(grid: Grid, G: MembraneTables, b: np.ndarray):
    """(p [k][j][i], g per entry, lambda) of the bordered system by a pinned SuperLU solve."""
    A, is_fluid = assemble(grid, G)
    ncell = int(np.prod(grid.shape))
    i0 = 0
    At = A.tolil(copy=True)
    At[i0, :] = 0.0
    At[i0, i0] = 1.0
    lu = spl.splu(sp.csc_matrix(At), permc_spec="COLAMD")
    bb = np.concatenate([b.ravel(), G.d])
    one = is_fluid.astype(np.float64)
    r1 = bb.copy(); r1[i0] = 0.0
    r2 = one.copy(); r2[i0] = 0.0
    q1, q2 = lu.solve(r1), lu.solve(r2)
    lam = float((bb[i0] - (A[i0] @ q1)[0]) / (1.0 - (A[i0] @ q2)[0]))
    x = q1 - lam * q2
    V = grid.volumes().ravel()
    mean = float(np.sum(V * x[:ncell]) / np.sum(V))
    return (x[:ncell] - mean).reshape(grid.shape), x[ncell:] - mean, lam


def residual(grid: Grid, G: MembraneTables, b: np.ndarray, p: np.ndarray, g: np.ndarray, lam: float = 0.0):
    """(r_fluid [k][j][i], r_ghost per entry) of r = b - lambda - A u."""
    A, _ = assemble(grid, G)
    ncell = int(np.prod(grid.shape))
    u = np.concatenate([p.ravel(), g])
    Au = A @ u
    rf = (b.ravel() - lam) - Au[:ncell]
    rg = G.d - Au[ncell:]
    return rf.reshape(grid.shape), rg


def relative_residual(grid: Grid, G: MembraneTables, b: np.ndarray, p: np.ndarray, g: np.ndarray) -> float:
    """||S P r|| / ||S P b|| over cells and entries (lambda drops out under the projection)."""
    V = grid.volumes()
    fv = float(np.sum(V))

    def pnorm(rf, rg):
        mu = float(np.sum(V * rf)) / fv
        return float(np.sqrt(np.sum((rf - mu) ** 2) + np.sum((G.scale * rg) ** 2)))

    rf, rg = residual(grid, G, b, p, g)
    return pnorm(rf, rg) / pnorm(b, np.zeros(len(G)))
