"""The discrete pressure Poisson system with ghost rows, its residual and gauge (oracle).

Paper: Sec. "Governing Equations and Numerical Methods" (the pressure Poisson
equation of the fractional-step method, second-order finite differences) and
Sec. "GPU Porting" item 2 (ghost-cell boundary condition).  Readings:

* Unknowns ("active rows"): the pressure p_i of every fluid cell and the value
  g_G of every ghost entry.  For closed bodies a ghost entry lives at its solid
  cell, so a full [k][j][i] array holds both (plain solid cells hold 0).
* Fluid row i:  sum_d c_{i,d} (v_nb - p_i) = b_i - lambda, where v_nb is the
  neighbour's pressure, or its ghost value when the neighbour is a ghost.
* Ghost row G:  g_G - sum_k w_k v_k = 0 (dp/dn = 0 at the boundary intercept:
  the ghost copies the interpolated value at its image point).
* lambda (one scalar on all fluid rows) absorbs the inconsistency that the
  non-symmetric ghost rows leave in a pure-Neumann problem; the gauge is the
  volume-weighted zero mean of p over fluid cells.  The bordered system
  [A 1_F; V_F^T 0][p; lambda] = [b; 0] has a unique solution.
* Residual r = b - A p on active rows (ghost rows: r_G = sum_k w_k v_k - g_G).
  Projected residual P r: the volume-weighted mean of r over fluid rows is
  removed from fluid rows.  Ghost rows are scaled by s_G (the sum of the
  coefficients of the fluid rows that reference them).  Relative residual =
  ||S P r||_2 / ||S P b||_2 over active rows.  The fluid-row mean of b does not
  change p (lambda absorbs it), so b is used as given on fluid rows and ignored
  elsewhere.

Parity status: pinned by DCT-II and separable eigen solves (no body), second
order on a manufactured solution, the grid-aligned wall that reduces to a
Neumann sub-box, and invariants (A 1 = 0, symmetry of V A without a body,
telescoping sums) -- tests/test_oracle_system.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .classify import IBLANK_FLUID, IBLANK_SOLID, GhostTable
from .grid import Grid


def _nb_terms(grid: Grid):
    """(axis, shift, coefficient array broadcast to [k][j][i]) for the six directions."""
    cx = lambda a: a[None, None, :]
    cy = lambda a: a[None, :, None]
    cz = lambda a: a[:, None, None]
    return [(2, -1, cx(grid.cxm)), (2, 1, cx(grid.cxp)), (1, -1, cy(grid.cym)), (1, 1, cy(grid.cyp)),
            (0, -1, cz(grid.czm)), (0, 1, cz(grid.czp))]


def _shifted(p: np.ndarray, axis: int, s: int) -> np.ndarray:
    """Neighbour values p[idx + s along axis]; zero outside (their coefficient is 0)."""
    out = np.zeros_like(p)
    src = [slice(None)] * 3
    dst = [slice(None)] * 3
    if s < 0:
        src[axis] = slice(0, -1); dst[axis] = slice(1, None)
    else:
        src[axis] = slice(1, None); dst[axis] = slice(0, -1)
    out[tuple(dst)] = p[tuple(src)]
    return out


def apply_fluid(grid: Grid, p: np.ndarray, slab: int = 32) -> np.ndarray:
    """(A p)_i = sum_d c_{i,d} (p_nb - p_i) on every cell of the full array.

    Evaluated slab by slab along z (each slab with one halo plane), so large grids need
    only a few slab-sized temporaries; every cell's arithmetic is the same.
    """
    nz = p.shape[0]
    out = np.empty_like(p)
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        a, b = max(0, k0 - 1), min(nz, k1 + 1)
        sub = p[a:b]
        zc = Grid.__new__(Grid)
        zc.czm, zc.czp = grid.czm[a:b], grid.czp[a:b]
        zc.cym, zc.cyp, zc.cxm, zc.cxp = grid.cym, grid.cyp, grid.cxm, grid.cxp
        acc = np.zeros_like(sub)
        for axis, s_, c in _nb_terms(zc):
            acc += c * (_shifted(sub, axis, s_) - sub)
        out[k0:k1] = acc[k0 - a:k0 - a + (k1 - k0)]
    return out


def ghost_values_interp(G: GhostTable, pfull: np.ndarray) -> np.ndarray:
    """sum_k w_k v_k per ghost entry (v read from the full array)."""
    flat = pfull.ravel()
    ref = np.where(G.ref >= 0, G.ref, 0)
    return np.sum(np.where(G.ref >= 0, G.w * flat[ref], 0.0), axis=1)


def residual(grid: Grid, iblank: np.ndarray, G: GhostTable, b: np.ndarray, pfull: np.ndarray, lam: float = 0.0):
    """(r_fluid [k][j][i] (0 off fluid rows), r_ghost per entry) for r = b - lambda - A p."""
    rf = apply_fluid(grid, pfull)
    np.subtract(b - lam if lam else b, rf, out=rf)
    rf[iblank != IBLANK_FLUID] = 0.0
    rg = (ghost_values_interp(G, pfull) - pfull.ravel()[G.cell]) + G.d if len(G) else np.zeros(0)
    return rf, rg


def _slabs(n, slab=64):
    return [(k0, min(n, k0 + slab)) for k0 in range(0, n, slab)]


def fluid_mean(grid: Grid, iblank: np.ndarray, v: np.ndarray) -> float:
    """Volume-weighted mean of v over fluid cells (summed slab by slab along z)."""
    num = den = 0.0
    for k0, k1 in _slabs(v.shape[0]):
        fluid = iblank[k0:k1] == IBLANK_FLUID
        V = grid.dz[k0:k1, None, None] * grid.dy[None, :, None] * grid.dx[None, None, :]
        num += float(np.sum(np.where(fluid, V * v[k0:k1], 0.0)))
        den += float(np.sum(np.where(fluid, V, 0.0)))
    return num / den


def projected_norm(grid: Grid, iblank: np.ndarray, G: GhostTable, rf: np.ndarray, rg: np.ndarray) -> float:
    """||S P r||_2 over active rows."""
    mu = fluid_mean(grid, iblank, rf)
    acc = 0.0
    for k0, k1 in _slabs(rf.shape[0]):
        pf = np.where(iblank[k0:k1] == IBLANK_FLUID, rf[k0:k1] - mu, 0.0)
        acc += float(np.sum(pf * pf))
    sg = G.scale * rg if len(G) else np.zeros(0)
    return float(np.sqrt(acc + np.sum(sg * sg)))


def relative_residual(grid: Grid, iblank: np.ndarray, G: GhostTable, b: np.ndarray, pfull: np.ndarray) -> float:
    """||S P (b - A p)|| / ||S P b||  (lambda drops out under the projection)."""
    den = projected_norm(grid, iblank, G, b, np.zeros(len(G)))    # fluid rows of b; ghost rows 0
    rf, rg = residual(grid, iblank, G, b, pfull)
    return projected_norm(grid, iblank, G, rf, rg) / den


def gauge(grid: Grid, iblank: np.ndarray, pfull: np.ndarray) -> np.ndarray:
    """Subtract the volume-weighted fluid mean from every active value; solid cells stay 0."""
    mu = fluid_mean(grid, iblank, pfull)
    active = iblank != IBLANK_SOLID
    return np.where(active, pfull - mu, 0.0)


# ----------------------------------------------------------------------------- assembly

def active_index(iblank: np.ndarray):
    """Linear cell indices of active rows (fluid or ghost), and the cell -> row map."""
    flat = iblank.ravel()
    cells = np.flatnonzero(flat != IBLANK_SOLID).astype(np.int64)
    row = np.full(flat.size, -1, dtype=np.int64)
    row[cells] = np.arange(cells.size)
    return cells, row


def assemble(grid: Grid, iblank: np.ndarray, G: GhostTable):
    """Sparse A over active rows (CSR), the row map and the fluid-row mask."""
    nz, ny, nx = grid.shape
    flat = iblank.ravel()
    cells, row = active_index(iblank)
    fluid_cells = np.flatnonzero(flat == IBLANK_FLUID).astype(np.int64)
    i = fluid_cells % nx; j = (fluid_cells // nx) % ny; k = fluid_cells // (nx * ny)
    rows, cols, vals = [], [], []
    diag = np.zeros(fluid_cells.size)
    for (di, dj, dk, c) in ((-1, 0, 0, grid.cxm[i]), (1, 0, 0, grid.cxp[i]), (0, -1, 0, grid.cym[j]),
                            (0, 1, 0, grid.cyp[j]), (0, 0, -1, grid.czm[k]), (0, 0, 1, grid.czp[k])):
        ok = c != 0.0
        nb = ((k + dk) * ny + (j + dj)) * nx + (i + di)
        nb = np.where(ok, nb, 0)
        rows.append(row[fluid_cells[ok]]); cols.append(row[nb[ok]]); vals.append(c[ok])
        diag -= c
    rows.append(row[fluid_cells]); cols.append(row[fluid_cells]); vals.append(diag)
    if len(G):
        grow = row[G.cell]
        rows.append(grow); cols.append(grow); vals.append(np.ones(len(G)))
        m = G.ref >= 0
        rows.append(np.repeat(grow, 8)[m.ravel()]); cols.append(row[G.ref[m]]); vals.append(-G.w[m])
    R = np.concatenate(rows); Cc = np.concatenate(cols); Vv = np.concatenate(vals)
    if np.any(Cc < 0):
        raise ValueError("a fluid row or ghost row references a plain solid cell")
    A = sp.csr_matrix((Vv, (R, Cc)), shape=(cells.size, cells.size))
    is_fluid = flat[cells] == IBLANK_FLUID
    return A, cells, is_fluid
