"""Advection-diffusion (Helmholtz-type) velocity systems of the fractional step, with no-slip
ghost rows (oracle).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU legs use
this module; the GPU library never calls it.

Paper: Sec. "Governing Equations and Numerical Methods" -- the fractional step splits the
momentum equation into an advection-diffusion step, solved with scheduled relaxed Jacobi
(SRJ) iterations, and the pressure Poisson equation; Sec. "Results and Discussions" -- the
advection-diffusion system is diagonally dominant and cheap next to the pressure solve;
Sec. "GPU Porting", item 2 -- the ghost-cell modules impose no-slip and no-penetration on
the immersed surface.  The paper gives no discretisation of the step.  Readings:

* Each velocity component u solves (I - alpha L) u = f: alpha = dt nu / 2 for Crank-Nicolson
  diffusion, the explicit terms (advection, the old diffusion half, the pressure gradient)
  gathered in f by the caller; L is the pressure system's 7-point operator with zero flux
  across the outer walls.  Fluid row i:
      D_i u_i - alpha sum_d c_{i,d} v_nb(i,d) = f_i,   D_i = 1 + alpha sum_d c_{i,d},
  v_nb the neighbour's value, or the ghost value across the body (closed bodies: the ghost
  cell; membranes: the entry of the neighbour on this cell's side of the cut link).
* Ghost rows impose the boundary value u_b at BI, the midpoint of GC and its image point:
  (u_G + u(IP)) / 2 = u_b with u(IP) from the image-point weights.  The stored weights w_k
  are already divided by 1 - w_s, w_s the row's own weight moved to the left-hand side, so
      (1 + w_s) u_G + (1 - w_s) sum_k w_k v_k = 2 u_b;
  a nearest-neighbour fallback row (w_s = 0, weight 1) reads u_G + v_nb = 2 u_b.  Membrane
  entries on both sides of a cell share its BI and so its u_b (no slip on either side).
  In terms of the pressure system's matrix A (fluid rows sum c (v - u), ghost rows
  g - sum w v): fluid rows of H are those of I - alpha A, ghost rows those of
  2 I - (1 - w_s) A.
* Convergence measure: ||S (b - H x)|| / ||S b|| over fluid and ghost rows, S = 1 on fluid
  rows and alpha s_G on ghost rows (s_G: the coefficients of the fluid rows that reference
  the entry, so S puts a ghost row on the scale at which it enters the fluid rows).
* Rigid boundary velocity: u_b = v0 + omega x (BI - centre) for the mesh holding the
  entry's closest triangle.

The oracle solves the system directly (sparse LU); the GPU path iterates to it.

Parity status: pinned by the DCT-II closed form with no body, second-order convergence to a
manufactured field with a body (planted ghost-row mistakes fail), exact constant fields on
closed bodies and membranes, and finite differences of the moving plate for the rigid
velocity (tests/test_oracle_helmholtz.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import membrane as OM
from .classify import GhostTable
from .grid import Grid
from .system import assemble


def _helmholtz_from(A, is_fluid: np.ndarray, ghost_row: np.ndarray, wself: np.ndarray, alpha: float):
    """H = diag(s) - diag(a) A with s = 1, a = alpha on fluid rows and s = 2,
    a = 1 - w_s on ghost rows (ghost_row: the row of each ghost entry)."""
    n = A.shape[0]
    s = np.where(is_fluid, 1.0, 0.0)
    a = np.where(is_fluid, alpha, 0.0)
    s[ghost_row] = 2.0
    a[ghost_row] = 1.0 - wself
    return (sp.diags(s) - sp.diags(a) @ A).tocsr(), s


def system_closed(grid: Grid, iblank: np.ndarray, G: GhostTable, alpha: float):
    """(H over the active cells, cells, is_fluid, row of each ghost)."""
    A, cells, is_fluid = assemble(grid, iblank, G)
    row = np.full(int(np.prod(grid.shape)), -1, dtype=np.int64)
    row[cells] = np.arange(cells.size)
    grow = row[G.cell]
    H, _ = _helmholtz_from(A, is_fluid, grow, G.wself, alpha)
    return H, cells, is_fluid, grow


def system_membrane(grid: Grid, G, alpha: float):
    """(H over [cells, entries], is_fluid, row of each entry)."""
    A, is_fluid = OM.assemble(grid, G)
    ncell = int(np.prod(grid.shape))
    grow = ncell + np.arange(len(G))
    H, _ = _helmholtz_from(A, is_fluid, grow, G.wself, alpha)
    return H, is_fluid, grow


def _rhs(n, f_rows, grow, ub):
    b = np.zeros(n)
    b[: f_rows.size] = f_rows
    b[grow] = 2.0 * np.asarray(ub, dtype=np.float64)
    return b


def solve_closed(grid: Grid, iblank: np.ndarray, G: GhostTable, alpha: float, f: np.ndarray, ub=None):
    """u [k][j][i]: fluid values, ghost values at the ghost cells, 0 elsewhere."""
    H, cells, is_fluid, grow = system_closed(grid, iblank, G, alpha)
    ubv = np.zeros(len(G)) if ub is None else ub
    b = np.where(is_fluid, np.asarray(f, dtype=np.float64).ravel()[cells], 0.0)
    b[grow] = 2.0 * np.asarray(ubv, dtype=np.float64)
    x = spl.spsolve(sp.csc_matrix(H), b)
    out = np.zeros(int(np.prod(grid.shape)))
    out[cells] = x
    return out.reshape(grid.shape)


def solve_membrane(grid: Grid, G, alpha: float, f: np.ndarray, ub=None):
    """(u [k][j][i] on every cell, u per entry)."""
    H, is_fluid, grow = system_membrane(grid, G, alpha)
    ncell = int(np.prod(grid.shape))
    ubv = np.zeros(len(G)) if ub is None else ub
    b = _rhs(H.shape[0], np.asarray(f, dtype=np.float64).ravel(), grow, ubv)
    x = spl.spsolve(sp.csc_matrix(H), b)
    return x[:ncell].reshape(grid.shape), x[ncell:]


def relative_residual_closed(grid: Grid, iblank: np.ndarray, G: GhostTable, alpha: float, f: np.ndarray,
                             u: np.ndarray, ub=None) -> float:
    """||S (b - H u)|| / ||S b|| (u: full array with the ghost values at the ghost cells)."""
    H, cells, is_fluid, grow = system_closed(grid, iblank, G, alpha)
    ubv = np.zeros(len(G)) if ub is None else ub
    b = np.where(is_fluid, np.asarray(f, dtype=np.float64).ravel()[cells], 0.0)
    b[grow] = 2.0 * np.asarray(ubv, dtype=np.float64)
    S = np.ones(cells.size)
    S[grow] = alpha * G.scale
    r = b - H @ np.asarray(u, dtype=np.float64).ravel()[cells]
    return float(np.linalg.norm(S * r) / np.linalg.norm(S * b))


def ghost_velocity(G: GhostTable, tri_off, motions) -> np.ndarray:
    """u_b (ng, 3) = v0 + omega x (BI - centre) for rigid motions per mesh (v0 (3),
    omega (3), centre (3)), the mesh being the one holding each entry's closest triangle."""
    M = np.asarray(motions, dtype=np.float64).reshape(-1, 9)
    m = np.searchsorted(np.asarray(tri_off), G.tri, side="right") - 1
    return point_velocity(G.bi, M[m])


def point_velocity(X: np.ndarray, M: np.ndarray) -> np.ndarray:
    """v0 + omega x (X - centre) per point, M (n, 9) the motion of each point's body."""
    r = X - M[:, 6:9]
    om = M[:, 3:6]
    return np.stack([M[:, 0] + (om[:, 1] * r[:, 2] - om[:, 2] * r[:, 1]),
                     M[:, 1] + (om[:, 2] * r[:, 0] - om[:, 0] * r[:, 2]),
                     M[:, 2] + (om[:, 0] * r[:, 1] - om[:, 1] * r[:, 0])], -1)
