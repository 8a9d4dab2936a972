"""Exact discrete solution of the bordered pressure system by library direct solvers (oracle).

The method's result has a plain definition: the unique (p, lambda) with
A p = b - lambda 1_F on every active row and sum_F V_i p_i = 0 (see
``oracle.system``).  The paper's own solver reaches it iteratively (BiCGStab
with scheduled relaxed Jacobi, Sec. "Governing Equations and Numerical
Methods"); the oracle writes the definition out and hands it to LAPACK
(dense, tiny grids) or SuperLU (sparse, up to ~32^3 cells).

* ``solve_dense``  -- the bordered matrix [A 1_F; V_F^T 0] by numpy.linalg.solve.
* ``solve_sparse`` -- row i0 (first fluid row) replaced by p_{i0} = 0; two
  solves with one SuperLU factorisation give q1 (rhs b) and q2 (rhs 1_F);
  then p = q1 - lambda q2 with lambda fixed by the original row i0, and the
  gauge is applied.  Algebraically identical to the bordered system.

Parity status: the dense and sparse paths are compared with each other and
both with the DCT solve of the no-body and grid-aligned-wall problems
(tests/test_oracle_system.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from .classify import GhostTable
from .grid import Grid
from .system import assemble, gauge


def _rhs(b: np.ndarray, cells: np.ndarray, is_fluid: np.ndarray, G: GhostTable) -> np.ndarray:
    """b on fluid rows, the ghost rows' right-hand sides d on ghost rows."""
    out = np.where(is_fluid, b.ravel()[cells], 0.0)
    if len(G):
        row = np.full(b.size, -1, dtype=np.int64)
        row[cells] = np.arange(cells.size)
        out[row[G.cell]] = G.d
    return out


def _scatter(shape, cells, x) -> np.ndarray:
    out = np.zeros(int(np.prod(shape)))
    out[cells] = x
    return out.reshape(shape)


def solve_dense(grid: Grid, iblank: np.ndarray, G: GhostTable, b: np.ndarray):
    """(p full array with ghost values, lambda) via the dense bordered system."""
    A, cells, is_fluid = assemble(grid, iblank, G)
    n = cells.size
    V = grid.volumes().ravel()[cells]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = A.toarray()
    M[:n, n] = is_fluid.astype(np.float64)
    M[n, :n] = np.where(is_fluid, V, 0.0)
    rhs = np.concatenate([_rhs(b, cells, is_fluid, G), [0.0]])
    x = np.linalg.solve(M, rhs)
    return _scatter(grid.shape, cells, x[:n]), float(x[n])


def solve_sparse(grid: Grid, iblank: np.ndarray, G: GhostTable, b: np.ndarray):
    """(p full array with ghost values, lambda) via a pinned SuperLU factorisation."""
    A, cells, is_fluid = assemble(grid, iblank, G)
    n = cells.size
    i0 = int(np.flatnonzero(is_fluid)[0])
    At = A.tolil(copy=True)
    At[i0, :] = 0.0
    At[i0, i0] = 1.0
    lu = spl.splu(sp.csc_matrix(At), permc_spec="COLAMD")
    bb = _rhs(b, cells, is_fluid, G)
    one = is_fluid.astype(np.float64)
    r1 = bb.copy(); r1[i0] = 0.0
    r2 = one.copy(); r2[i0] = 0.0
    q1 = lu.solve(r1)
    q2 = lu.solve(r2)
    a1 = A[i0] @ q1
    a2 = A[i0] @ q2
    lam = float((bb[i0] - a1[0]) / (1.0 - a2[0]))
    x = q1 - lam * q2
    p = gauge(grid, iblank, _scatter(grid.shape, cells, x))
    return p, lam


class BoxSolver:
    """Exact inverse of the no-body Neumann operator on the full box (a preconditioner).

    Along each axis the 1-D operator L = W^-1 S (W = diag of cell widths, S
    symmetric) is diagonalised through the symmetric W^1/2 L W^-1/2 by
    numpy.linalg.eigh; the 3-D operator is the Kronecker sum, inverted on
    everything but the constant mode.
    """

    def __init__(self, grid: Grid):
        self.shape = grid.shape
        self.ops = []
        for f, cm, cp in ((grid.zf, grid.czm, grid.czp), (grid.yf, grid.cym, grid.cyp), (grid.xf, grid.cxm, grid.cxp)):
            n = cm.size
            L = np.diag(-(cm + cp)) + np.diag(cm[1:], -1) + np.diag(cp[:-1], 1)
            w = np.sqrt(np.diff(f))
            Ssym = (w[:, None] * L) / w[None, :]
            Ssym = 0.5 * (Ssym + Ssym.T)
            lam, Q = np.linalg.eigh(Ssym)
            self.ops.append((lam, Q / w[:, None], Q.T * w[None, :]))   # (eigs, W^-1/2 Q, Q^T W^1/2)
        lz, ly, lx = self.ops[0][0], self.ops[1][0], self.ops[2][0]
        tot = lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
        small = np.abs(tot) < 1e-9 * np.max(np.abs(tot))
        self.inv = np.where(small, 0.0, 1.0 / np.where(small, 1.0, tot))

    def solve(self, r: np.ndarray) -> np.ndarray:
        """Each axis transform is one matrix contraction along that axis (np.tensordot, a
        BLAS matrix product): forward transforms z, y, x, the scaling by the inverse
        eigenvalue sums, then the inverse transforms."""
        x = r.reshape(self.shape)
        x = np.tensordot(self.ops[0][2], x, axes=([1], [0]))                     # z
        x = np.tensordot(self.ops[1][2], x, axes=([1], [1])).transpose(1, 0, 2)  # y
        x = np.tensordot(x, self.ops[2][2], axes=([2], [1]))                     # x
        x = x * self.inv
        x = np.tensordot(self.ops[0][1], x, axes=([1], [0]))
        x = np.tensordot(self.ops[1][1], x, axes=([1], [1])).transpose(1, 0, 2)
        x = np.tensordot(x, self.ops[2][1], axes=([2], [1]))
        return np.ascontiguousarray(x)


def solve_gmres(grid: Grid, iblank: np.ndarray, G: GhostTable, b: np.ndarray,
                rtol: float = 1e-13, restart: int = 200, maxiter: int = 20):
    """(p, lambda) of the bordered system by scipy GMRES, right-preconditioned with the
    no-body box inverse on fluid rows and the identity on ghost rows.  Grids well past
    the reach of sparse LU (64^3 and up); the result is certified by its residual."""
    A, cells, is_fluid = assemble(grid, iblank, G)
    n = cells.size
    V = grid.volumes().ravel()[cells]
    ncell = int(np.prod(grid.shape))
    scale = float(ncell) / float(np.sum(np.where(is_fluid, V, 0.0)))
    Bm = sp.bmat([[A, sp.csr_matrix(is_fluid.astype(np.float64)[:, None])],
                  [sp.csr_matrix((np.where(is_fluid, V, 0.0) * scale)[None, :]), None]]).tocsr()
    box = BoxSolver(grid)
    fl_cells = cells[is_fluid]

    def msolve(r):
        full = np.zeros(ncell)
        full[fl_cells] = r[:n][is_fluid]
        z = box.solve(full).ravel()
        out = np.empty(n + 1)
        out[:n] = z[cells]
        out[:n][~is_fluid] += r[:n][~is_fluid]
        out[n] = r[n]
        return out

    rhs = np.concatenate([_rhs(b, cells, is_fluid, G), [0.0]])
    M = spl.LinearOperator((n + 1, n + 1), msolve)
    x, info = spl.gmres(Bm, rhs, M=M, rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter)
    p = gauge(grid, iblank, _scatter(grid.shape, cells, x[:n]))
    if info != 0:
        # GMRES's own stopping test can stall just above rtol at the FP64 floor (it depends on
        # the platform's BLAS rounding); accept the iterate when the defining residual is at
        # the floor, judged by the plain operator itself.
        from .system import relative_residual
        rr = relative_residual(grid, iblank, G, b, p)
        if not rr <= 1e-12:
            raise RuntimeError("oracle GMRES did not converge (info=%d, relative residual %g)" % (info, rr))
    # lambda from its definition: every fluid row reads b_i - (A p)_i = lambda
    from .system import residual, fluid_mean
    rf, _ = residual(grid, iblank, G, b, p, 0.0)
    return p, fluid_mean(grid, iblank, rf)
