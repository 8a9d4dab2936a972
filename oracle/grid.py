"""Cell-centred stretched Cartesian grid and its 7-point coefficients (oracle).

Paper: Sec. "Governing Equations and Numerical Methods" (second-order finite
differences on a Cartesian grid) and Sec. "Fluid-Structure Interaction in Bat"
(uniform near the body, stretched towards the outer boundaries).

Reading (the paper gives no stencil formula): the finite-volume form divided by
the cell volume,

    (A p)_i = sum_{d in +-x,+-y,+-z} c_{i,d} (p_nb(i,d) - p_i),
    c_{i,+x} = 1 / (dx_i * (x_{i+1} - x_i)),   c_{i,-x} = 1 / (dx_i * (x_i - x_{i-1})),

with c = 0 across the outer walls (homogeneous Neumann).  Parity: pinned by the
DCT-II solve, the separable eigen solve and second-order convergence on a
manufactured solution (tests/test_oracle_system.py).
"""
from __future__ import annotations

import numpy as np


def centres(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    return 0.5 * (f[:-1] + f[1:])


def widths(f: np.ndarray) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    return f[1:] - f[:-1]


def coeffs_1d(f: np.ndarray):
    """(c_minus, c_plus) per cell along one axis; zero across the walls."""
    c = centres(f)
    w = widths(f)
    n = w.size
    cm = np.zeros(n)
    cp = np.zeros(n)
    if n > 1:
        dc = c[1:] - c[:-1]
        cm[1:] = 1.0 / (w[1:] * dc)
        cp[:-1] = 1.0 / (w[:-1] * dc)
    return cm, cp


class Grid:
    """Face coordinates along x, y, z and derived 1-D arrays; arrays are [k][j][i]."""

    def __init__(self, xf, yf, zf):
        self.xf = np.asarray(xf, dtype=np.float64)
        self.yf = np.asarray(yf, dtype=np.float64)
        self.zf = np.asarray(zf, dtype=np.float64)
        self.nx, self.ny, self.nz = self.xf.size - 1, self.yf.size - 1, self.zf.size - 1
        self.xc, self.yc, self.zc = centres(self.xf), centres(self.yf), centres(self.zf)
        self.dx, self.dy, self.dz = widths(self.xf), widths(self.yf), widths(self.zf)
        self.cxm, self.cxp = coeffs_1d(self.xf)
        self.cym, self.cyp = coeffs_1d(self.yf)
        self.czm, self.czp = coeffs_1d(self.zf)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def volumes(self) -> np.ndarray:
        return self.dz[:, None, None] * self.dy[None, :, None] * self.dx[None, None, :]

    def centre(self, lin) -> np.ndarray:
        """Cell-centre coordinates (x, y, z) of linear indices l = (k*ny + j)*nx + i."""
        lin = np.asarray(lin, dtype=np.int64)
        i = lin % self.nx
        j = (lin // self.nx) % self.ny
        k = lin // (self.nx * self.ny)
        return np.stack([self.xc[i], self.yc[j], self.zc[k]], axis=-1)
