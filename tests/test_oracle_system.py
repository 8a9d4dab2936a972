"""Pins of the oracle's discrete pressure system and its solvers.

Independent references: the DCT-II diagonalisation of the uniform
cell-centred Neumann Laplacian (scipy.fft), second-order convergence to
manufactured solutions (no body, and a sphere with dp/dn = 0), the exact
reduction of a grid-aligned wall to a Neumann sub-box, and invariants.
Planted-mistake tests show that the pins fail when the oracle is wrong.
"""
import numpy as np
import pytest
import scipy.fft as fft

import synth
from oracle import classify as C
from oracle import solve as SV
from oracle import system as S
from oracle.grid import Grid


def _dct_solve(b: np.ndarray, h) -> np.ndarray:
    """Closed form: eigenvalues sum_axes (2 cos(pi k/n) - 2)/h^2 of the DCT-II basis."""
    nz, ny, nx = b.shape
    lam = [(2 * np.cos(np.pi * np.arange(n) / n) - 2) / hh ** 2 for n, hh in zip((nz, ny, nx), h)]
    L = lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]
    bh = fft.dctn(b, type=2, norm="ortho")
    L[0, 0, 0] = 1.0
    ph = bh / L
    ph[0, 0, 0] = 0.0
    return fft.idctn(ph, type=2, norm="ortho")


def _no_body(grid):
    ib = np.zeros(grid.shape, dtype=np.uint8)
    return ib, C.GhostTable(0)


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 20, 16)])
def test_uniform_no_body_matches_dct(shape):
    nz, ny, nx = shape
    g = Grid(synth.faces_uniform(nx), synth.faces_uniform(ny), synth.faces_uniform(nz))
    b = synth.rhs_divergence(g.xf, g.yf, g.zf, 9)
    ib, G = _no_body(g)
    p, lam = SV.solve_sparse(g, ib, G, b)
    ref = _dct_solve(b - b.mean(), (1 / nz, 1 / ny, 1 / nx))
    assert abs(lam) < 1e-10
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) < 1e-11
    pg, _ = SV.solve_gmres(g, ib, G, b)
    assert np.linalg.norm(pg - ref) / np.linalg.norm(ref) < 1e-11


@pytest.mark.parametrize("ratio", [1.0, 2.0])
def test_manufactured_second_order_no_body(ratio):
    errs = []
    for n in (8, 16, 32):
        f = synth.faces_tanh(n, ratio)
        g = Grid(f, f, f)
        Z, Y, X = np.meshgrid(g.zc, g.yc, g.xc, indexing="ij")
        pex = np.cos(np.pi * X) * np.cos(np.pi * Y) * np.cos(np.pi * Z)
        b = -3 * np.pi ** 2 * pex
        ib, G = _no_body(g)
        p, _ = SV.solve_gmres(g, ib, G, b)
        V = g.volumes()
        pe = pex - np.sum(V * pex) / np.sum(V)
        errs.append(np.sqrt(np.sum(V * (p - pe) ** 2)))          # volume-weighted L2
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r2 < 4.3 and 3.4 < r1 < 4.6, errs


def _sphere_mms(n, ratio, mesh, R=0.18, R1=0.28, R2=0.45, c=0.5):
    """Potential flow past a sphere, u = (z-c)(1 + R^3/(2 r^3)): harmonic, du/dr = 0 at r = R.

    p = chi(r) u with chi = 1 inside r < R1 and a quintic blend to 0 at R2, so b = lap p
    vanishes near the body (no cut-cell sliver enters the compatibility) and p = 0 near
    the outer walls.  The body is felt only through the ghost-cell rows.
    """
    f = synth.faces_tanh(n, ratio)
    g = Grid(f, f, f)
    ib, G = C.classify(g, [mesh])
    Z, Y, X = np.meshgrid(g.zc, g.yc, g.xc, indexing="ij")
    r = np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2)
    w = Z - c
    fr = 1 + R ** 3 / (2 * r ** 3)
    fp = -1.5 * R ** 3 / r ** 4
    D = R2 - R1
    s = np.clip((r - R1) / D, 0, 1)
    chi = 1 - (10 * s ** 3 - 15 * s ** 4 + 6 * s ** 5)
    chp = -30 * s ** 2 * (1 - s) ** 2 / D
    chpp = -(60 * s - 180 * s ** 2 + 120 * s ** 3) / D ** 2
    pex = chi * w * fr
    b = 2 * chp * w * (fr / r + fp) + w * fr * (chpp + 2 * chp / r)
    p, lam = SV.solve_gmres(g, ib, G, b)
    fl = ib == 0
    V = g.volumes()
    pe = pex - np.sum(V[fl] * pex[fl]) / np.sum(V[fl])
    return np.sqrt(np.sum(V[fl] * (p - pe)[fl] ** 2)), lam


_MMS_MESH = synth.octa_sphere(5, (0.5, 0.5, 0.5), 0.18)


@pytest.mark.parametrize("ratio", [1.0, 2.0])
def test_manufactured_sphere_neumann_converges(ratio):
    e16, _ = _sphere_mms(16, ratio, _MMS_MESH)
    e32, _ = _sphere_mms(32, ratio, _MMS_MESH)
    assert e16 / e32 > 4.0, (e16, e32)          # at least second order in volume-weighted L2
    assert e32 < 3e-3, e32


@pytest.mark.parametrize("mistake", ["mirror_inward", "no_reflection"])
def test_planted_wrong_image_point_fails_the_sphere_pin(monkeypatch, mistake):
    """The same pin with a wrong image point must fail: IP = 3 GC - 2 BI, or IP = GC."""
    orig = C.closest_points

    def wrong(P, meshes, chunk=64):
        BI, t = orig(P, meshes, chunk)
        return (P + (P - BI) if mistake == "mirror_inward" else P.copy()), t
    monkeypatch.setattr(C, "closest_points", wrong)
    e16, _ = _sphere_mms(16, 1.0, _MMS_MESH)
    e32, _ = _sphere_mms(32, 1.0, _MMS_MESH)
    assert not (e16 / e32 > 4.0 and e32 < 3e-3)


def test_grid_aligned_wall_is_neumann_sub_box():
    n = 16
    f = synth.faces_uniform(n)
    g = Grid(f, f, f)
    m = synth.box_mesh((0.5, -1.0, -1.0), (2.0, 2.0, 2.0))
    ib, G = C.classify(g, [m])
    b = synth.rhs_divergence(f, f, f, 4)
    p, lam = SV.solve_sparse(g, ib, G, b)
    sub = b[:, :, : n // 2]
    ref = _dct_solve(sub - sub.mean(), (1 / n, 1 / n, 1 / n))
    assert abs(lam - sub.mean()) < 1e-10
    assert np.linalg.norm(p[:, :, : n // 2] - ref) / np.linalg.norm(ref) < 1e-11
    # ghost values copy their mirror cell
    assert np.allclose(p.ravel()[G.cell], p.ravel()[G.cell - 1], rtol=0, atol=1e-11 * np.abs(p).max())


def test_invariants_no_body():
    f = synth.faces_tanh(10, 2.0)
    g = Grid(f, synth.faces_tanh(12, 1.5), synth.faces_uniform(9))
    ib, G = _no_body(g)
    A, cells, isf = S.assemble(g, ib, G)
    V = g.volumes().ravel()
    VA = (A.multiply(V[:, None])).toarray()
    assert np.allclose(VA, VA.T, rtol=0, atol=1e-9 * np.abs(VA).max())        # symmetric
    rng = np.random.default_rng(0)
    x = rng.normal(size=A.shape[0])
    assert abs(V @ (A @ x)) < 1e-10 * np.abs(V * (A @ x)).sum()            # telescoping fluxes
    assert np.allclose(A @ np.ones(A.shape[0]), 0, atol=1e-9)


def test_invariants_with_body_and_solvers_agree():
    for n, ratio in ((8, 1.0), (12, 2.0)):
        f = synth.faces_tanh(n, ratio)
        g = Grid(f, f, f)
        ib, G = C.classify(g, [synth.octa_sphere(3, (0.5, 0.5, 0.5), 0.3)])
        assert len(G) > 0
        A, cells, isf = S.assemble(g, ib, G)
        assert np.allclose(A @ np.ones(A.shape[0]), 0, atol=1e-9 * abs(A).max())
        b = synth.rhs_divergence(f, f, f, 1)
        pd, ld = SV.solve_dense(g, ib, G, b)
        ps, ls = SV.solve_sparse(g, ib, G, b)
        pg, lg = SV.solve_gmres(g, ib, G, b)
        fl = ib == 0
        for q in (ps, pg):
            assert np.linalg.norm((q - pd)[fl]) / np.linalg.norm(pd[fl]) < 1e-11
        assert abs(ls - ld) < 1e-9 * max(1, abs(ld)) and abs(lg - ld) < 1e-9 * max(1, abs(ld))
        assert S.relative_residual(g, ib, G, b, pd) < 1e-12
        # the fluid mean of b is absorbed by lambda: p does not change
        ps2, ls2 = SV.solve_sparse(g, ib, G, b + 3.0)
        assert np.linalg.norm((ps2 - ps)[fl]) / np.linalg.norm(ps[fl]) < 1e-10
        assert abs(ls2 - (ls + 3.0)) < 1e-9


def test_planted_dropped_term_fails_dct(monkeypatch):
    """Dropping one neighbour term of the stencil must break the DCT pin."""
    g = Grid(synth.faces_uniform(8), synth.faces_uniform(8), synth.faces_uniform(8))
    g.cyp = g.cyp * 0.0
    b = synth.rhs_divergence(g.xf, g.yf, g.zf, 9)
    ib, G = _no_body(g)
    p, _ = SV.solve_sparse(g, ib, G, b)
    ref = _dct_solve(b - b.mean(), (1 / 8, 1 / 8, 1 / 8))
    assert np.linalg.norm(p - ref) / np.linalg.norm(ref) > 1e-3
