"""The finest level's smoother, one or two sweeps, against red-black Gauss-Seidel written out.

ibm_smoother_apply loads e and r into the finest level and runs the sweeps exactly as a
V-cycle does (the fused z-march kernel in FP32, the two colour passes in FP64).  The
reference here restates one sweep from its definition: the fluid cells of one colour at a
time, red ((i + j + k) even) then black, take e += omega ((A e)_i - (r_i - mu)) / D_i with A
the oracle's fluid operator and D_i the sum of the cell's coefficients; then every ghost row is
re-evaluated from the values the sweep left, e_G = sum_k w_k e_k + r_G (Jacobi among ghosts).
Cells that are neither fluid nor ghost keep their loaded value bit for bit.

Grids span several x-y tiles of the fused sweep (128 x 14 cells) with ragged edges and
several z-chunks, with bodies across tile borders, so a wrong colour, ring cell or chunk
seam shows as an O(1) difference.  Tolerances: the FP32 path rounds the coefficients and every
product (a few units of 2^-24 per term, values O(1)); the FP64 path forms its relaxation
factor omega res / D in FP32 (relative 2^-22 of the update)."""
import numpy as np
import pytest

import synth
from oracle.grid import Grid
from oracle.system import apply_fluid
from tests.gpu_util import require_gpu, torch

pytestmark = pytest.mark.gpu
OMEGA = 1.3
TOL = {0: 5e-6, 1: 5e-5, 2: 5e-5}


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _diag(g: Grid) -> np.ndarray:
    return ((g.cxm + g.cxp)[None, None, :] + (g.cym + g.cyp)[None, :, None]) + (g.czm + g.czp)[:, None, None]


def _reference(g, ex, e, r, mu, nsweeps):
    ib = ex["iblank"]
    D = _diag(g)
    kk, jj, ii = np.indices(ib.shape)
    red = (ii + jj + kk) % 2 == 0
    fluid = ib == 0
    ghost = ib == 3
    ng = int(np.sum(ghost))
    cell, ref, w = ex["cell"][:ng], ex["ref"][:ng], ex["w"][:ng]
    for _ in range(nsweeps):
        for colour in (red, ~red):
            upd = fluid & colour
            Ae = apply_fluid(g, e)
            e = np.where(upd, e + OMEGA * (Ae - (r - mu)) / np.where(upd, D, 1.0), e)
        if ng:
            flat = e.ravel().copy()
            vals = np.where(ref >= 0, flat[np.maximum(ref, 0)], 0.0)
            flat[cell] = np.sum(np.where(ref >= 0, w, 0.0) * vals, axis=1) + r.ravel()[cell]
            e = flat.reshape(e.shape)
    return e


def _inputs(g: Grid, ib: np.ndarray, seed: int):
    """e ~ U(-1, 1); r = D u on fluid rows and u on ghost rows (a value relation), u ~ U(-1, 1);
    both rounded to FP32 (so every path loads the same values); a shift mu of the order of the
    smallest diagonal."""
    rng = np.random.default_rng(seed)
    D = _diag(g)
    e = rng.uniform(-1.0, 1.0, g.shape).astype(np.float32).astype(np.float64)
    u = rng.uniform(-1.0, 1.0, g.shape)
    r = np.where(ib == 3, u, D * u).astype(np.float32).astype(np.float64)
    mu = float(np.float32(0.3 * D.min()))
    return e, r, mu


def _check(ctx, xf, yf, zf, meshes, seed, precisions=(0, 1, 2), sweeps=(1, 2)):
    pkg, c = ctx
    g = Grid(xf, yf, zf)
    T = pkg.Tables(c, xf, yf, zf, meshes)
    ex = {k: v.cpu().numpy() for k, v in T.export().items()}
    ib = ex["iblank"]
    e, r, mu = _inputs(g, ib, seed)
    et, rt = torch.from_numpy(e).cuda(), torch.from_numpy(r).cuda()
    other = (ib != 0) & (ib != 3)
    for ns in sweeps:
        ref = _reference(g, ex, e, r, mu, ns)
        for prec in precisions:
            out = pkg.ibm_smoother_apply(c.h, T.h, prec, ns, OMEGA, et, rt, mu).cpu().numpy()
            assert np.all(np.isfinite(out)), (prec, ns)
            assert np.array_equal(out[other], e[other]), (prec, ns)
            for name, sel in (("fluid", ib == 0), ("ghost", ib == 3)):
                if np.any(sel):
                    err = np.max(np.abs(out[sel] - ref[sel]) / (1.0 + np.abs(ref[sel])))
                    assert err <= TOL[prec], (name, prec, ns, err)
    T.close()


def test_multi_tile_two_bodies_across_tile_borders(ctx):
    """200 x 45 x 37 cells: 2 x 4 tiles, both ragged, bodies over the x = 128 and y = 14, 28
    tile borders; z split into chunks by the sweep's schedule."""
    xf, yf, zf = synth.faces_tanh(200, 1.5), synth.faces_uniform(45), synth.faces_tanh(37, 1.2)
    meshes = [synth.octa_sphere(4, (xf[128], yf[14], 0.5 * (zf[17] + zf[18])), 0.17),
              synth.octa_sphere(3, (xf[60], yf[29], zf[9]), 0.09)]
    _check(ctx, xf, yf, zf, meshes, 31)


def test_single_ragged_tile(ctx):
    """37 x 20 x 9 cells: one tile in x (37 of 128 columns), two in y (the second ragged), a
    body across most of the nine planes."""
    xf, yf, zf = synth.faces_tanh(37, 2.0), synth.faces_uniform(20), synth.faces_uniform(9)
    _check(ctx, xf, yf, zf, [synth.octa_sphere(3, (0.5, 0.45, 0.5), 0.3)], 32)


def test_no_body_wide(ctx):
    """300 x 29 x 17 cells, no body: three tiles in x, the last ragged; pure Neumann walls."""
    _check(ctx, synth.faces_uniform(300), synth.faces_tanh(29, 2.0), synth.faces_uniform(17), [], 33)
