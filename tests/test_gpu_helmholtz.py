"""Advection-diffusion (Helmholtz) velocity solve on the GPU against the oracle: closed bodies
and membranes, every precision mode, after reclassification; the rigid boundary velocity bit for
bit; the 256^3 stretched-grid case by sampled rows; argument errors."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import helmholtz as OH
from oracle import membrane as OM
from oracle.grid import Grid
from tests.gpu_util import require_gpu, torch

pytestmark = pytest.mark.gpu
TOL = 1e-10
PARITY = 1e-8


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _err(a, b, sel):
    return float(np.linalg.norm((a - b)[sel]) / np.linalg.norm(b[sel]))


def _alpha(grid, aS):
    """alpha with alpha S = aS, S the largest coefficient sum of a cell (the diagonal
    dominance of the system: the fluid rows' Jacobi radius is aS / (1 + aS))."""
    S = (np.max(grid.cxm + grid.cxp) + np.max(grid.cym + grid.cyp)) + np.max(grid.czm + grid.czp)
    return aS / S


@pytest.mark.parametrize("aS", [0.5, 3.0])
def test_closed_body_matches_oracle(ctx, aS):
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(34, 2.0), synth.faces_uniform(30), synth.faces_tanh(32, 1.5)
    grid = Grid(xf, yf, zf)
    alpha = _alpha(grid, aS)
    meshes = [synth.ellipsoid(4, (0.21, 0.13, 0.12), 23.0, (0.49, 0.51, 0.5))]
    ib, G = OC.classify(grid, meshes)
    f = synth.smooth_field(xf, yf, zf, 3) + 0.1 * synth.counter_normal(6, 0, np.arange(grid.nx * grid.ny * grid.nz)).reshape(grid.shape)
    ub = synth.counter_normal(7, 0, np.arange(len(G)))
    u_o = OH.solve_closed(grid, ib, G, alpha, f, ub)
    T = pkg.Tables(c, xf, yf, zf, meshes)
    act = ib != 1                                  # fluid and ghost cells
    fd, ubd = torch.from_numpy(f).cuda(), torch.from_numpy(ub).cuda()
    for prec in (0, 1, 2):
        u = torch.zeros_like(fd)
        rep = T.helmholtz_solve(alpha, fd, u, ubd, TOL, pkg.HelmholtzOpts(precision=prec))
        ug = u.cpu().numpy()
        assert rep["status"] == "IBM_OK" and rep["rel_resid"] <= TOL
        assert _err(ug, u_o, act) <= PARITY, (prec, _err(ug, u_o, act), rep["cycles"])
        assert OH.relative_residual_closed(grid, ib, G, alpha, f, ug, ub) <= 10 * TOL
        assert np.all(ug[ib == 1] == 0.0)
    T.close()


def test_membrane_with_rigid_velocity(ctx):
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(30, 2.0), synth.faces_uniform(28), synth.faces_tanh(29, 1.5)
    grid = Grid(xf, yf, zf)
    m = synth.plate(0.13, chord=0.5, span=0.35, nq_x=6, nq_y=5, heave=0.05, pitch_deg=25.0,
                    center=(0.503, 0.491, 0.517))
    meshes = [m]
    _, G = OM.classify(grid, meshes)
    motion = synth.plate_velocity(0.13, heave=0.05, pitch_deg=25.0, center=(0.503, 0.491, 0.517))[None]
    ub_o = OH.ghost_velocity(G, [0, m.ntris], motion)
    T = pkg.Tables(c, xf, yf, zf, meshes)
    ub = T.boundary_velocity_rigid(motion)
    assert np.array_equal(ub.cpu().numpy(), ub_o.T)
    alpha = _alpha(grid, 1.0)
    f = synth.smooth_field(xf, yf, zf, 8)
    fd = torch.from_numpy(f).cuda()
    for comp in range(3):
        u_o, _ = OH.solve_membrane(grid, G, alpha, f, ub_o[:, comp])
        for prec in (0, 1, 2):
            u = torch.zeros_like(fd)
            rep = T.helmholtz_solve(alpha, fd, u, ub[comp].contiguous(), TOL, pkg.HelmholtzOpts(precision=prec))
            assert rep["status"] == "IBM_OK"
            err = _err(u.cpu().numpy(), u_o, np.ones(grid.shape, dtype=bool))
            assert err <= PARITY, (comp, prec, err)
    T.close()


def test_after_reclassification(ctx):
    pkg, c = ctx
    f1 = synth.faces_tanh(28, 2.0)
    grid = Grid(f1, f1, f1)
    mA = [synth.octa_sphere(3, (0.45, 0.5, 0.5), 0.2)]
    mB = [synth.octa_sphere(3, (0.55, 0.48, 0.52), 0.2)]
    alpha = _alpha(grid, 1.0)
    f = synth.smooth_field(f1, f1, f1, 9)
    fd = torch.from_numpy(f).cuda()
    T = pkg.Tables(c, f1, f1, f1, mA)
    u = torch.zeros_like(fd)
    T.helmholtz_solve(alpha, fd, u, None, TOL)
    T.reclassify(mB)
    ib, G = OC.classify(grid, mB)
    u_o = OH.solve_closed(grid, ib, G, alpha, f, None)
    u = torch.zeros_like(fd)
    rep = T.helmholtz_solve(alpha, fd, u, None, TOL)
    assert rep["status"] == "IBM_OK"
    assert _err(u.cpu().numpy(), u_o, ib != 1) <= PARITY
    T.close()


def test_stretched_256_sampled_rows(ctx):
    """256^3 stretched grid with the 8192-triangle ellipsoid (the pressure benchmark's grid and
    body): the returned field satisfies sampled fluid rows, written out with the oracle's
    coefficients, to the solve's tolerance."""
    pkg, c = ctx
    pr = synth.cfg2(256)
    grid = Grid(pr.xf, pr.yf, pr.zf)
    f = synth.smooth_field(pr.xf, pr.yf, pr.zf, 12)
    fd = torch.from_numpy(f).cuda()
    T = pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes)
    alpha = 0.5 / 1000 * 0.5 / 256                 # dt nu / 2 with dt = 0.5 h, nu = 1 / 1000
    for prec in (0, 1, 2):
        u = torch.zeros_like(fd)
        rep = T.helmholtz_solve(alpha, fd, u, None, TOL, pkg.HelmholtzOpts(precision=prec))
        assert rep["status"] == "IBM_OK", rep
        ug = u.cpu().numpy()
        ib = T.export()["iblank"].cpu().numpy()
        nz, ny, nx = grid.shape
        rng = np.random.default_rng(1)
        kk, jj, ii = rng.integers(1, nz - 1, 4000), rng.integers(1, ny - 1, 4000), rng.integers(1, nx - 1, 4000)
        ok = np.ones(ii.size, dtype=bool)
        for dk, dj, di in ((0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
            ok &= ib[kk + dk, jj + dj, ii + di] == 0
        kk, jj, ii = kk[ok], jj[ok], ii[ok]
        s = (grid.cxm[ii] * ug[kk, jj, ii - 1] + grid.cxp[ii] * ug[kk, jj, ii + 1] + grid.cym[jj] * ug[kk, jj - 1, ii]
             + grid.cyp[jj] * ug[kk, jj + 1, ii] + grid.czm[kk] * ug[kk - 1, jj, ii] + grid.czp[kk] * ug[kk + 1, jj, ii])
        D = 1.0 + alpha * ((grid.cxm[ii] + grid.cxp[ii]) + (grid.cym[jj] + grid.cyp[jj]) + (grid.czm[kk] + grid.czp[kk]))
        r = f[kk, jj, ii] - (D * ug[kk, jj, ii] - alpha * s)
        assert ii.size > 3000
        assert np.sqrt(np.mean(r * r)) <= 10 * TOL * np.sqrt(np.mean(f[ib == 0] ** 2)), prec
    T.close()


def test_argument_errors(ctx):
    pkg, c = ctx
    f1 = synth.faces_uniform(16)
    T = pkg.Tables(c, f1, f1, f1, [synth.octa_sphere(2, (0.5, 0.5, 0.5), 0.2)])
    fd = torch.ones((16, 16, 16), dtype=torch.float64, device="cuda")
    u = torch.zeros_like(fd)
    for alpha, opts in ((-1.0, None), (0.1, pkg.HelmholtzOpts(precision=3)), (0.1, pkg.HelmholtzOpts(srj_steps=0))):
        with pytest.raises(pkg.IbmError):
            T.helmholtz_solve(alpha, fd, u, None, TOL, opts)
    with pytest.raises(pkg.IbmError):
        T.boundary_velocity_rigid(np.zeros((2, 9)))   # one motion per mesh
    rep = T.helmholtz_solve(1e-4, torch.zeros_like(fd), u, None, TOL)
    assert rep["status"] == "IBM_OK" and float(u.abs().max()) == 0.0
    T.close()
