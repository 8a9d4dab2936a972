"""ibm_residual_norm_noalloc: the allocation-free residual check, through the C ABI.

Callers that cannot allocate device memory once they are running (a flow solver working
inside a fixed device arena, where cudaMalloc would synchronise the device and stall the
overlap of compute and communication, or could fail mid-run) use this entry point to check
a pressure field.  This file is collected last on purpose, so a failure here comes after
every other test has run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-3     # agreement of two FP64 evaluations of a ~1e-6 residual norm


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_04335_gb300 as pkg
    return torch, pkg


def _closed_case():
    xf, yf, zf = synth.faces_tanh(48, 2.0), synth.faces_uniform(40), synth.faces_tanh(44, 1.5)
    return xf, yf, zf, [synth.octa_sphere(4, (0.5, 0.5, 0.5), 0.22)]


def _noalloc(pkg, xf, yf, zf, ex, rhs, p, d=None):
    return pkg.ibm_residual_norm_noalloc(xf, yf, zf, ex["iblank"], ex["cell"], ex["ref"], ex["w"], ex["scale"],
                                         rhs, p, d=d)


def test_noalloc_residual_matches_solver_on_two_calls_in_a_row():
    torch, pkg = _setup()
    from oracle import classify as OC
    from oracle import system as OSys
    from oracle.grid import Grid

    xf, yf, zf, meshes = _closed_case()
    b = synth.rhs_divergence(xf, yf, zf, 21)
    with pkg.Context(0) as ctx:
        T = pkg.Tables(ctx, xf, yf, zf, meshes)
        ex = T.export()
        rhs = torch.from_numpy(b).cuda()
        g = Grid(xf, yf, zf)
        ib, G = OC.classify(g, meshes)
        for prec in (0, 1):
            # a partly converged field: its residual (~1e-6) is far above the FP64 rounding
            # noise, so both implementations must agree closely
            p = torch.zeros_like(rhs)
            rep = T.solve(rhs, p, 1e-5, pkg.SolveOpts(precision=prec))      # the existing entry point
            torch.cuda.synchronize()
            r1 = _noalloc(pkg, xf, yf, zf, ex, rhs, p)
            r2 = _noalloc(pkg, xf, yf, zf, ex, rhs, p)
            assert r1 == r2                                            # two calls in a row agree exactly
            assert abs(r1[0] - rep["rel_resid"]) <= RTOL * rep["rel_resid"], (r1, rep["rel_resid"])
            ro = OSys.relative_residual(g, ib, G, b, p.cpu().numpy())
            assert abs(r1[0] - ro) <= RTOL * ro, (r1, ro)
            # the converged field passes the same 1e-10 bound the parity tests use
            p = torch.zeros_like(rhs)
            T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=prec))
            torch.cuda.synchronize()
            rc = _noalloc(pkg, xf, yf, zf, ex, rhs, p)
            assert rc[0] <= 1.05e-10, rc
        # a different field right after: the shared scratch keeps no stale sums
        pz = torch.zeros_like(rhs)
        r0 = _noalloc(pkg, xf, yf, zf, ex, rhs, pz)
        assert abs(r0[0] - 1.0) < 1e-12
        T.close()


def test_noalloc_rhs_with_a_large_fluid_mean():
    """b + 3: the compatibility constant absorbs the mean, the solve still reaches 1e-10, and
    the two-pass norm reports that (a one-pass variance would cancel to rounding noise)."""
    torch, pkg = _setup()
    from oracle import classify as OC
    from oracle import system as OSys
    from oracle.grid import Grid

    xf, yf, zf, meshes = _closed_case()
    b = synth.rhs_divergence(xf, yf, zf, 22) + 3.0
    g = Grid(xf, yf, zf)
    ib, G = OC.classify(g, meshes)
    with pkg.Context(0) as ctx:
        T = pkg.Tables(ctx, xf, yf, zf, meshes)
        ex = T.export()
        rhs = torch.from_numpy(b).cuda()
        for prec in (0, 1, 2):
            p = torch.zeros_like(rhs)
            rep = T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=prec))
            torch.cuda.synchronize()
            rc = _noalloc(pkg, xf, yf, zf, ex, rhs, p)
            ro = OSys.relative_residual(g, ib, G, b, p.cpu().numpy())
            assert rep["rel_resid"] <= 1e-10
            assert rc[0] <= 1.05e-10, (prec, rc)
            assert abs(rc[0] - ro) <= 0.05 * ro, (prec, rc, ro)
            # ||S P b|| does not see the mean: it equals the norm of the zero-mean field
            bz = torch.from_numpy(b - 3.0).cuda()
            rz = _noalloc(pkg, xf, yf, zf, ex, bz, torch.zeros_like(rhs))
            assert abs(rc[2] - rz[2]) <= 1e-12 * rz[2]
        T.close()


def test_noalloc_ghost_rows_with_a_neumann_datum():
    """A moving-boundary datum d = kappa q on the ghost rows enters the ghost-row residual."""
    torch, pkg = _setup()
    from oracle import classify as OC
    from oracle import system as OSys
    from oracle.grid import Grid

    xf, yf, zf, meshes = _closed_case()
    b = synth.rhs_divergence(xf, yf, zf, 23)
    g = Grid(xf, yf, zf)
    ib, G = OC.classify(g, meshes)
    q = np.random.default_rng(31).standard_normal(len(G))
    OC.set_neumann(G, q)
    with pkg.Context(0) as ctx:
        T = pkg.Tables(ctx, xf, yf, zf, meshes)
        T.set_neumann(torch.from_numpy(q).cuda())
        ex = T.export()
        rhs = torch.from_numpy(b).cuda()
        for tol in (1e-5, 1e-10):
            p = torch.zeros_like(rhs)
            rep = T.solve(rhs, p, tol, pkg.SolveOpts(precision=1))
            torch.cuda.synchronize()
            rc = _noalloc(pkg, xf, yf, zf, ex, rhs, p, d=ex["d"])
            ro = OSys.relative_residual(g, ib, G, b, p.cpu().numpy())
            bound = RTOL if tol > 1e-8 else 0.05
            assert abs(rc[0] - ro) <= bound * ro, (tol, rc, ro)
            assert abs(rc[0] - rep["rel_resid"]) <= bound * rep["rel_resid"], (tol, rc, rep["rel_resid"])
            if tol == 1e-10:
                assert rc[0] <= 1.05e-10
                # without the datum the same field reads as far from converged
                r_nod = _noalloc(pkg, xf, yf, zf, ex, rhs, p)
                assert r_nod[0] > 1e3 * rc[0]
        T.close()


def test_noalloc_rejects_membrane_tables():
    """Membrane entries live past the cell array (ncell + e) and their cells are fluid: the
    call returns IBM_ERR_INVALID_ARG without reading p there."""
    torch, pkg = _setup()
    f = synth.faces_tanh(26, 2.0)
    meshes = [synth.plate(0.3, nq_x=10, nq_y=6)]
    b = synth.rhs_divergence(f, f, f, 4)
    with pkg.Context(0) as ctx:
        T = pkg.Tables(ctx, f, f, f, meshes)
        assert T.nghost > 0
        ex = T.export()
        rhs = torch.from_numpy(b).cuda()
        p = torch.zeros_like(rhs)
        with pytest.raises(pkg.IbmError) as e:
            _noalloc(pkg, f, f, f, ex, rhs, p)
        assert e.value.status == 1
        # the error word is cleared by the next call: a closed-body call right after succeeds
        xf, yf, zf, cm = _closed_case()
        C = pkg.Tables(ctx, xf, yf, zf, cm)
        exc = C.export()
        bc = torch.from_numpy(synth.rhs_divergence(xf, yf, zf, 5)).cuda()
        r = _noalloc(pkg, xf, yf, zf, exc, bc, torch.zeros_like(bc))
        assert abs(r[0] - 1.0) < 1e-12
        C.close()
        T.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch, pkg = _setup()
    f = synth.faces_uniform(2049)
    g2 = synth.faces_uniform(2)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    ib = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.IbmError) as e:
        pkg.ibm_residual_norm_noalloc(f, g2, g2, ib, None, None, None, None, dummy, dummy)
    assert e.value.status == 9
