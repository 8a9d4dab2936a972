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


def test_noalloc_residual_matches_solver_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_04335_gb300 as pkg
    from oracle import classify as OC
    from oracle import system as OSys
    from oracle.grid import Grid

    xf, yf, zf = synth.faces_tanh(48, 2.0), synth.faces_uniform(40), synth.faces_tanh(44, 1.5)
    meshes = [synth.octa_sphere(4, (0.5, 0.5, 0.5), 0.22)]
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
            r1 = pkg.ibm_residual_norm_noalloc(xf, yf, zf, ex["iblank"], ex["cell"], ex["ref"], ex["w"],
                                               ex["scale"], rhs, p)
            r2 = pkg.ibm_residual_norm_noalloc(xf, yf, zf, ex["iblank"], ex["cell"], ex["ref"], ex["w"],
                                               ex["scale"], rhs, p)
            assert r1 == r2                                            # two calls in a row agree exactly
            assert abs(r1[0] - rep["rel_resid"]) <= RTOL * rep["rel_resid"], (r1, rep["rel_resid"])
            ro = OSys.relative_residual(g, ib, G, b, p.cpu().numpy())
            assert abs(r1[0] - ro) <= RTOL * ro, (r1, ro)
            # the converged field passes the same 1e-10 bound the parity tests use
            p = torch.zeros_like(rhs)
            T.solve(rhs, p, 1e-10, pkg.SolveOpts(precision=prec))
            torch.cuda.synchronize()
            rc = pkg.ibm_residual_norm_noalloc(xf, yf, zf, ex["iblank"], ex["cell"], ex["ref"], ex["w"],
                                               ex["scale"], rhs, p)
            assert rc[0] <= 1.05e-10, rc
        # a different field right after: the shared scratch keeps no stale sums
        pz = torch.zeros_like(rhs)
        r0 = pkg.ibm_residual_norm_noalloc(xf, yf, zf, ex["iblank"], ex["cell"], ex["ref"], ex["w"], ex["scale"],
                                           rhs, pz)
        assert abs(r0[0] - 1.0) < 1e-12
        T.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_04335_gb300 as pkg
    f = synth.faces_uniform(2049)
    g2 = synth.faces_uniform(2)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    ib = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.IbmError) as e:
        pkg.ibm_residual_norm_noalloc(f, g2, g2, ib, None, None, None, None, dummy, dummy)
    assert e.value.status == 9
