"""Batched solves of uneven problems (one launch per V-cycle stage) vs the oracle and the
single-problem path; the autotuner returns a schedule that converges."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import solve as OS
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


def _batch(nprob=6, seed=3, lo=20, hi=44):
    return synth.cfg5(nprob, seed, lo, hi)


@pytest.mark.parametrize("prec", [1, 0])
def test_batched_matches_oracle_and_single(ctx, prec):
    pkg, c = ctx
    probs = _batch()
    tabs, rhs, ps = [], [], []
    for pr in probs:
        tabs.append(pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes))
        rhs.append(torch.from_numpy(pr.rhs()).cuda())
        ps.append(torch.zeros_like(rhs[-1]))
    status, reps = pkg.poisson_solve_batched(c.h, [t.h for t in tabs], rhs, TOL, ps,
                                             pkg.SolveOpts(precision=prec))
    assert status == "IBM_OK"
    cyc = [r["cycles"] for r in reps]
    for q, pr in enumerate(probs):
        assert reps[q]["rel_resid"] <= TOL
        g = Grid(pr.xf, pr.yf, pr.zf)
        ib, G = OC.classify(g, pr.meshes)
        po, lam = (OS.solve_sparse if pr.ncells <= 40000 else OS.solve_gmres)(g, ib, G, pr.rhs())
        fl = ib == 0
        pb = ps[q].cpu().numpy()
        assert np.linalg.norm((pb - po)[fl]) / np.linalg.norm(po[fl]) <= PARITY
        # the single-problem path reaches the same solution
        p1 = torch.zeros_like(rhs[q])
        tabs[q].solve(rhs[q], p1, TOL, pkg.SolveOpts(precision=prec))
        assert np.linalg.norm((p1.cpu().numpy() - pb)[fl]) / np.linalg.norm(pb[fl]) <= PARITY
    assert len(set(cyc)) >= 1
    for t in tabs:
        t.close()


def test_batched_with_an_already_converged_problem(ctx):
    pkg, c = ctx
    probs = _batch(3, 9, 16, 30)
    tabs = [pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes) for pr in probs]
    rhs = [torch.from_numpy(pr.rhs()).cuda() for pr in probs]
    rhs[1].zero_()                                  # b = 0: p = 0 is already the solution
    ps = [torch.zeros_like(r) for r in rhs]
    status, reps = pkg.poisson_solve_batched(c.h, [t.h for t in tabs], rhs, TOL, ps, pkg.SolveOpts(precision=1))
    assert status == "IBM_OK"
    assert reps[1]["cycles"] == 0 and reps[0]["cycles"] > 0 and reps[2]["cycles"] > 0
    assert float(ps[1].abs().max()) == 0.0
    for t in tabs:
        t.close()


def test_autotune_returns_a_converging_schedule(ctx):
    pkg, c = ctx
    f = synth.faces_tanh(40, 2.0)
    T = pkg.Tables(c, f, f, f, [synth.ellipsoid(4)])
    rhs = torch.from_numpy(synth.rhs_divergence(f, f, f, 2)).cuda()
    work = torch.zeros_like(rhs)
    opts, ms = pkg.ibm_autotune(c.h, T.h, 1, rhs, work, TOL)
    assert 1.0 < opts.omega < 2.0 and opts.nu1 + opts.nu2 >= 1 and ms > 0 and opts.krylov in (0, 2)
    p = torch.zeros_like(rhs)
    rep = T.solve(rhs, p, TOL, opts)
    assert rep["rel_resid"] <= TOL
    T.close()


def test_batched_every_mode_membranes_and_krylov(ctx):
    """The batched path runs each problem's single-problem step: double-FP32 refinement, GCR
    acceleration and membrane tables batch like the rest, and every problem matches its own
    single solve (1e-8) at a residual within tol."""
    pkg, c = ctx
    probs = _batch(3, 5, 16, 28)
    tabs = [pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes) for pr in probs]
    f = synth.faces_tanh(24, 2.0)
    tabs.append(pkg.Tables(c, f, f, f, [synth.plate(0.25, nq_x=10, nq_y=6)]))
    rhs = [torch.from_numpy(pr.rhs()).cuda() for pr in probs]
    rhs.append(torch.from_numpy(synth.rhs_divergence(f, f, f, 3)).cuda())
    for o in (pkg.SolveOpts(precision=2), pkg.SolveOpts(precision=1, krylov=4), pkg.SolveOpts(precision=0)):
        ps = [torch.zeros_like(r) for r in rhs]
        status, reps = pkg.poisson_solve_batched(c.h, [t.h for t in tabs], rhs, TOL, ps, o)
        assert status == "IBM_OK", o
        for q, t in enumerate(tabs):
            assert reps[q]["rel_resid"] <= TOL and reps[q]["cycles"] > 0
            p1 = torch.zeros_like(rhs[q])
            t.solve(rhs[q], p1, TOL, o)
            assert float((p1 - ps[q]).norm() / p1.norm()) <= PARITY, (o, q)
    for t in tabs:
        t.close()
