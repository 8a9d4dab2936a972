"""Batched solves of uneven problems (lockstep: one launch per V-cycle stage over every
problem; or the stream pool) vs the oracle and the single-problem path; the autotuner returns
a schedule that converges."""
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


def _wide_problem():
    """136 x 40 x 24 cubic cells: two 128-cell tiles of the fused sweep in x."""
    h = 1.0 / 40
    return synth.Problem("wide", np.arange(137) * h, np.arange(41) * h, np.arange(25) * h,
                         [synth.octa_sphere(3, (1.2, 0.5, 0.3), 0.12)], 4242)


def _solve_all(pkg, c, tabs, rhs, opts):
    ps = [torch.zeros_like(r) for r in rhs]
    status, reps = pkg.poisson_solve_batched(c.h, [t.h for t in tabs], rhs, TOL, ps, opts)
    assert status == "IBM_OK"
    return [x.cpu().numpy() for x in ps], reps


@pytest.mark.parametrize("prec", [1, 2])
def test_lockstep_gives_each_problem_its_own_solve(ctx, prec):
    """The lockstep schedule (one launch per V-cycle stage over every problem, the default for
    mixed precision on closed bodies) runs each block on the single-problem kernels' bodies:
    every problem's pressure, cycle count and lambda equal its own poisson_solve's, and the
    stream-pool schedule's, bit for bit.  The batch mixes level counts (edges 20-44) and a
    problem two sweep tiles wide."""
    pkg, c = ctx
    probs = _batch(5, 11, 20, 44) + [_wide_problem()]
    tabs = [pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes) for pr in probs]
    rhs = [torch.from_numpy(pr.rhs()).cuda() for pr in probs]
    pl, rl = _solve_all(pkg, c, tabs, rhs, pkg.SolveOpts(precision=prec))
    pp, rp = _solve_all(pkg, c, tabs, rhs, pkg.SolveOpts(precision=prec, batch_schedule=1))
    for q in range(len(probs)):
        p1 = torch.zeros_like(rhs[q])
        r1 = tabs[q].solve(rhs[q], p1, TOL, pkg.SolveOpts(precision=prec))
        assert rl[q]["rel_resid"] <= TOL
        assert rl[q]["cycles"] == r1["cycles"] == rp[q]["cycles"]
        assert rl[q]["lambda"] == r1["lambda"] == rp[q]["lambda"]
        assert np.array_equal(pl[q], p1.cpu().numpy()), probs[q].name
        assert np.array_equal(pl[q], pp[q]), probs[q].name
    for t in tabs:
        t.close()


def test_lockstep_splits_launches_of_more_than_48_problems(ctx):
    """50 problems: each stage takes two launches (48 + 2 problems); every problem still gets
    its own solve's bits."""
    pkg, c = ctx
    probs = _batch(50, 21, 12, 20)
    tabs = [pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes) for pr in probs]
    rhs = [torch.from_numpy(pr.rhs()).cuda() for pr in probs]
    pl, rl = _solve_all(pkg, c, tabs, rhs, pkg.SolveOpts(precision=1))
    for q in range(len(probs)):
        assert rl[q]["rel_resid"] <= TOL
    for q in (0, 1, 47, 48, 49):
        p1 = torch.zeros_like(rhs[q])
        r1 = tabs[q].solve(rhs[q], p1, TOL, pkg.SolveOpts(precision=1))
        assert rl[q]["cycles"] == r1["cycles"]
        assert np.array_equal(pl[q], p1.cpu().numpy()), q
    with pytest.raises(pkg.IbmError):
        pkg.poisson_solve_batched(c.h, [tabs[0].h], [rhs[0]], TOL, [torch.zeros_like(rhs[0])],
                                  pkg.SolveOpts(precision=1, batch_schedule=2))
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
