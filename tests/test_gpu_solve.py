"""GPU pressure solve vs the oracle: relative L2 <= 1e-8 after the gauge, both at 1e-10.

Precision modes: 0 FP64, 1 FP32 multigrid in FP64 refinement, 2 FP32 multigrid in
double-FP32 refinement; every mode must meet the same bar."""
import numpy as np
import pytest

import synth
from oracle import classify as OC
from oracle import solve as OS
from oracle import system as OSys
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


def _solve_gpu(pkg, T, b, prec, **kw):
    rhs = torch.from_numpy(b).cuda()
    p = torch.zeros_like(rhs)
    rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec, **kw))
    return p.cpu().numpy(), rep


def _lambda_tol(b, fl):
    """lambda's bar: 1e-8 of the rms of b's projected fluid values.  The solver's lambda is the
    sum of the fluid means of its residuals, the last one taken from the converged residual, so
    its error is of the order of that residual's mean (1e-10 relative), far inside this bar."""
    bf = b[fl]
    return 1e-8 * float(np.sqrt(np.mean((bf - bf.mean()) ** 2)))


def _parity(ctx, xf, yf, zf, meshes, seed, oracle="gmres", modes=(0, 1, 2), b=None, **kw):
    pkg, c = ctx
    g = Grid(xf, yf, zf)
    ib, G = OC.classify(g, meshes)
    if b is None:
        b = synth.rhs_divergence(xf, yf, zf, seed)
    p_o, lam_o = (OS.solve_gmres(g, ib, G, b, restart=40) if oracle == "gmres" else OS.solve_sparse(g, ib, G, b))
    T = pkg.Tables(c, xf, yf, zf, meshes)
    fl = ib == 0
    out = {}
    for mode in modes:
        # a mode is a precision, or (precision, extra solve options)
        prec, extra = (mode, {}) if isinstance(mode, int) else mode
        p, rep = _solve_gpu(pkg, T, b, prec, **kw, **extra)
        assert rep["status"] == "IBM_OK" and rep["rel_resid"] <= TOL
        # the residual the oracle computes for the GPU's p, on the oracle's own tables
        assert OSys.relative_residual(g, ib, G, b, p) <= 1.05 * TOL
        err = np.linalg.norm((p - p_o)[fl]) / np.linalg.norm(p_o[fl])
        assert err <= PARITY, (prec, err, rep)
        if len(G):
            gerr = np.max(np.abs(p.ravel()[G.cell] - p_o.ravel()[G.cell])) / np.max(np.abs(p_o[fl]))
            assert gerr <= 10 * PARITY
        assert abs(rep["lambda"] - lam_o) <= _lambda_tol(b, fl), (prec, rep["lambda"], lam_o)
        out[prec if not extra else (prec, tuple(sorted(extra.items())))] = (err, rep)
    T.close()
    return out


def test_sphere_stretched_24_sparse_oracle(ctx):
    f = synth.faces_tanh(24, 2.0)
    _parity(ctx, f, f, f, [synth.octa_sphere(4, (0.5, 0.48, 0.52), 0.22)], 1, "sparse")


def test_cfg1_sphere_64(ctx):
    p = synth.cfg1(64)
    _parity(ctx, p.xf, p.yf, p.zf, p.meshes, p.seed)


def test_ragged_stretched_ellipsoid(ctx):
    xf, yf, zf = synth.faces_tanh(37, 2.0), synth.faces_tanh(29, 1.5), synth.faces_uniform(41)
    _parity(ctx, xf, yf, zf, [synth.ellipsoid(4, (0.25, 0.12, 0.1), 33.0, (0.45, 0.5, 0.5))], 7)


def test_multi_tile_stretched_ellipsoid(ctx):
    """160 x 96 x 80 tanh-stretched cells around the 256^3 case's ellipsoid: the fused sweep's
    128 x 14 tiles number 2 x 7 (ragged in x and y) with z-chunks, so its inter-tile rings and
    the one-wave grid are compared element by element with the oracle in every mode."""
    xf, yf, zf = synth.faces_tanh(160, 2.0), synth.faces_tanh(96, 2.0), synth.faces_tanh(80, 2.0)
    _parity(ctx, xf, yf, zf, [synth.ellipsoid(5, (0.2, 0.08, 0.08), 20.0, (0.5, 0.5, 0.5))], 2)


def test_multi_tile_mean_carrying_rhs(ctx):
    """b + 3 (a large fluid mean, absorbed by lambda) on a 130 x 68 x 66 grid (ragged in every
    tile direction): same pressure as for b, lambda shifted by 3."""
    xf, yf, zf = synth.faces_tanh(130, 1.5), synth.faces_uniform(68), synth.faces_tanh(66, 2.0)
    b = synth.rhs_divergence(xf, yf, zf, 12) + 3.0
    _parity(ctx, xf, yf, zf, [synth.octa_sphere(4, (0.47, 0.52, 0.5), 0.21)], 12, b=b)


def test_coarse_bf16_storage(ctx):
    """BF16 storage of the z-march coarse levels' e and r (modes 1 and 2): 160 x 130 x 112
    stretched cells, so level 1 (80 x 65 x 56) has more than 2^18 cells and is stored in BF16,
    with ragged tiles on it; the refined pressure meets the same bar against the oracle."""
    xf, yf, zf = synth.faces_tanh(160, 1.5), synth.faces_uniform(130), synth.faces_tanh(112, 1.5)
    out = _parity(ctx, xf, yf, zf, [synth.ellipsoid(5, (0.2, 0.1, 0.08), 30.0, (0.48, 0.5, 0.5))], 14, modes=(1, 2),
                  coarse_bf16=1)
    pkg, c = ctx
    T = pkg.Tables(c, xf, yf, zf, [synth.ellipsoid(5, (0.2, 0.1, 0.08), 30.0, (0.48, 0.5, 0.5))])
    rhs = torch.from_numpy(synth.rhs_divergence(xf, yf, zf, 14)).cuda()
    p = torch.zeros_like(rhs)
    with pytest.raises(pkg.IbmError):   # FP64 multigrid has no BF16 form
        T.solve(rhs, p, TOL, pkg.SolveOpts(precision=0, coarse_bf16=1))
    T.close()
    assert all(rep["cycles"] <= 12 for _, rep in out.values()), out


def test_sweep_chunk_gives_the_same_bits(ctx):
    """The z extent of the fused sweep's tiles (sweep_chunk: the cost model's, 8, 13 planes;
    13 leaves a ragged last chunk) changes which CTA computes which plane, not the arithmetic:
    the solves' pressures are equal bit for bit, in both mixed modes, and solve the system."""
    pkg, c = ctx
    xf, yf, zf = synth.faces_tanh(150, 1.5), synth.faces_uniform(40), synth.faces_tanh(58, 2.0)
    meshes = [synth.octa_sphere(4, (0.52, 0.48, 0.5), 0.2)]
    T = pkg.Tables(c, xf, yf, zf, meshes)
    rhs = torch.from_numpy(synth.rhs_divergence(xf, yf, zf, 17)).cuda()
    for prec in (1, 2):
        out = []
        for chunk in (0, 8, 13):
            p = torch.zeros_like(rhs)
            rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=prec, sweep_chunk=chunk))
            assert rep["status"] == "IBM_OK" and rep["rel_resid"] <= TOL, (prec, chunk, rep)
            out.append((p, rep["cycles"]))
        assert all(torch.equal(out[0][0], q) and out[0][1] == k for q, k in out[1:]), prec
    p = torch.zeros_like(rhs)
    with pytest.raises(pkg.IbmError):
        T.solve(rhs, p, TOL, pkg.SolveOpts(precision=1, sweep_chunk=300))
    T.close()


def test_no_body_ragged(ctx):
    _parity(ctx, synth.faces_uniform(33), synth.faces_tanh(24, 2.0), synth.faces_uniform(20), [], 3)


def test_cfg2_full_256_elementwise(ctx):
    """The full 256^3 stretched grid around the ellipsoid: every mode, and mode 1 with BF16
    coarse storage, against the oracle's GMRES solution element by element (1e-8 relative L2
    over fluid cells after the gauge)."""
    pr = synth.cfg2(256)
    _parity(ctx, pr.xf, pr.yf, pr.zf, pr.meshes, pr.seed, modes=(0, 1, 2, (1, {"coarse_bf16": 1})))


def test_cfg2_full_256_residual_property(ctx):
    """At the full 256^3 size the oracle cannot solve in seconds; it certifies the GPU result
    by evaluating its own residual of the GPU's p (any size), for both precisions."""
    pkg, c = ctx
    pr = synth.cfg2(256)
    g = Grid(pr.xf, pr.yf, pr.zf)
    ib, G = OC.classify(g, pr.meshes)
    b = pr.rhs()
    T = pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes)
    ps = {}
    for prec in (0, 1, 2):
        p, rep = _solve_gpu(pkg, T, b, prec)
        assert rep["status"] == "IBM_OK"
        assert OSys.relative_residual(g, ib, G, b, p) <= 1.05 * TOL
        ps[prec] = p
    fl = ib == 0
    for prec in (1, 2):
        assert np.linalg.norm((ps[0] - ps[prec])[fl]) / np.linalg.norm(ps[0][fl]) <= PARITY
    T.close()


def test_paper_shape_301x385x129_residual_property(ctx):
    """The paper's weak-scaling subdomain shape (odd, ragged against every tile size): the
    oracle's residual of the GPU's p in every precision mode, and the modes against each
    other."""
    pkg, c = ctx
    pr = synth.cfg_paper_shape()
    g = Grid(pr.xf, pr.yf, pr.zf)
    ib, G = OC.classify(g, pr.meshes)
    b = pr.rhs()
    T = pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes)
    ex = T.export()
    assert np.array_equal(ex["iblank"].cpu().numpy(), ib)
    assert np.array_equal(ex["cell"].cpu().numpy(), G.cell)
    ps = {}
    for prec in (0, 1, 2):
        p, rep = _solve_gpu(pkg, T, b, prec)
        assert rep["status"] == "IBM_OK"
        assert OSys.relative_residual(g, ib, G, b, p) <= 1.05 * TOL
        ps[prec] = p
    fl = ib == 0
    for prec in (1, 2):
        assert np.linalg.norm((ps[0] - ps[prec])[fl]) / np.linalg.norm(ps[0][fl]) <= PARITY
    T.close()


def test_warm_start_and_not_converged(ctx):
    pkg, c = ctx
    f = synth.faces_uniform(20)
    m = [synth.octa_sphere(3, (0.5, 0.5, 0.5), 0.2)]
    T = pkg.Tables(c, f, f, f, m)
    b = synth.rhs_divergence(f, f, f, 5)
    p, rep = _solve_gpu(pkg, T, b, 0)
    rhs = torch.from_numpy(b).cuda()
    pw = torch.from_numpy(p).cuda()
    rep2 = T.solve(rhs, pw, TOL, pkg.SolveOpts(precision=0))
    assert rep2["cycles"] <= 1
    p3 = torch.zeros_like(rhs)
    rep3 = T.solve(rhs, p3, TOL, pkg.SolveOpts(precision=0, max_cycles=1), raise_on_error=False)
    assert rep3["status"] == "IBM_ERR_NOT_CONVERGED"
    # double-FP32 outer loop: a converged warm start needs no refinement step either
    rep4 = T.solve(rhs, torch.from_numpy(p).cuda(), TOL, pkg.SolveOpts(precision=2))
    assert rep4["status"] == "IBM_OK" and rep4["cycles"] <= 1
    T.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_graph_replay_is_bit_identical_and_deterministic(ctx, prec):
    """Replaying the captured cycle gives the same bits as direct launches, run after run
    (fixed reduction trees, Jacobi ghost updates, ping-pong sweeps)."""
    pkg, c = ctx
    f = synth.faces_tanh(40, 2.0)
    T = pkg.Tables(c, f, synth.faces_uniform(36), f, [synth.octa_sphere(4, (0.5, 0.5, 0.5), 0.2)])
    b = synth.rhs_divergence(f, synth.faces_uniform(36), f, 11)
    outs = []
    for g in (0, 1, 1, 0):
        p, rep = _solve_gpu(pkg, T, b, prec, use_graph=g)
        outs.append((p, rep["history"].copy()))
    for p, hst in outs[1:]:
        assert np.array_equal(p, outs[0][0])
        assert np.array_equal(hst, outs[0][1])
    T.close()


def test_cfg4_1024_twelve_spheres_single_gpu(ctx):
    """1024^3 uniform grid, 12 random spheres: classification bit-exact (full iblank, ghost list,
    sampled image-point rows), mixed solve to 1e-10 certified by the oracle's own residual of the
    GPU pressure, device memory reported."""
    pkg, c = ctx
    pr = synth.cfg4(1024)
    g = Grid(pr.xf, pr.yf, pr.zf)
    ib = OC.iblank_closed(g, pr.meshes)
    ghosts = OC.mark_ghosts(ib)
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    T = pkg.Tables(c, pr.xf, pr.yf, pr.zf, pr.meshes)
    ex = T.export()
    assert np.array_equal(ex["iblank"].cpu().numpy(), ib)
    assert np.array_equal(ex["cell"].cpu().numpy(), ghosts)
    rng = np.random.default_rng(4)
    sample = np.sort(rng.choice(ghosts.size, size=min(2000, ghosts.size), replace=False))
    Gs = OC.ghost_tables(g, ib, ghosts[sample], pr.meshes)
    for k, o in (("bi", Gs.bi), ("ip", Gs.ip), ("w", Gs.w), ("scale", Gs.scale), ("ref", Gs.ref), ("base", Gs.base)):
        assert np.array_equal(ex[k].cpu().numpy()[sample], o), k
    b = pr.rhs()
    rhs = torch.from_numpy(b).cuda()
    p = torch.zeros_like(rhs)
    rep = T.solve(rhs, p, TOL, pkg.SolveOpts(precision=1))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used_gb = (free0 - free1) / 1e9
    print("1024^3: ghosts %d, cycles %d, %.1f ms, device memory for tables + solver %.1f GB"
          % (T.nghost, rep["cycles"], rep["ms_total"], used_gb))
    assert rep["status"] == "IBM_OK"
    G = OC.ghost_tables(g, ib, ghosts, pr.meshes)          # every ghost row, from the oracle alone
    ph = p.cpu().numpy()
    del p, rhs
    assert OSys.relative_residual(g, ib, G, b, ph) <= 1.05 * TOL
    T.close()
