"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def classify_both(pkg, ctx, xf, yf, zf, meshes, oracle_ghosts=True):
    """GPU tables (exported to host numpy) and oracle tables for the same inputs."""
    from oracle import classify as OC
    from oracle.grid import Grid
    g = Grid(xf, yf, zf)
    T = pkg.Tables(ctx, xf, yf, zf, meshes)
    ex = {k: v.cpu().numpy() for k, v in T.export().items()}
    if oracle_ghosts:
        ib, G = OC.classify(g, meshes)
    else:
        ib = OC.iblank_closed(g, meshes)
        OC.mark_ghosts(ib)
        G = None
    return g, T, ex, ib, G


def assert_tables_equal(ex, ib, G, bitexact_fp=True):
    assert np.array_equal(ex["iblank"], ib), "iblank: %d cells differ" % int(np.sum(ex["iblank"] != ib))
    if G is None:
        return
    assert np.array_equal(ex["cell"], G.cell)
    assert np.array_equal(ex["base"], G.base)
    assert np.array_equal(ex["flags"], G.flags)
    assert np.array_equal(ex["ref"], G.ref)
    assert np.array_equal(ex["tri"].astype(np.int64), G.tri)
    for k, o in (("bi", G.bi), ("ip", G.ip), ("w", G.w), ("scale", G.scale), ("kappa", G.kappa),
                 ("wself", G.wself)):
        if bitexact_fp:
            assert np.array_equal(ex[k], o), "%s: max diff %g" % (k, np.max(np.abs(ex[k] - o)) if o.size else 0)
        else:
            assert np.allclose(ex[k], o, rtol=1e-14, atol=1e-15)
