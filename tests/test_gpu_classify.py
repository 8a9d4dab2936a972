"""GPU iblanking / ghost / image-point tables vs the oracle: bit-exact (integer and FP64)."""
import numpy as np
import pytest

import synth
from tests.gpu_util import assert_tables_equal, classify_both, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2605_04335_gb300 as pkg
    c = pkg.Context(0)
    yield pkg, c
    c.close()


def _run(ctx, xf, yf, zf, meshes, oracle_ghosts=True):
    pkg, c = ctx
    g, T, ex, ib, G = classify_both(pkg, c, xf, yf, zf, meshes, oracle_ghosts)
    assert_tables_equal(ex, ib, G)
    assert T.nghost == (len(G) if G is not None else T.nghost)
    T.close()
    return ex


def test_sphere_stretched_24(ctx):
    f = synth.faces_tanh(24, 2.0)
    ex = _run(ctx, f, f, f, [synth.octa_sphere(4, (0.5, 0.48, 0.52), 0.22)])
    assert np.sum(ex["iblank"] & 1) > 100


def test_cfg1_sphere_64(ctx):
    p = synth.cfg1(64)
    _run(ctx, p.xf, p.yf, p.zf, p.meshes)


def test_ragged_ellipsoid_and_union(ctx):
    xf, yf, zf = synth.faces_tanh(37, 2.0), synth.faces_tanh(29, 1.5), synth.faces_uniform(41)
    ms = [synth.ellipsoid(4, (0.25, 0.12, 0.1), 33.0, (0.45, 0.5, 0.5)),
          synth.octa_sphere(3, (0.8, 0.7, 0.25), 0.12)]
    _run(ctx, xf, yf, zf, ms)


def test_ties_box_through_centres(ctx):
    n = 12
    f = synth.faces_uniform(n)
    c = 0.5 * (f[:-1] + f[1:])
    m = synth.box_mesh((c[2], c[3], c[1]), (c[8], c[9], c[10]))
    _run(ctx, f, f, f, [m])


def test_ties_rotated_cube_vertices_on_columns(ctx):
    n = 16
    f = synth.faces_uniform(n)
    h = 1.0 / n
    cc, r = 0.5 + h / 2, 4 * h
    V = np.array([[cc - r, cc, 0.23], [cc, cc - r, 0.23], [cc + r, cc, 0.23], [cc, cc + r, 0.23],
                  [cc - r, cc, 0.71], [cc, cc - r, 0.71], [cc + r, cc, 0.71], [cc, cc + r, 0.71]])
    m = synth.Mesh(V, synth.box_mesh((0, 0, 0), (1, 1, 1)).tris, 1)
    _run(ctx, f, f, f, [m])


def test_wall_slab_mirror(ctx):
    f = synth.faces_uniform(16)
    ex = _run(ctx, f, f, f, [synth.box_mesh((0.5, -1.0, -1.0), (2.0, 2.0, 2.0))])
    assert np.all(np.sum(ex["w"] == 1.0, axis=1) == 1)


def test_no_body(ctx):
    pkg, c = ctx
    f = synth.faces_uniform(10)
    T = pkg.Tables(c, f, f, f, [])
    assert (T.nghost, T.nsolid, T.nfluid) == (0, 0, 1000)
    assert not np.any(T.export()["iblank"].cpu().numpy())
    T.close()


def test_cfg2_full_256(ctx):
    p = synth.cfg2(256)
    _run(ctx, p.xf, p.yf, p.zf, p.meshes)


def test_invalid_inputs(ctx):
    pkg, c = ctx
    f = synth.faces_uniform(8)
    with pytest.raises(pkg.IbmError):
        pkg.Tables(c, f[::-1], f, f, [])              # decreasing faces
    with pytest.raises(pkg.IbmError):
        pkg.Tables(c, f * 10, f, f, [])               # outside [-4, 4]
    bad = synth.octa_sphere(2)
    bad.tris = bad.tris.copy()
    bad.tris[0, 0] = 10 ** 6
    with pytest.raises(pkg.IbmError):
        pkg.Tables(c, f, f, f, [bad])                 # vertex index out of range
