"""Seeded input generators: meshes are closed and outward, the RHS telescopes to zero."""
import numpy as np
import pytest

import synth


def _edges_manifold(tris):
    from collections import Counter
    e = Counter()
    for a, b, c in tris:
        for u, v in ((a, b), (b, c), (c, a)):
            e[(int(u), int(v))] += 1
    # every directed edge once, and its reverse once: closed, consistently oriented
    return all(n == 1 and e.get((v, u), 0) == 1 for (u, v), n in e.items())


def _signed_volume(m):
    V = m.verts[m.tris]
    return float(np.sum(np.einsum("ij,ij->i", V[:, 0], np.cross(V[:, 1], V[:, 2]))) / 6.0)


@pytest.mark.parametrize("level,count", [(4, 2048), (5, 8192)])
def test_octa_sphere_counts_closed_outward(level, count):
    m = synth.octa_sphere(level, (0.5, 0.5, 0.5), 0.15)
    assert m.ntris == count
    assert _edges_manifold(m.tris)
    vol = _signed_volume(synth.octa_sphere(level, (0.0, 0.0, 0.0), 0.15))
    assert 0.97 * (4 / 3) * np.pi * 0.15 ** 3 < vol < (4 / 3) * np.pi * 0.15 ** 3
    r = np.linalg.norm(m.verts - 0.5, axis=1)
    assert np.allclose(r, 0.15, rtol=0, atol=1e-15)


def test_ellipsoid_box_plate():
    e = synth.ellipsoid(5)
    assert e.ntris == 8192 and _edges_manifold(e.tris)
    b = synth.box_mesh((0.1, 0.2, 0.3), (0.6, 0.7, 0.9))
    assert _edges_manifold(b.tris)
    assert abs(_signed_volume(b) - 0.5 * 0.5 * 0.6) < 1e-15
    p = synth.plate(0.0)
    assert p.ntris == 20000 and p.closed == 0


def test_tanh_faces():
    f = synth.faces_tanh(256, 2.0)
    d = np.diff(f)
    assert f[0] == 0.0 and f[-1] == 1.0 and np.all(d > 0)
    assert abs(d.max() / d.min() - 2.0) < 0.02


def test_rhs_telescopes():
    f = synth.faces_tanh(20, 2.0)
    g = synth.faces_uniform(12)
    b = synth.rhs_divergence(f, g, f, 3)
    V = np.diff(f)[:, None, None] * np.diff(g)[None, :, None] * np.diff(f)[None, None, :]
    assert abs(np.sum(V * b)) < 1e-12 * np.sum(np.abs(V * b))


def test_counter_rng_is_chunk_free_and_normal():
    a = synth.counter_normal(7, 0, np.arange(100000, dtype=np.uint64))
    b = synth.counter_normal(7, 0, np.arange(50000, 100000, dtype=np.uint64))
    assert np.array_equal(a[50000:], b)
    assert abs(a.mean()) < 0.02 and abs(a.std() - 1) < 0.02


def test_configs_build():
    p = synth.cfg1(16)
    assert p.shape == (16, 16, 16) and p.meshes[0].ntris == 2048
    batch = synth.cfg5(48)
    assert len(batch) == 48
    sizes = np.array([q.shape for q in batch])
    assert sizes.min() >= 64 and sizes.max() <= 192
    s = synth.random_spheres(12, 4, 1.0 / 1024)
    assert len(s) == 12


def test_plate_motion_matches_the_poses():
    """The rigid kinematics of the flapping plate against central differences of its own
    vertex positions in time (velocity from omega, acceleration from a0, alpha and omega)."""
    t, h = 0.37, 1e-4
    V = [synth.plate(t + s * h, nq_x=4, nq_y=3).verts for s in (-1, 0, 1)]
    acc_fd = (V[2] - 2 * V[1] + V[0]) / (h * h)
    m = synth.plate_motion(t)
    a0, al, om, c = m[0:3], m[3:6], m[6:9], m[9:12]
    r = V[1] - c
    acc = a0 + np.cross(al, r) + np.cross(om, np.cross(om, r))
    assert np.max(np.abs(acc - acc_fd)) < 1e-4 * np.max(np.abs(acc))
    vel_fd = (V[2] - V[0]) / (2 * h)
    vel_rot = np.cross(om, r)
    heave_v = vel_fd - vel_rot                        # the centre's velocity, equal at every vertex
    assert np.max(np.abs(heave_v - heave_v[0])) < 1e-6
