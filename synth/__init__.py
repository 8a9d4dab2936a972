"""Seeded synthetic inputs for the ghost-cell immersed-boundary pressure Poisson solve.

This module is shared by the tests, the benchmark and the smoke check.  It only
*creates inputs* -- grid face coordinates, triangulated body meshes and the
right-hand side -- and holds none of the solver's arithmetic (no stencil, no
classification, no image points, no multigrid).  Both the CPU oracle and the
CUDA library receive what it produces as plain arrays.

Workloads (the paper's own geometries and kinematics are not available, so
these stand in for them at the paper's grid scales, O(10M)-O(1B) points,
Sec. "Results and Discussions"):

* ``cfg1``: 64^3 uniform grid, sphere r=0.15 at the centre (2048-triangle
  octahedral geodesic mesh), seed 1.
* ``cfg2``: 256^3 tanh-stretched grid (max/min spacing ratio 2), prolate
  ellipsoid 0.2/0.08/0.08 with 8192 triangles rotated 20 deg about z, seed 2.
* ``cfg3``: 512^3 stretched grid, 20,000-triangle zero-thickness plate
  0.4 x 0.2, heave 0.1 sin(2 pi t), pitch 30 deg cos(2 pi t), 8 phases.
* ``cfg4``: 1024^3 uniform grid, 12 random non-overlapping spheres.
* ``cfg5``: 48 independent uneven grids (edges drawn from U{64..192}), each
  with a sphere or an ellipsoid.

Random numbers come from a counter-based splitmix64 generator (S. Vigna's
public-domain mixer) keyed by (seed, stream, index), so any element can be
regenerated independently and the arrays do not depend on chunking.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied elementwise to uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, stream: int, index) -> np.ndarray:
    """Counter-based 64-bit random words: mix(mix(seed*G + stream) + (index+1)*G)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix64(np.uint64((seed * 0x9E3779B97F4A7C15 + stream) & _MASK64))
        return _mix64(key + (idx + np.uint64(1)) * _GOLDEN)


def counter_uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in (0, 1]: (top 53 bits + 1) * 2^-53."""
    w = counter_u64(seed, stream, index)
    return ((w >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def counter_normal(seed: int, stream: int, index) -> np.ndarray:
    """Standard normal samples by Box-Muller (cosine branch) on two counter streams."""
    u1 = counter_uniform(seed, 2 * stream, index)
    u2 = counter_uniform(seed, 2 * stream + 1, index)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------- grids

def faces_uniform(n: int) -> np.ndarray:
    """n+1 uniform face coordinates on [0, 1]."""
    return np.arange(n + 1, dtype=np.float64) / n


def faces_tanh(n: int, ratio: float = 2.0) -> np.ndarray:
    """n+1 face coordinates on [0, 1], clustered at 0.5 by a tanh map.

    x_f(s) = 1/2 + atanh(tanh(beta) * (2 s - 1)) / (2 beta), s = i/n.  The
    spacing is finest at the centre and coarsest at the walls; their ratio is
    cosh(beta)^2, so beta = acosh(sqrt(ratio)).  The end faces are pinned to
    exactly 0 and 1.
    """
    if ratio <= 1.0:
        return faces_uniform(n)
    beta = math.acosh(math.sqrt(ratio))
    s = np.arange(n + 1, dtype=np.float64) / n
    x = 0.5 + np.arctanh(np.tanh(beta) * (2.0 * s - 1.0)) / (2.0 * beta)
    x[0], x[-1] = 0.0, 1.0
    if n % 2 == 0:
        x[n // 2] = 0.5
    return x


# ----------------------------------------------------------------------------- meshes

@dataclass
class Mesh:
    """Triangulated surface. ``closed`` = 1 for a solid body, 0 for a membrane."""
    verts: np.ndarray          # (V, 3) float64
    tris: np.ndarray           # (T, 3) int32, counter-clockwise seen from outside
    closed: int = 1

    @property
    def ntris(self) -> int:
        return int(self.tris.shape[0])


def octa_sphere(level: int, center=(0.5, 0.5, 0.5), radius: float = 0.15) -> Mesh:
    """Octahedral geodesic sphere: 8 * 4**level triangles (2048 at level 4).

    Each subdivision splits a triangle into four through its edge midpoints;
    every new vertex is pushed out to the unit sphere before the next level.
    """
    v = [(1.0, 0, 0), (-1.0, 0, 0), (0, 1.0, 0), (0, -1.0, 0), (0, 0, 1.0), (0, 0, -1.0)]
    verts = [np.array(p, dtype=np.float64) for p in v]
    tris = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4), (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    for _ in range(level):
        cache: dict = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                m = m / math.sqrt(float(m @ m))
                cache[key] = len(verts)
                verts.append(m)
            return cache[key]

        nt = []
        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = nt
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    return Mesh(V, np.array(tris, dtype=np.int32), 1)


def ellipsoid(level: int, semi=(0.2, 0.08, 0.08), rot_z_deg: float = 20.0,
              center=(0.5, 0.5, 0.5)) -> Mesh:
    """Unit octahedral sphere scaled by the semi-axes, rotated about z, translated."""
    s = octa_sphere(level, (0.0, 0.0, 0.0), 1.0)
    V = s.verts * np.asarray(semi, dtype=np.float64)
    a = math.radians(rot_z_deg)
    R = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    V = V @ R.T + np.asarray(center, dtype=np.float64)
    return Mesh(V, s.tris.copy(), 1)


def box_mesh(lo, hi) -> Mesh:
    """Axis-aligned box as 12 outward-oriented triangles."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    V = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    T = np.array([[0, 2, 1], [0, 3, 2], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                  [2, 3, 7], [2, 7, 6], [1, 2, 6], [1, 6, 5], [0, 4, 7], [0, 7, 3]], dtype=np.int32)
    return Mesh(V, T, 1)


def overlapping_bodies(zc: float = 0.47) -> list:
    """A box [0.1, 0.9]^2 x [0.1, zc] and a 512-triangle sphere (radius 0.23) centred on its top
    face: two closed bodies whose surfaces cut through each other (the solid is their union)."""
    return [box_mesh((0.1, 0.1, 0.1), (0.9, 0.9, zc)), octa_sphere(3, (0.5, 0.5, zc), 0.23)]


def plate(t: float, chord: float = 0.4, span: float = 0.2, nq_x: int = 100, nq_y: int = 100,
          heave: float = 0.1, pitch_deg: float = 30.0, center=(0.5, 0.5, 0.5)) -> Mesh:
    """Zero-thickness flapping plate (membrane) at phase t.

    A chord x span rectangle in the xy-plane split into nq_x * nq_y quads, two
    triangles each (normal +z), rotated about y by pitch_deg * cos(2 pi t) and
    translated to center + (0, 0, heave * sin(2 pi t)).
    """
    xs = (np.arange(nq_x + 1) / nq_x - 0.5) * chord
    ys = (np.arange(nq_y + 1) / nq_y - 0.5) * span
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    vid = np.arange((nq_y + 1) * (nq_x + 1)).reshape(nq_y + 1, nq_x + 1)
    a = vid[:-1, :-1].ravel(); b = vid[:-1, 1:].ravel(); c = vid[1:, 1:].ravel(); d = vid[1:, :-1].ravel()
    T = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)]).astype(np.int32)
    th = math.radians(pitch_deg) * math.cos(2.0 * math.pi * t)
    R = np.array([[math.cos(th), 0.0, math.sin(th)], [0.0, 1.0, 0.0], [-math.sin(th), 0.0, math.cos(th)]])
    off = np.asarray(center, dtype=np.float64) + np.array([0.0, 0.0, heave * math.sin(2.0 * math.pi * t)])
    return Mesh(V @ R.T + off, T, 0)


def plate_motion(t: float, heave: float = 0.1, pitch_deg: float = 30.0, center=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Rigid-body kinematics of `plate` at phase t (time in periods): the acceleration of its
    centre, its angular acceleration and angular velocity (about y), and the centre.  Twelve
    numbers, the layout ibm_neumann_rigid takes per mesh."""
    w = 2.0 * math.pi
    th0 = math.radians(pitch_deg)
    c = np.asarray(center, dtype=np.float64) + np.array([0.0, 0.0, heave * math.sin(w * t)])
    a0 = np.array([0.0, 0.0, -heave * w * w * math.sin(w * t)])
    alpha = np.array([0.0, -th0 * w * w * math.cos(w * t), 0.0])
    omega = np.array([0.0, -th0 * w * math.sin(w * t), 0.0])
    return np.concatenate([a0, alpha, omega, c])


def plate_velocity(t: float, heave: float = 0.1, pitch_deg: float = 30.0, center=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Rigid-body velocity of `plate` at phase t (time in periods): the velocity of its centre,
    its angular velocity (about y) and the centre.  Nine numbers, the layout
    ibm_boundary_velocity_rigid takes per mesh."""
    w = 2.0 * math.pi
    th0 = math.radians(pitch_deg)
    c = np.asarray(center, dtype=np.float64) + np.array([0.0, 0.0, heave * math.sin(w * t)])
    v0 = np.array([0.0, 0.0, heave * w * math.cos(w * t)])
    omega = np.array([0.0, -th0 * w * math.sin(w * t), 0.0])
    return np.concatenate([v0, omega, c])


def random_spheres(count: int = 12, seed: int = 4, h: float = 1.0 / 1024, level: int = 4,
                   rmin: float = 0.03, rmax: float = 0.08) -> list:
    """Non-overlapping spheres by rejection sampling (surface gap >= 8 h)."""
    out = []
    draw = 0
    while len(out) < count:
        u = counter_uniform(seed, 7, np.arange(draw, draw + 4, dtype=np.uint64))
        draw += 4
        r = rmin + (rmax - rmin) * u[0]
        lo, hi = r + 0.05, 1.0 - r - 0.05
        c = lo + (hi - lo) * u[1:4]
        if all(np.linalg.norm(c - c2) >= r + r2 + 8 * h for c2, r2 in out):
            out.append((c, r))
        if draw > 400000:
            raise RuntimeError("random_spheres: could not place spheres")
    return [octa_sphere(level, tuple(c), r) for c, r in out]


# ----------------------------------------------------------------------------- rhs

def _velocity_planes(seed: int, k0: int, k1: int, nx: int, ny: int):
    """Cell velocities (u, v, w) of planes [k0, k1), each (k1-k0, ny, nx)."""
    idx = np.arange(k0 * nx * ny, k1 * nx * ny, dtype=np.uint64)
    shp = (k1 - k0, ny, nx)
    return tuple(counter_normal(seed, c, idx).reshape(shp) for c in range(3))


def smooth_field(xf: np.ndarray, yf: np.ndarray, zf: np.ndarray, seed: int, modes: int = 3) -> np.ndarray:
    """A smooth seeded cell field [nz][ny][nx]: the product over the axes of
    1 + sum_m a_m cos(k_m x + phi_m) at the cell centres, with a_m, k_m, phi_m drawn from
    the counter generator (stream 10 + axis)."""
    out = None
    for ax, f in enumerate((xf, yf, zf)):
        f = np.asarray(f, dtype=np.float64)
        x = 0.5 * (f[:-1] + f[1:])
        u = counter_uniform(seed, 10 + ax, np.arange(3 * modes))
        g = np.ones_like(x)
        for m in range(modes):
            g = g + (0.5 * u[3 * m] / modes) * np.cos((1.0 + 6.0 * u[3 * m + 1]) * x + 6.283185307179586 * u[3 * m + 2])
        out = g if out is None else np.multiply.outer(g, out)
    return np.ascontiguousarray(out)


def rhs_divergence(xf: np.ndarray, yf: np.ndarray, zf: np.ndarray, seed: int, threads: int = 0) -> np.ndarray:
    """Discrete divergence of a seeded N(0,1) cell-centred velocity field.

    Cell velocity (u, v, w) at linear index l = (k*ny + j)*nx + i is drawn from
    streams 0, 1, 2.  Face velocity is the mean of the two adjacent cells, wall
    faces carry zero.  Returns b[k, j, i] = sum over axes of (face difference)
    / (cell width), on every cell (the solver itself only reads fluid rows).
    Planes are generated in independent slabs (in parallel threads); the values do
    not depend on the slabbing.
    """
    from concurrent.futures import ThreadPoolExecutor
    nx, ny, nz = len(xf) - 1, len(yf) - 1, len(zf) - 1
    dx, dy, dz = np.diff(xf), np.diff(yf), np.diff(zf)
    b = np.zeros((nz, ny, nx), dtype=np.float64)
    slab = max(1, min(nz, (1 << 22) // max(1, nx * ny)))

    def work(k0):
        k1 = min(nz, k0 + slab)
        a = max(0, k0 - 1)
        u, v, w = _velocity_planes(seed, a, k1, nx, ny)
        o = k0 - a                                       # offset of plane k0 in the slab
        uu, vv = u[o:], v[o:]
        fu = np.zeros((k1 - k0, ny, nx + 1)); fu[:, :, 1:-1] = 0.5 * (uu[:, :, :-1] + uu[:, :, 1:])
        fv = np.zeros((k1 - k0, ny + 1, nx)); fv[:, 1:-1, :] = 0.5 * (vv[:, :-1, :] + vv[:, 1:, :])
        out = (fu[:, :, 1:] - fu[:, :, :-1]) / dx[None, None, :] + (fv[:, 1:, :] - fv[:, :-1, :]) / dy[None, :, None]
        # z faces k-1/2 .. k+1/2 of planes k0 .. k1-1 (wall faces 0)
        fw = np.zeros((k1 - k0 + 1, ny, nx))
        ww = w                                            # planes a .. k1-1
        for q in range(k1 - k0 + 1):
            k = k0 + q                                    # face k-1/2, between planes k-1 and k
            if 0 < k < nz:
                if k < k1:
                    fw[q] = 0.5 * (ww[k - 1 - a] + ww[k - a])
        if k1 < nz:
            wn = _velocity_planes(seed, k1, k1 + 1, nx, ny)[2][0]
            fw[k1 - k0] = 0.5 * (ww[k1 - 1 - a] + wn)
        out += (fw[1:] - fw[:-1]) / dz[k0:k1, None, None]
        b[k0:k1] = out

    starts = list(range(0, nz, slab))
    nt = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=nt) as ex:
        list(ex.map(work, starts))
    return b


# ----------------------------------------------------------------------------- configs

@dataclass
class Problem:
    name: str
    xf: np.ndarray
    yf: np.ndarray
    zf: np.ndarray
    meshes: list
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (len(self.zf) - 1, len(self.yf) - 1, len(self.xf) - 1)

    @property
    def ncells(self) -> int:
        nz, ny, nx = self.shape
        return nx * ny * nz

    def rhs(self) -> np.ndarray:
        return rhs_divergence(self.xf, self.yf, self.zf, self.seed)


def cfg1(n: int = 64) -> Problem:
    f = faces_uniform(n)
    return Problem("sphere64_uniform", f, f.copy(), f.copy(), [octa_sphere(4, (0.5, 0.5, 0.5), 0.15)], 1)


def cfg2(n: int = 256, ratio: float = 2.0) -> Problem:
    f = faces_tanh(n, ratio)
    return Problem("ellipsoid256_stretched", f, f.copy(), f.copy(),
                   [ellipsoid(5, (0.2, 0.08, 0.08), 20.0, (0.5, 0.5, 0.5))], 2)


def cfg_paper_shape(ratio: float = 2.0) -> Problem:
    """The paper's weak-scaling subdomain shape, 301 x 385 x 129 cells (about 15M). The box's
    extents are proportional to the cell counts, [0, 301/385] x [0, 1] x [0, 129/385], so the
    cells are as isotropic as the paper's grid near the body; the same tanh stretching on every
    axis; the 8192-triangle ellipsoid of cfg2 at the box centre; right-hand side seed 6."""
    sx, sz = 301.0 / 385.0, 129.0 / 385.0
    return Problem("ellipsoid_301x385x129_stretched", sx * faces_tanh(301, ratio), faces_tanh(385, ratio),
                   sz * faces_tanh(129, ratio), [ellipsoid(5, (0.2, 0.08, 0.08), 20.0, (0.5 * sx, 0.5, 0.5 * sz))], 6)


def cfg3(n: int = 512, phase: int = 0, nphase: int = 8, ratio: float = 2.0) -> Problem:
    f = faces_tanh(n, ratio)
    return Problem("plate512_stretched_phase%d" % phase, f, f.copy(), f.copy(),
                   [plate(phase / nphase)], 3, {"phase": phase})


def cfg4(n: int = 1024, placement_n: int = 1024) -> Problem:
    """12 random spheres (placed for a placement_n^3 grid: surface gaps >= 8 / placement_n) on an
    n^3 uniform grid; the default keeps the 1024^3 workload's spheres at every n."""
    f = faces_uniform(n)
    return Problem("spheres12_%d_uniform" % n, f, f.copy(), f.copy(), random_spheres(12, 4, 1.0 / placement_n), 4)


def cfg5(count: int = 48, seed: int = 5, lo: int = 64, hi: int = 192) -> list:
    """Batch of uneven problems: per solve edges ~ U{lo..hi}, sphere or ellipsoid."""
    out = []
    for s in range(count):
        u = counter_uniform(seed, 11, np.arange(s * 16, s * 16 + 16, dtype=np.uint64))
        n = [lo + min(int(u[a] * (hi - lo + 1)), hi - lo) for a in range(3)]
        if u[3] < 0.5:
            m = octa_sphere(4, (0.5, 0.5, 0.5), 0.1 + 0.1 * u[4])
        else:
            m = ellipsoid(4, (0.12 + 0.1 * u[5], 0.05 + 0.05 * u[6], 0.05 + 0.05 * u[7]),
                          90.0 * u[8], (0.5, 0.5, 0.5))
        out.append(Problem("batch%02d" % s, faces_uniform(n[0]), faces_uniform(n[1]),
                           faces_uniform(n[2]), [m], 1000 * seed + s))
    return out
