"""ctypes binding of include/ibm_poisson.h: argument marshalling only.

Every function keeps the C name and forwards plain pointers and sizes; device buffers are
torch CUDA tensors (PyTorch supplies device memory and streams, nothing else).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

IBM_OK = 0
IBM_ERR_NOT_CONVERGED = 5
STATUS = {0: "IBM_OK", 1: "IBM_ERR_INVALID_ARG", 2: "IBM_ERR_OOM", 3: "IBM_ERR_CUDA", 4: "IBM_ERR_NO_FLUID",
          5: "IBM_ERR_NOT_CONVERGED", 6: "IBM_ERR_DIVERGED", 7: "IBM_ERR_TIMEOUT", 8: "IBM_ERR_NOT_IMPLEMENTED",
          9: "IBM_ERR_CAPACITY", 10: "IBM_ERR_MESH_NOT_CLOSED"}


class IbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = "%s failed: %s" % (where, STATUS.get(status, status))
        if status == 3 and _LIB is not None:
            msg += " (" + _LIB.ibm_last_cuda_error().decode() + ")"
        super().__init__(msg)
        self.status = status


class ibm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("xf", C.c_void_p), ("yf", C.c_void_p), ("zf", C.c_void_p)]


class ibm_mesh(C.Structure):
    _fields_ = [("nverts", C.c_int32), ("ntris", C.c_int32), ("verts", C.c_void_p), ("tris", C.c_void_p),
                ("closed", C.c_int32)]


class ibm_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32), ("max_cycles", C.c_int32),
                ("inner_cycles", C.c_int32), ("use_graph", C.c_int32), ("omega", C.c_double),
                ("krylov", C.c_int32), ("method", C.c_int32), ("srj_steps", C.c_int32),
                ("coarse_bf16", C.c_int32), ("sweep_chunk", C.c_int32), ("batch_schedule", C.c_int32)]


class ibm_helmholtz_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("srj_steps", C.c_int32), ("max_cycles", C.c_int32)]


class ibm_solve_info(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("history_len", C.c_int32), ("rel_resid", C.c_double),
                ("lambda_", C.c_double), ("ms_total", C.c_double), ("resid_history", C.c_void_p),
                ("history_cap", C.c_int32)]


def library_path() -> str:
    return os.path.join(_HERE, "lib", "libibmpoisson.so")


def load_library():
    """Load the CUDA library; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise ImportError("libibmpoisson.so not built: run __graft_entry__.build() (%s)" % path)
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "ibm_status_str": (C.c_char_p, [I32]),
        "ibm_last_cuda_error": (C.c_char_p, []),
        "ibm_ctx_create": (I32, [C.POINTER(P), I32, C.c_char_p]),
        "ibm_ctx_destroy": (I32, [P]),
        "ibm_classify": (I32, [P, C.POINTER(ibm_grid), C.POINTER(ibm_mesh), I32, C.POINTER(P), P]),
        "ibm_reclassify": (I32, [P, P, C.POINTER(ibm_mesh), I32, P]),
        "ibm_tables_destroy": (I32, [P]),
        "ibm_tables_counts": (I32, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
        "ibm_tables_export": (I32, [P, P, P, P, P, P, P, P, P, P, P]),
        "ibm_tables_export_membrane": (I32, [P, P, P, P, P]),
        "ibm_tables_export_neumann": (I32, [P, P, P, P, P]),
        "ibm_set_neumann": (I32, [P, P, P]),
        "ibm_neumann_rigid": (I32, [P, C.POINTER(C.c_double), I32, P]),
        "ibm_tables_export_self_weight": (I32, [P, P, P]),
        "ibm_helmholtz_opts_default": (None, [C.POINTER(ibm_helmholtz_opts)]),
        "ibm_helmholtz_solve": (I32, [P, P, D, P, P, D, P, C.POINTER(ibm_helmholtz_opts), C.POINTER(ibm_solve_info), P]),
        "ibm_boundary_velocity_rigid": (I32, [P, C.POINTER(C.c_double), I32, P, P]),
        "ibm_helmholtz_sweeps_timed": (I32, [P, P, D, I32, I32, P, P, P, C.POINTER(C.c_double)]),
        "ibm_surface_forces": (I32, [P, C.POINTER(ibm_mesh), I32, P, P, C.POINTER(C.c_double), P, P, P, P]),
        "ibm_solve_opts_default": (None, [C.POINTER(ibm_solve_opts)]),
        "poisson_solve": (I32, [P, P, P, D, P, C.POINTER(ibm_solve_opts), C.POINTER(ibm_solve_info), P]),
        "ibm_smoother_sweeps": (I32, [P, P, I32, I32, P]),
        "ibm_smoother_sweeps_timed": (I32, [P, P, I32, I32, P, C.POINTER(C.c_double)]),
        "ibm_ctx_launch_count": (I32, [P, C.POINTER(I64)]),
        "ibm_ctx_set_sweep_wait_limit": (I32, [P, I32]),
        "ibm_smoother_apply": (I32, [P, P, I32, I32, D, P, P, D, P, P]),
        "ibm_measure_fp64_rate": (I32, [P, C.POINTER(C.c_double), P]),
        "ibm_residual_norm_noalloc": (I32, [C.POINTER(ibm_grid), P, I64, P, P, P, P, P, P, P,
                                            C.POINTER(C.c_double), P]),
        "poisson_solve_batched": (I32, [P, I32, P, P, D, P, C.POINTER(ibm_solve_opts), P, P]),
        "ibm_autotune": (I32, [P, P, I32, P, P, D, C.POINTER(ibm_solve_opts), C.POINTER(C.c_double), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, where: str):
    if status != IBM_OK:
        raise IbmError(status, where)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------- C-named calls

def ibm_ctx_create(device: int = 0, tune_cache: str | None = None):
    """Context on `device`; tune_cache: path of the autotuner's JSON cache file, or None."""
    lib = load_library()
    h = C.c_void_p()
    path = None if tune_cache is None else os.fsencode(tune_cache)
    _check(lib.ibm_ctx_create(C.byref(h), device, path), "ibm_ctx_create")
    return h


def ibm_ctx_destroy(ctx):
    _check(load_library().ibm_ctx_destroy(ctx), "ibm_ctx_destroy")


def _mesh_array(meshes, keep):
    arr = (ibm_mesh * max(1, len(meshes)))()
    for q, m in enumerate(meshes):
        v = np.ascontiguousarray(m.verts, dtype=np.float64)
        t = np.ascontiguousarray(m.tris, dtype=np.int32)
        keep += [v, t]
        arr[q] = ibm_mesh(v.shape[0], t.shape[0], v.ctypes.data, t.ctypes.data, int(m.closed))
    return arr


def ibm_classify(ctx, xf, yf, zf, meshes, stream=None):
    """Classify the grid (host face arrays) against meshes (objects with verts, tris, closed)."""
    lib = load_library()
    keep = []
    f = [np.ascontiguousarray(a, dtype=np.float64) for a in (xf, yf, zf)]
    keep += f
    g = ibm_grid(f[0].size - 1, f[1].size - 1, f[2].size - 1, f[0].ctypes.data, f[1].ctypes.data, f[2].ctypes.data)
    arr = _mesh_array(meshes, keep)
    h = C.c_void_p()
    _check(lib.ibm_classify(ctx, C.byref(g), arr, len(meshes), C.byref(h), _stream(stream)), "ibm_classify")
    return h


def ibm_reclassify(ctx, tables, meshes, stream=None):
    """Reclassify existing tables for new meshes on the same grid (reuses their memory)."""
    keep = []
    arr = _mesh_array(meshes, keep)
    _check(load_library().ibm_reclassify(ctx, tables, arr, len(meshes), _stream(stream)), "ibm_reclassify")


def ibm_tables_counts(tables):
    v = [C.c_int64() for _ in range(4)]
    _check(load_library().ibm_tables_counts(tables, *[C.byref(x) for x in v]), "ibm_tables_counts")
    return tuple(int(x.value) for x in v)


def ibm_tables_export(tables, iblank=None, cell=None, bi=None, ip=None, base=None, flags=None, ref=None, w=None,
                      scale=None, stream=None):
    _check(load_library().ibm_tables_export(tables, _ptr(iblank), _ptr(cell), _ptr(bi), _ptr(ip), _ptr(base),
                                            _ptr(flags), _ptr(ref), _ptr(w), _ptr(scale), _stream(stream)),
           "ibm_tables_export")


def ibm_set_neumann(tables, q=None, stream=None):
    """Moving-boundary datum: q (CUDA float64, one per ghost row) the pressure's derivative
    along each row's direction; None clears it."""
    _check(load_library().ibm_set_neumann(tables, _ptr(q), _stream(stream)), "ibm_set_neumann")


def ibm_neumann_rigid(tables, motions, stream=None):
    """Datum from rigid-body kinematics: motions (nmesh x 12 floats per mesh: a0, angular
    acceleration, angular velocity, centre)."""
    m = np.ascontiguousarray(np.asarray(motions, dtype=np.float64).reshape(-1, 12))
    _check(load_library().ibm_neumann_rigid(tables, m.ctypes.data_as(C.POINTER(C.c_double)), int(m.shape[0]),
                                            _stream(stream)), "ibm_neumann_rigid")


def ibm_surface_forces(tables, meshes, p, f_node, q=None, motions=None, p_side=None, flags=None, stream=None):
    """Surface pressure per triangle side and nodal pressure forces (see the header): p the
    cell pressures, f_node (nvert, 3) out; q (per triangle) or motions (per mesh, 12 floats),
    not both; p_side (ntri, 2) and flags (ntri,) optional outputs.  All tensors CUDA."""
    keep = []
    arr = _mesh_array(meshes, keep)
    mo = None
    if motions is not None:
        m = np.ascontiguousarray(np.asarray(motions, dtype=np.float64).reshape(-1, 12))
        keep.append(m)
        mo = m.ctypes.data_as(C.POINTER(C.c_double))
    _check(load_library().ibm_surface_forces(tables, arr, len(meshes), _ptr(p), _ptr(q), mo, _ptr(p_side),
                                             _ptr(flags), _ptr(f_node), _stream(stream)), "ibm_surface_forces")


def ibm_tables_destroy(tables):
    _check(load_library().ibm_tables_destroy(tables), "ibm_tables_destroy")


@dataclass
class SolveOpts:
    precision: int = 0
    nu1: int = 2
    nu2: int = 2
    max_cycles: int = 100
    inner_cycles: int = 2
    use_graph: int = 1
    omega: float = 1.3
    krylov: int = -1
    method: int = 0
    srj_steps: int = 8
    coarse_bf16: int = 0
    sweep_chunk: int = 0
    batch_schedule: int = 0


def _c_opts(o: SolveOpts) -> ibm_solve_opts:
    return ibm_solve_opts(o.precision, o.nu1, o.nu2, o.max_cycles, o.inner_cycles, o.use_graph, o.omega, o.krylov,
                          o.method, o.srj_steps, o.coarse_bf16, o.sweep_chunk, o.batch_schedule)


def poisson_solve(ctx, tables, rhs, tol, p, opts: SolveOpts | None = None, stream=None, history_cap: int = 256,
                  raise_on_error: bool = True):
    """Solve in place: rhs, p are CUDA float64 tensors [nz, ny, nx].  Returns a dict report."""
    lib = load_library()
    o = opts or SolveOpts()
    co = _c_opts(o)
    hist = np.zeros(max(1, history_cap))
    info = ibm_solve_info(0, 0, 0.0, 0.0, 0.0, hist.ctypes.data, history_cap)
    s = lib.poisson_solve(ctx, tables, _ptr(rhs), float(tol), _ptr(p), C.byref(co), C.byref(info), _stream(stream))
    rep = {"status": STATUS.get(s, s), "cycles": info.cycles, "rel_resid": info.rel_resid, "lambda": info.lambda_,
           "ms_total": info.ms_total, "history": hist[:info.history_len].copy()}
    if raise_on_error and s != IBM_OK:
        raise IbmError(s, "poisson_solve (%s)" % rep)
    return rep


@dataclass
class HelmholtzOpts:
    precision: int = 2
    srj_steps: int = 8
    max_cycles: int = 100


def ibm_helmholtz_solve(ctx, tables, alpha, f, u, ub=None, tol=1e-10, opts: HelmholtzOpts | None = None, stream=None,
                        history_cap: int = 256, raise_on_error: bool = True):
    """Advection-diffusion velocity solve in place: f, u CUDA float64 [nz, ny, nx]; ub the
    boundary values per ghost entry (CUDA float64) or None.  Returns a dict report."""
    lib = load_library()
    o = opts or HelmholtzOpts()
    co = ibm_helmholtz_opts(o.precision, o.srj_steps, o.max_cycles)
    hist = np.zeros(max(1, history_cap))
    info = ibm_solve_info(0, 0, 0.0, 0.0, 0.0, hist.ctypes.data, history_cap)
    s = lib.ibm_helmholtz_solve(ctx, tables, float(alpha), _ptr(f), _ptr(ub), float(tol), _ptr(u), C.byref(co),
                                C.byref(info), _stream(stream))
    rep = {"status": STATUS.get(s, s), "cycles": info.cycles, "rel_resid": info.rel_resid, "ms_total": info.ms_total,
           "history": hist[:info.history_len].copy()}
    if raise_on_error and s != IBM_OK:
        raise IbmError(s, "ibm_helmholtz_solve (%s)" % rep)
    return rep


def ibm_helmholtz_sweeps_timed(ctx, tables, alpha, precision, nsweeps, f, u, stream=None) -> float:
    """Mean duration (ms) of one launch of the Helmholtz sweep kernel, CUDA events on `stream`."""
    ms = C.c_double()
    _check(load_library().ibm_helmholtz_sweeps_timed(ctx, tables, float(alpha), int(precision), int(nsweeps), _ptr(f),
                                                     _ptr(u), _stream(stream), C.byref(ms)),
           "ibm_helmholtz_sweeps_timed")
    return float(ms.value)


def ibm_boundary_velocity_rigid(tables, motions, ub, stream=None):
    """Rigid boundary velocity per ghost entry into ub (CUDA float64 (3, nghost)): motions
    (nmesh x 9: v0, omega, centre)."""
    m = np.ascontiguousarray(np.asarray(motions, dtype=np.float64).reshape(-1, 9))
    _check(load_library().ibm_boundary_velocity_rigid(tables, m.ctypes.data_as(C.POINTER(C.c_double)),
                                                      int(m.shape[0]), _ptr(ub), _stream(stream)),
           "ibm_boundary_velocity_rigid")


def ibm_smoother_sweeps(ctx, tables, precision: int, nsweeps: int, stream=None):
    _check(load_library().ibm_smoother_sweeps(ctx, tables, precision, nsweeps, _stream(stream)), "ibm_smoother_sweeps")


def ibm_smoother_sweeps_timed(ctx, tables, precision: int, nsweeps: int, stream=None) -> float:
    """Mean duration (ms) of one fine-level sweep's kernel(s), CUDA events on `stream`."""
    ms = C.c_double()
    _check(load_library().ibm_smoother_sweeps_timed(ctx, tables, precision, nsweeps, _stream(stream), C.byref(ms)),
           "ibm_smoother_sweeps_timed")
    return float(ms.value)


def ibm_ctx_set_sweep_wait_limit(ctx, tries: int):
    """Test hook: tries of the fused sweep's first wait per item (0: give up at once; -1: normal)."""
    _check(load_library().ibm_ctx_set_sweep_wait_limit(ctx, int(tries)), "ibm_ctx_set_sweep_wait_limit")


def ibm_smoother_apply(ctx, tables, precision: int, nsweeps: int, omega: float, e, r, mu: float, stream=None):
    """Test hook: nsweeps finest-level smoother sweeps on caller data (e, r: float64 CUDA
    tensors of the grid's [k][j][i] shape); returns the resulting e as a new tensor."""
    e = e.contiguous()
    r = r.contiguous()
    out = e.new_empty(e.shape)
    _check(load_library().ibm_smoother_apply(ctx, tables, int(precision), int(nsweeps), float(omega), _ptr(e), _ptr(r),
                                             float(mu), _ptr(out), _stream(stream)), "ibm_smoother_apply")
    return out


def ibm_measure_fp64_rate(ctx, stream=None) -> float:
    """FP64 fused multiply-adds per second of the device (a throughput kernel, best of three)."""
    v = C.c_double()
    _check(load_library().ibm_measure_fp64_rate(ctx, C.byref(v), _stream(stream)), "ibm_measure_fp64_rate")
    return float(v.value)


def ibm_ctx_launch_count(ctx) -> int:
    v = C.c_int64()
    _check(load_library().ibm_ctx_launch_count(ctx, C.byref(v)), "ibm_ctx_launch_count")
    return int(v.value)


def ibm_residual_norm_noalloc(xf, yf, zf, iblank, cell, ref, w, scale, rhs, p, d=None, stream=None):
    """Relative projected residual of p, computed by the library without allocating device
    memory (for callers that cannot allocate after start-up).  Device arrays are torch CUDA
    tensors in the layout ibm_tables_export produces (closed bodies only); d the ghost rows'
    data as export()["d"] gives it, or None.  Returns (rel, ||SPr||, ||SPb||)."""
    f = [np.ascontiguousarray(a, dtype=np.float64) for a in (xf, yf, zf)]
    g = ibm_grid(f[0].size - 1, f[1].size - 1, f[2].size - 1, f[0].ctypes.data, f[1].ctypes.data, f[2].ctypes.data)
    out = (C.c_double * 3)()
    ng = int(cell.numel()) if cell is not None else 0
    _check(load_library().ibm_residual_norm_noalloc(C.byref(g), _ptr(iblank), ng, _ptr(cell), _ptr(ref), _ptr(w),
                                                    _ptr(scale), _ptr(d), _ptr(rhs), _ptr(p), out, _stream(stream)),
           "ibm_residual_norm_noalloc")
    return float(out[0]), float(out[1]), float(out[2])


def poisson_solve_batched(ctx, tables, rhs_list, tol, p_list, opts: "SolveOpts | None" = None, stream=None,
                          history_cap: int = 64, raise_on_error: bool = True):
    """Batched solve of independent problems (tables handles, CUDA float64 tensors).
    Returns (status name, list of per-problem report dicts)."""
    lib = load_library()
    n = len(tables)
    o = opts or SolveOpts()
    co = _c_opts(o)
    T = (C.c_void_p * max(1, n))(*[t.value if hasattr(t, "value") else t for t in tables])
    R = (C.c_void_p * max(1, n))(*[r.data_ptr() for r in rhs_list])
    Pp = (C.c_void_p * max(1, n))(*[x.data_ptr() for x in p_list])
    hists = [np.zeros(max(1, history_cap)) for _ in range(n)]
    infos = (ibm_solve_info * max(1, n))()
    for q in range(n):
        infos[q] = ibm_solve_info(0, 0, 0.0, 0.0, 0.0, hists[q].ctypes.data, history_cap)
    s = lib.poisson_solve_batched(ctx, n, T, R, float(tol), Pp, C.byref(co), infos, _stream(stream))
    reps = [{"cycles": infos[q].cycles, "rel_resid": infos[q].rel_resid, "lambda": infos[q].lambda_,
             "ms_total": infos[q].ms_total, "history": hists[q][:infos[q].history_len].copy()} for q in range(n)]
    if raise_on_error and s != IBM_OK:
        raise IbmError(s, "poisson_solve_batched")
    return STATUS.get(s, s), reps


def ibm_autotune(ctx, tables, precision: int, rhs, p_work, tol: float = 1e-10, stream=None):
    """Fastest smoother schedule for this problem: (SolveOpts, ms)."""
    best = ibm_solve_opts()
    ms = C.c_double()
    _check(load_library().ibm_autotune(ctx, tables, precision, _ptr(rhs), _ptr(p_work), float(tol), C.byref(best),
                                       C.byref(ms), _stream(stream)), "ibm_autotune")
    return SolveOpts(best.precision, best.nu1, best.nu2, best.max_cycles, best.inner_cycles, best.use_graph,
                     best.omega, best.krylov, best.method, best.srj_steps, best.coarse_bf16, best.sweep_chunk,
                     best.batch_schedule), float(ms.value)


# ----------------------------------------------------------------------------- conveniences

class Context:
    def __init__(self, device: int = 0, tune_cache: str | None = None):
        self.h = ibm_ctx_create(device, tune_cache)

    def close(self):
        if self.h is not None:
            ibm_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Tables:
    """Classified grid owned by a Context; export() returns torch CUDA tensors."""

    def __init__(self, ctx: Context, xf, yf, zf, meshes, stream=None):
        self.ctx = ctx
        self.shape = (len(zf) - 1, len(yf) - 1, len(xf) - 1)
        self.h = ibm_classify(ctx.h, xf, yf, zf, meshes, stream)
        self.membrane = len(meshes) > 0 and not int(meshes[0].closed)
        self.ncell, self.nfluid, self.nghost, self.nsolid = ibm_tables_counts(self.h)

    def export(self, stream=None) -> dict:
        import torch
        dev = torch.device("cuda")
        ng = max(self.nghost, 1)
        out = {"iblank": torch.empty(self.shape, dtype=torch.uint8, device=dev),
               "cell": torch.empty(ng, dtype=torch.int64, device=dev),
               "bi": torch.empty((ng, 3), dtype=torch.float64, device=dev),
               "ip": torch.empty((ng, 3), dtype=torch.float64, device=dev),
               "base": torch.empty((ng, 3), dtype=torch.int32, device=dev),
               "flags": torch.empty(ng, dtype=torch.int32, device=dev),
               "ref": torch.empty((ng, 8), dtype=torch.int64, device=dev),
               "w": torch.empty((ng, 8), dtype=torch.float64, device=dev),
               "scale": torch.empty(ng, dtype=torch.float64, device=dev)}
        ibm_tables_export(self.h, **out, stream=stream)
        out["kappa"] = torch.empty(ng, dtype=torch.float64, device=dev)
        out["tri"] = torch.empty(ng, dtype=torch.int32, device=dev)
        out["d"] = torch.empty(ng, dtype=torch.float64, device=dev)
        _check(load_library().ibm_tables_export_neumann(self.h, _ptr(out["kappa"]), _ptr(out["tri"]), _ptr(out["d"]),
                                                        _stream(stream)), "ibm_tables_export_neumann")
        out["wself"] = torch.empty(ng, dtype=torch.float64, device=dev)
        _check(load_library().ibm_tables_export_self_weight(self.h, _ptr(out["wself"]), _stream(stream)),
               "ibm_tables_export_self_weight")
        if self.membrane:
            out["cut"] = torch.empty(self.shape, dtype=torch.uint8, device=dev)
            out["cside"] = torch.empty(self.shape, dtype=torch.uint8, device=dev)
            out["side"] = torch.empty(ng, dtype=torch.uint8, device=dev)
            _check(load_library().ibm_tables_export_membrane(self.h, _ptr(out["cut"]), _ptr(out["cside"]),
                                                             _ptr(out["side"]), _stream(stream)),
                   "ibm_tables_export_membrane")
        if self.nghost == 0:
            for k in list(out):
                if k not in ("iblank", "cut", "cside"):
                    out[k] = out[k][:0]
        return out

    def set_neumann(self, q=None, stream=None):
        """Per-ghost pressure derivative along each row's direction (None: fixed body)."""
        ibm_set_neumann(self.h, q, stream)

    def neumann_rigid(self, motions, stream=None):
        """Datum from rigid-body kinematics per mesh (a0, alpha, omega, centre)."""
        ibm_neumann_rigid(self.h, motions, stream)

    def helmholtz_solve(self, alpha, f, u, ub=None, tol=1e-10, opts: HelmholtzOpts | None = None, stream=None, **kw):
        """Advection-diffusion velocity solve (one component) on these tables, in place."""
        return ibm_helmholtz_solve(self.ctx.h, self.h, alpha, f, u, ub, tol, opts, stream, **kw)

    def boundary_velocity_rigid(self, motions, stream=None):
        """(3, nghost) CUDA tensor of rigid boundary velocities (motions: nmesh x 9)."""
        import torch
        ub = torch.empty((3, max(self.nghost, 1)), dtype=torch.float64, device="cuda")
        ibm_boundary_velocity_rigid(self.h, motions, ub, stream)
        return ub[:, :self.nghost]

    def surface_forces(self, meshes, p, q=None, motions=None, stream=None) -> dict:
        """Side pressures (ntri, 2), flags (ntri,) and nodal forces (nvert, 3) of the meshes of
        the last classification, from the cell pressures p (CUDA float64)."""
        import torch
        dev = p.device
        ntri = sum(int(np.asarray(m.tris).reshape(-1, 3).shape[0]) for m in meshes)
        nvert = sum(int(np.asarray(m.verts).reshape(-1, 3).shape[0]) for m in meshes)
        out = {"p_side": torch.empty((ntri, 2), dtype=torch.float64, device=dev),
               "flags": torch.empty(ntri, dtype=torch.uint8, device=dev),
               "f_node": torch.empty((nvert, 3), dtype=torch.float64, device=dev)}
        ibm_surface_forces(self.h, meshes, p, out["f_node"], q=q, motions=motions, p_side=out["p_side"],
                           flags=out["flags"], stream=stream)
        return out

    def reclassify(self, meshes, stream=None):
        """New body positions on the same grid, in the tables' own memory."""
        ibm_reclassify(self.ctx.h, self.h, meshes, stream)
        self.membrane = len(meshes) > 0 and not int(meshes[0].closed)
        self.ncell, self.nfluid, self.nghost, self.nsolid = ibm_tables_counts(self.h)

    def solve(self, rhs, p, tol=1e-10, opts: SolveOpts | None = None, stream=None, **kw):
        return poisson_solve(self.ctx.h, self.h, rhs, tol, p, opts, stream, **kw)

    def close(self):
        if self.h is not None:
            ibm_tables_destroy(self.h)
            self.h = None
