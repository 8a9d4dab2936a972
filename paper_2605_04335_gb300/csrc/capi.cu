// extern "C" entry points of libibmpoisson (declared and documented in include/ibm_poisson.h).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "ibm_internal.cuh"

namespace ibm {

static thread_local std::string g_last_error;

void set_cuda_error(cudaError_t e, const char *where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

ibm_status check(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return IBM_OK;
  set_cuda_error(e, where);
  cudaGetLastError();   // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA;
}

ibm_status classify_impl(ibm_ctx *ctx, const ibm_grid *grid, const ibm_mesh *meshes, int nmesh, ibm_tables **out,
                         cudaStream_t st);
ibm_status reclassify_impl(ibm_ctx *ctx, ibm_tables *t, const ibm_mesh *meshes, int nmesh, cudaStream_t st);
ibm_status solve_impl(ibm_ctx *ctx, ibm_tables *t, const double *rhs, double tol, double *p_user,
                      const ibm_solve_opts *opts, ibm_solve_info *info, cudaStream_t st);
ibm_status sweeps_impl(ibm_ctx *ctx, ibm_tables *t, int precision, int nsweeps, cudaStream_t st,
                       double *kernel_ms);
ibm_status smoother_apply_impl(ibm_ctx *ctx, ibm_tables *t, int precision, int nsweeps, double omega,
                               const double *e_in, const double *r_in, double mu, double *e_out, cudaStream_t st);
ibm_status measure_fp64_impl(ibm_ctx *ctx, double *dfma_per_s, cudaStream_t st);
ibm_status neumann_set_impl(ibm_tables *T, const double *q, cudaStream_t st);
ibm_status neumann_rigid_impl(ibm_tables *T, const double *motions, int nmesh, cudaStream_t st);
ibm_status helmholtz_solve_impl(ibm_ctx *ctx, ibm_tables *t, double alpha, const double *f_user, const double *ub,
                                double tol, double *u_user, const ibm_helmholtz_opts *opts, ibm_solve_info *info,
                                cudaStream_t st, double *time_ms = nullptr, int n_timed = 0);
ibm_status boundary_velocity_rigid_impl(ibm_tables *T, const double *motions, int nmesh, double *ub,
                                        cudaStream_t st);
ibm_status helmholtz_sweeps_timed_impl(ibm_ctx *ctx, ibm_tables *t, double alpha, int precision, int nsweeps,
                                       const double *f_user, double *u_user, cudaStream_t st, double *ms);
ibm_status surface_forces_impl(ibm_tables *T, const ibm_mesh *meshes, int nmesh, const double *p,
                               const double *q_tri, const double *motions, double *p_side, uint8_t *flags,
                               double *f_node, cudaStream_t st);
ibm_status solve_batched_impl(ibm_ctx *ctx, int n, ibm_tables *const *ts, const double *const *rhs, double tol,
                              double *const *p_user, const ibm_solve_opts *opts, ibm_solve_info *infos,
                              cudaStream_t st);

// ---------------------------------------------------------------------- tune cache
//
// A JSON file of autotuned schedules, one entry per line:
//   {"ibm_tune_cache": 1, "entries": [
//   {"key": "...", "omega": 1.3, "nu1": 2, "nu2": 2, "inner_cycles": 2, "krylov": 0, "ms": 8.1},
//   ...
//   ]}
// Key: the grid (cell counts and a 64-bit FNV-1a hash of the face coordinates' bytes), the
// precision mode and whether the tables hold membranes.  The body's position is not part of
// it, so one entry serves every time step of a moving body.

struct TuneEntry {
  std::string key;
  double omega = 1.3, ms = 0.0;
  int nu1 = 2, nu2 = 2, inner = 2, krylov = -1, chunk = 0;
};

static std::string tune_key(const ibm_tables *t, int precision) {
  uint64_t h = 1469598103934665603ULL;
  auto mix = [&](const std::vector<double> &v) {
    const unsigned char *b = reinterpret_cast<const unsigned char *>(v.data());
    for (size_t q = 0; q < v.size() * sizeof(double); ++q) { h ^= b[q]; h *= 1099511628211ULL; }
  };
  mix(t->xf); mix(t->yf); mix(t->zf);
  char buf[128];
  std::snprintf(buf, sizeof buf, "grid=%dx%dx%d faces=%016llx precision=%d membrane=%d", t->nx, t->ny, t->nz,
                (unsigned long long)h, precision, t->membrane ? 1 : 0);
  return buf;
}

// value of "name": in one entry line (number), false if absent
static bool json_num(const std::string &line, const char *name, double *v) {
  const std::string pat = std::string("\"") + name + "\":";
  size_t q = line.find(pat);
  if (q == std::string::npos) return false;
  const char *p = line.c_str() + q + pat.size();
  char *end = nullptr;
  *v = std::strtod(p, &end);
  return end != p;
}

// entries of the cache file (a missing or unreadable file reads as empty; lines that do not
// parse are skipped)
static std::vector<TuneEntry> tune_read(const std::string &path) {
  std::vector<TuneEntry> out;
  std::ifstream f(path);
  std::string line;
  while (f && std::getline(f, line)) {
    size_t a = line.find("{\"key\": \"");
    if (a == std::string::npos) continue;
    a += 9;
    size_t b = line.find('"', a);
    if (b == std::string::npos) continue;
    TuneEntry e;
    e.key = line.substr(a, b - a);
    double nu1, nu2, inner, kry;
    if (!json_num(line, "omega", &e.omega) || !json_num(line, "nu1", &nu1) || !json_num(line, "nu2", &nu2) ||
        !json_num(line, "inner_cycles", &inner) || !json_num(line, "krylov", &kry) || !json_num(line, "ms", &e.ms))
      continue;
    e.nu1 = (int)nu1; e.nu2 = (int)nu2; e.inner = (int)inner; e.krylov = (int)kry;
    double chunk = 0;
    if (json_num(line, "sweep_chunk", &chunk)) e.chunk = (int)chunk;
    out.push_back(e);
  }
  return out;
}

// the whole file, rewritten through a temporary file and a rename
static bool tune_write(const std::string &path, const std::vector<TuneEntry> &es) {
  const std::string tmp = path + ".tmp";
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return false;
    f << "{\"ibm_tune_cache\": 1, \"entries\": [\n";
    char buf[512];
    for (size_t q = 0; q < es.size(); ++q) {
      const TuneEntry &e = es[q];
      std::snprintf(buf, sizeof buf,
                    "{\"key\": \"%s\", \"omega\": %.17g, \"nu1\": %d, \"nu2\": %d, \"inner_cycles\": %d, "
                    "\"krylov\": %d, \"sweep_chunk\": %d, \"ms\": %.6g}%s\n",
                    e.key.c_str(), e.omega, e.nu1, e.nu2, e.inner, e.krylov, e.chunk, e.ms,
                    q + 1 < es.size() ? "," : "");
      f << buf;
    }
    f << "]}\n";
    if (!f) return false;
  }
  return std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace ibm

extern "C" {

const char *ibm_status_str(ibm_status s) {
  switch (s) {
    case IBM_OK: return "ok";
    case IBM_ERR_INVALID_ARG: return "invalid argument";
    case IBM_ERR_OOM: return "out of device memory";
    case IBM_ERR_CUDA: return "CUDA error";
    case IBM_ERR_NO_FLUID: return "no fluid cell";
    case IBM_ERR_NOT_CONVERGED: return "not converged";
    case IBM_ERR_DIVERGED: return "diverged";
    case IBM_ERR_TIMEOUT: return "device wait timed out";
    case IBM_ERR_NOT_IMPLEMENTED: return "not implemented";
    case IBM_ERR_CAPACITY: return "capacity exceeded";
    case IBM_ERR_MESH_NOT_CLOSED: return "closed mesh not watertight";
  }
  return "unknown status";
}

const char *ibm_last_cuda_error(void) { return ibm::g_last_error.c_str(); }

ibm_status ibm_ctx_create(ibm_ctx **out, int32_t device, const char *tune_cache_path) {
  if (!out) return IBM_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  IBM_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(device));
  ibm_ctx *c = new ibm_ctx();
  c->device = device;
  if (tune_cache_path) c->tune_cache = tune_cache_path;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (c->sm_count > 0) c->wave = 8 * c->sm_count;
  cudaError_t e = cudaMalloc((void **)&c->partials, sizeof(double) * ibm::REDUCE_BLOCKS * 8);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->scal, sizeof(double) * ibm::NSCAL);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&c->hscal, sizeof(double) * ibm::NSCAL);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->errflag, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->errflag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    ibm_ctx_destroy(c);
    return ibm::check(e, "ibm_ctx_create");
  }
  cudaMemset(c->scal, 0, sizeof(double) * ibm::NSCAL);
  *out = c;
  return IBM_OK;
}

ibm_status ibm_ctx_destroy(ibm_ctx *c) {
  if (!c) return IBM_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (c->partials) cudaFree(c->partials);
  if (c->scal) cudaFree(c->scal);
  if (c->hscal) cudaFreeHost(c->hscal);
  if (c->errflag) cudaFree(c->errflag);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaStream_t q : c->bstream) if (q) cudaStreamDestroy(q);
  for (cudaEvent_t q : c->bevent) if (q) cudaEventDestroy(q);
  if (c->bscal) cudaFree(c->bscal);
  if (c->bhscal) cudaFreeHost(c->bhscal);
  if (c->bpart) cudaFree(c->bpart);
  if (c->lk_count) cudaFree(c->lk_count);
  if (c->lk_tail) cudaFree(c->lk_tail);
  delete c;
  return IBM_OK;
}

ibm_status ibm_classify(ibm_ctx *ctx, const ibm_grid *grid, const ibm_mesh *meshes, int32_t nmesh, ibm_tables **out,
                        void *stream) {
  if (out) *out = nullptr;
  return ibm::classify_impl(ctx, grid, meshes, nmesh, out, (cudaStream_t)stream);
}

ibm_status ibm_reclassify(ibm_ctx *ctx, ibm_tables *t, const ibm_mesh *meshes, int32_t nmesh, void *stream) {
  return ibm::reclassify_impl(ctx, t, meshes, nmesh, (cudaStream_t)stream);
}

ibm_status ibm_tables_destroy(ibm_tables *t) {
  if (!t) return IBM_ERR_INVALID_ARG;
  if (t->ctx) cudaSetDevice(t->ctx->device);
  cudaDeviceSynchronize();
  for (int q = 0; q < 5; ++q) ibm::free_hierarchy(t->hier[q]);
  void *ps[] = {t->iblank, t->gcell, t->gbi, t->gip, t->gw, t->gscale, t->gbase, t->gflags, t->gref, t->axis,
                t->scratch, t->cut, t->cside, t->gside, t->gkeys, t->gkappa, t->gd, t->gtri, t->fbuf, t->gwself};
  for (void *p : ps) if (p) cudaFree(p);
  delete t;
  return IBM_OK;
}

ibm_status ibm_set_neumann(ibm_tables *t, const double *q_dev, void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  return ibm::neumann_set_impl(t, q_dev, (cudaStream_t)stream);
}

ibm_status ibm_neumann_rigid(ibm_tables *t, const double *motions, int32_t nmesh, void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  return ibm::neumann_rigid_impl(t, motions, nmesh, (cudaStream_t)stream);
}

ibm_status ibm_tables_export_self_weight(const ibm_tables *t, double *wself_dev, void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (t->nghost > 0 && wself_dev)
    IBM_TRY(cudaMemcpyAsync(wself_dev, t->gwself, sizeof(double) * t->nghost, cudaMemcpyDeviceToDevice, st));
  IBM_TRY(cudaStreamSynchronize(st));
  return IBM_OK;
}

void ibm_helmholtz_opts_default(ibm_helmholtz_opts *o) {
  if (!o) return;
  o->precision = 2;
  o->srj_steps = 8;
  o->max_cycles = 100;
}

ibm_status ibm_helmholtz_solve(ibm_ctx *ctx, ibm_tables *t, double alpha, const double *f_dev, const double *ub_dev,
                               double tol, double *u_dev, const ibm_helmholtz_opts *opts, ibm_solve_info *info,
                               void *stream) {
  if (!ctx || !t || t->ctx != ctx) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  return ibm::helmholtz_solve_impl(ctx, t, alpha, f_dev, ub_dev, tol, u_dev, opts, info, (cudaStream_t)stream);
}

ibm_status ibm_helmholtz_sweeps_timed(ibm_ctx *ctx, ibm_tables *t, double alpha, int32_t precision, int32_t nsweeps,
                                      const double *f_dev, double *u_dev, void *stream, double *kernel_ms) {
  if (!ctx || !t || t->ctx != ctx) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  return ibm::helmholtz_sweeps_timed_impl(ctx, t, alpha, precision, nsweeps, f_dev, u_dev, (cudaStream_t)stream,
                                          kernel_ms);
}

ibm_status ibm_boundary_velocity_rigid(ibm_tables *t, const double *motions, int32_t nmesh, double *ub_dev,
                                       void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  return ibm::boundary_velocity_rigid_impl(t, motions, nmesh, ub_dev, (cudaStream_t)stream);
}

ibm_status ibm_surface_forces(ibm_tables *t, const ibm_mesh *meshes, int32_t nmesh, const double *p_dev,
                              const double *q_tri_dev, const double *motions, double *p_side_dev, uint8_t *flags_dev,
                              double *f_node_dev, void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  if (t->nx < 2 || t->ny < 2 || t->nz < 2) return IBM_ERR_INVALID_ARG;
  return ibm::surface_forces_impl(t, meshes, nmesh, p_dev, q_tri_dev, motions, p_side_dev, flags_dev, f_node_dev,
                                  (cudaStream_t)stream);
}

ibm_status ibm_tables_export_neumann(const ibm_tables *t, double *kappa_dev, int32_t *tri_dev, double *d_dev,
                                     void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const long long ng = t->nghost;
  if (ng > 0) {
    if (kappa_dev) IBM_TRY(cudaMemcpyAsync(kappa_dev, t->gkappa, sizeof(double) * ng, cudaMemcpyDeviceToDevice, st));
    if (tri_dev) IBM_TRY(cudaMemcpyAsync(tri_dev, t->gtri, sizeof(int32_t) * ng, cudaMemcpyDeviceToDevice, st));
    if (d_dev) {
      if (t->has_datum) IBM_TRY(cudaMemcpyAsync(d_dev, t->gd, sizeof(double) * ng, cudaMemcpyDeviceToDevice, st));
      else IBM_TRY(cudaMemsetAsync(d_dev, 0, sizeof(double) * ng, st));
    }
  }
  IBM_TRY(cudaStreamSynchronize(st));
  return IBM_OK;
}

ibm_status ibm_tables_export_membrane(const ibm_tables *t, uint8_t *cut_dev, uint8_t *side_dev, uint8_t *gside_dev,
                                      void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  if (!t->membrane) return IBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  if (cut_dev) IBM_TRY(cudaMemcpyAsync(cut_dev, t->cut, t->ncell, cudaMemcpyDeviceToDevice, st));
  if (side_dev) IBM_TRY(cudaMemcpyAsync(side_dev, t->cside, t->ncell, cudaMemcpyDeviceToDevice, st));
  if (gside_dev && t->nghost > 0) IBM_TRY(cudaMemcpyAsync(gside_dev, t->gside, t->nghost, cudaMemcpyDeviceToDevice, st));
  IBM_TRY(cudaStreamSynchronize(st));
  return IBM_OK;
}

ibm_status ibm_tables_counts(const ibm_tables *t, int64_t *ncell, int64_t *nfluid, int64_t *nghost, int64_t *nsolid) {
  if (!t) return IBM_ERR_INVALID_ARG;
  if (ncell) *ncell = t->ncell;
  if (nfluid) *nfluid = t->nfluid;
  if (nghost) *nghost = t->nghost;
  if (nsolid) *nsolid = t->nsolid;
  return IBM_OK;
}

ibm_status ibm_tables_export(const ibm_tables *t, uint8_t *iblank_dev, int64_t *cell_dev, double *bi_dev,
                             double *ip_dev, int32_t *base_dev, int32_t *flags_dev, int64_t *ref_dev, double *w_dev,
                             double *scale_dev, void *stream) {
  if (!t) return IBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  IBM_TRY(cudaSetDevice(t->ctx->device));
  const long long ng = t->nghost;
  if (iblank_dev) IBM_TRY(cudaMemcpyAsync(iblank_dev, t->iblank, t->ncell, cudaMemcpyDeviceToDevice, st));
  if (ng > 0) {
    if (cell_dev) IBM_TRY(cudaMemcpyAsync(cell_dev, t->gcell, 8 * ng, cudaMemcpyDeviceToDevice, st));
    if (bi_dev) IBM_TRY(cudaMemcpyAsync(bi_dev, t->gbi, 24 * ng, cudaMemcpyDeviceToDevice, st));
    if (ip_dev) IBM_TRY(cudaMemcpyAsync(ip_dev, t->gip, 24 * ng, cudaMemcpyDeviceToDevice, st));
    if (base_dev) IBM_TRY(cudaMemcpyAsync(base_dev, t->gbase, 12 * ng, cudaMemcpyDeviceToDevice, st));
    if (flags_dev) IBM_TRY(cudaMemcpyAsync(flags_dev, t->gflags, 4 * ng, cudaMemcpyDeviceToDevice, st));
    if (ref_dev) IBM_TRY(cudaMemcpyAsync(ref_dev, t->gref, 64 * ng, cudaMemcpyDeviceToDevice, st));
    if (w_dev) IBM_TRY(cudaMemcpyAsync(w_dev, t->gw, 64 * ng, cudaMemcpyDeviceToDevice, st));
    if (scale_dev) IBM_TRY(cudaMemcpyAsync(scale_dev, t->gscale, 8 * ng, cudaMemcpyDeviceToDevice, st));
  }
  IBM_TRY(cudaStreamSynchronize(st));
  return IBM_OK;
}

void ibm_solve_opts_default(ibm_solve_opts *o) {
  if (!o) return;
  o->precision = 0;
  o->nu1 = 2;
  o->nu2 = 2;
  o->max_cycles = 100;
  o->inner_cycles = 2;
  o->use_graph = 1;
  o->omega = 1.3;
  o->krylov = -1;
  o->method = 0;
  o->srj_steps = 8;
  o->coarse_bf16 = 0;
  o->sweep_chunk = 0;
  o->batch_schedule = 0;
}

ibm_status poisson_solve(ibm_ctx *ctx, const ibm_tables *t, const double *rhs_dev, double tol, double *p_dev,
                         const ibm_solve_opts *opts, ibm_solve_info *info, void *stream) {
  if (!ctx || !t || !rhs_dev || !p_dev || !(tol >= 0.0) || t->ctx != ctx) return IBM_ERR_INVALID_ARG;
  ibm_solve_opts o;
  ibm_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.precision >= 0 && o.precision <= 2) || o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1 || o.max_cycles < 0 ||
      o.inner_cycles < 1 || !(o.omega > 0.0 && o.omega < 2.0) || o.krylov < -1 || o.krylov > 8 || o.method < 0 ||
      o.method > 1 || o.srj_steps < 1 || o.srj_steps > 64 || (o.method == 1 && o.precision != 0) ||
      o.coarse_bf16 < 0 || o.coarse_bf16 > 1 || (o.coarse_bf16 && (o.precision == 0 || t->membrane)) ||
      o.sweep_chunk < 0 || o.sweep_chunk > 256 || o.batch_schedule < 0 || o.batch_schedule > 1)
    return IBM_ERR_INVALID_ARG;
  if (info && info->history_cap > 0 && !info->resid_history) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  auto t0 = std::chrono::steady_clock::now();
  ibm_status s = ibm::solve_impl(ctx, const_cast<ibm_tables *>(t), rhs_dev, tol, p_dev, &o, info, (cudaStream_t)stream);
  if (info) info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

ibm_status ibm_smoother_sweeps(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, int32_t nsweeps, void *stream) {
  if (!ctx || !t || t->ctx != ctx || precision < 0 || precision > 2 || nsweeps < 0) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  return ibm::sweeps_impl(ctx, const_cast<ibm_tables *>(t), precision, nsweeps, (cudaStream_t)stream, nullptr);
}

ibm_status ibm_smoother_sweeps_timed(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, int32_t nsweeps,
                                     void *stream, double *kernel_ms) {
  if (!ctx || !t || t->ctx != ctx || precision < 0 || precision > 2 || nsweeps < 1 || !kernel_ms)
    return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  return ibm::sweeps_impl(ctx, const_cast<ibm_tables *>(t), precision, nsweeps, (cudaStream_t)stream, kernel_ms);
}

ibm_status ibm_smoother_apply(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, int32_t nsweeps, double omega,
                              const double *e_dev, const double *r_dev, double mu, double *e_out_dev, void *stream) {
  if (!ctx || !t || t->ctx != ctx || precision < 0 || precision > 2 || nsweeps < 0 || !(omega > 0.0 && omega < 2.0) ||
      !e_dev || !r_dev || !e_out_dev || !std::isfinite(mu))
    return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  return ibm::smoother_apply_impl(ctx, const_cast<ibm_tables *>(t), precision, nsweeps, omega, e_dev, r_dev, mu,
                                  e_out_dev, (cudaStream_t)stream);
}

ibm_status ibm_measure_fp64_rate(ibm_ctx *ctx, double *dfma_per_s, void *stream) {
  if (!ctx || !dfma_per_s) return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  return ibm::measure_fp64_impl(ctx, dfma_per_s, (cudaStream_t)stream);
}

static bool valid_opts(const ibm_solve_opts &o) {
  return o.precision >= 0 && o.precision <= 2 && o.nu1 >= 0 && o.nu2 >= 0 && o.nu1 + o.nu2 >= 1 &&
         o.max_cycles >= 0 && o.inner_cycles >= 1 && o.omega > 0.0 && o.omega < 2.0 && o.krylov >= -1 &&
         o.krylov <= 8 && o.method == 0 &&   // batched: the multigrid solver
         (o.coarse_bf16 == 0 || (o.coarse_bf16 == 1 && o.precision != 0)) && o.sweep_chunk >= 0 &&
         o.sweep_chunk <= 256 && o.batch_schedule >= 0 && o.batch_schedule <= 1;
}

ibm_status poisson_solve_batched(ibm_ctx *ctx, int32_t n, const ibm_tables *const *tables,
                                 const double *const *rhs_dev, double tol, double *const *p_dev,
                                 const ibm_solve_opts *opts, ibm_solve_info *infos, void *stream) {
  if (!ctx || n < 0 || (n > 0 && (!tables || !rhs_dev || !p_dev)) || !(tol >= 0.0)) return IBM_ERR_INVALID_ARG;
  for (int p = 0; p < n; ++p) {
    if (!tables[p] || tables[p]->ctx != ctx || !rhs_dev[p] || !p_dev[p]) return IBM_ERR_INVALID_ARG;
    if (opts && opts->coarse_bf16 && tables[p]->membrane) return IBM_ERR_INVALID_ARG;
    for (int q = 0; q < p; ++q)
      if (tables[q] == tables[p]) return IBM_ERR_INVALID_ARG;   // each problem owns its work arrays
    if (infos && infos[p].history_cap > 0 && !infos[p].resid_history) return IBM_ERR_INVALID_ARG;
  }
  ibm_solve_opts o;
  ibm_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!valid_opts(o)) return IBM_ERR_INVALID_ARG;
  if (n == 0) return IBM_OK;
  IBM_TRY(cudaSetDevice(ctx->device));
  if (infos)
    for (int p = 0; p < n; ++p) { infos[p].cycles = 0; infos[p].history_len = 0; }
  auto t0 = std::chrono::steady_clock::now();
  ibm_status s = ibm::solve_batched_impl(ctx, n, const_cast<ibm_tables *const *>(tables), rhs_dev, tol, p_dev, &o,
                                         infos, (cudaStream_t)stream);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int p = 0; p < n; ++p) infos[p].ms_total = ms;
  return s;
}

ibm_status ibm_autotune(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, const double *rhs_dev,
                        double *p_work_dev, double tol, ibm_solve_opts *best, double *best_ms, void *stream) {
  if (!ctx || !t || t->ctx != ctx || !rhs_dev || !p_work_dev || !best || precision < 0 || precision > 2 ||
      !(tol > 0.0))
    return IBM_ERR_INVALID_ARG;
  IBM_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::string key;
  if (!ctx->tune_cache.empty()) {
    key = ibm::tune_key(t, precision);
    for (const ibm::TuneEntry &e : ibm::tune_read(ctx->tune_cache))
      if (e.key == key) {
        ibm_solve_opts_default(best);
        best->precision = precision;
        best->omega = e.omega; best->nu1 = e.nu1; best->nu2 = e.nu2; best->inner_cycles = e.inner;
        best->krylov = e.krylov;
        best->sweep_chunk = e.chunk;
        if (best_ms) *best_ms = e.ms;
        return IBM_OK;
      }
  }
  const double omegas[3] = {1.2, 1.3, 1.4};
  const int nus[3][2] = {{1, 1}, {2, 1}, {2, 2}};
  const int inners_mixed[3] = {1, 2, 3}, inner_fp64[1] = {1};
  const int *inners = precision != 0 ? inners_mixed : inner_fp64;
  const int ninner = precision != 0 ? 3 : 1;
  // Krylov acceleration: none, GCR(2), and the automatic choice when it differs (GCR(8) on
  // membrane tables)
  int krylovs[3] = {0, 2, 0}, nkry = 2;
  if (t->membrane) krylovs[nkry++] = 8;
  const size_t bytes = sizeof(double) * (size_t)t->ncell;
  cudaEvent_t e0, e1;
  IBM_TRY(cudaEventCreate(&e0));
  IBM_TRY(cudaEventCreate(&e1));
  double best_t = 1e300;
  ibm_solve_opts cand;
  ibm_solve_opts_default(&cand);
  cand.precision = precision;
  ibm_status last = IBM_OK;
  for (double om : omegas)
    for (auto &nu : nus)
      for (int q = 0; q < ninner; ++q)
        for (int kq = 0; kq < nkry; ++kq) {
          cand.omega = om; cand.nu1 = nu[0]; cand.nu2 = nu[1]; cand.inner_cycles = inners[q];
          cand.krylov = krylovs[kq];
          float ms_best = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {      // first run builds graphs; keep the faster
            cudaMemsetAsync(p_work_dev, 0, bytes, st);
            cudaEventRecord(e0, st);
            ibm_solve_info info{};
            ibm_status s = ibm::solve_impl(ctx, const_cast<ibm_tables *>(t), rhs_dev, tol, p_work_dev, &cand, &info, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            if (s != IBM_OK) { last = s; ms_best = 1e30f; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_best = std::min(ms_best, ms);
          }
          if (ms_best < best_t) { best_t = ms_best; *best = cand; }
        }
  // the tiles' z extent for the best schedule: the cost model's chunking, then fixed chunks
  if (best_t < 1e29) {
    const int chunks[3] = {128, 64, 32};
    cand = *best;
    for (int c : chunks) {
      cand.sweep_chunk = c;
      float ms_best = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaMemsetAsync(p_work_dev, 0, bytes, st);
        cudaEventRecord(e0, st);
        ibm_solve_info info{};
        ibm_status s = ibm::solve_impl(ctx, const_cast<ibm_tables *>(t), rhs_dev, tol, p_work_dev, &cand, &info, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        if (s != IBM_OK) { ms_best = 1e30f; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_best = std::min(ms_best, ms);
      }
      if (ms_best < best_t) { best_t = ms_best; *best = cand; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_t >= 1e29) return last != IBM_OK ? last : IBM_ERR_NOT_CONVERGED;
  if (best_ms) *best_ms = best_t;
  if (!key.empty()) {
    std::vector<ibm::TuneEntry> es = ibm::tune_read(ctx->tune_cache);
    ibm::TuneEntry e;
    e.key = key; e.omega = best->omega; e.nu1 = best->nu1; e.nu2 = best->nu2; e.inner = best->inner_cycles;
    e.krylov = best->krylov; e.chunk = best->sweep_chunk; e.ms = best_t;
    es.push_back(e);
    if (!ibm::tune_write(ctx->tune_cache, es)) return IBM_ERR_INVALID_ARG;
  }
  return IBM_OK;
}

ibm_status ibm_ctx_set_sweep_wait_limit(ibm_ctx *ctx, int32_t tries) {
  if (!ctx) return IBM_ERR_INVALID_ARG;
  ctx->sweep_first_wait = tries < 0 ? -1 : tries;
  return IBM_OK;
}

ibm_status ibm_ctx_launch_count(const ibm_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return IBM_ERR_INVALID_ARG;
  *count = ctx->launches;
  return IBM_OK;
}

}  // extern "C"
