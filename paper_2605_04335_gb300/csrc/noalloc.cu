// ibm_residual_norm_noalloc: relative projected residual of a pressure field, computed
// without allocating any device memory (declared in include/ibm_poisson.h).
//
// Who needs this: a flow solver that hands the library a fixed device arena up front and
// forbids further cudaMalloc (cudaMalloc / cudaFree synchronise the whole device, which
// breaks a pipeline that overlaps the pressure solve with halo exchange, and an allocation
// that fails mid-run cannot be recovered inside a time-step loop), or a caller that is
// checking a result from code paths where allocating is not allowed.  Everything it needs
// beyond the caller's own inputs and outputs lives in one file-scope device array of fixed
// size, shared by every call on a device.
//
// The projected norms are formed in two passes over the grid: the first reduces the
// volume-weighted fluid sums of r and b (their fluid means), the second the squared
// deviations from those means.  A one-pass form (sum r^2 - 2 mu sum r + N mu^2) cancels
// catastrophically when r or b carries a large fluid mean, which the solver accepts (the
// compatibility constant absorbs it).
#include <cmath>
#include <mutex>

#include <cudaTypedefs.h>

#include "ibm_internal.cuh"

namespace {

// Limits of the static scratch: cells per axis and reduction blocks.
constexpr int NA_MAX_AXIS = 2048;
constexpr int NA_BLOCKS = 304;
constexpr int NA_THREADS = 256;
constexpr int NA_NP1 = 5;                          // first pass: sum V r, sum V b, V_F, N_F, sum (s r_G)^2
constexpr int NA_NP2 = 2;                          // second pass: sum (r - mu_r)^2, sum (b - mu_b)^2
// layout (doubles): pass-1 partials | pass-2 partials | results (8) | error word | per axis:
// faces, widths, c-, c+
constexpr size_t NA_OFF_P2 = (size_t)NA_BLOCKS * NA_NP1;
constexpr size_t NA_OFF_RES = NA_OFF_P2 + (size_t)NA_BLOCKS * NA_NP2;
constexpr size_t NA_OFF_ERR = NA_OFF_RES + 8;
constexpr size_t NA_OFF_AXIS = NA_OFF_ERR + 8;
constexpr size_t NA_AXIS_STRIDE = 4 * (size_t)(NA_MAX_AXIS + 1);
constexpr size_t NA_TOTAL = NA_OFF_AXIS + 3 * NA_AXIS_STRIDE;   // ~ 0.2 MB
// result slots: 0 relative residual, 1 ||S P r||, 2 ||S P b||, 3 mu_r, 4 mu_b

static __device__ __align__(256) double g_na_scratch[NA_TOTAL];

// Per-device address of g_na_scratch, looked up with that device current the first time a
// call runs in a (device, CUDA context) pair.  A new context on the device (after
// cudaDeviceReset) looks it up again, so a stale address is never passed to a kernel.
constexpr int NA_MAX_DEVICES = 64;
struct NaSlot {
  CUcontext ctx = nullptr;
  double *ptr = nullptr;
};
static NaSlot g_na_slot[NA_MAX_DEVICES];
static std::mutex g_na_mutex;

PFN_cuCtxGetCurrent_v4000 ctx_get_current() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&fn, 4000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
  }
  return fn;
}

cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  e = cudaSetDevice(dev);   // initialises the device's primary context and makes it current
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  CUcontext cur = nullptr;
  auto get = ctx_get_current();
  if (!get || get(&cur) != CUDA_SUCCESS) return cudaErrorInitializationError;
  NaSlot &s = g_na_slot[dev];
  if (!s.ptr || s.ctx != cur) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    s.ptr = (double *)p;
    s.ctx = cur;
  }
  *out = s.ptr;
  return cudaSuccess;
}

// widths and the 7-point coefficients of one axis from its faces (already in scratch)
__global__ void k_na_axis(double *ax, int n) {
  const double *f = ax;
  double *w = ax + (NA_MAX_AXIS + 1), *cm = w + (NA_MAX_AXIS + 1), *cp = cm + (NA_MAX_AXIS + 1);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ci = 0.5 * (f[i] + f[i + 1]), wi = f[i + 1] - f[i];
  w[i] = wi;
  cm[i] = i > 0 ? 1.0 / (wi * (ci - 0.5 * (f[i - 1] + f[i]))) : 0.0;
  cp[i] = i < n - 1 ? 1.0 / (wi * (0.5 * (f[i + 1] + f[i + 2]) - ci)) : 0.0;
}

struct NaArgs {
  int nx, ny, nz;
  const uint8_t *ib;
  const double *b, *p;
  long long ng;
  const long long *gcell, *gref;
  const double *gw, *gscale, *gd;
};

// (A p)_l on fluid cell l at (i, j, k): sum_d c_d (p_nb - p_l), zero flux across the walls
__device__ __forceinline__ double na_apply(const double *scr, const NaArgs &a, long long l, int i, int j, int k) {
  const double *ax = scr + NA_OFF_AXIS, *ay = ax + NA_AXIS_STRIDE, *az = ay + NA_AXIS_STRIDE;
  const int S1 = NA_MAX_AXIS + 1;
  const long long sy = a.nx, sz = (long long)a.nx * a.ny;
  const double pc = a.p[l];
  double s = 0.0;
  if (i > 0) s += ax[2 * S1 + i] * (a.p[l - 1] - pc);
  if (i < a.nx - 1) s += ax[3 * S1 + i] * (a.p[l + 1] - pc);
  if (j > 0) s += ay[2 * S1 + j] * (a.p[l - sy] - pc);
  if (j < a.ny - 1) s += ay[3 * S1 + j] * (a.p[l + sy] - pc);
  if (k > 0) s += az[2 * S1 + k] * (a.p[l - sz] - pc);
  if (k < a.nz - 1) s += az[3 * S1 + k] * (a.p[l + sz] - pc);
  return s;
}

__device__ __forceinline__ double na_volume(const double *scr, int i, int j, int k) {
  const double *ax = scr + NA_OFF_AXIS, *ay = ax + NA_AXIS_STRIDE, *az = ay + NA_AXIS_STRIDE;
  const int S1 = NA_MAX_AXIS + 1;
  return ax[S1 + i] * ay[S1 + j] * az[S1 + k];
}

template <int NP>
__device__ __forceinline__ void na_block_store(double (&acc)[NP], double *dst) {
  __shared__ double sm[NP][NA_THREADS];
  for (int q = 0; q < NP; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int st = NA_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < NP; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + st];
    __syncthreads();
  }
  // every block writes all of its partials, so no value of an earlier call survives
  if (threadIdx.x == 0)
    for (int q = 0; q < NP; ++q) dst[blockIdx.x * NP + q] = sm[q][0];
}

// First pass.  Fluid rows: sum V r, sum V b, sum V, N_F.  Ghost rows (closed bodies):
// r_G = d_G - (g_G - sum_k w_k v_k), scaled by s_G, squared and summed.  A row whose cell is
// not a ghost cell of a closed body (iblank 3), or whose indices leave the grid (membrane
// entries live at ncell + e), sets the error word and is skipped without reading p there.
__global__ void k_na_pass1(double *scr, NaArgs a) {
  double acc[NA_NP1] = {0, 0, 0, 0, 0};
  const long long ncell = (long long)a.nx * a.ny * a.nz, sz = (long long)a.nx * a.ny;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, ts = (long long)gridDim.x * blockDim.x;
  for (long long l = t0; l < ncell; l += ts) {
    if (a.ib[l] != 0) continue;
    const int i = (int)(l % a.nx), j = (int)((l / a.nx) % a.ny), k = (int)(l / sz);
    const double V = na_volume(scr, i, j, k);
    const double r = a.b[l] - na_apply(scr, a, l, i, j, k);
    acc[0] += V * r;
    acc[1] += V * a.b[l];
    acc[2] += V;
    acc[3] += 1.0;
  }
  bool bad = false;
  for (long long g = t0; g < a.ng; g += ts) {
    const long long gc = a.gcell[g];
    if (gc < 0 || gc >= ncell || a.ib[gc] != 3) { bad = true; continue; }
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      const long long q = a.gref[8 * g + c];
      if (q < 0) continue;
      if (q >= ncell) { bad = true; continue; }
      s += a.gw[8 * g + c] * a.p[q];
    }
    double rg = s - a.p[gc];
    if (a.gd) rg += a.gd[g];
    rg *= a.gscale[g];
    acc[4] += rg * rg;
  }
  if (bad) scr[NA_OFF_ERR] = 1.0;
  na_block_store<NA_NP1>(acc, scr);
}

// fixed-order sums of the first pass: the fluid means of r and b
__global__ void k_na_means(double *scr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[NA_NP1] = {0, 0, 0, 0, 0};
  for (int blk = 0; blk < NA_BLOCKS; ++blk)
    for (int q = 0; q < NA_NP1; ++q) t[q] += scr[blk * NA_NP1 + q];
  double *res = scr + NA_OFF_RES;
  res[3] = t[2] > 0.0 ? t[0] / t[2] : 0.0;
  res[4] = t[2] > 0.0 ? t[1] / t[2] : 0.0;
  res[5] = t[4];
}

// Second pass: sum over fluid rows of (r - mu_r)^2 and (b - mu_b)^2
__global__ void k_na_pass2(double *scr, NaArgs a) {
  double acc[NA_NP2] = {0, 0};
  const double mr = scr[NA_OFF_RES + 3], mb = scr[NA_OFF_RES + 4];
  const long long ncell = (long long)a.nx * a.ny * a.nz, sz = (long long)a.nx * a.ny;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < ncell;
       l += (long long)gridDim.x * blockDim.x) {
    if (a.ib[l] != 0) continue;
    const int i = (int)(l % a.nx), j = (int)((l / a.nx) % a.ny), k = (int)(l / sz);
    const double dr = (a.b[l] - na_apply(scr, a, l, i, j, k)) - mr, db = a.b[l] - mb;
    acc[0] += dr * dr;
    acc[1] += db * db;
  }
  na_block_store<NA_NP2>(acc, scr + NA_OFF_P2);
}

// results: relative residual, ||S P r||, ||S P b||
__global__ void k_na_finalize(double *scr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[NA_NP2] = {0, 0};
  for (int blk = 0; blk < NA_BLOCKS; ++blk)
    for (int q = 0; q < NA_NP2; ++q) t[q] += scr[NA_OFF_P2 + blk * NA_NP2 + q];
  double *res = scr + NA_OFF_RES;
  res[1] = sqrt(t[0] + res[5]);
  res[2] = sqrt(t[1]);
  res[0] = res[2] > 0.0 ? res[1] / res[2] : 0.0;
}

}  // namespace

extern "C" ibm_status ibm_residual_norm_noalloc(const ibm_grid *grid, const uint8_t *iblank_dev, int64_t nghost,
                                                const int64_t *ghost_cell_dev, const int64_t *ghost_ref_dev,
                                                const double *ghost_w_dev, const double *ghost_scale_dev,
                                                const double *ghost_d_dev, const double *rhs_dev,
                                                const double *p_dev, double *result, void *stream) {
  if (!grid || !iblank_dev || !rhs_dev || !p_dev || !result || nghost < 0 ||
      (nghost > 0 && (!ghost_cell_dev || !ghost_ref_dev || !ghost_w_dev || !ghost_scale_dev)))
    return IBM_ERR_INVALID_ARG;
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  const double *f[3] = {grid->xf, grid->yf, grid->zf};
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 2 || !f[a]) return IBM_ERR_INVALID_ARG;
    if (n[a] > NA_MAX_AXIS) return IBM_ERR_CAPACITY;   // the static scratch holds 2048 cells per axis
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *scr = nullptr;
  IBM_TRY(scratch_for_current_device(&scr));
  IBM_TRY(cudaMemsetAsync(scr + NA_OFF_ERR, 0, sizeof(double), st));   // the error word starts clear
  for (int a = 0; a < 3; ++a) {
    double *ax = scr + NA_OFF_AXIS + a * NA_AXIS_STRIDE;
    IBM_TRY(cudaMemcpyAsync(ax, f[a], sizeof(double) * (n[a] + 1), cudaMemcpyHostToDevice, st));
    k_na_axis<<<(n[a] + 127) / 128, 128, 0, st>>>(ax, n[a]);
  }
  NaArgs a;
  a.nx = n[0]; a.ny = n[1]; a.nz = n[2];
  a.ib = iblank_dev; a.b = rhs_dev; a.p = p_dev;
  a.ng = nghost;
  a.gcell = (const long long *)ghost_cell_dev; a.gref = (const long long *)ghost_ref_dev;
  a.gw = ghost_w_dev; a.gscale = ghost_scale_dev; a.gd = ghost_d_dev;
  k_na_pass1<<<NA_BLOCKS, NA_THREADS, 0, st>>>(scr, a);
  k_na_means<<<1, 32, 0, st>>>(scr);
  k_na_pass2<<<NA_BLOCKS, NA_THREADS, 0, st>>>(scr, a);
  k_na_finalize<<<1, 32, 0, st>>>(scr);
  IBM_TRY(cudaGetLastError());
  double out[NA_OFF_AXIS - NA_OFF_RES];
  IBM_TRY(cudaMemcpyAsync(out, scr + NA_OFF_RES, sizeof(out), cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  if (out[NA_OFF_ERR - NA_OFF_RES] != 0.0) return IBM_ERR_INVALID_ARG;
  result[0] = out[0]; result[1] = out[1]; result[2] = out[2];
  return IBM_OK;
}
