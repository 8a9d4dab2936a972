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
#include <cmath>
#include <mutex>

#include "ibm_internal.cuh"

namespace {

// Limits of the static scratch: cells per axis and reduction blocks.
constexpr int NA_MAX_AXIS = 2048;
constexpr int NA_BLOCKS = 304;
constexpr int NA_THREADS = 256;
constexpr int NA_NPART = 9;                        // partial sums per block
// layout (doubles): block partials | results (4) | per axis: faces, widths, c-, c+
constexpr size_t NA_OFF_RES = (size_t)NA_BLOCKS * NA_NPART;
constexpr size_t NA_OFF_AXIS = NA_OFF_RES + 8;
constexpr size_t NA_AXIS_STRIDE = 4 * (size_t)(NA_MAX_AXIS + 1);
constexpr size_t NA_TOTAL = NA_OFF_AXIS + 3 * NA_AXIS_STRIDE;   // ~ 0.2 MB

static __device__ __align__(256) double g_na_scratch[NA_TOTAL];

// per-device address of g_na_scratch, looked up once per device with that device current
constexpr int NA_MAX_DEVICES = 64;
static double *g_na_ptr[NA_MAX_DEVICES] = {nullptr};
static std::mutex g_na_mutex;

cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = (double *)p;
  }
  *out = g_na_ptr[dev];
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

// per block: sum V r, sum r, sum r^2, sum V b, sum b, sum b^2, sum V, N_F, sum (s r_G)^2
__global__ void k_na_partials(double *scr, int nx, int ny, int nz, const uint8_t *ib, const double *b,
                              const double *p, long long ng, const long long *gcell, const long long *gref,
                              const double *gw, const double *gscale) {
  __shared__ double sm[NA_NPART][NA_THREADS];
  const double *ax = scr + NA_OFF_AXIS, *ay = ax + NA_AXIS_STRIDE, *az = ay + NA_AXIS_STRIDE;
  const int S1 = NA_MAX_AXIS + 1;
  double acc[NA_NPART] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const long long ncell = (long long)nx * ny * nz, sy = nx, sz = (long long)nx * ny;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < ncell; l += (long long)gridDim.x * blockDim.x) {
    if (ib[l] != 0) continue;
    const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / sz);
    const double pc = p[l];
    double s = 0.0;
    if (i > 0) s += ax[2 * S1 + i] * (p[l - 1] - pc);
    if (i < nx - 1) s += ax[3 * S1 + i] * (p[l + 1] - pc);
    if (j > 0) s += ay[2 * S1 + j] * (p[l - sy] - pc);
    if (j < ny - 1) s += ay[3 * S1 + j] * (p[l + sy] - pc);
    if (k > 0) s += az[2 * S1 + k] * (p[l - sz] - pc);
    if (k < nz - 1) s += az[3 * S1 + k] * (p[l + sz] - pc);
    const double V = ax[S1 + i] * ay[S1 + j] * az[S1 + k];
    const double r = b[l] - s, bl = b[l];
    acc[0] += V * r; acc[1] += r; acc[2] += r * r;
    acc[3] += V * bl; acc[4] += bl; acc[5] += bl * bl;
    acc[6] += V; acc[7] += 1.0;
  }
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      const long long q = gref[8 * g + c];
      if (q >= 0) s += gw[8 * g + c] * p[q];
    }
    const double rg = gscale[g] * (s - p[gcell[g]]);
    acc[8] += rg * rg;
  }
  for (int q = 0; q < NA_NPART; ++q) sm[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int st = NA_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < NA_NPART; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + st];
    __syncthreads();
  }
  // every block writes all of its partials, so no value of an earlier call survives
  if (threadIdx.x == 0)
    for (int q = 0; q < NA_NPART; ++q) scr[blockIdx.x * NA_NPART + q] = sm[q][0];
}

// fixed-order sum of the partials; results: relative residual, ||S P r||, ||S P b||
__global__ void k_na_finalize(double *scr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t[NA_NPART] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int blk = 0; blk < NA_BLOCKS; ++blk)
    for (int q = 0; q < NA_NPART; ++q) t[q] += scr[blk * NA_NPART + q];
  const double vf = t[6], nf = t[7];
  const double mr = t[0] / vf, mb = t[3] / vf;
  double nr = t[2] - 2.0 * mr * t[1] + nf * mr * mr;
  double nb = t[5] - 2.0 * mb * t[4] + nf * mb * mb;
  nr = (nr > 0.0 ? nr : 0.0) + t[8];
  nb = nb > 0.0 ? nb : 0.0;
  double *res = scr + NA_OFF_RES;
  res[1] = sqrt(nr);
  res[2] = sqrt(nb);
  res[0] = res[2] > 0.0 ? res[1] / res[2] : 0.0;
}

}  // namespace

extern "C" ibm_status ibm_residual_norm_noalloc(const ibm_grid *grid, const uint8_t *iblank_dev, int64_t nghost,
                                                const int64_t *ghost_cell_dev, const int64_t *ghost_ref_dev,
                                                const double *ghost_w_dev, const double *ghost_scale_dev,
                                                const double *rhs_dev, const double *p_dev, double *result,
                                                void *stream) {
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
  for (int a = 0; a < 3; ++a) {
    double *ax = scr + NA_OFF_AXIS + a * NA_AXIS_STRIDE;
    IBM_TRY(cudaMemcpyAsync(ax, f[a], sizeof(double) * (n[a] + 1), cudaMemcpyHostToDevice, st));
    k_na_axis<<<(n[a] + 127) / 128, 128, 0, st>>>(ax, n[a]);
  }
  k_na_partials<<<NA_BLOCKS, NA_THREADS, 0, st>>>(scr, n[0], n[1], n[2], iblank_dev, rhs_dev, p_dev, nghost,
                                                  (const long long *)ghost_cell_dev, (const long long *)ghost_ref_dev,
                                                  ghost_w_dev, ghost_scale_dev);
  k_na_finalize<<<1, 32, 0, st>>>(scr);
  IBM_TRY(cudaGetLastError());
  IBM_TRY(cudaMemcpyAsync(result, scr + NA_OFF_RES, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  return IBM_OK;
}
