// Geometric multigrid for the ghost-cell pressure Poisson system.
//
// Paper (arxiv 2605.04335) Sec. "Governing Equations and Numerical Methods": the pressure
// Poisson equation of the fractional-step method, second-order finite differences on a
// Cartesian grid.  The paper's own solver is BiCGStab with scheduled relaxed Jacobi; this
// library reaches the same discrete solution with V-cycles:
//
//  * smoother: red-black Gauss-Seidel on fluid rows (colour (i+j+k) mod 2), followed on the
//    finest level by a Jacobi update of every ghost row g_G = sum_k w_k v_k (+ rhs);
//  * coarse levels: n_c = ceil(n/2) per axis, coarse cell fluid iff any child is fluid,
//    coefficients rediscretised on the coarse faces and scaled by the area fraction of
//    open fine faces (both neighbours fluid); no ghost rows (staircase Neumann);
//  * restriction: volume-weighted sum of fluid children's residuals / coarse volume,
//    followed by removal of the coarse level's volume-weighted fluid mean;
//  * prolongation: trilinear in physical coordinates over fluid coarse cells, renormalised;
//  * coarsest level (<= 128 cells): exact bordered solve [A 1; V' 0] by a precomputed inverse.
//
// Element type T is float or double; the fine-level residual, the refinement update and
// the gauge are FP64, or pairs of floats in the double-FP32 outer loop (precision mode 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cudaTypedefs.h>

#include "ibm_internal.cuh"
#include "dfloat.cuh"
#include "zmarch.cuh"

namespace ibm {

constexpr int MAX_COARSE = 128;

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr long long GHOST_CORNER = 1LL << 62;   // flag on a ghost-row source that is itself a ghost

template <typename T>
struct LV {          // kernel-side view of one level
  int nx, ny, nz, px;
  long long sy, sz;
  const uint8_t *mask;
  const T *cxm, *cxp, *cym, *cyp, *czm, *czp;
  const T *fx, *fy, *fz;     // nullptr on the finest level
  const double *dx, *dy, *dz;
  const T *wx, *wy, *wz;     // widths in T
  const T *sdx, *sdy, *sdz;  // finest level: separable diagonal parts (else nullptr)
};

template <typename T>
LV<T> view(const Level &L) {
  LV<T> v;
  v.nx = L.g.nx; v.ny = L.g.ny; v.nz = L.g.nz; v.px = L.g.px; v.sy = L.g.sy; v.sz = L.g.sz;
  v.mask = L.mask;
  const T *c = (const T *)L.c1d;
  v.cxm = c; v.cxp = c + L.g.nx; v.cym = c + 2 * L.g.nx; v.cyp = v.cym + L.g.ny;
  v.czm = v.cyp + L.g.ny; v.czp = v.czm + L.g.nz;
  v.fx = (const T *)L.fx; v.fy = (const T *)L.fy; v.fz = (const T *)L.fz;
  v.dx = L.w1d; v.dy = L.w1d + L.g.nx; v.dz = L.w1d + L.g.nx + L.g.ny;
  const T *w = (const T *)L.wT;
  v.wx = w; v.wy = w ? w + L.g.nx : nullptr; v.wz = w ? w + L.g.nx + L.g.ny : nullptr;
  const T *d = (const T *)L.sdiag;
  v.sdx = d; v.sdy = d ? d + L.g.nx : nullptr; v.sdz = d ? d + L.g.nx + L.g.ny : nullptr;
  return v;
}

template <typename T>
__device__ __forceinline__ long long vidx(const LV<T> &v, int i, int j, int k) {
  return ((long long)(k + 1) * (v.ny + 2) + (j + 1)) * v.px + (i + OX);
}

// six face coefficients of cell (i,j,k) at padded index id
template <typename T>
__device__ __forceinline__ void coefs(const LV<T> &v, int i, int j, int k, long long id, T c[6]) {
  c[0] = v.cxm[i]; c[1] = v.cxp[i]; c[2] = v.cym[j]; c[3] = v.cyp[j]; c[4] = v.czm[k]; c[5] = v.czp[k];
  if (v.fx) {
    c[0] *= v.fx[id - 1]; c[1] *= v.fx[id];
    c[2] *= v.fy[id - v.sy]; c[3] *= v.fy[id];
    c[4] *= v.fz[id - v.sz]; c[5] *= v.fz[id];
  }
}

template <typename T>
__device__ __forceinline__ T stencil_sum(const LV<T> &v, const T *e, long long id, const T c[6]) {
  return c[0] * e[id - 1] + c[1] * e[id + 1] + c[2] * e[id - v.sy] + c[3] * e[id + v.sy] +
         c[4] * e[id - v.sz] + c[5] * e[id + v.sz];
}

// ------------------------------------------------------------------ hierarchy setup kernels

template <typename T>
__global__ void k_axis_level(const double *f, int n, T *cm, T *cp, double *w, double *c, T *wt = nullptr,
                             T *sd = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ci = 0.5 * (f[i] + f[i + 1]), wi = f[i + 1] - f[i];
  double m = 0.0, p = 0.0;
  if (i > 0) m = 1.0 / (wi * (ci - 0.5 * (f[i - 1] + f[i])));
  if (i < n - 1) p = 1.0 / (wi * (0.5 * (f[i + 1] + f[i + 2]) - ci));
  cm[i] = (T)m; cp[i] = (T)p; w[i] = wi; c[i] = ci;
  if (wt) wt[i] = (T)wi;
  if (sd) sd[i] = (T)m + (T)p;
}

// prolongation weights from coarse (cc, nc) to fine (cf, nf) along one axis
__global__ void k_prolong_axis(const double *cf, int nf, const double *cc, int nc, int8_t *off, float *t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  int I = i >> 1;
  double xf = cf[i], X = cc[I];
  int nb = xf < X ? I - 1 : (xf > X ? I + 1 : I);
  if (nb < 0 || nb >= nc || nb == I) { off[i] = 0; t[i] = 0.0f; return; }
  off[i] = (int8_t)(nb - I);
  t[i] = (float)((xf - X) / (cc[nb] - X));
}

__global__ void k_mask0(const uint8_t *ib, int nx, int ny, int nz, uint8_t *mask, LevelGeom g) {
  long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)nx * ny * nz) return;
  int i = (int)(l % nx); long long r = l / nx; int j = (int)(r % ny); int k = (int)(r / ny);
  mask[pidx(g, i, j, k)] = ib[l];
}

__global__ void k_mask_coarse(const uint8_t *mf, LevelGeom gf, uint8_t *mc, LevelGeom gc) {
  long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)gc.nx * gc.ny * gc.nz) return;
  int I = (int)(l % gc.nx); long long r = l / gc.nx; int J = (int)(r % gc.ny); int K = (int)(r / gc.ny);
  uint8_t m = 1;
  for (int c = 0; c < 8; ++c) {
    int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
    if (i < gf.nx && j < gf.ny && k < gf.nz && mf[pidx(gf, i, j, k)] == 0) m = 0;
  }
  mc[pidx(gc, I, J, K)] = m;
}

// area fraction of open fine faces on each +x/+y/+z coarse face.
// Fine open fraction: level 0 from the mask (both sides fluid), else the fine fraction.
template <typename T>
__global__ void k_fractions(const uint8_t *mf, const T *ffx, const T *ffy, const T *ffz, LevelGeom gf,
                            const double *dxf, const double *dyf, const double *dzf, LevelGeom gc,
                            const double *dxc, const double *dyc, const double *dzc, T *fx, T *fy, T *fz) {
  long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)gc.nx * gc.ny * gc.nz) return;
  int I = (int)(l % gc.nx); long long r = l / gc.nx; int J = (int)(r % gc.ny); int K = (int)(r / gc.ny);
  long long ic = pidx(gc, I, J, K);
  auto open_f = [&](int i, int j, int k, int axis) -> double {
    long long id = pidx(gf, i, j, k);
    if (ffx == nullptr) {
      long long s = axis == 0 ? 1 : (axis == 1 ? gf.sy : gf.sz);
      return (mf[id] == 0 && mf[id + s] == 0) ? 1.0 : 0.0;
    }
    const T *f = axis == 0 ? ffx : (axis == 1 ? ffy : ffz);
    return (double)f[id];
  };
  // +x face: fine face between 2I+1 and 2I+2
  double sx = 0.0, sy = 0.0, sz = 0.0;
  if (I + 1 < gc.nx && 2 * I + 2 < gf.nx) {
    for (int b = 0; b < 2; ++b) for (int a = 0; a < 2; ++a) {
      int j = 2 * J + a, k = 2 * K + b;
      if (j < gf.ny && k < gf.nz) sx += open_f(2 * I + 1, j, k, 0) * dyf[j] * dzf[k];
    }
    sx /= dyc[J] * dzc[K];
  }
  if (J + 1 < gc.ny && 2 * J + 2 < gf.ny) {
    for (int b = 0; b < 2; ++b) for (int a = 0; a < 2; ++a) {
      int i = 2 * I + a, k = 2 * K + b;
      if (i < gf.nx && k < gf.nz) sy += open_f(i, 2 * J + 1, k, 1) * dxf[i] * dzf[k];
    }
    sy /= dxc[I] * dzc[K];
  }
  if (K + 1 < gc.nz && 2 * K + 2 < gf.nz) {
    for (int b = 0; b < 2; ++b) for (int a = 0; a < 2; ++a) {
      int i = 2 * I + a, j = 2 * J + b;
      if (i < gf.nx && j < gf.ny) sz += open_f(i, j, 2 * K + 1, 2) * dxf[i] * dyf[j];
    }
    sz /= dxc[I] * dyc[J];
  }
  fx[ic] = (T)sx; fy[ic] = (T)sy; fz[ic] = (T)sz;
}

__global__ void k_fluid_stats(const uint8_t *mask, LevelGeom g, const double *dx, const double *dy,
                              const double *dz, double *out) {
  __shared__ double s[2][256];
  double v = 0.0, c = 0.0;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < (long long)g.nx * g.ny * g.nz;
       l += (long long)gridDim.x * blockDim.x) {
    int i = (int)(l % g.nx); long long r = l / g.nx; int j = (int)(r % g.ny); int k = (int)(r / g.ny);
    if (mask[pidx(g, i, j, k)] == 0) { v += dx[i] * dy[j] * dz[k]; c += 1.0; }
  }
  s[0][threadIdx.x] = v; s[1][threadIdx.x] = c;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) { s[0][threadIdx.x] += s[0][threadIdx.x + st]; s[1][threadIdx.x] += s[1][threadIdx.x + st]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[2 * blockIdx.x] = s[0][0]; out[2 * blockIdx.x + 1] = s[1][0]; }
}

// Coarsest level: gather fluid cells, assemble the bordered matrix [A 1; V'/vbar 0] and
// invert it by Gauss-Jordan with partial pivoting (one block, setup only).
template <typename T>
__global__ void k_coarsest_setup(LV<T> v, int *cidx, int *ncount, double *M, double *Minv, int cap) {
  __shared__ int n_s;
  __shared__ int piv_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    int n = 0;
    for (int k = 0; k < v.nz; ++k) for (int j = 0; j < v.ny; ++j) for (int i = 0; i < v.nx; ++i) {
      long long id = vidx(v, i, j, k);
      if (v.mask[id] == 0 && n < cap) cidx[n++] = (int)id;
    }
    n_s = n;
    *ncount = n;
  }
  __syncthreads();
  const int n = n_s, m = n + 1;
  for (int q = tid; q < m * m; q += nt) { M[q] = 0.0; Minv[q] = (q / m == q % m) ? 1.0 : 0.0; }
  __syncthreads();
  double vbar = 0.0;
  for (int q = 0; q < n; ++q) {
    long long id = cidx[q];
    int i = (int)(id % v.px) - OX; long long r = id / v.px; int j = (int)(r % (v.ny + 2)) - 1; int k = (int)(r / (v.ny + 2)) - 1;
    vbar += v.dx[i] * v.dy[j] * v.dz[k];
  }
  vbar /= (n > 0 ? n : 1);
  for (int q = tid; q < n; q += nt) {
    long long id = cidx[q];
    int i = (int)(id % v.px) - OX; long long r = id / v.px; int j = (int)(r % (v.ny + 2)) - 1; int k = (int)(r / (v.ny + 2)) - 1;
    T c[6];
    coefs(v, i, j, k, id, c);
    const long long nb[6] = {id - 1, id + 1, id - v.sy, id + v.sy, id - v.sz, id + v.sz};
    double diag = 0.0;
    for (int d = 0; d < 6; ++d) {
      if (c[d] == (T)0) continue;
      diag -= (double)c[d];
      for (int s2 = 0; s2 < n; ++s2)
        if (cidx[s2] == nb[d]) { M[q * m + s2] += (double)c[d]; break; }
    }
    M[q * m + q] += diag;
    M[q * m + n] = 1.0;
    M[n * m + q] = v.dx[i] * v.dy[j] * v.dz[k] / vbar;
  }
  __syncthreads();
  for (int col = 0; col < m; ++col) {
    if (tid == 0) {
      int p = col;
      double best = fabs(M[col * m + col]);
      for (int rr = col + 1; rr < m; ++rr)
        if (fabs(M[rr * m + col]) > best) { best = fabs(M[rr * m + col]); p = rr; }
      piv_s = p;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != col)
      for (int q = tid; q < m; q += nt) {
        double a = M[col * m + q]; M[col * m + q] = M[p * m + q]; M[p * m + q] = a;
        double b = Minv[col * m + q]; Minv[col * m + q] = Minv[p * m + q]; Minv[p * m + q] = b;
      }
    __syncthreads();
    const double inv = 1.0 / M[col * m + col];
    __syncthreads();
    for (int q = tid; q < m; q += nt) { M[col * m + q] *= inv; Minv[col * m + q] *= inv; }
    __syncthreads();
    for (int rr = tid; rr < m; rr += nt) {
      if (rr == col) continue;
      double f = M[rr * m + col];
      if (f == 0.0) continue;
      for (int q = 0; q < m; ++q) { M[rr * m + q] -= f * M[col * m + q]; Minv[rr * m + q] -= f * Minv[col * m + q]; }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ solve kernels

// one colour of red-black Gauss-Seidel on fluid rows: e_i += omega (sum - D e_i - rhs) / D
template <typename T>
__global__ void k_rbgs(LV<T> v, T *e, const T *r, const double *shift, int colour, T omega) {
  int ti = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y, k = blockIdx.z;
  int i = 2 * ti + ((j + k + colour) & 1);
  if (i >= v.nx) return;
  long long id = vidx(v, i, j, k);
  if (v.mask[id] != 0) return;
  T c[6];
  coefs(v, i, j, k, id, c);
  T D = v.sdx ? (v.sdx[i] + v.sdy[j]) + v.sdz[k] : ((c[0] + c[1]) + (c[2] + c[3])) + (c[4] + c[5]);
  if (D == (T)0) return;
  T rhs = r[id] - (shift ? (T)(*shift) : (T)0);
  T res = stencil_sum(v, e, id, c) - D * e[id] - rhs;
  // FP32 relaxation step: the fixed point (res = 0 in T) is unchanged, FP64 work stays minimal
  e[id] += (T)__fdividef((float)omega * (float)res, (float)D);
}

// ghost rows (Jacobi): gnew = sum_k w_k e[src_k] (+ rhs at the ghost cell)
template <typename T, typename W>
__global__ void k_ghost_eval(const long long *src, const long long *dst, const W *w, long long ng, const T *e,
                             const T *rhs, T *gtmp) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  T s = (T)0;
  for (int c = 0; c < 8; ++c) {
    long long q = src[8 * g + c];
    if (q >= 0) s += (T)w[8 * g + c] * e[q & ~GHOST_CORNER];
  }
  if (rhs) s += rhs[dst[g]];
  gtmp[g] = s;
}

// ghost rows right after a ping-pong sweep, in one launch: fluid sources from the new
// array, ghost sources from the previous one (whose ghost values the sweep copied
// unchanged), so no thread reads a value another thread writes (Jacobi among ghosts)
template <typename T, typename W>
__global__ void k_ghost_pp(const long long *src, const long long *dst, const W *w, long long ng, T *enew,
                           const T *eold, const T *rhs) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  T s = (T)0;
  for (int c = 0; c < 8; ++c) {
    long long q = src[8 * g + c];
    if (q < 0) continue;
    const T v = (q & GHOST_CORNER) ? eold[q & ~GHOST_CORNER] : enew[q];
    s += (T)w[8 * g + c] * v;
  }
  if (rhs) s += rhs[dst[g]];
  enew[dst[g]] = s;
}

template <typename T>
__global__ void k_ghost_store(const long long *dst, long long ng, const T *gtmp, T *e) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < ng) e[dst[g]] = gtmp[g];
}

// residual of level f restricted to level c: rc = sum_{fluid children} V_f r_f / V_c, and
// block partial sums of V_c rc for the coarse projection
template <typename T>
__global__ void k_restrict(LV<T> f, const T *e, const T *r, const double *shift, LV<T> cv, T *rc, double *partials) {
  __shared__ double sm[256];
  double acc_all = 0.0;
  const long long nc = (long long)cv.nx * cv.ny * cv.nz;
  const T sh = shift ? (T)(*shift) : (T)0;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nc; l += (long long)gridDim.x * blockDim.x) {
    int I = (int)(l % cv.nx); long long q = l / cv.nx; int J = (int)(q % cv.ny); int K = (int)(q / cv.ny);
    long long ic = vidx(cv, I, J, K);
    if (cv.mask[ic] != 0) { rc[ic] = (T)0; continue; }
    T acc = (T)0;
    for (int c = 0; c < 8; ++c) {
      int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
      if (i >= f.nx || j >= f.ny || k >= f.nz) continue;
      long long id = vidx(f, i, j, k);
      if (f.mask[id] != 0) continue;
      T cf[6];
      coefs(f, i, j, k, id, cf);
      T D = f.sdx ? (f.sdx[i] + f.sdy[j]) + f.sdz[k] : ((cf[0] + cf[1]) + (cf[2] + cf[3])) + (cf[4] + cf[5]);
      T res = (r[id] - sh) - (stencil_sum(f, e, id, cf) - D * e[id]);
      acc += (f.wx[i] * f.wy[j]) * f.wz[k] * res;
    }
    T vc = (cv.wx[I] * cv.wy[J]) * cv.wz[K];
    rc[ic] = acc / vc;
    acc_all += (double)acc;
  }
  sm[threadIdx.x] = acc_all;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

// deterministic sum of nb partials (stride `stride`, offset `off`) in one block
__device__ double block_sum_partials(const double *p, int nb, int stride, int off) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += p[b * stride + off];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  double out = sm[0];
  __syncthreads();
  return out;
}

__global__ void k_finalize_shift(const double *partials, int nb, double fluid_vol, double *shift) {
  double s = block_sum_partials(partials, nb, 1, 0);
  if (threadIdx.x == 0) *shift = fluid_vol > 0 ? s / fluid_vol : 0.0;
}

template <typename T>
__global__ void k_prolong(LV<T> cv, const T *ec, LV<T> f, T *ef, const int8_t *offx, const int8_t *offy,
                          const int8_t *offz, const float *tx, const float *ty, const float *tz) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y, k = blockIdx.z;
  if (i >= f.nx) return;
  long long id = vidx(f, i, j, k);
  if (f.mask[id] != 0) return;
  int I = i >> 1, J = j >> 1, K = k >> 1;
  float wx[2] = {1.0f - tx[i], tx[i]}, wy[2] = {1.0f - ty[j], ty[j]}, wz[2] = {1.0f - tz[k], tz[k]};
  int ox = offx[i], oy = offy[j], oz = offz[k];
  T s = (T)0;
  float ws = 0.0f;
  for (int c = 0; c < 8; ++c) {
    int a = c & 1, b = (c >> 1) & 1, d = (c >> 2) & 1;
    float w = (wx[a] * wy[b]) * wz[d];
    if (w == 0.0f) continue;
    long long ic = vidx(cv, I + a * ox, J + b * oy, K + d * oz);
    if (cv.mask[ic] != 0) continue;
    s += (T)w * ec[ic];
    ws += w;
  }
  if (ws > 0.0f) ef[id] += s * (T)(1.0f / ws);
}

// bordered coarsest solve: [e; lambda] = Minv [r; 0]
template <typename T>
__global__ void k_coarsest(const double *Minv, const int *cidx, const int *ncount, const T *r, T *e) {
  __shared__ double rs[MAX_COARSE + 1];
  const int n = *ncount, m = n + 1;
  for (int q = threadIdx.x; q < n; q += blockDim.x) rs[q] = (double)r[cidx[q]];
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += Minv[q * m + c] * rs[c];
    e[cidx[q]] = (T)s;
  }
}

// FP64 fine residual r = b - lambda - A p on fluid rows; optional FP32 copy; block partials
// (sum V r, sum r, sum r^2) at partials[3 b + {0,1,2}].  FP64 arithmetic is kept to the
// stencil itself (GB300 issues FP64 at 1/57 of the FP32 rate): the diagonal is separable,
// row invariants are hoisted, and the norm/mean partial sums run in FP32 per thread.
__global__ void k_residual64(LV<double> v, const double *p, const double *b, const double *lambda, float *r32,
                             double *partials) {
  __shared__ double sm[3][REDUCE_THREADS];
  const double lam = *lambda;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  double A0 = 0.0, A1 = 0.0, A2 = 0.0;
  const long long rows = (long long)v.ny * v.nz;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = (int)(row % v.ny), k = (int)(row / v.ny);
    const double cym = v.cym[j], cyp = v.cyp[j], czm = v.czm[k], czp = v.czp[k];
    const double syz = v.sdy[j] + v.sdz[k];
    const float dydz = (float)(v.dy[j] * v.dz[k]);
    for (int i = threadIdx.x; i < v.nx; i += blockDim.x) {
      long long id = vidx(v, i, j, k);
      if (v.mask[id] != 0) continue;
      if (p == nullptr) {            // residual of p = 0: b - lambda
        const float rf0 = (float)(b[id] - lam);
        if (r32) r32[id] = rf0;
        a0 = fmaf((float)v.dx[i] * dydz, rf0, a0);
        a1 += rf0;
        a2 = fmaf(rf0, rf0, a2);
        continue;
      }
      const double pc = p[id];
      double s = v.cxm[i] * p[id - 1];
      s = fma(v.cxp[i], p[id + 1], s);
      s = fma(cym, p[id - v.sy], s);
      s = fma(cyp, p[id + v.sy], s);
      s = fma(czm, p[id - v.sz], s);
      s = fma(czp, p[id + v.sz], s);
      s = fma(-(v.sdx[i] + syz), pc, s);           // (A p)_i
      const double res = (b[id] - lam) - s;
      const float rf = (float)res;
      if (r32) r32[id] = rf;
      a0 = fmaf((float)v.dx[i] * dydz, rf, a0);
      a1 += rf;
      a2 = fmaf(rf, rf, a2);
    }
    // fold the FP32 row partials into FP64 every row (bounded FP32 error)
    A0 += a0; A1 += a1; A2 += a2;
    a0 = a1 = a2 = 0.f;
  }
  sm[0][threadIdx.x] = A0; sm[1][threadIdx.x] = A1; sm[2][threadIdx.x] = A2;
  __syncthreads();
  for (int st = REDUCE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partials[3 * blockIdx.x + q] = sm[q][0];
}

// ghost rows r_G = sum w v - g; block partials of (s_G r_G)^2 at gpart[b]
__global__ void k_ghost_resid64(const long long *src, const long long *dst, const double *w, const double *scale,
                                long long ng, const double *p, float *r32, double *gpart) {
  __shared__ double sm[REDUCE_THREADS];
  double a = 0.0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      long long q = src[8 * g + c];
      if (q >= 0) s += w[8 * g + c] * p[q & ~GHOST_CORNER];
    }
    double rg = s - p[dst[g]];
    if (r32) r32[dst[g]] = (float)rg;
    double sr = scale[g] * rg;
    a += sr * sr;
  }
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int st = REDUCE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) gpart[blockIdx.x] = sm[0];
}

// mu = sum V r / V_F; ||S P r||^2 = sum r^2 - 2 mu sum r + N_F mu^2 + sum (s r_G)^2;
// lambda += mu when update_lambda
__global__ void k_finalize_resid(const double *partials, int nb, const double *gpart, int ngb, double *scal,
                                 int update_lambda) {
  double sv = block_sum_partials(partials, nb, 3, 0);
  double s1 = block_sum_partials(partials, nb, 3, 1);
  double s2 = block_sum_partials(partials, nb, 3, 2);
  double sg = ngb > 0 ? block_sum_partials(gpart, ngb, 1, 0) : 0.0;
  if (threadIdx.x == 0) {
    double mu = sv / scal[S_FLUIDVOL];
    double n2 = s2 - 2.0 * mu * s1 + scal[S_NF] * mu * mu;
    scal[S_MU] = mu;
    scal[S_NORM2] = (n2 > 0.0 ? n2 : 0.0) + sg;
    if (update_lambda) scal[S_LAMBDA] += mu;
  }
}

__global__ void k_update_p(double *p, const float *e, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    p[q] += (double)e[q];
}

__global__ void k_gauge_sum(LV<double> v, const double *p, double *partials) {
  __shared__ double sm[REDUCE_THREADS];
  double a = 0.0;
  const long long rows = (long long)v.ny * v.nz;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    int j = (int)(row % v.ny), k = (int)(row / v.ny);
    for (int i = threadIdx.x; i < v.nx; i += blockDim.x) {
      long long id = vidx(v, i, j, k);
      if (v.mask[id] == 0) a += v.dx[i] * v.dy[j] * v.dz[k] * p[id];
    }
  }
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int st = REDUCE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

__global__ void k_gauge_finalize(const double *partials, int nb, double *scal) {
  double s = block_sum_partials(partials, nb, 1, 0);
  if (threadIdx.x == 0) scal[S_MEANP] = s / scal[S_FLUIDVOL];
}

// pack user [k][j][i] arrays into padded arrays; unpack with the gauge applied
__global__ void k_pack(const double *src, LevelGeom g, double *dst) {
  long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)g.nx * g.ny * g.nz) return;
  int i = (int)(l % g.nx); long long r = l / g.nx; int j = (int)(r % g.ny); int k = (int)(r / g.ny);
  dst[pidx(g, i, j, k)] = src[l];
}

__global__ void k_unpack_gauge(const double *src, const uint8_t *mask, LevelGeom g, const double *scal, double *dst) {
  long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)g.nx * g.ny * g.nz) return;
  int i = (int)(l % g.nx); long long r = l / g.nx; int j = (int)(r % g.ny); int k = (int)(r / g.ny);
  long long id = pidx(g, i, j, k);
  dst[l] = mask[id] == 1 ? 0.0 : src[id] - scal[S_MEANP];
}

// mask solid cells of the packed p to zero (they are never read, keep them finite)
__global__ void k_zero_solid(double *p, const uint8_t *mask, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    if (mask[q] == 1) p[q] = 0.0;
}

// ------------------------------------------------------------------ double-FP32 outer loop

// Fine-level view for the double-FP32 kernels.  h and l hold the split fine data, 4n floats
// each (n = nx + ny + nz): cxm cxp cym cyp czm czp (2n), sdx sdy sdz (n), dx dy dz (n).
struct DfView {
  int nx, ny, nz, px;
  long long sy, sz;
  const uint8_t *mask;
  const float *h, *l;
};

// split n doubles into hi/lo floats
__global__ void k_split_df(const double *src, int n, float *h, float *l) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) dfl::split(src[q], h[q], l[q]);
}

// r = b - lambda - A p on fluid rows with pairs of floats (see dfloat.cuh); FP32 copy of r;
// block partials (sum V r, sum r, sum r^2) at partials[3 b + {0,1,2}] as k_residual64.
// ph == nullptr: residual of p = 0.
__global__ void __launch_bounds__(REDUCE_THREADS) k_residual_df(DfView v, const float *ph, const float *pl,
                                                               const float *bh, const float *bl,
                                                               const double *lambda, float *r32, double *partials) {
  __shared__ double sm[3][REDUCE_THREADS];
  float lh, ll;
  dfl::split(*lambda, lh, ll);
  const int nx = v.nx, ny = v.ny, nz = v.nz, n = nx + ny + nz;
  const float *H = v.h, *L = v.l;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  double A0 = 0.0, A1 = 0.0, A2 = 0.0;
  int nrow = 0;
  const long long rows = (long long)ny * nz;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = (int)(row % ny), k = (int)(row / ny);
    const float cymh = H[2 * nx + j], cyml = L[2 * nx + j], cyph = H[2 * nx + ny + j], cypl = L[2 * nx + ny + j];
    const float czmh = H[2 * nx + 2 * ny + k], czml = L[2 * nx + 2 * ny + k];
    const float czph = H[2 * nx + 2 * ny + nz + k], czpl = L[2 * nx + 2 * ny + nz + k];
    float syh, syl;   // sdy_j + sdz_k
    dfl::two_sum(H[2 * n + nx + j], H[2 * n + nx + ny + k], syh, syl);
    syl += L[2 * n + nx + j] + L[2 * n + nx + ny + k];
    const float dydz = H[3 * n + nx + j] * H[3 * n + nx + ny + k];
    const long long base = (long long)(k + 1) * v.sz + (long long)(j + 1) * v.sy + OX;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long id = base + i;
      if (v.mask[id] != 0) continue;
      float sh, sl;
      dfl::two_sum(bh[id], -lh, sh, sl);
      sl += bl[id] - ll;
      if (ph) {
        float dh, dl;   // diagonal sdx_i + sdy_j + sdz_k
        dfl::two_sum(H[2 * n + i], syh, dh, dl);
        dl += L[2 * n + i] + syl;
        dfl::acc_prod(dh, dl, ph[id], pl[id], sh, sl);
        dfl::acc_prod(-H[i], -L[i], ph[id - 1], pl[id - 1], sh, sl);
        dfl::acc_prod(-H[nx + i], -L[nx + i], ph[id + 1], pl[id + 1], sh, sl);
        dfl::acc_prod(-cymh, -cyml, ph[id - v.sy], pl[id - v.sy], sh, sl);
        dfl::acc_prod(-cyph, -cypl, ph[id + v.sy], pl[id + v.sy], sh, sl);
        dfl::acc_prod(-czmh, -czml, ph[id - v.sz], pl[id - v.sz], sh, sl);
        dfl::acc_prod(-czph, -czpl, ph[id + v.sz], pl[id + v.sz], sh, sl);
      }
      const float rf = sh + sl;
      if (r32) r32[id] = rf;
      a0 = fmaf(H[3 * n + i] * dydz, rf, a0);
      a1 += rf;
      a2 = fmaf(rf, rf, a2);
    }
    // fold the FP32 partials into FP64 every 8 rows (bounded FP32 error)
    if (++nrow == 8) {
      A0 += a0; A1 += a1; A2 += a2;
      a0 = a1 = a2 = 0.f;
      nrow = 0;
    }
  }
  A0 += a0; A1 += a1; A2 += a2;
  sm[0][threadIdx.x] = A0; sm[1][threadIdx.x] = A1; sm[2][threadIdx.x] = A2;
  __syncthreads();
  for (int st = REDUCE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partials[3 * blockIdx.x + q] = sm[q][0];
}

// ghost rows r_G = sum w v - g in FP64 from the split values; block partials of (s_G r_G)^2
__global__ void k_ghost_resid_df(const long long *src, const long long *dst, const double *w, const double *scale,
                                 long long ng, const float *ph, const float *pl, float *r32, double *gpart) {
  __shared__ double sm[REDUCE_THREADS];
  double a = 0.0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      long long q = src[8 * g + c];
      if (q >= 0) {
        q &= ~GHOST_CORNER;
        s += w[8 * g + c] * dfl::join(ph[q], pl[q]);
      }
    }
    const long long d = dst[g];
    const double rg = s - dfl::join(ph[d], pl[d]);
    if (r32) r32[d] = (float)rg;
    const double sr = scale[g] * rg;
    a += sr * sr;
  }
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int st = REDUCE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) gpart[blockIdx.x] = sm[0];
}

// ghost values g = sum w v from the split values (into gtmp), then stored split (Jacobi)
__global__ void k_ghost_eval_df(const long long *src, const double *w, long long ng, const float *ph,
                                const float *pl, double *gtmp) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  double s = 0.0;
  for (int c = 0; c < 8; ++c) {
    long long q = src[8 * g + c];
    if (q >= 0) {
      q &= ~GHOST_CORNER;
      s += w[8 * g + c] * dfl::join(ph[q], pl[q]);
    }
  }
  gtmp[g] = s;
}

__global__ void k_ghost_store_df(const long long *dst, long long ng, const double *gtmp, float *ph, float *pl) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < ng) dfl::split(gtmp[g], ph[dst[g]], pl[dst[g]]);
}

// p += e (FP32 correction) on every padded cell, four at a time (n4 = ntot / 4)
__global__ void k_update_df(float4 *ph, float4 *pl, const float4 *e, long long n4) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += (long long)gridDim.x * blockDim.x) {
    float4 h = ph[q], l = pl[q];
    const float4 x = e[q];
    float *hv = &h.x, *lv = &l.x;
    const float *xv = &x.x;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float s, t;
      dfl::two_sum(hv[u], xv[u], s, t);
      t += lv[u];
      dfl::two_sum(s, t, hv[u], lv[u]);
    }
    ph[q] = h;
    pl[q] = l;
  }
}

// pack a user [k][j][i] array into split padded arrays; cells with mask == 1 (plain solid)
// are set to zero when mask is given
__global__ void k_pack_df(const double *src, LevelGeom g, float *dh, float *dl, const uint8_t *mask) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)g.nx * g.ny * g.nz) return;
  int i = (int)(q % g.nx); long long r = q / g.nx; int j = (int)(r % g.ny); int k = (int)(r / g.ny);
  const long long id = pidx(g, i, j, k);
  float h, l;
  dfl::split(src[q], h, l);
  if (mask && mask[id] == 1) h = l = 0.f;
  dh[id] = h;
  dl[id] = l;
}

// block partials of sum V p over fluid cells; V and the products as pairs of floats
__global__ void __launch_bounds__(REDUCE_THREADS) k_gauge_sum_df(DfView v, const float *ph, const float *pl,
                                                                double *partials) {
  __shared__ double sm[REDUCE_THREADS];
  const int nx = v.nx, ny = v.ny, n = nx + ny + v.nz;
  const float *H = v.h + 3 * n, *L = v.l + 3 * n;   // widths
  float sh = 0.f, sl = 0.f;
  const long long rows = (long long)ny * v.nz;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = (int)(row % ny), k = (int)(row / ny);
    float ah = 0.f, al = 0.f, yzh, yzl;   // dy_j dz_k
    dfl::acc_prod(H[nx + j], L[nx + j], H[nx + ny + k], L[nx + ny + k], ah, al);
    dfl::fast_two_sum(ah, al, yzh, yzl);
    const long long base = (long long)(k + 1) * v.sz + (long long)(j + 1) * v.sy + OX;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const long long id = base + i;
      if (v.mask[id] != 0) continue;
      float vh = 0.f, vl = 0.f, Vh, Vl;
      dfl::acc_prod(H[i], L[i], yzh, yzl, vh, vl);
      dfl::fast_two_sum(vh, vl, Vh, Vl);
      dfl::acc_prod(Vh, Vl, ph[id], pl[id], sh, sl);
    }
  }
  sm[threadIdx.x] = dfl::join(sh, sl);
  __syncthreads();
  for (int st = REDUCE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

// (grid-stride: the mean is split once per thread)
__global__ void k_unpack_gauge_df(const float *ph, const float *pl, const uint8_t *mask, LevelGeom g,
                                  const double *scal, double *dst) {
  float mh, ml;
  dfl::split(scal[S_MEANP], mh, ml);
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    int i = (int)(q % g.nx); long long r = q / g.nx; int j = (int)(r % g.ny); int k = (int)(r / g.ny);
    const long long id = pidx(g, i, j, k);
    if (mask[id] == 1) { dst[q] = 0.0; continue; }
    float s, t;
    dfl::two_sum(ph[id], -mh, s, t);
    t += pl[id] - ml;
    dst[q] = dfl::join(s, t);
  }
}

__global__ void k_ghost_src(const long long *ref, const long long *cell, long long ng, LevelGeom g, long long *src,
                            long long *dst, const double *w, float *w32, const uint8_t *ib) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= ng * 8) return;
  auto tp = [&](long long l) {
    int i = (int)(l % g.nx); long long r = l / g.nx; int j = (int)(r % g.ny); int k = (int)(r / g.ny);
    return pidx(g, i, j, k);
  };
  long long l = ref[q];
  src[q] = l >= 0 ? (tp(l) | (ib[l] == 3 ? GHOST_CORNER : 0LL)) : -1;
  w32[q] = (float)w[q];
  if ((q & 7) == 0) dst[q >> 3] = tp(cell[q >> 3]);
}

template <typename T>
cudaError_t alloc_zero(void **p, long long n, cudaStream_t st) {
  cudaError_t e = cudaMalloc(p, (size_t)(n ? n : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(*p, 0, (size_t)(n ? n : 1) * sizeof(T), st);
}

}  // namespace

void free_hierarchy(Hierarchy *h) {
  if (!h) return;
  std::vector<void *> ps;
  for (Level &L : h->lv) {
    void *q[] = {L.mask, L.e, L.r, L.fx, L.fy, L.fz, L.c1d, L.w1d, L.cen, L.poff, L.pt, L.wT, L.sdiag};
    ps.insert(ps.end(), q, q + 13);
  }
  void *q[] = {h->p64, h->b64, h->minv, h->cidx, h->dncoarse, h->c64, h->cdf, h->gsrc, h->gdst, h->gw64, h->gw32,
               h->gtmp, h->e_alt, h->tm_base[0], h->tm_base[1]};
  ps.insert(ps.end(), q, q + 15);
  std::sort(ps.begin(), ps.end());
  ps.erase(std::unique(ps.begin(), ps.end()), ps.end());
  for (void *p : ps) if (p) cudaFree(p);
  if (h->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)h->graph_exec);
  delete h;
}

// ------------------------------------------------------------------ hierarchy build

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
  }
  return fn;
}

// 3-D tensor map over a padded level array; box (bx, by, 1); zero fill outside
static bool make_map(CUtensorMap *m, void *base, CUtensorMapDataType dt, int elem, const LevelGeom &g, int bx, int by) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)(g.ny + 2), (cuuint64_t)(g.nz + 2)};
  cuuint64_t strides[2] = {(cuuint64_t)g.px * elem, (cuuint64_t)g.px * (g.ny + 2) * elem};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T>
static void setup_zmarch(Hierarchy *h, void *e0, void *r0) {
  Level &L0 = h->lv[0];
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  bool ok = make_map(&h->tm_e[0], e0, dt, sizeof(T), L0.g, zm::BX, zm::EY) &&
            make_map(&h->tm_e[1], h->e_alt, dt, sizeof(T), L0.g, zm::BX, zm::EY) &&
            make_map(&h->tm_r, r0, dt, sizeof(T), L0.g, zm::BX, zm::RY) &&
            make_map(&h->tm_m, L0.mask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, L0.g, zm::BXM, zm::RY);
  h->tm_base[0] = e0;
  h->tm_base[1] = h->e_alt;
  // the FP64 smoother is bound by the FP64 pipe, not by memory: it keeps the two-pass kernel,
  // whose small blocks give the occupancy that hides FP64 latency
  h->zmarch = sizeof(T) == 4 && ok &&
              cudaFuncSetAttribute(zm::k_sweep_zmarch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(zm::Smem<T>)) == cudaSuccess;
  int per_sm = 0;
  if (h->zmarch && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zm::k_sweep_zmarch<T>, zm::THREADS,
                                                                 sizeof(zm::Smem<T>)) == cudaSuccess && per_sm > 0)
    h->zm_per_sm = per_sm;
  else
    h->zmarch = false;
}

template <typename T>
static ibm_status build_hierarchy_t(ibm_tables *t, cudaStream_t st, Hierarchy **out) {
  Hierarchy *h = new Hierarchy();
  h->elem = sizeof(T);
  auto fail = [&](cudaError_t e, const char *w) { free_hierarchy(h); return check(e, w); };
#define HTRY(call) do { cudaError_t e__ = (call); if (e__ != cudaSuccess) return fail(e__, #call); } while (0)
  std::vector<double> fx(t->xf), fy(t->yf), fz(t->zf);
  double *dfaces = nullptr;
  while (true) {
    Level L;
    L.g = make_geom((int)fx.size() - 1, (int)fy.size() - 1, (int)fz.size() - 1);
    const int nx = L.g.nx, ny = L.g.ny, nz = L.g.nz;
    HTRY(alloc_zero<uint8_t>((void **)&L.mask, L.g.ntot, st));
    HTRY(cudaMemsetAsync(L.mask, 1, L.g.ntot, st));
    HTRY(alloc_zero<T>(&L.e, L.g.ntot, st));
    HTRY(alloc_zero<T>(&L.r, L.g.ntot, st));
    HTRY(cudaMalloc(&L.c1d, sizeof(T) * 2 * (nx + ny + nz)));
    HTRY(cudaMalloc((void **)&L.w1d, sizeof(double) * (nx + ny + nz)));
    HTRY(cudaMalloc((void **)&L.cen, sizeof(double) * (nx + ny + nz)));
    HTRY(cudaMalloc(&L.wT, sizeof(T) * (nx + ny + nz)));
    const bool finest = h->lv.empty();
    if (finest) HTRY(cudaMalloc(&L.sdiag, sizeof(T) * (nx + ny + nz)));
    HTRY(cudaMalloc((void **)&dfaces, sizeof(double) * (nx + ny + nz + 3)));
    HTRY(cudaMemcpyAsync(dfaces, fx.data(), sizeof(double) * (nx + 1), cudaMemcpyHostToDevice, st));
    HTRY(cudaMemcpyAsync(dfaces + nx + 1, fy.data(), sizeof(double) * (ny + 1), cudaMemcpyHostToDevice, st));
    HTRY(cudaMemcpyAsync(dfaces + nx + ny + 2, fz.data(), sizeof(double) * (nz + 1), cudaMemcpyHostToDevice, st));
    T *c = (T *)L.c1d, *wt = (T *)L.wT, *sd = (T *)L.sdiag;
    k_axis_level<T><<<nblk(nx, 128), 128, 0, st>>>(dfaces, nx, c, c + nx, L.w1d, L.cen, wt, sd);
    k_axis_level<T><<<nblk(ny, 128), 128, 0, st>>>(dfaces + nx + 1, ny, c + 2 * nx, c + 2 * nx + ny, L.w1d + nx,
                                                    L.cen + nx, wt + nx, sd ? sd + nx : nullptr);
    k_axis_level<T><<<nblk(nz, 128), 128, 0, st>>>(dfaces + nx + ny + 2, nz, c + 2 * nx + 2 * ny,
                                                    c + 2 * nx + 2 * ny + nz, L.w1d + nx + ny, L.cen + nx + ny,
                                                    wt + nx + ny, sd ? sd + nx + ny : nullptr);
    HTRY(cudaGetLastError());
    HTRY(cudaStreamSynchronize(st));
    cudaFree(dfaces);
    dfaces = nullptr;
    h->lv.push_back(L);
    const long long cells = (long long)nx * ny * nz;
    if (cells <= MAX_COARSE || (nx == 1 && ny == 1 && nz == 1)) break;
    auto coarsen = [](const std::vector<double> &f) {
      int n = (int)f.size() - 1, nc = (n + 1) / 2;
      std::vector<double> c(nc + 1);
      for (int I = 0; I < nc; ++I) c[I] = f[2 * I];
      c[nc] = f[n];
      return c;
    };
    fx = coarsen(fx); fy = coarsen(fy); fz = coarsen(fz);
  }
  const int nl = (int)h->lv.size();
  // masks, fractions, prolongation tables
  {
    Level &L0 = h->lv[0];
    const long long n0 = (long long)L0.g.nx * L0.g.ny * L0.g.nz;
    k_mask0<<<nblk(n0, 256), 256, 0, st>>>(t->iblank, L0.g.nx, L0.g.ny, L0.g.nz, L0.mask, L0.g);
  }
  for (int l = 0; l + 1 < nl; ++l) {
    Level &F = h->lv[l], &C = h->lv[l + 1];
    const long long nc = (long long)C.g.nx * C.g.ny * C.g.nz;
    k_mask_coarse<<<nblk(nc, 256), 256, 0, st>>>(F.mask, F.g, C.mask, C.g);
    HTRY(alloc_zero<T>(&C.fx, C.g.ntot, st));
    HTRY(alloc_zero<T>(&C.fy, C.g.ntot, st));
    HTRY(alloc_zero<T>(&C.fz, C.g.ntot, st));
    const double *wf = F.w1d, *wc = C.w1d;
    k_fractions<T><<<nblk(nc, 256), 256, 0, st>>>(F.mask, (const T *)F.fx, (const T *)F.fy, (const T *)F.fz, F.g, wf,
                                                  wf + F.g.nx, wf + F.g.nx + F.g.ny, C.g, wc, wc + C.g.nx,
                                                  wc + C.g.nx + C.g.ny, (T *)C.fx, (T *)C.fy, (T *)C.fz);
    const int nf = F.g.nx + F.g.ny + F.g.nz;
    HTRY(cudaMalloc((void **)&F.poff, nf));
    HTRY(cudaMalloc((void **)&F.pt, sizeof(float) * nf));
    k_prolong_axis<<<nblk(F.g.nx, 128), 128, 0, st>>>(F.cen, F.g.nx, C.cen, C.g.nx, F.poff, F.pt);
    k_prolong_axis<<<nblk(F.g.ny, 128), 128, 0, st>>>(F.cen + F.g.nx, F.g.ny, C.cen + C.g.nx, C.g.ny,
                                                      F.poff + F.g.nx, F.pt + F.g.nx);
    k_prolong_axis<<<nblk(F.g.nz, 128), 128, 0, st>>>(F.cen + F.g.nx + F.g.ny, F.g.nz, C.cen + C.g.nx + C.g.ny, C.g.nz,
                                                      F.poff + F.g.nx + F.g.ny, F.pt + F.g.nx + F.g.ny);
    HTRY(cudaGetLastError());
  }
  // fluid volume per level
  {
    double *tmp = nullptr;
    HTRY(cudaMalloc((void **)&tmp, sizeof(double) * 2 * 152));
    std::vector<double> hv(2 * 152);
    for (int l = 0; l < nl; ++l) {
      Level &L = h->lv[l];
      k_fluid_stats<<<152, 256, 0, st>>>(L.mask, L.g, L.w1d, L.w1d + L.g.nx, L.w1d + L.g.nx + L.g.ny, tmp);
      cudaError_t e = cudaMemcpyAsync(hv.data(), tmp, sizeof(double) * 2 * 152, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { cudaFree(tmp); return fail(e, "fluid stats"); }
      double v = 0.0, c = 0.0;
      for (int b = 0; b < 152; ++b) { v += hv[2 * b]; c += hv[2 * b + 1]; }
      L.fluid_vol = v;
      L.nfluid = (long long)c;
    }
    cudaFree(tmp);
  }
  // coarsest bordered inverse
  {
    Level &Lc = h->lv[nl - 1];
    const int m = MAX_COARSE + 1;
    double *M = nullptr;
    int *nc = nullptr;
    HTRY(cudaMalloc((void **)&M, sizeof(double) * m * m));
    HTRY(cudaMalloc((void **)&h->minv, sizeof(double) * m * m));
    HTRY(cudaMalloc((void **)&h->cidx, sizeof(int) * (MAX_COARSE + 1)));
    HTRY(cudaMalloc((void **)&nc, sizeof(int) * 2));
    h->dncoarse = nc;
    k_coarsest_setup<T><<<1, 256, 0, st>>>(view<T>(Lc), h->cidx, nc, M, h->minv, MAX_COARSE);
    HTRY(cudaGetLastError());
    HTRY(cudaMemcpyAsync(&h->ncoarse, nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    HTRY(cudaStreamSynchronize(st));
    cudaFree(M);
  }
  // fine FP64 arrays and solver-side ghost rows
  {
    Level &L0 = h->lv[0];
    HTRY(alloc_zero<double>((void **)&h->p64, L0.g.ntot, st));
    HTRY(alloc_zero<double>((void **)&h->b64, L0.g.ntot, st));
    const long long ng = t->nghost;
    HTRY(cudaMalloc((void **)&h->gsrc, sizeof(long long) * 8 * (ng ? ng : 1)));
    HTRY(cudaMalloc((void **)&h->gdst, sizeof(long long) * (ng ? ng : 1)));
    HTRY(cudaMalloc((void **)&h->gw32, sizeof(float) * 8 * (ng ? ng : 1)));
    HTRY(cudaMalloc((void **)&h->gtmp, sizeof(double) * (ng ? ng : 1)));
    h->gw64 = nullptr;
    if (ng) k_ghost_src<<<nblk(8 * ng, 256), 256, 0, st>>>(t->gref, t->gcell, ng, L0.g, h->gsrc, h->gdst, t->gw, h->gw32,
                                                         t->iblank);
    HTRY(cudaGetLastError());
    HTRY(alloc_zero<T>(&h->e_alt, L0.g.ntot, st));
    HTRY(cudaStreamSynchronize(st));
    if (sizeof(T) == 8) setup_zmarch<T>(h, h->p64, h->b64);
    else setup_zmarch<T>(h, L0.e, L0.r);
  }
#undef HTRY
  *out = h;
  return IBM_OK;
}

// ------------------------------------------------------------------ solve driver

namespace {

struct Solver {
  ibm_ctx *ctx;
  ibm_tables *t;
  Hierarchy *h;
  cudaStream_t st;
  int nu1, nu2;
  double omega;
  int *d_ncoarse;
  bool dfo = false;   // double-FP32 outer loop (precision mode 2)
};

template <typename T>
void ghost_update(Solver &S, T *e, const T *ghost_rhs) {
  const long long ng = S.t->nghost;
  if (ng <= 0) return;
  if (sizeof(T) == 8)
    k_ghost_eval<T, double><<<nblk(ng, 128), 128, 0, S.st>>>(S.h->gsrc, S.h->gdst, S.t->gw, ng, e, ghost_rhs,
                                                              (T *)S.h->gtmp);
  else
    k_ghost_eval<T, float><<<nblk(ng, 128), 128, 0, S.st>>>(S.h->gsrc, S.h->gdst, S.h->gw32, ng, e, ghost_rhs,
                                                             (T *)S.h->gtmp);
  k_ghost_store<T><<<nblk(ng, 128), 128, 0, S.st>>>(S.h->gdst, ng, (const T *)S.h->gtmp, e);
  S.ctx->launches += 2;
}

template <typename T>
void sweep_zmarch(Solver &S, T *&e, const double *shift) {
  Hierarchy *h = S.h;
  Level &L0 = h->lv[0];
  const int which = (e == (T *)h->tm_base[0]) ? 0 : 1;
  T *other = (T *)h->tm_base[1 - which];
  LV<T> v = view<T>(L0);
  zm::Args<T> a;
  a.nx = L0.g.nx; a.ny = L0.g.ny; a.nz = L0.g.nz; a.px = L0.g.px; a.sy = L0.g.sy; a.sz = L0.g.sz;
  a.cxm = v.cxm; a.cxp = v.cxp; a.cym = v.cym; a.cyp = v.cyp; a.czm = v.czm; a.czp = v.czp;
  a.sdx = v.sdx; a.sdy = v.sdy; a.sdz = v.sdz;
  a.shift = shift;
  a.omega = (float)S.omega;
  a.out = other;
  a.err = S.ctx->errflag;
  const int gx = (a.nx + zm::TX - 1) / zm::TX, gy = (a.ny + zm::TY - 1) / zm::TY;
  const int per_sm = std::max(1, h->zm_per_sm);
  const long long target = (long long)per_sm * (S.ctx->sm_count > 0 ? S.ctx->sm_count : 152);
  // one wave: tiles x chunks <= resident CTAs (a second, partly filled wave would idle most SMs)
  int chunks = (int)std::max<long long>(1, std::min<long long>(a.nz, target / (gx * gy)));
  a.kz = (a.nz + chunks - 1) / chunks;
  chunks = (a.nz + a.kz - 1) / a.kz;
  dim3 grid(gx, gy, chunks);
  zm::k_sweep_zmarch<T><<<grid, zm::THREADS, sizeof(zm::Smem<T>), S.st>>>(h->tm_e[which], h->tm_r, h->tm_m, a);
  S.ctx->launches += 1;
  e = other;
}

template <typename T>
void smooth_level(Solver &S, int l, T *&e, const T *r, const double *shift, bool fine, const T *ghost_rhs, int sweeps) {
  Level &L = S.h->lv[l];
  LV<T> v = view<T>(L);
  dim3 grid(nblk((L.g.nx + 1) / 2, 128), L.g.ny, L.g.nz);
  for (int s = 0; s < sweeps; ++s) {
    if (fine && S.h->zmarch) {
      T *old = e;
      sweep_zmarch<T>(S, e, shift);
      const long long ng = S.t->nghost;
      if (ng > 0) {
        if (sizeof(T) == 8)
          k_ghost_pp<T, double><<<nblk(ng, 128), 128, 0, S.st>>>(S.h->gsrc, S.h->gdst, S.t->gw, ng, e, old, ghost_rhs);
        else
          k_ghost_pp<T, float><<<nblk(ng, 128), 128, 0, S.st>>>(S.h->gsrc, S.h->gdst, S.h->gw32, ng, e, old, ghost_rhs);
        S.ctx->launches += 1;
      }
      continue;
    } else {
      for (int colour = 0; colour < 2; ++colour)
        k_rbgs<T><<<grid, 128, 0, S.st>>>(v, e, r, shift, colour, (T)S.omega);
      S.ctx->launches += 2;
    }
    if (fine) ghost_update<T>(S, e, ghost_rhs);
  }
}

// V-cycle for level l: e_l (in/out) approximately solves A_l e_l = r_l - shift_l.  On the
// finest level e is the hierarchy's own pointer: the fused sweep swaps it between two buffers.
template <typename T>
void vcycle(Solver &S, int l, T *&e, const T *r, const double *shift, const T *ghost_rhs) {
  Hierarchy *h = S.h;
  const int nl = (int)h->lv.size();
  if (l == nl - 1) {
    k_coarsest<T><<<1, 128, 0, S.st>>>(h->minv, h->cidx, S.d_ncoarse, r, e);
    S.ctx->launches += 1;
    return;
  }
  const bool fine = (l == 0);
  smooth_level<T>(S, l, e, r, shift, fine, ghost_rhs, S.nu1);
  Level &F = h->lv[l], &C = h->lv[l + 1];
  const long long nc = (long long)C.g.nx * C.g.ny * C.g.nz;
  const int nb = (int)std::min<long long>(nblk(nc, 256), REDUCE_BLOCKS);
  T *ec = (T *)C.e, *rc = (T *)C.r;
  k_restrict<T><<<nb, 256, 0, S.st>>>(view<T>(F), e, r, shift, view<T>(C), rc, S.ctx->partials);
  double *cshift = S.ctx->scal + S_LEVEL_SHIFT + (l + 1);
  k_finalize_shift<<<1, 256, 0, S.st>>>(S.ctx->partials, nb, C.fluid_vol, cshift);
  cudaMemsetAsync(ec, 0, sizeof(T) * C.g.ntot, S.st);
  vcycle<T>(S, l + 1, ec, rc, cshift, nullptr);
  dim3 gp(nblk(F.g.nx, 128), F.g.ny, F.g.nz);
  const int nxf = F.g.nx, nyf = F.g.ny;
  k_prolong<T><<<gp, 128, 0, S.st>>>(view<T>(C), ec, view<T>(F), e, F.poff, F.poff + nxf, F.poff + nxf + nyf, F.pt,
                                     F.pt + nxf, F.pt + nxf + nyf);
  S.ctx->launches += 3;   // restrict, finalize shift, prolong
  // the corrected fluid values make the ghost rows stale: refresh them before post-smoothing
  if (fine) ghost_update<T>(S, e, ghost_rhs);
  smooth_level<T>(S, l, e, r, shift, fine, ghost_rhs, S.nu2);
}

LV<double> fine_view64(Hierarchy *h) {
  Level &L0 = h->lv[0];
  LV<double> v;
  v.nx = L0.g.nx; v.ny = L0.g.ny; v.nz = L0.g.nz; v.px = L0.g.px; v.sy = L0.g.sy; v.sz = L0.g.sz;
  v.mask = L0.mask;
  v.fx = v.fy = v.fz = nullptr;
  v.dx = L0.w1d; v.dy = L0.w1d + v.nx; v.dz = L0.w1d + v.nx + v.ny;
  const double *c = h->c64;
  v.cxm = c; v.cxp = c + v.nx; v.cym = c + 2 * v.nx; v.cyp = v.cym + v.ny; v.czm = v.cyp + v.ny; v.czp = v.czm + v.nz;
  const double *d = c + 2 * (v.nx + v.ny + v.nz);
  v.sdx = d; v.sdy = d + v.nx; v.sdz = d + v.nx + v.ny;
  v.wx = v.wy = v.wz = nullptr;
  return v;
}

DfView fine_view_df(Hierarchy *h) {
  Level &L0 = h->lv[0];
  DfView v;
  v.nx = L0.g.nx; v.ny = L0.g.ny; v.nz = L0.g.nz; v.px = L0.g.px; v.sy = L0.g.sy; v.sz = L0.g.sz;
  v.mask = L0.mask;
  const int n = v.nx + v.ny + v.nz;
  v.h = h->cdf;
  v.l = h->cdf + 4 * n;
  return v;
}

// split views of the outer arrays in double-FP32 mode
inline float *hi_of(double *a) { return reinterpret_cast<float *>(a); }
inline float *lo_of(double *a, long long ntot) { return reinterpret_cast<float *>(a) + ntot; }

void fine_residual(Solver &S, const double *p, float *r32, bool update_lambda);

// the outer residual, its norms and the lambda update; with_p == false: residual of p = 0
void outer_residual(Solver &S, bool with_p, float *r32, bool update_lambda) {
  if (!S.dfo) return fine_residual(S, with_p ? S.h->p64 : nullptr, r32, update_lambda);
  Hierarchy *h = S.h;
  const long long ntot = h->lv[0].g.ntot;
  double *part = S.ctx->partials;
  float *ph = with_p ? hi_of(h->p64) : nullptr, *pl = lo_of(h->p64, ntot);
  k_residual_df<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, S.st>>>(fine_view_df(h), ph, pl, hi_of(h->b64),
                                                           lo_of(h->b64, ntot), S.ctx->scal + S_LAMBDA, r32, part);
  const long long ng = S.t->nghost;
  const int ngb = 152;
  double *gpart = part + 3 * REDUCE_BLOCKS;
  const bool gh = ng > 0 && with_p;
  if (gh)
    k_ghost_resid_df<<<ngb, REDUCE_THREADS, 0, S.st>>>(h->gsrc, h->gdst, S.t->gw, S.t->gscale, ng, hi_of(h->p64),
                                                       pl, r32, gpart);
  k_finalize_resid<<<1, 256, 0, S.st>>>(part, REDUCE_BLOCKS, gpart, gh ? ngb : 0, S.ctx->scal,
                                        update_lambda ? 1 : 0);
  S.ctx->launches += gh ? 3 : 2;
}

void fine_residual(Solver &S, const double *p, float *r32, bool update_lambda) {
  LV<double> v = fine_view64(S.h);
  double *part = S.ctx->partials;
  k_residual64<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, S.st>>>(v, p, S.h->b64, S.ctx->scal + S_LAMBDA, r32, part);
  const long long ng = S.t->nghost;
  const int ngb = 152;
  double *gpart = part + 3 * REDUCE_BLOCKS;
  const bool gh = ng > 0 && p != nullptr;
  if (gh)
    k_ghost_resid64<<<ngb, REDUCE_THREADS, 0, S.st>>>(S.h->gsrc, S.h->gdst, S.t->gw, S.t->gscale, ng, p, r32, gpart);
  k_finalize_resid<<<1, 256, 0, S.st>>>(part, REDUCE_BLOCKS, gpart, gh ? ngb : 0, S.ctx->scal,
                                        update_lambda ? 1 : 0);
  S.ctx->launches += gh ? 3 : 2;
}

}  // namespace

ibm_status build_hierarchy(ibm_tables *t, int precision, cudaStream_t st) {
  if (t->hier[precision]) return IBM_OK;
  Hierarchy *h = nullptr;
  ibm_status s = precision == 0 ? build_hierarchy_t<double>(t, st, &h) : build_hierarchy_t<float>(t, st, &h);
  if (s != IBM_OK) return s;
  // FP64 fine coefficients
  Level &L0 = h->lv[0];
  const int n = L0.g.nx + L0.g.ny + L0.g.nz;
  double *c64 = nullptr, *df = nullptr;
  IBM_TRY(cudaMalloc((void **)&c64, sizeof(double) * 3 * n));
  IBM_TRY(cudaMalloc((void **)&df, sizeof(double) * (n + 3)));
  IBM_TRY(cudaMemcpyAsync(df, t->xf.data(), sizeof(double) * (L0.g.nx + 1), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(df + L0.g.nx + 1, t->yf.data(), sizeof(double) * (L0.g.ny + 1), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(df + L0.g.nx + L0.g.ny + 2, t->zf.data(), sizeof(double) * (L0.g.nz + 1),
                          cudaMemcpyHostToDevice, st));
  double *w = nullptr, *c = nullptr;
  IBM_TRY(cudaMalloc((void **)&w, sizeof(double) * n));
  IBM_TRY(cudaMalloc((void **)&c, sizeof(double) * n));
  const int nx = L0.g.nx, ny = L0.g.ny, nz = L0.g.nz;
  double *sd = c64 + 2 * n;
  k_axis_level<double><<<nblk(nx, 128), 128, 0, st>>>(df, nx, c64, c64 + nx, w, c, nullptr, sd);
  k_axis_level<double><<<nblk(ny, 128), 128, 0, st>>>(df + nx + 1, ny, c64 + 2 * nx, c64 + 2 * nx + ny, w + nx, c + nx,
                                                      nullptr, sd + nx);
  k_axis_level<double><<<nblk(nz, 128), 128, 0, st>>>(df + nx + ny + 2, nz, c64 + 2 * nx + 2 * ny,
                                                      c64 + 2 * nx + 2 * ny + nz, w + nx + ny, c + nx + ny, nullptr,
                                                      sd + nx + ny);
  h->c64 = c64;
  if (precision == 2) {
    // split coefficients, diagonal parts (3n doubles of c64) and widths (n of w1d)
    float *cdf = nullptr;
    IBM_TRY(cudaMalloc((void **)&cdf, sizeof(float) * 8 * n));
    h->cdf = cdf;
    k_split_df<<<nblk(3 * n, 128), 128, 0, st>>>(c64, 3 * n, cdf, cdf + 4 * n);
    k_split_df<<<nblk(n, 128), 128, 0, st>>>(L0.w1d, n, cdf + 3 * n, cdf + 7 * n);
  }
  IBM_TRY(cudaGetLastError());
  IBM_TRY(cudaStreamSynchronize(st));
  cudaFree(df); cudaFree(w); cudaFree(c);
  t->hier[precision] = h;
  return IBM_OK;
}

ibm_status solve_impl(ibm_ctx *ctx, ibm_tables *t, const double *rhs, double tol, double *p_user,
                      const ibm_solve_opts *opts, ibm_solve_info *info, cudaStream_t st) {
  const int prec = opts->precision;
  ibm_status s = build_hierarchy(t, prec, st);
  if (s != IBM_OK) return s;
  Hierarchy *h = t->hier[prec];
  Level &L0 = h->lv[0];
  const long long n0 = (long long)L0.g.nx * L0.g.ny * L0.g.nz;
  Solver S{ctx, t, h, st, opts->nu1, opts->nu2, opts->omega, h->dncoarse};
  S.dfo = prec == 2;
  const long long ntot = L0.g.ntot;
  // inputs
  if (S.dfo) {
    k_pack_df<<<nblk(n0, 256), 256, 0, st>>>(rhs, L0.g, hi_of(h->b64), lo_of(h->b64, ntot), nullptr);
    k_pack_df<<<nblk(n0, 256), 256, 0, st>>>(p_user, L0.g, hi_of(h->p64), lo_of(h->p64, ntot), L0.mask);
    ctx->launches += 2;
  } else {
    k_pack<<<nblk(n0, 256), 256, 0, st>>>(rhs, L0.g, h->b64);
    k_pack<<<nblk(n0, 256), 256, 0, st>>>(p_user, L0.g, h->p64);
    k_zero_solid<<<1216, 256, 0, st>>>(h->p64, L0.mask, L0.g.ntot);
    ctx->launches += 3;
  }
  double hs[NSCAL] = {0};
  hs[S_FLUIDVOL] = L0.fluid_vol;
  hs[S_NF] = (double)L0.nfluid;
  IBM_TRY(cudaMemcpyAsync(ctx->scal, hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  // ||S P b||: residual of p = 0 with lambda = 0
  outer_residual(S, false, nullptr, false);
  IBM_TRY(cudaMemcpyAsync(ctx->hscal, ctx->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(ctx->hscal[S_NORM2]);
  const double denom = bnorm > 0 ? bnorm : 1.0;
  // initial ghost values consistent with p, and the initial residual
  const long long ng = t->nghost;
  if (ng > 0 && S.dfo) {
    k_ghost_eval_df<<<nblk(ng, 128), 128, 0, st>>>(h->gsrc, t->gw, ng, hi_of(h->p64), lo_of(h->p64, ntot), h->gtmp);
    k_ghost_store_df<<<nblk(ng, 128), 128, 0, st>>>(h->gdst, ng, h->gtmp, hi_of(h->p64), lo_of(h->p64, ntot));
    ctx->launches += 2;
  } else if (ng > 0) {
    k_ghost_eval<double, double><<<nblk(ng, 128), 128, 0, st>>>(h->gsrc, h->gdst, t->gw, ng, h->p64, nullptr, h->gtmp);
    k_ghost_store<double><<<nblk(ng, 128), 128, 0, st>>>(h->gdst, ng, h->gtmp, h->p64);
    ctx->launches += 2;
  }
  IBM_TRY(cudaGetLastError());
  int cycles = 0;
  double rel = 0.0;
  int hl = 0;
  ibm_status result = IBM_ERR_NOT_CONVERGED;
  float *r32 = prec != 0 ? (float *)L0.r : nullptr;
  outer_residual(S, true, r32, true);
  IBM_TRY(cudaMemcpyAsync(ctx->hscal, ctx->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  rel = std::sqrt(ctx->hscal[S_NORM2]) / denom;
  double rel0 = rel;
  if (rel <= tol) result = IBM_OK;
  // one cycle: V-cycle (FP64) or FP32 V-cycle(s) + FP64 update (mixed), then the FP64 fine
  // residual with its norms.  Launched directly, or captured once as a CUDA graph (on the
  // context's capture stream) and replayed; the pointer swaps of the fused sweep cancel
  // over a cycle when its number of fine sweeps is even, so the graph stays valid.
  auto body = [&](cudaStream_t bs) {
    S.st = bs;
    if (prec == 0) {
      vcycle<double>(S, 0, h->p64, h->b64, ctx->scal + S_LAMBDA, nullptr);
      fine_residual(S, h->p64, nullptr, true);
    } else {
      float *&e32 = reinterpret_cast<float *&>(L0.e);
      for (int q = 0; q < std::max(1, opts->inner_cycles); ++q) {
        if (q == 0) cudaMemsetAsync(e32, 0, sizeof(float) * L0.g.ntot, bs);
        vcycle<float>(S, 0, e32, r32, ctx->scal + S_MU, r32);
      }
      if (S.dfo)
        k_update_df<<<1216, 256, 0, bs>>>(reinterpret_cast<float4 *>(hi_of(h->p64)),
                                          reinterpret_cast<float4 *>(lo_of(h->p64, ntot)),
                                          reinterpret_cast<const float4 *>(e32), ntot / 4);
      else
        k_update_p<<<1216, 256, 0, bs>>>(h->p64, e32, L0.g.ntot);
      ctx->launches += 1;
      outer_residual(S, true, r32, true);
    }
    S.st = st;
  };
  const long long sweeps_per_cycle =
      (long long)(opts->nu1 + opts->nu2) * (prec != 0 ? std::max(1, opts->inner_cycles) : 1);
  const bool graph = opts->use_graph && ctx->cap_stream && (!h->zmarch || sweeps_per_cycle % 2 == 0);
  long long graph_launches = 0;
  if (graph) {
    const long long key = ((long long)opts->nu1 << 48) ^ ((long long)opts->nu2 << 40) ^
                          ((long long)opts->inner_cycles << 32) ^ (long long)(opts->omega * 1e6);
    if (!h->graph_exec || h->graph_key != key) {
      if (h->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)h->graph_exec);
      h->graph_exec = nullptr;
      cudaGraph_t g = nullptr;
      const long long l0 = ctx->launches;
      IBM_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      body(ctx->cap_stream);
      cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
      if (ce != cudaSuccess) return check(ce, "graph capture");
      cudaGraphExec_t ge = nullptr;
      ce = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return check(ce, "graph instantiate");
      h->graph_exec = ge;
      h->graph_key = key;
      h->graph_launches = ctx->launches - l0;
      ctx->launches = l0;
    }
    graph_launches = h->graph_launches;
  }
  while (result != IBM_OK && cycles < opts->max_cycles) {
    if (graph) {
      IBM_TRY(cudaGraphLaunch((cudaGraphExec_t)h->graph_exec, st));
      ctx->launches += graph_launches;
    } else {
      body(st);
    }
    IBM_TRY(cudaGetLastError());
    IBM_TRY(cudaMemcpyAsync(ctx->hscal, ctx->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, st));
    IBM_TRY(cudaStreamSynchronize(st));
    ++cycles;
    rel = std::sqrt(ctx->hscal[S_NORM2]) / denom;
    if (info && info->resid_history && hl < info->history_cap) info->resid_history[hl++] = rel;
    if (!std::isfinite(rel) || rel > 1e6 * std::max(rel0, 1.0)) { result = IBM_ERR_DIVERGED; break; }
    if (rel <= tol) result = IBM_OK;
  }
  // gauge and unpack
  if (S.dfo)
    k_gauge_sum_df<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, st>>>(fine_view_df(h), hi_of(h->p64), lo_of(h->p64, ntot),
                                                             ctx->partials);
  else
    k_gauge_sum<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, st>>>(fine_view64(h), h->p64, ctx->partials);
  k_gauge_finalize<<<1, 256, 0, st>>>(ctx->partials, REDUCE_BLOCKS, ctx->scal);
  if (S.dfo)
    k_unpack_gauge_df<<<1216, 256, 0, st>>>(hi_of(h->p64), lo_of(h->p64, ntot), L0.mask, L0.g, ctx->scal, p_user);
  else
    k_unpack_gauge<<<nblk(n0, 256), 256, 0, st>>>(h->p64, L0.mask, L0.g, ctx->scal, p_user);
  ctx->launches += 3;
  IBM_TRY(cudaGetLastError());
  IBM_TRY(cudaMemcpyAsync(ctx->hscal, ctx->scal, sizeof(double) * NSCAL, cudaMemcpyDeviceToHost, st));
  int herr = 0;
  IBM_TRY(cudaMemcpyAsync(&herr, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  if (herr) {
    IBM_TRY(cudaMemsetAsync(ctx->errflag, 0, sizeof(int), st));
    result = IBM_ERR_TIMEOUT;
  }
  if (info) {
    info->cycles = cycles;
    info->history_len = hl;
    info->rel_resid = rel;
    info->lambda = ctx->hscal[S_LAMBDA];
  }
  return result;
}

ibm_status sweeps_impl(ibm_ctx *ctx, ibm_tables *t, int precision, int nsweeps, cudaStream_t st) {
  ibm_status s = build_hierarchy(t, precision, st);
  if (s != IBM_OK) return s;
  Hierarchy *h = t->hier[precision];
  Solver S{ctx, t, h, st, 1, 1, 1.0, h->dncoarse};
  Level &L0 = h->lv[0];
  if (precision == 0)
    smooth_level<double>(S, 0, h->p64, h->b64, ctx->scal + S_LAMBDA, true, nullptr, nsweeps);
  else
    smooth_level<float>(S, 0, reinterpret_cast<float *&>(L0.e), (const float *)L0.r, ctx->scal + S_MU, true,
                        (const float *)L0.r, nsweeps);
  IBM_TRY(cudaGetLastError());
  return IBM_OK;
}

}  // namespace ibm

#include "batch.cuh"
