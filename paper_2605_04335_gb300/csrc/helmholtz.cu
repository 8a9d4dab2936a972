// Advection-diffusion (Helmholtz-type) velocity solve of the fractional step, with no-slip
// ghost rows, by scheduled relaxed Jacobi (SRJ): Sec. "Governing Equations and Numerical
// Methods" (the momentum equation split into an advection-diffusion step solved with SRJ and
// the pressure Poisson equation), Sec. "Results and Discussions" (the diagonally dominant
// advection-diffusion system), Sec. "GPU Porting" item 2 (no-slip on the immersed surface).
//
// System (the paper gives no discretisation; reading): one velocity component u solves
//   fluid row i:  D_i u_i - alpha sum_d c_{i,d} v_nb = f_i,  D_i = 1 + alpha sum_d c_{i,d}
//                 (c: the pressure system's 7-point coefficients, zero across the walls;
//                 v_nb the neighbour, the ghost cell or, across a cut membrane link, the
//                 neighbour's entry on this cell's side)
//   ghost row G:  (1 + w_s) u_G + (1 - w_s) sum_k w_k v_k = 2 u_b
//                 (the boundary value at BI, the midpoint of the ghost centre and its image
//                 point; w_k the image-point weights divided by 1 - w_s, w_s the row's own
//                 weight moved to the left-hand side, 0 if none)
// SRJ cycle: K Jacobi sweeps of the fluid rows with relaxation factors w_k = 1 / lambda_k,
// lambda_k the Chebyshev nodes of [1 - rho, 1 + rho], rho = alpha S / (1 + alpha S) with S
// the largest sum of a cell's coefficients: the fluid rows' Jacobi spectrum lies in that
// interval (diagonal dominance); the step divides by D through an FP32 reciprocal (it scales
// the step only, so the fixed point is unchanged).  After every sweep the ghost rows are
// re-evaluated from the new fluid values (Jacobi among ghosts).  Precision 0 runs the cycles
// in FP64; precisions 1 and 2 run each cycle in FP32 on the correction equation H e = r
// inside iterative refinement, whose residual and update are FP64 (1) or double-FP32 pairs
// with error-free transformations on the FP32 pipe (2).  Convergence: ||S r|| / ||S b|| over
// fluid and ghost rows, S = alpha s_G on ghost rows (s_G the pressure system's row scale), 1 elsewhere.
//
// Layout: the finest level of the FP64 multigrid hierarchy of the tables (padded arrays,
// mask, ghost sources, membrane entry slots and cut-cell lists) is shared with the pressure
// solver; the velocity work arrays live in the hierarchy's own workspace.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "ibm_internal.cuh"

namespace ibm {

ibm_status build_hierarchy(ibm_tables *t, int precision, cudaStream_t st);

namespace {

constexpr int HZ_BLOCKS = REDUCE_BLOCKS;   // fixed grid of the norm kernels: deterministic sums
constexpr int HZ_THREADS = 256;
constexpr int TX = 32, TY = 8, KCH = 16;   // sweep tile (x, y) and z-planes per block

inline unsigned nb_of(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
struct HzView {
  int nx, ny, nz;
  long long sy, sz;
  const uint8_t *mask;
  const T *cxm, *cxp, *cym, *cyp, *czm, *czp;   // alpha x the face coefficients, per axis
  const T *sdx, *sdy, *sdz;                     // alpha x their per-axis sums
};

// relaxation divisor: 1 / D as an FP32 reciprocal (it scales the Jacobi step only, so the
// iteration's fixed point does not depend on its rounding)
template <typename T> __device__ __forceinline__ T relax_rcp(T D);
template <> __device__ __forceinline__ float relax_rcp<float>(float D) { return __frcp_rn(D); }
template <> __device__ __forceinline__ double relax_rcp<double>(double D) { return (double)__frcp_rn((float)D); }

// one Jacobi step of the fluid rows with relaxation w: un = u + w (f - H u) / D, each block a
// 32 x 8 tile marching KCH planes in z with the z-neighbours in registers; the next plane's
// value, mask and right-hand side are loaded one plane ahead
template <typename T>
__global__ void __launch_bounds__(TX *TY) k_hz_sweep(HzView<T> v, const T *u, T *un, const T *f, T w) {
  const int i = blockIdx.x * TX + threadIdx.x, j = blockIdx.y * TY + threadIdx.y;
  if (i >= v.nx || j >= v.ny) return;
  const int k0 = blockIdx.z * KCH, k1 = min(v.nz, k0 + KCH);
  const long long sy = v.sy, sz = v.sz;
  long long id = ((long long)(k0 + 1) * (v.ny + 2) + (j + 1)) * sy + (i + OX);
  const T cxm = v.cxm[i], cxp = v.cxp[i], cym = v.cym[j], cyp = v.cyp[j], dxy = (T)1 + (v.sdx[i] + v.sdy[j]);
  T zm = u[id - sz], zc = u[id], zp = u[id + sz], fc = f[id];
  uint8_t m = v.mask[id];
  for (int k = k0; k < k1; ++k, id += sz) {
    T zpp = 0, fn = 0;
    uint8_t mn = 1;
    if (k + 1 < k1) {   // planes k + 2 and k + 3 of the padded array exist when k + 1 < nz
      zpp = u[id + 2 * sz];
      fn = f[id + sz];
      mn = v.mask[id + sz];
    }
    const T xl = u[id - 1], xr = u[id + 1], yl = u[id - sy], yr = u[id + sy];
    T s = cxm * xl;
    s = fma(cxp, xr, s);
    s = fma(cym, yl, s);
    s = fma(cyp, yr, s);
    s = fma(v.czm[k], zm, s);
    s = fma(v.czp[k], zp, s);
    const T D = dxy + v.sdz[k];
    const T res = fma(-D, zc, fc) + s;
    if (m == 0) un[id] = fma(w * relax_rcp(D), res, zc);
    zm = zc;
    zc = zp;
    zp = zpp;
    fc = fn;
    m = mn;
  }
}

// the same step at the membrane cut cells (their links read the entries through cut_nb)
template <typename T>
__global__ void k_hz_sweep_cut(HzView<T> v, const long long *cut_id, const long long *cut_nb, const int *cut_ijk,
                               const long long *cnt, const T *u, T *un, const T *f, T w) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt[1];
       t += (long long)gridDim.x * blockDim.x) {
    const long long id = cut_id[t];
    const int i = cut_ijk[3 * t], j = cut_ijk[3 * t + 1], k = cut_ijk[3 * t + 2];
    const T c[6] = {v.cxm[i], v.cxp[i], v.cym[j], v.cyp[j], v.czm[k], v.czp[k]};
    T s = 0;
    for (int d = 0; d < 6; ++d) s = fma(c[d], u[cut_nb[6 * t + d]], s);
    const T D = ((T)1 + (v.sdx[i] + v.sdy[j])) + v.sdz[k];
    const T res = fma(-D, u[id], f[id]) + s;
    un[id] = fma(w * relax_rcp(D), res, u[id]);
  }
}

// ghost rows from the new fluid values and the previous ghost values:
// u_G = (b_G - (1 - w_s) sum w v) / (1 + w_s), b_G = f at the ghost's slot
template <typename T>
__global__ void k_hz_ghost(const long long *src, const long long *dst, const double *gw, const double *ws,
                           long long ng, T *un, const T *u, const T *f) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  T s = 0;
  for (int c = 0; c < 8; ++c) {
    const long long q = src[8 * g + c];
    if (q < 0) continue;
    const T v = (q & GHOST_CORNER) ? u[q & ~GHOST_CORNER] : un[q];
    s += (T)gw[8 * g + c] * v;
  }
  const T w = (T)ws[g];
  un[dst[g]] = (f[dst[g]] - ((T)1 - w) * s) / ((T)1 + w);
}

// FP64 residual r = b - H u of the regular fluid rows (coefficients pre-scaled by alpha);
// block partials of sum r^2 (and of sum b^2 when with_b); r32 (if given) receives r in FP32
__global__ void __launch_bounds__(HZ_THREADS) k_hz_resid(HzView<double> v, const double *u, const double *f,
                                                         float *r32, double *part, bool with_b) {
  __shared__ double sr[HZ_THREADS], sb[HZ_THREADS];
  double ar = 0.0, ab = 0.0;
  const long long rows = (long long)v.ny * v.nz;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = (int)(row % v.ny), k = (int)(row / v.ny);
    const long long base = ((long long)(k + 1) * (v.ny + 2) + (j + 1)) * v.sy + OX;
    const double cym = v.cym[j], cyp = v.cyp[j], czm = v.czm[k], czp = v.czp[k], syz = v.sdy[j] + v.sdz[k];
    for (int i = threadIdx.x; i < v.nx; i += blockDim.x) {
      const long long id = base + i;
      if (v.mask[id] != 0) continue;
      double acc = v.cxm[i] * u[id - 1];
      acc = fma(v.cxp[i], u[id + 1], acc);
      acc = fma(cym, u[id - v.sy], acc);
      acc = fma(cyp, u[id + v.sy], acc);
      acc = fma(czm, u[id - v.sz], acc);
      acc = fma(czp, u[id + v.sz], acc);
      const double D = 1.0 + (v.sdx[i] + syz);
      const double r = fma(-D, u[id], f[id]) + acc;
      if (r32) r32[id] = (float)r;
      ar += r * r;
      if (with_b) ab += f[id] * f[id];
    }
  }
  sr[threadIdx.x] = ar;
  sb[threadIdx.x] = ab;
  __syncthreads();
  for (int st = HZ_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) { sr[threadIdx.x] += sr[threadIdx.x + st]; sb[threadIdx.x] += sb[threadIdx.x + st]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = sr[0]; part[2 * blockIdx.x + 1] = sb[0]; }
}

// residual of the cut cells and of the ghost rows (scaled by alpha s_G), one block-partial
// pair per block after the regular rows' partials
// values of the refinement loop's u and f: FP64 arrays, or double-FP32 pairs (hi + lo)
struct Fp64Vals {
  const double *u, *f;
  __device__ double U(long long q) const { return u[q]; }
  __device__ double F(long long q) const { return f[q]; }
};
struct DfVals {
  const float *uh, *ul, *fh, *fl;
  __device__ double U(long long q) const { return dfl::join(uh[q], ul[q]); }
  __device__ double F(long long q) const { return dfl::join(fh[q], fl[q]); }
};

template <typename Vals>
__global__ void __launch_bounds__(HZ_THREADS) k_hz_resid_rest(
    HzView<double> v, const long long *cut_id, const long long *cut_nb, const int *cut_ijk, const long long *cnt,
    const long long *src, const long long *dst, const double *gw, const double *ws, const double *gscale,
    long long ng, Vals x, double alpha, float *r32, double *part, bool with_b) {
  __shared__ double sr[HZ_THREADS], sb[HZ_THREADS];
  double ar = 0.0, ab = 0.0;
  const long long ncut = cnt ? cnt[1] : 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ncut + ng;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < ncut) {
      const long long id = cut_id[t];
      const int i = cut_ijk[3 * t], j = cut_ijk[3 * t + 1], k = cut_ijk[3 * t + 2];
      const double c[6] = {v.cxm[i], v.cxp[i], v.cym[j], v.cyp[j], v.czm[k], v.czp[k]};
      double acc = 0.0;
      for (int d = 0; d < 6; ++d) acc = fma(c[d], x.U(cut_nb[6 * t + d]), acc);
      const double D = 1.0 + ((v.sdx[i] + v.sdy[j]) + v.sdz[k]);
      const double fi = x.F(id);
      const double r = fma(-D, x.U(id), fi) + acc;
      if (r32) r32[id] = (float)r;
      ar += r * r;
      if (with_b) ab += fi * fi;
    } else {
      const long long g = t - ncut;
      double s = 0.0;
      for (int c = 0; c < 8; ++c) {
        const long long q = src[8 * g + c];
        if (q >= 0) s += gw[8 * g + c] * x.U(q & ~GHOST_CORNER);
      }
      const long long id = dst[g];
      const double fi = x.F(id);
      const double r = fi - ((1.0 + ws[g]) * x.U(id) + (1.0 - ws[g]) * s);
      if (r32) r32[id] = (float)r;
      const double sc = alpha * gscale[g];
      ar += (sc * r) * (sc * r);
      if (with_b) ab += (sc * fi) * (sc * fi);
    }
  }
  sr[threadIdx.x] = ar;
  sb[threadIdx.x] = ab;
  __syncthreads();
  for (int st = HZ_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) { sr[threadIdx.x] += sr[threadIdx.x + st]; sb[threadIdx.x] += sb[threadIdx.x + st]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = sr[0]; part[2 * blockIdx.x + 1] = sb[0]; }
}

// out[0] = sum of the r^2 partials, out[1] = sum of the b^2 partials (fixed order): nreg
// pairs of the regular rows at part, nrest pairs of the other rows at part + 2 HZ_BLOCKS
__global__ void k_hz_norms(const double *part, int nreg, int nrest, double *out) {
  __shared__ double sr[HZ_THREADS], sb[HZ_THREADS];
  double ar = 0.0, ab = 0.0;
  for (int b = threadIdx.x; b < nreg + nrest; b += blockDim.x) {
    const int q = b < nreg ? b : HZ_BLOCKS + (b - nreg);
    ar += part[2 * q];
    ab += part[2 * q + 1];
  }
  sr[threadIdx.x] = ar;
  sb[threadIdx.x] = ab;
  __syncthreads();
  for (int st = HZ_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) { sr[threadIdx.x] += sr[threadIdx.x + st]; sb[threadIdx.x] += sb[threadIdx.x + st]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sr[0]; out[1] = sb[0]; }
}

// double-FP32 residual of the regular fluid rows (precision 2): u, f and alpha x the
// coefficients as hi + lo float pairs, r = f - D u + sum c v by error-free transformations
// on the FP32 pipe (the residual error is a few units of 2^-48 x sum |c| |v|); r32 receives
// r; block partials of sum r^2 (and sum f^2 when with_b)
struct HzDf {
  const float *ch, *cl;   // alpha x coefficients and sums (layout of HzView), hi and lo parts
};

__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &sh, float &sl) {
  float s, e;
  dfl::two_sum(ah, bh, s, e);
  e += al + bl;
  dfl::fast_two_sum(s, e, sh, sl);
}

__global__ void __launch_bounds__(HZ_THREADS) k_hz_resid_df(HzView<double> v, HzDf c, const float *uh,
                                                            const float *ul, const float *fh, const float *fl,
                                                            float *r32, double *part, bool with_b) {
  __shared__ double sr[HZ_THREADS], sb[HZ_THREADS];
  const int nx = v.nx, ny = v.ny, nz = v.nz, na = nx + ny + nz;
  const long long sy = v.sy, sz = v.sz;
  // coefficient offsets in the layout cxm cxp cym cyp czm czp (2 na) then sdx sdy sdz (na)
  const float *cxmh = c.ch, *cxml = c.cl, *cxph = c.ch + nx, *cxpl = c.cl + nx;
  const float *cyh = c.ch + 2 * nx, *cyl = c.cl + 2 * nx, *czh = c.ch + 2 * nx + 2 * ny, *czl = c.cl + 2 * nx + 2 * ny;
  const float *sdh = c.ch + 2 * na, *sdl = c.cl + 2 * na;
  double dr = 0.0, db = 0.0;
  // one warp per row, each lane four consecutive cells (16-byte loads: rows start at OX = 4 of
  // a 16-float pitch, so every group is aligned); the halo and padding masks are non-zero
  const int lane = threadIdx.x & 31;
  const long long rows = (long long)ny * nz, wstep = (long long)gridDim.x * (HZ_THREADS / 32);
  const int ngroups = (nx + 3) / 4;
  for (long long row = blockIdx.x * (long long)(HZ_THREADS / 32) + (threadIdx.x >> 5); row < rows; row += wstep) {
    const int j = (int)(row % ny), k = (int)(row / ny);
    const long long base = ((long long)(k + 1) * (ny + 2) + (j + 1)) * sy + OX;
    const float cymh = cyh[j], cyml = cyl[j], cyph = cyh[ny + j], cypl = cyl[ny + j];
    const float czmh = czh[k], czml = czl[k], czph = czh[nz + k], czpl = czl[nz + k];
    float dyzh, dyzl, t1h, t1l;
    df_add(1.0f, 0.0f, sdh[nx + j], sdl[nx + j], t1h, t1l);
    df_add(t1h, t1l, sdh[nx + ny + k], sdl[nx + ny + k], dyzh, dyzl);
    float ar = 0.f, ab = 0.f;
    for (int g = lane; g < ngroups; g += 32) {
      const long long id = base + 4 * g;
      const uchar4 m4 = *reinterpret_cast<const uchar4 *>(v.mask + id);
      const uint8_t mk[4] = {m4.x, m4.y, m4.z, m4.w};
      if (mk[0] && mk[1] && mk[2] && mk[3]) continue;
      const float4 ch4 = *reinterpret_cast<const float4 *>(uh + id), cl4 = *reinterpret_cast<const float4 *>(ul + id);
      const float4 f4h = *reinterpret_cast<const float4 *>(fh + id), f4l = *reinterpret_cast<const float4 *>(fl + id);
      const float Ch[6] = {uh[id - 1], ch4.x, ch4.y, ch4.z, ch4.w, uh[id + 4]};
      const float Cl[6] = {ul[id - 1], cl4.x, cl4.y, cl4.z, cl4.w, ul[id + 4]};
      const float Fh[4] = {f4h.x, f4h.y, f4h.z, f4h.w}, Fl[4] = {f4l.x, f4l.y, f4l.z, f4l.w};
      float R[4];
      // neighbours in y and z, one pair of 16-byte loads each, consumed one at a time
      float acc_h[4], acc_l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { acc_h[q] = Fh[q]; acc_l[q] = Fl[q]; }
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) {
        const long long off = nb == 0 ? -sy : (nb == 1 ? sy : (nb == 2 ? -sz : sz));
        const float4 h4 = *reinterpret_cast<const float4 *>(uh + id + off);
        const float4 l4 = *reinterpret_cast<const float4 *>(ul + id + off);
        const float H[4] = {h4.x, h4.y, h4.z, h4.w}, L[4] = {l4.x, l4.y, l4.z, l4.w};
        const float cH = nb == 0 ? cymh : (nb == 1 ? cyph : (nb == 2 ? czmh : czph));
        const float cL = nb == 0 ? cyml : (nb == 1 ? cypl : (nb == 2 ? czml : czpl));
#pragma unroll
        for (int q = 0; q < 4; ++q) dfl::acc_prod(cH, cL, H[q], L[q], acc_h[q], acc_l[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = min(4 * g + q, nx - 1);
        float Dh, Dl;
        df_add(dyzh, dyzl, sdh[i], sdl[i], Dh, Dl);
        dfl::acc_prod(-Dh, -Dl, Ch[q + 1], Cl[q + 1], acc_h[q], acc_l[q]);
        dfl::acc_prod(cxmh[i], cxml[i], Ch[q], Cl[q], acc_h[q], acc_l[q]);
        dfl::acc_prod(cxph[i], cxpl[i], Ch[q + 2], Cl[q + 2], acc_h[q], acc_l[q]);
        R[q] = acc_h[q] + acc_l[q];
        if (mk[q] == 0) {
          ar = fmaf(R[q], R[q], ar);
          if (with_b) { const float b = Fh[q] + Fl[q]; ab = fmaf(b, b, ab); }
        }
      }
      if (r32)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (mk[q] == 0) r32[id + q] = R[q];
    }
    dr += dfl::widen(ar);   // per row: the float sums of a lane's few groups
    if (with_b) db += dfl::widen(ab);
  }
  sr[threadIdx.x] = dr;
  sb[threadIdx.x] = db;
  __syncthreads();
  for (int st = HZ_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) { sr[threadIdx.x] += sr[threadIdx.x + st]; sb[threadIdx.x] += sb[threadIdx.x + st]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = sr[0]; part[2 * blockIdx.x + 1] = sb[0]; }
}

// (uh, ul) += e on every slot (double-FP32 update)
__global__ void k_hz_update_df(float *uh, float *ul, const float *e, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    float s, t;
    dfl::two_sum(uh[q], e[q], s, t);
    t += ul[q];
    dfl::fast_two_sum(s, t, uh[q], ul[q]);
  }
}

__global__ void k_hz_pack_df(const double *f, const double *u, long long ncell, int nx, int ny, LevelGeom g,
                             const uint8_t *mask, float *fh, float *fl, float *uh, float *ul) {
  // grid: (x blocks, ny, nz); no divisions
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const long long l = ((long long)k * ny + j) * nx + i;
  const long long id = pidx(g, i, j, k);
  const uint8_t m = mask[id];
  dfl::split(fluid_row(m) ? f[l] : 0.0, fh[id], fl[id]);
  dfl::split((fluid_row(m) || m == 3) ? u[l] : 0.0, uh[id], ul[id]);
}

__global__ void k_hz_ghost_rhs_df(const long long *dst, const double *ub, long long ng, float *fh, float *fl) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < ng) dfl::split(ub ? 2.0 * ub[g] : 0.0, fh[dst[g]], fl[dst[g]]);
}

__global__ void k_hz_unpack_df(const float *uh, const float *ul, long long ncell, int nx, int ny, LevelGeom g,
                               const uint8_t *mask, double *u) {
  // grid: (x blocks, ny, nz); no divisions
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const long long l = ((long long)k * ny + j) * nx + i;
  const long long id = pidx(g, i, j, k);
  const uint8_t m = mask[id];
  u[l] = (fluid_row(m) || m == 3) ? dfl::join(uh[id], ul[id]) : 0.0;
}

// user layout -> padded: f on fluid rows (0 elsewhere), u on fluid and ghost cells
__global__ void k_hz_pack(const double *f, const double *u, long long ncell, int nx, int ny, LevelGeom g,
                          const uint8_t *mask, double *fp, double *up) {
  // grid: (x blocks, ny, nz); no divisions
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const long long l = ((long long)k * ny + j) * nx + i;
  const long long id = pidx(g, i, j, k);
  const uint8_t m = mask[id];
  fp[id] = fluid_row(m) ? f[l] : 0.0;
  up[id] = (fluid_row(m) || m == 3) ? u[l] : 0.0;
}

// ghost-row right-hand sides 2 u_b at the ghosts' slots
__global__ void k_hz_ghost_rhs(const long long *dst, const double *ub, long long ng, double *fp) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < ng) fp[dst[g]] = ub ? 2.0 * ub[g] : 0.0;
}

__global__ void k_hz_unpack(const double *up, long long ncell, int nx, int ny, LevelGeom g, const uint8_t *mask,
                            double *u) {
  // grid: (x blocks, ny, nz); no divisions
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= nx) return;
  const long long l = ((long long)k * ny + j) * nx + i;
  const long long id = pidx(g, i, j, k);
  const uint8_t m = mask[id];
  u[l] = (fluid_row(m) || m == 3) ? up[id] : 0.0;
}

// u += e on every slot (e is zero off the active rows)
__global__ void k_hz_update(double *u, const float *e, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    u[q] += (double)e[q];
}

// alpha x the FP64 coefficients and their sums, in FP64 and as a double-FP32 pair (a32 the
// high part, the FP32 coefficients of the correction sweeps)
__global__ void k_scale_coefs(const double *c, long long n, double alpha, double *a64, float *a32, float *a32lo) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double x = alpha * c[q];
  a64[q] = x;
  dfl::split(x, a32[q], a32lo[q]);
}

// rigid boundary velocity of every ghost entry: u_b = v0 + omega x (BI - c) for the mesh of
// its closest triangle; out[d * ng + g]
constexpr int MAX_RIGID_V = 32;
struct RigidVel {
  int n;
  int off[MAX_RIGID_V + 1];
  double m[MAX_RIGID_V][9];   // v0 (3), omega (3), centre (3)
};

__global__ void k_rigid_velocity(const double *bi, const int *tri, long long ng, RigidVel M, double *out) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  int lo = 0, hi = M.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (M.off[mid] <= tri[g]) lo = mid; else hi = mid;
  }
  const double *mm = M.m[lo], *om = mm + 3;
  const double r[3] = {bi[3 * g] - mm[6], bi[3 * g + 1] - mm[7], bi[3 * g + 2] - mm[8]};
  out[g] = mm[0] + (om[1] * r[2] - om[2] * r[1]);
  out[ng + g] = mm[1] + (om[2] * r[0] - om[0] * r[2]);
  out[2 * ng + g] = mm[2] + (om[0] * r[1] - om[1] * r[0]);
}

// the largest sum of one cell's face coefficients along one axis (host, from the faces)
double axis_max_sum(const std::vector<double> &f) {
  const int n = (int)f.size() - 1;
  double best = 0.0;
  for (int i = 0; i < n; ++i) {
    const double ci = 0.5 * (f[i] + f[i + 1]), wi = f[i + 1] - f[i];
    double s = 0.0;
    if (i > 0) s += 1.0 / (wi * (ci - 0.5 * (f[i - 1] + f[i])));
    if (i < n - 1) s += 1.0 / (wi * (0.5 * (f[i + 1] + f[i + 2]) - ci));
    best = std::max(best, s);
  }
  return best;
}

struct HzWork {
  double *u[2], *f, *ac64;   // ac: alpha x coefficients and sums
  float *e[2], *r32, *ac32, *ac32lo;
  double *part, *norms;
};

}  // namespace

// time_ms non-null: after the setup, time n_timed launches of the sweep kernel alone (CUDA
// events on st around each launch; mean in *time_ms) instead of solving
ibm_status helmholtz_solve_impl(ibm_ctx *ctx, ibm_tables *t, double alpha, const double *f_user, const double *ub,
                                double tol, double *u_user, const ibm_helmholtz_opts *opts, ibm_solve_info *info,
                                cudaStream_t st, double *time_ms = nullptr, int n_timed = 0) {
  const auto t0 = std::chrono::steady_clock::now();
  ibm_helmholtz_opts o;
  ibm_helmholtz_opts_default(&o);
  if (opts) o = *opts;
  if (!f_user || !u_user || !(alpha >= 0.0) || !std::isfinite(alpha) || !(tol > 0.0) || o.precision < 0 ||
      o.precision > 2 || o.srj_steps < 1 || o.srj_steps > 64 || o.max_cycles < 1)
    return IBM_ERR_INVALID_ARG;
  if (t->ny > 65535 || t->nz > 65535) return IBM_ERR_CAPACITY;   // launch grid rows and planes
  ibm_status s = build_hierarchy(t, 0, st);
  if (s != IBM_OK) return s;
  Hierarchy *h = t->hier[0];
  Level &L0 = h->lv[0];
  const LevelGeom &G = L0.g;
  const long long nslot = h->nslot, ncell = t->ncell, ng = t->nghost;
  const int nx = G.nx, ny = G.ny, nz = G.nz, na = nx + ny + nz;
  // workspace: u (2), f in FP64; e (2), r in FP32; FP32 coefficients; partials; norms
  const long long want = nslot;
  const size_t na3 = ((3 * (size_t)na + 31) / 32) * 32;   // keeps the FP32 arrays 256-byte aligned
  const size_t bytes = sizeof(double) * (3 * (size_t)want + 2 * (size_t)HZ_BLOCKS * 2 + 8 + na3) +
                       sizeof(float) * (3 * (size_t)want + 2 * na3 + 64);
  if (!h->helm_buf || h->helm_n != want + na) {
    if (h->helm_buf) { IBM_TRY(cudaStreamSynchronize(st)); cudaFree(h->helm_buf); }
    h->helm_buf = nullptr;
    h->helm_n = 0;
    IBM_TRY(cudaMalloc(&h->helm_buf, bytes));
    IBM_TRY(cudaMemsetAsync(h->helm_buf, 0, bytes, st));   // halos and inactive cells stay 0
    h->helm_n = want + na;
    h->helm_layout = -1;
  }
  HzWork W;
  {
    double *d = (double *)h->helm_buf;
    W.u[0] = d; W.u[1] = d + want; W.f = d + 2 * want;
    W.part = d + 3 * want;
    W.norms = W.part + 2 * 2 * HZ_BLOCKS;
    W.ac64 = W.norms + 8;
    float *fl = (float *)(W.ac64 + na3);
    W.e[0] = fl; W.e[1] = fl + want; W.r32 = fl + 2 * want; W.ac32 = fl + 3 * want;
    W.ac32lo = W.ac32 + na3;
  }
  // views of the finest level: alpha x the hierarchy's FP64 coefficients, and FP32 copies
  long long launches = 0;
  k_scale_coefs<<<nb_of(3 * na, 256), 256, 0, st>>>(h->c64, 3 * na, alpha, W.ac64, W.ac32, W.ac32lo);
  ++launches;
  HzView<double> v64;
  {
    const double *c = W.ac64;
    v64.nx = nx; v64.ny = ny; v64.nz = nz; v64.sy = G.sy; v64.sz = G.sz; v64.mask = L0.mask;
    v64.cxm = c; v64.cxp = c + nx; v64.cym = c + 2 * nx; v64.cyp = v64.cym + ny;
    v64.czm = v64.cyp + ny; v64.czp = v64.czm + nz;
    v64.sdx = c + 2 * na; v64.sdy = v64.sdx + nx; v64.sdz = v64.sdy + ny;
  }
  HzView<float> v32;
  {
    const float *c = W.ac32;
    v32.nx = nx; v32.ny = ny; v32.nz = nz; v32.sy = G.sy; v32.sz = G.sz; v32.mask = L0.mask;
    v32.cxm = c; v32.cxp = c + nx; v32.cym = c + 2 * nx; v32.cyp = v32.cym + ny;
    v32.czm = v32.cyp + ny; v32.czp = v32.czm + nz;
    v32.sdx = c + 2 * na; v32.sdy = v32.sdx + nx; v32.sdz = v32.sdy + ny;
  }
  // pack f, u and the ghost rows' right-hand sides
  // precision 2: u and f as double-FP32 pairs in the same bytes (hi parts, then lo parts).
  // The packs write the cells only; halo and padding slots must read 0 in either view, so
  // the arrays are cleared whenever the layout changes.
  const bool df = o.precision == 2;
  const dim3 cell_grid(nb_of(nx, 256), ny, nz);   // pack / unpack: one thread per cell of a row
  float *uh = (float *)W.u[0], *ul = uh + want, *fh = (float *)W.f, *fl = fh + want;
  if (h->helm_layout != (df ? 1 : 0)) {
    IBM_TRY(cudaMemsetAsync(W.u[0], 0, sizeof(double) * 3 * (size_t)want, st));   // u[0], u[1], f
    h->helm_layout = df ? 1 : 0;
  }
  if (df)
    k_hz_pack_df<<<cell_grid, 256, 0, st>>>(f_user, u_user, ncell, nx, ny, G, L0.mask, fh, fl, uh, ul);
  else
    k_hz_pack<<<cell_grid, 256, 0, st>>>(f_user, u_user, ncell, nx, ny, G, L0.mask, W.f, W.u[0]);
  ++launches;
  if (ng > 0) {
    if (df) k_hz_ghost_rhs_df<<<nb_of(ng, 128), 128, 0, st>>>(h->gdst, ub, ng, fh, fl);
    else k_hz_ghost_rhs<<<nb_of(ng, 128), 128, 0, st>>>(h->gdst, ub, ng, W.f);
    ++launches;
  }
  const bool cuts = t->membrane && h->cut_id;
  const unsigned cut_blocks = cuts ? std::max(1u, std::min(nb_of(h->cutcap, 256), (unsigned)ctx->wave)) : 0;
  // SRJ relaxation factors: 1 / Chebyshev nodes of [1 - rho, 1 + rho]
  const double S = axis_max_sum(t->xf) + axis_max_sum(t->yf) + axis_max_sum(t->zf);
  const double rho = alpha * S / (1.0 + alpha * S);
  const int K = o.srj_steps;
  std::vector<double> om(K);
  for (int k = 0; k < K; ++k) om[k] = 1.0 / (1.0 + rho * std::cos(3.141592653589793 * (2.0 * k + 1.0) / (2.0 * K)));
  const dim3 sweep_grid(nb_of(nx, TX), nb_of(ny, TY), nb_of(nz, KCH)), sweep_block(TX, TY);
  const int rest_blocks = (int)std::max<long long>(1, std::min<long long>(HZ_BLOCKS, nb_of((cuts ? h->cutcap : 0) + ng, HZ_THREADS)));
  // the double-FP32 residual keeps 80 registers: three resident blocks per SM, one wave
  const int df_blocks = std::max(1, std::min(HZ_BLOCKS, 3 * std::max(1, ctx->sm_count)));
  // residual r = b - H u (FP64) with its norm, and the norm of b on the first call
  auto residual = [&](const double *u, float *r32, bool with_b) -> ibm_status {
    const long long *cnt = cuts ? h->d_cnt : nullptr;
    if (df) {
      const float *xh = (const float *)u, *xl = xh + want;
      k_hz_resid_df<<<df_blocks, HZ_THREADS, 0, st>>>(v64, HzDf{W.ac32, W.ac32lo}, xh, xl, fh, fl, r32, W.part, with_b);
      k_hz_resid_rest<DfVals><<<rest_blocks, HZ_THREADS, 0, st>>>(
          v64, h->cut_id, h->cut_nb, h->cut_ijk, cnt, h->gsrc, h->gdst, t->gw, t->gwself, t->gscale, ng,
          DfVals{xh, xl, fh, fl}, alpha, r32, W.part + 2 * HZ_BLOCKS, with_b);
    } else {
      k_hz_resid<<<HZ_BLOCKS, HZ_THREADS, 0, st>>>(v64, u, W.f, r32, W.part, with_b);
      k_hz_resid_rest<Fp64Vals><<<rest_blocks, HZ_THREADS, 0, st>>>(
          v64, h->cut_id, h->cut_nb, h->cut_ijk, cnt, h->gsrc, h->gdst, t->gw, t->gwself, t->gscale, ng,
          Fp64Vals{u, W.f}, alpha, r32, W.part + 2 * HZ_BLOCKS, with_b);
    }
    k_hz_norms<<<1, HZ_THREADS, 0, st>>>(W.part, df ? df_blocks : HZ_BLOCKS, rest_blocks, W.norms);
    launches += 3;
    IBM_TRY(cudaMemcpyAsync(ctx->hscal, W.norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    IBM_TRY(cudaStreamSynchronize(st));
    return IBM_OK;
  };
  // one SRJ cycle of K relaxed Jacobi steps on (u, rhs); returns the index of the current buffer
  auto srj_cycle = [&](auto *buf0, auto *buf1, const auto *rhs, auto view, int cur) -> int {
    using T = std::remove_const_t<std::remove_pointer_t<decltype(buf0)>>;
    T *b[2] = {buf0, buf1};
    for (int k = 0; k < K; ++k) {
      T *u = b[cur], *un = b[1 - cur];
      k_hz_sweep<T><<<sweep_grid, sweep_block, 0, st>>>(view, u, un, rhs, (T)om[k]);
      ++launches;
      if (cuts) {
        k_hz_sweep_cut<T><<<cut_blocks, 256, 0, st>>>(view, h->cut_id, h->cut_nb, h->cut_ijk, h->d_cnt, u, un, rhs,
                                                     (T)om[k]);
        ++launches;
      }
      if (ng > 0) {
        k_hz_ghost<T><<<nb_of(ng, 128), 128, 0, st>>>(h->gsrc, h->gdst, t->gw, t->gwself, ng, un, u, rhs);
        ++launches;
      }
      cur = 1 - cur;
    }
    return cur;
  };
  if (time_ms) {   // the sweep kernel alone, on the packed field (FP32: the correction arrays)
    std::vector<cudaEvent_t> ev(2 * (size_t)n_timed);
    for (auto &e : ev) IBM_TRY(cudaEventCreate(&e));
    for (int q = 0; q < n_timed; ++q) {
      IBM_TRY(cudaEventRecord(ev[2 * q], st));
      if (o.precision == 0)
        k_hz_sweep<double><<<sweep_grid, sweep_block, 0, st>>>(v64, W.u[q & 1], W.u[1 - (q & 1)], W.f, om[0]);
      else
        k_hz_sweep<float><<<sweep_grid, sweep_block, 0, st>>>(v32, W.e[q & 1], W.e[1 - (q & 1)], W.r32,
                                                              (float)om[0]);
      IBM_TRY(cudaEventRecord(ev[2 * q + 1], st));
    }
    IBM_TRY(cudaGetLastError());
    IBM_TRY(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (int q = 0; q < n_timed; ++q) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]);
      tot += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    *time_ms = tot / std::max(1, n_timed);
    ctx->launches += launches + n_timed;
    return IBM_OK;
  }
  ibm_status ret = IBM_OK;
  int cycles = 0, hist = 0;
  double rel = 0.0;
  if ((s = residual(W.u[0], o.precision >= 1 ? W.r32 : nullptr, true)) != IBM_OK) return s;
  const double bnorm = std::sqrt(ctx->hscal[1]);
  double r0 = std::sqrt(ctx->hscal[0]);
  int cur = 0;
  if (!std::isfinite(bnorm) || !std::isfinite(r0)) {
    ret = IBM_ERR_DIVERGED;
    rel = r0 / bnorm;
  } else if (bnorm == 0.0) {
    IBM_TRY(cudaMemsetAsync(W.u[0], 0, sizeof(double) * want, st));
    rel = 0.0;
  } else {
    rel = r0 / bnorm;
    while (rel > tol) {
      if (cycles >= o.max_cycles) { ret = IBM_ERR_NOT_CONVERGED; break; }
      if (o.precision == 0) {
        cur = srj_cycle(W.u[0], W.u[1], (const double *)W.f, v64, cur);
        if ((s = residual(W.u[cur], nullptr, false)) != IBM_OK) return s;
      } else {
        IBM_TRY(cudaMemsetAsync(W.e[0], 0, sizeof(float) * want, st));
        const int ec = srj_cycle(W.e[0], W.e[1], (const float *)W.r32, v32, 0);
        if (df) k_hz_update_df<<<ctx->wave, 256, 0, st>>>(uh, ul, W.e[ec], want);
        else k_hz_update<<<ctx->wave, 256, 0, st>>>(W.u[cur], W.e[ec], want);
        ++launches;
        if ((s = residual(W.u[cur], W.r32, false)) != IBM_OK) return s;
      }
      ++cycles;
      const double rn = std::sqrt(ctx->hscal[0]);
      rel = rn / bnorm;
      if (info && info->resid_history && hist < info->history_cap) info->resid_history[hist++] = rel;
      if (!std::isfinite(rel) || rn > 1e6 * std::max(r0, bnorm)) { ret = IBM_ERR_DIVERGED; break; }
    }
  }
  if (df) k_hz_unpack_df<<<cell_grid, 256, 0, st>>>(uh, ul, ncell, nx, ny, G, L0.mask, u_user);
  else k_hz_unpack<<<cell_grid, 256, 0, st>>>(W.u[cur], ncell, nx, ny, G, L0.mask, u_user);
  ++launches;
  IBM_TRY(cudaGetLastError());
  IBM_TRY(cudaStreamSynchronize(st));
  ctx->launches += launches;
  if (info) {
    info->cycles = cycles;
    info->history_len = hist;
    info->rel_resid = rel;
    info->lambda = 0.0;
    info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return ret;
}

ibm_status helmholtz_sweeps_timed_impl(ibm_ctx *ctx, ibm_tables *t, double alpha, int precision, int nsweeps,
                                       const double *f_user, double *u_user, cudaStream_t st, double *ms) {
  if (!ms || nsweeps < 1 || nsweeps > 4096) return IBM_ERR_INVALID_ARG;
  ibm_helmholtz_opts o;
  ibm_helmholtz_opts_default(&o);
  o.precision = precision;
  return helmholtz_solve_impl(ctx, t, alpha, f_user, nullptr, 1.0, u_user, &o, nullptr, st, ms, nsweeps);
}

ibm_status boundary_velocity_rigid_impl(ibm_tables *T, const double *motions, int nmesh, double *ub,
                                        cudaStream_t st) {
  if (nmesh < 1 || nmesh + 1 != (int)T->mesh_tri_off.size() || !motions || !ub) return IBM_ERR_INVALID_ARG;
  if (nmesh > MAX_RIGID_V) return IBM_ERR_CAPACITY;
  RigidVel M;
  M.n = nmesh;
  for (int m = 0; m <= nmesh; ++m) M.off[m] = T->mesh_tri_off[m];
  for (int m = 0; m < nmesh; ++m)
    for (int q = 0; q < 9; ++q) M.m[m][q] = motions[9 * m + q];
  const long long ng = T->nghost;
  if (ng > 0) {
    k_rigid_velocity<<<nb_of(ng, 256), 256, 0, st>>>(T->gbi, T->gtri, ng, M, ub);
    T->ctx->launches += 1;
  }
  IBM_TRY(cudaGetLastError());
  return IBM_OK;
}

}  // namespace ibm
