// Iblanking, ghost cells, boundary intercepts, image points and interpolation rows.
//
// Paper (arxiv 2605.04335) Sec. "GPU Porting": item 1 classifies the grid's voxels as
// interior or exterior of the triangulated body ("iblanking"); item 2 applies the
// internal boundary condition with the ghost-cell method.  The paper gives no formulas;
// this file implements the library's definition (stated in include/ibm_poisson.h):
//
//  * exact inside test on the integer lattice 2^-24: a centre is inside a closed mesh iff
//    an odd number of triangles cross its vertical line strictly below it; a triangle
//    covers a column by the half-open (top-left) rule of its xy-projection; centres on
//    the surface are fluid;
//  * ghost = solid cell with a fluid face-neighbour;
//  * BI = closest surface point (lowest triangle index on exact ties), IP = 2 BI - GC,
//    trilinear weights on the cell-centre lattice with invalid (plain solid) corners
//    dropped and renormalised, nearest-neighbour fallback, own weight moved left.
//
// This translation unit is compiled with -fmad=false: every floating-point expression
// is evaluated with separately rounded operations in the order written, and divisions
// are IEEE, so the FP64 outputs are reproducible bit for bit by any implementation that
// evaluates the same expressions in the same order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ibm_internal.cuh"

namespace ibm {
namespace {

constexpr double SNAP_SCALE = 16777216.0;   // 2^24
constexpr double COORD_LIMIT = 4.0;
constexpr double WEIGHT_SUM_MIN = 1e-3;
constexpr double SELF_WEIGHT_MAX = 1.0 - 1e-12;

__device__ __forceinline__ long long snapd(double x) { return __double2ll_rn(x * SNAP_SCALE); }

// first index with a[idx] > v (a ascending, n entries)
template <typename T>
__device__ __forceinline__ int upper_bound_dev(const T *a, int n, T v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] > v) hi = mid; else lo = mid + 1;
  }
  return lo;
}
// first index with a[idx] >= v
template <typename T>
__device__ __forceinline__ int lower_bound_dev(const T *a, int n, T v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] >= v) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ long long orient2d(long long ax, long long ay, long long bx, long long by,
                                              long long qx, long long qy) {
  return (bx - ax) * (qy - ay) - (by - ay) * (qx - ax);
}

__device__ __forceinline__ bool top_left(long long px, long long py, long long qx, long long qy) {
  return (qx > px) || (qx == px && py > qy);
}

// -------------------------------------------------------------------------- grid (step a1)

// centres, snapped centres, widths and the 7-point coefficients of one axis
__global__ void k_axis(const double *f, int n, double *c, long long *cs, double *w, double *cm, double *cp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ci = 0.5 * (f[i] + f[i + 1]);
  c[i] = ci;
  cs[i] = snapd(ci);
  double wi = f[i + 1] - f[i];
  w[i] = wi;
  double m = 0.0, p = 0.0;
  if (i > 0) {
    double cl = 0.5 * (f[i - 1] + f[i]);
    m = 1.0 / (wi * (ci - cl));
  }
  if (i < n - 1) {
    double cr = 0.5 * (f[i + 1] + f[i + 2]);
    p = 1.0 / (wi * (cr - ci));
  }
  cm[i] = m;
  cp[i] = p;
}

// -------------------------------------------------------------------------- inside test

struct Tri {
  long long a[3], b[3], c[3];   // snapped, counter-clockwise in xy when area > 0
  long long area;               // twice the projected area (> 0), or 0 if vertical
  int i0, i1, j0, j1, k0, k1;   // covered column / plane ranges (half-open)
  int kind;                     // 0 none, 1 projected, 2 vertical
};

__global__ void k_tri_setup(const double *verts, const int *tris, int ntri, const long long *Xs, int nx,
                            const long long *Ys, int ny, const long long *Zs, int nz, Tri *out,
                            long long *count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  Tri T;
  long long v[3][3];
  for (int q = 0; q < 3; ++q)
    for (int d = 0; d < 3; ++d) v[q][d] = snapd(verts[3 * tris[3 * t + q] + d]);
  for (int d = 0; d < 3; ++d) { T.a[d] = v[0][d]; T.b[d] = v[1][d]; T.c[d] = v[2][d]; }
  long long area = orient2d(T.a[0], T.a[1], T.b[0], T.b[1], T.c[0], T.c[1]);
  long long xl = min(T.a[0], min(T.b[0], T.c[0])), xh = max(T.a[0], max(T.b[0], T.c[0]));
  long long yl = min(T.a[1], min(T.b[1], T.c[1])), yh = max(T.a[1], max(T.b[1], T.c[1]));
  long long zl = min(T.a[2], min(T.b[2], T.c[2])), zh = max(T.a[2], max(T.b[2], T.c[2]));
  T.i0 = lower_bound_dev(Xs, nx, xl); T.i1 = upper_bound_dev(Xs, nx, xh);
  T.j0 = lower_bound_dev(Ys, ny, yl); T.j1 = upper_bound_dev(Ys, ny, yh);
  T.k0 = lower_bound_dev(Zs, nz, zl); T.k1 = upper_bound_dev(Zs, nz, zh);
  long long cnt = 0;
  T.kind = 0;
  if (area != 0) {
    if (area < 0) {
      for (int d = 0; d < 3; ++d) { long long s = T.b[d]; T.b[d] = T.c[d]; T.c[d] = s; }
      area = -area;
    }
    T.kind = 1;
    if (T.i1 > T.i0 && T.j1 > T.j0) cnt = (long long)(T.i1 - T.i0) * (T.j1 - T.j0);
  } else {
    long long abx = T.b[0] - T.a[0], aby = T.b[1] - T.a[1], abz = T.b[2] - T.a[2];
    long long acx = T.c[0] - T.a[0], acy = T.c[1] - T.a[1], acz = T.c[2] - T.a[2];
    long long nxv = aby * acz - abz * acy, nyv = abz * acx - abx * acz;
    if ((nxv != 0 || nyv != 0) && T.i1 > T.i0 && T.j1 > T.j0 && T.k1 > T.k0) {
      T.kind = 2;
      cnt = (long long)(T.i1 - T.i0) * (T.j1 - T.j0) * (T.k1 - T.k0);
    }
  }
  T.area = area;
  out[t] = T;
  count[t] = cnt;
}

// exclusive scan of n int64 counts in one block; out has n+1 entries
__global__ void k_scan_single(const long long *in, long long *out, int n) {
  __shared__ long long part[1024];
  int tid = threadIdx.x, nt = blockDim.x;
  int per = (n + nt - 1) / nt;
  int b = tid * per, e = min(n, b + per);
  long long s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    long long run = 0;
    for (int i = 0; i < nt; ++i) { long long v = part[i]; part[i] = run; run += v; }
    out[n] = run;
  }
  __syncthreads();
  long long run = part[tid];
  for (int i = b; i < e; ++i) { out[i] = run; run += in[i]; }
}

__device__ __forceinline__ bool in_closed_tri2d(long long pu0, long long pv0, long long pu1, long long pv1,
                                                long long pu2, long long pv2, long long qu, long long qv) {
  long long e0 = orient2d(pu0, pv0, pu1, pv1, qu, qv);
  long long e1 = orient2d(pu1, pv1, pu2, pv2, qu, qv);
  long long e2 = orient2d(pu2, pv2, pu0, pv0, qu, qv);
  return (e0 >= 0 && e1 >= 0 && e2 >= 0) || (e0 <= 0 && e1 <= 0 && e2 <= 0);
}

__global__ void k_tri_pairs(const Tri *tris, const long long *off, int ntri, long long total,
                            const long long *Xs, const long long *Ys, const long long *Zs, int nx, int ny,
                            int nz, int words, unsigned *toggles, unsigned *onsurf) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    int t = upper_bound_dev(off, ntri + 1, p) - 1;
    const Tri &T = tris[t];
    long long local = p - off[t];
    int ni = T.i1 - T.i0, nj = T.j1 - T.j0;
    int i = T.i0 + (int)(local % ni);
    long long rest = local / ni;
    int j = T.j0 + (int)(rest % nj);
    long long col = (long long)j * nx + i;
    long long qx = Xs[i], qy = Ys[j];
    if (T.kind == 1) {
      long long wa = orient2d(T.b[0], T.b[1], T.c[0], T.c[1], qx, qy);
      long long wb = orient2d(T.c[0], T.c[1], T.a[0], T.a[1], qx, qy);
      long long wc = orient2d(T.a[0], T.a[1], T.b[0], T.b[1], qx, qy);
      bool cov = (wa > 0 || (wa == 0 && top_left(T.b[0], T.b[1], T.c[0], T.c[1]))) &&
                 (wb > 0 || (wb == 0 && top_left(T.c[0], T.c[1], T.a[0], T.a[1]))) &&
                 (wc > 0 || (wc == 0 && top_left(T.a[0], T.a[1], T.b[0], T.b[1])));
      if (!cov) continue;
      __int128 N = (__int128)wa * T.a[2] + (__int128)wb * T.b[2] + (__int128)wc * T.c[2];
      __int128 D = (__int128)T.area;
      __int128 q = N / D;
      __int128 r = N - q * D;
      if (r != 0 && N < 0) q -= 1;          // floor division (D > 0)
      long long qz = (long long)q;
      int ks = upper_bound_dev(Zs, nz, qz);  // first centre strictly above the crossing
      atomicXor(&toggles[col * words + (ks >> 5)], 1u << (ks & 31));
      if (r == 0 && ks >= 1 && Zs[ks - 1] == qz)
        atomicOr(&onsurf[col * words + ((ks - 1) >> 5)], 1u << ((ks - 1) & 31));
    } else if (T.kind == 2) {
      int k = T.k0 + (int)(rest / nj);
      // the projection is a segment: the column must lie on its line
      long long p0x = T.a[0], p0y = T.a[1], p1x = T.b[0], p1y = T.b[1];
      if (p0x == p1x && p0y == p1y) { p1x = T.c[0]; p1y = T.c[1]; }
      if (orient2d(p0x, p0y, p1x, p1y, qx, qy) != 0) continue;
      long long abx = T.b[0] - T.a[0], abz = T.b[2] - T.a[2], acx = T.c[0] - T.a[0], acz = T.c[2] - T.a[2];
      long long nyv = abz * acx - abx * acz;
      bool use_x = nyv != 0;
      long long qu = use_x ? qx : qy, qv = Zs[k];
      long long u0 = use_x ? T.a[0] : T.a[1], u1 = use_x ? T.b[0] : T.b[1], u2 = use_x ? T.c[0] : T.c[1];
      if (in_closed_tri2d(u0, T.a[2], u1, T.b[2], u2, T.c[2], qu, qv))
        atomicOr(&onsurf[col * words + (k >> 5)], 1u << (k & 31));
    }
  }
}

// per column: prefix parity of the toggles; solid where odd and not on the surface.
// Clears the column's bit words for the next mesh.  A watertight surface crosses every
// vertical line an even number of times (each crossing counted once by the top-left rule),
// so an odd total over the column -- the parity of all its toggle bits, the slot above the
// top centre included -- marks a surface with a hole on that line: *leak is set.
__global__ void k_parity(unsigned *toggles, unsigned *onsurf, int words, int nx, int ny, int nz, int i0, int i1,
                         int j0, int j1, uint8_t *iblank, unsigned *leak) {
  int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
  int j = j0 + blockIdx.y;
  if (i >= i1 || j >= j1) return;
  long long col = (long long)j * nx + i;
  unsigned par = 0, total = 0;
  for (int w = 0; w < words; ++w) {
    unsigned tg = toggles[col * words + w], os = onsurf[col * words + w];
    total ^= (unsigned)__popc(tg) & 1u;
    if (tg == 0 && os == 0 && par == 0) continue;
    toggles[col * words + w] = 0u;
    onsurf[col * words + w] = 0u;
    for (int b = 0; b < 32; ++b) {
      int k = w * 32 + b;
      if (k >= nz) break;
      par ^= (tg >> b) & 1u;
      if (par && !((os >> b) & 1u)) iblank[((long long)k * ny + j) * nx + i] = 1;
    }
  }
  if (total) atomicOr(leak, 1u);
}

// -------------------------------------------------------------------------- ghost marking

constexpr int GM_THREADS = 256;
constexpr int GM_PER = 16;   // cells per thread; contiguous runs keep the output sorted

__device__ __forceinline__ bool is_ghost(const uint8_t *ib, int nx, int ny, int nz, long long l) {
  if ((ib[l] & 1) == 0) return false;
  int i = (int)(l % nx);
  long long r = l / nx;
  int j = (int)(r % ny);
  int k = (int)(r / ny);
  long long sy = nx, sz = (long long)nx * ny;
  if (i > 0 && (ib[l - 1] & 1) == 0) return true;
  if (i < nx - 1 && (ib[l + 1] & 1) == 0) return true;
  if (j > 0 && (ib[l - sy] & 1) == 0) return true;
  if (j < ny - 1 && (ib[l + sy] & 1) == 0) return true;
  if (k > 0 && (ib[l - sz] & 1) == 0) return true;
  if (k < nz - 1 && (ib[l + sz] & 1) == 0) return true;
  return false;
}

__global__ void k_ghost_count(const uint8_t *ib, int nx, int ny, int nz, long long ncell, long long *bcount) {
  __shared__ int s[GM_THREADS];
  long long base = (long long)blockIdx.x * GM_THREADS * GM_PER + (long long)threadIdx.x * GM_PER;
  int c = 0;
  for (int q = 0; q < GM_PER; ++q) {
    long long l = base + q;
    if (l < ncell && is_ghost(ib, nx, ny, nz, l)) ++c;
  }
  s[threadIdx.x] = c;
  __syncthreads();
  for (int st = GM_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) bcount[blockIdx.x] = s[0];
}

__global__ void k_ghost_scatter(const uint8_t *ib, int nx, int ny, int nz, long long ncell, const long long *boff,
                                long long *gcell) {
  __shared__ int s[GM_THREADS];
  long long base = (long long)blockIdx.x * GM_THREADS * GM_PER + (long long)threadIdx.x * GM_PER;
  unsigned bits = 0;
  int c = 0;
  for (int q = 0; q < GM_PER; ++q) {
    long long l = base + q;
    if (l < ncell && is_ghost(ib, nx, ny, nz, l)) { bits |= 1u << q; ++c; }
  }
  s[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < GM_THREADS; ++t) { int v = s[t]; s[t] = run; run += v; }
  }
  __syncthreads();
  long long o = boff[blockIdx.x] + s[threadIdx.x];
  for (int q = 0; q < GM_PER; ++q)
    if (bits & (1u << q)) gcell[o++] = base + q;
}

__global__ void k_ghost_bits(uint8_t *ib, const long long *gcell, long long ng) {
  long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < ng) ib[gcell[g]] |= 2;
}

__global__ void k_count_cells(const uint8_t *ib, long long n, unsigned long long *cnt) {
  __shared__ unsigned long long s[2][256];
  unsigned long long f = 0, so = 0;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n; l += (long long)gridDim.x * blockDim.x) {
    uint8_t v = ib[l];
    if (v == 0) ++f; else if (v == 1) ++so;
  }
  s[0][threadIdx.x] = f; s[1][threadIdx.x] = so;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) { s[0][threadIdx.x] += s[0][threadIdx.x + st]; s[1][threadIdx.x] += s[1][threadIdx.x + st]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { atomicAdd(&cnt[0], s[0][0]); atomicAdd(&cnt[1], s[1][0]); }
}

// -------------------------------------------------------------------------- image points

// Closest point of P on triangle ABC and its squared distance.  Interior: the stationary
// point of |P - (A + u ab + v ac)|^2 (normal equations [a b; b c][u v]' = [d e]') when it
// lies in the triangle; otherwise the best projection onto the edges AB, BC, CA.
__device__ void closest_on_tri(const double P[3], const double *A, const double *B, const double *C, double Q[3],
                               double &d2) {
  double abx = B[0] - A[0], aby = B[1] - A[1], abz = B[2] - A[2];
  double acx = C[0] - A[0], acy = C[1] - A[1], acz = C[2] - A[2];
  double apx = P[0] - A[0], apy = P[1] - A[1], apz = P[2] - A[2];
  double a = (abx * abx + aby * aby) + abz * abz;
  double b = (abx * acx + aby * acy) + abz * acz;
  double c = (acx * acx + acy * acy) + acz * acz;
  double d = (abx * apx + aby * apy) + abz * apz;
  double e = (acx * apx + acy * apy) + acz * apz;
  double det = a * c - b * b;
  double su = c * d - b * e;
  double sv = a * e - b * d;
  if (det > 0 && su >= 0 && sv >= 0 && su + sv <= det) {
    double u = su / det, v = sv / det;
    Q[0] = (A[0] + u * abx) + v * acx;
    Q[1] = (A[1] + u * aby) + v * acy;
    Q[2] = (A[2] + u * abz) + v * acz;
  } else {
    const double *E0[3] = {A, B, C};
    const double *E1[3] = {B, C, A};
    double best = 0.0;
    for (int s = 0; s < 3; ++s) {
      const double *P0 = E0[s], *P1 = E1[s];
      double ex = P1[0] - P0[0], ey = P1[1] - P0[1], ez = P1[2] - P0[2];
      double px = P[0] - P0[0], py = P[1] - P0[1], pz = P[2] - P0[2];
      double num = (ex * px + ey * py) + ez * pz;
      double den = (ex * ex + ey * ey) + ez * ez;
      double q0, q1, q2;
      if (num <= 0 || den <= 0) { q0 = P0[0]; q1 = P0[1]; q2 = P0[2]; }
      else if (num >= den) { q0 = P1[0]; q1 = P1[1]; q2 = P1[2]; }
      else {
        double t = num / den;
        q0 = P0[0] + t * ex; q1 = P0[1] + t * ey; q2 = P0[2] + t * ez;
      }
      double dx = P[0] - q0, dy = P[1] - q1, dz = P[2] - q2;
      double de = (dx * dx + dy * dy) + dz * dz;
      if (s == 0 || de < best) { best = de; Q[0] = q0; Q[1] = q1; Q[2] = q2; }
    }
  }
  double dx = P[0] - Q[0], dy = P[1] - Q[1], dz = P[2] - Q[2];
  d2 = (dx * dx + dy * dy) + dz * dz;
}

__device__ __forceinline__ float box_dist2(const float p[3], float4 lo, float4 hi) {
  float dx = fmaxf(fmaxf(lo.x - p[0], 0.0f), p[0] - hi.x);
  float dy = fmaxf(fmaxf(lo.y - p[1], 0.0f), p[1] - hi.y);
  float dz = fmaxf(fmaxf(lo.z - p[2], 0.0f), p[2] - hi.z);
  return dx * dx + dy * dy + dz * dz;
}

// Uniform cubic bins (edge h, origin lo, nb[d] per axis) over the triangles' bounding box:
// each triangle is listed in every bin that its box, widened by BIN_MARGIN, meets.  A search
// that has visited every bin within distance L of a point has therefore seen every triangle
// within L of it.
struct TriBins {
  double lo[3];
  double h, inv;
  int nb[3];
  const long long *off;   // nb[0] nb[1] nb[2] + 1 offsets into tri
  const int *tri;         // triangle indices, bin by bin
  const uint2 *range;     // per triangle: first (x) and last (y) bin per axis, one byte each
};

// does triangle t's bin range meet the box of bins [l, h] (per axis)?  first: the range's
// first bin inside the box
__device__ __forceinline__ bool range_meets(uint2 rg, const int l[3], const int h[3], int first[3]) {
  bool ok = true;
  for (int d = 0; d < 3; ++d) {
    const int a = (int)((rg.x >> (8 * d)) & 0xffu), b = (int)((rg.y >> (8 * d)) & 0xffu);
    first[d] = max(a, l[d]);
    ok = ok && first[d] <= min(b, h[d]);
  }
  return ok;
}
constexpr double BIN_MARGIN = 1e-9;

// bins met by the box [l, h] widened by BIN_MARGIN (clamped to the grid)
__device__ __forceinline__ void box_bin_range(const double l[3], const double h[3], const TriBins &B, int i0[3],
                                              int i1[3]) {
  for (int d = 0; d < 3; ++d) {
    const double a = floor((l[d] - B.lo[d] - BIN_MARGIN) * B.inv), b = floor((h[d] - B.lo[d] + BIN_MARGIN) * B.inv);
    const double top = (double)(B.nb[d] - 1);
    i0[d] = (int)fmin(fmax(a, 0.0), top);
    i1[d] = (int)fmin(fmax(b, 0.0), top);
  }
}

__device__ __forceinline__ void tri_bin_range(const double *v, const TriBins &B, int i0[3], int i1[3]) {
  double l[3], h[3];
  for (int d = 0; d < 3; ++d) {
    l[d] = fmin(v[d], fmin(v[3 + d], v[6 + d]));
    h[d] = fmax(v[d], fmax(v[3 + d], v[6 + d]));
  }
  box_bin_range(l, h, B, i0, i1);
}

__global__ void k_bin_count(const double *tv, int ntri, TriBins B, long long *cnt, uint2 *range) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  int i0[3], i1[3];
  tri_bin_range(tv + 9 * t, B, i0, i1);
  range[t] = make_uint2((unsigned)i0[0] | ((unsigned)i0[1] << 8) | ((unsigned)i0[2] << 16),
                        (unsigned)i1[0] | ((unsigned)i1[1] << 8) | ((unsigned)i1[2] << 16));
  for (int k = i0[2]; k <= i1[2]; ++k)
    for (int j = i0[1]; j <= i1[1]; ++j)
      for (int i = i0[0]; i <= i1[0]; ++i)
        atomicAdd(reinterpret_cast<unsigned long long *>(cnt) + ((long long)k * B.nb[1] + j) * B.nb[0] + i, 1ULL);
}

// the order inside a bin is arbitrary: the search's result does not depend on it
__global__ void k_bin_fill(const double *tv, int ntri, TriBins B, const long long *off, long long *cur, int *tri) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  int i0[3], i1[3];
  tri_bin_range(tv + 9 * t, B, i0, i1);
  for (int k = i0[2]; k <= i1[2]; ++k)
    for (int j = i0[1]; j <= i1[1]; ++j)
      for (int i = i0[0]; i <= i1[0]; ++i) {
        const long long b = ((long long)k * B.nb[1] + j) * B.nb[0] + i;
        tri[off[b] + (long long)atomicAdd(reinterpret_cast<unsigned long long *>(cur) + b, 1ULL)] = t;
      }
}

struct GhostArgs {
  int nx, ny, nz;
  const double *xc, *yc, *zc;
  const double *cxm, *cxp, *cym, *cyp, *czm, *czp;
  const uint8_t *ib;
  const double *tv;        // ntri x 9 vertex coordinates
  const float4 *blo, *bhi; // triangle boxes, outward-rounded to float
  const float4 *cen;       // triangle centroids (float)
  TriBins bins;
  long long ng;
  const long long *gcell;
  double *bi, *ip, *w, *scale;
  int *base, *flags;
  long long *ref;
  double *kappa;           // Neumann coefficient of each row
  int *tri;                // closest triangle of each ghost
  double *wself;           // the row's own weight where moved to the left-hand side, else 0
};

__device__ __forceinline__ void base_t(const double *c, int n, double v, int &i0, double &t) {
  int b = upper_bound_dev(c, n, v) - 1;
  b = b < 0 ? 0 : (b > n - 2 ? n - 2 : b);
  i0 = b;
  double tt = (v - c[b]) / (c[b + 1] - c[b]);
  t = tt < 0.0 ? 0.0 : (tt > 1.0 ? 1.0 : tt);
}

// one warp per ghost: the lanes split the triangle loops, then a warp reduction picks the
// minimum squared distance (lowest triangle index on exact ties), the same result as a
// sequential scan; lane 0 finishes the row
__device__ __forceinline__ void warp_argmin(double &d, int &t, float &f) {
  for (int o = 16; o > 0; o >>= 1) {
    double od = __shfl_xor_sync(0xffffffffu, d, o);
    int ot = __shfl_xor_sync(0xffffffffu, t, o);
    if (od < d || (od == d && ot < t)) { d = od; t = ot; }
  }
  (void)f;
}

// per-warp candidate list of the closest-triangle search (shared memory)
constexpr int CAND_MAX = 64;
constexpr int TABLE_THREADS = 128;

// The closest triangle to P (minimum squared distance, lowest index on exact ties) and the
// closest point Q on it: the warp visits the bins in Chebyshev shells around P's bin (first
// the whole 3 x 3 x 3 block, then r = 2, 3, ...) and stops once every unvisited bin lies
// farther than the best distance found (plus a margin covering the float boxes).  In a
// shell a triangle is taken once, from the first bin of its range inside the visited block,
// and only if no earlier shell met its range.  The nearest centroid bounds the distance
// first; triangles whose box is not farther than the bound are gathered into the warp's
// list cq and evaluated exactly, spread over the lanes.  Every triangle that could be the
// minimum or tie with it is evaluated, so the result equals a scan over all triangles.
// Every lane returns the result.
__device__ void find_closest(const GhostArgs &a, const double P[3], int lane, double &best, int &bidx, double Q[3],
                             int *cq) {
  const TriBins &B = a.bins;
  const float Pf[3] = {(float)P[0], (float)P[1], (float)P[2]};
  int c[3];
  for (int d = 0; d < 3; ++d)
    c[d] = (int)fmin(fmax(floor((P[d] - B.lo[d]) * B.inv), 0.0), (double)(B.nb[d] - 1));
  double lb = 1e300, lq[3] = {0.0, 0.0, 0.0};   // this lane's best
  int lt = 0x7fffffff;
  best = 1e300;
  bidx = 0x7fffffff;
  double thr = 1e300;
  auto consider = [&](int t) {
    double d2, Qt[3];
    closest_on_tri(P, a.tv + 9 * t, a.tv + 9 * t + 3, a.tv + 9 * t + 6, Qt, d2);
    if (d2 < lb || (d2 == lb && t < lt)) {
      lb = d2; lt = t;
      lq[0] = Qt[0]; lq[1] = Qt[1]; lq[2] = Qt[2];
    }
  };
  for (int r = 1;; ++r) {
    const int w = 2 * r + 1;
    const long long ncube = (long long)w * w * w;
    int vl[3], vh[3], pl[3], ph[3];   // visited block after this shell, and before it
    for (int d = 0; d < 3; ++d) {
      vl[d] = max(c[d] - r, 0); vh[d] = min(c[d] + r, B.nb[d] - 1);
      pl[d] = max(c[d] - r + 1, 0); ph[d] = min(c[d] + r - 1, B.nb[d] - 1);
    }
    auto shell_bin = [&](long long q, int bc[3]) -> long long {   // bin of cube cell q, or -1
      const int dx = (int)(q % w) - r, dy = (int)((q / w) % w) - r, dz = (int)(q / ((long long)w * w)) - r;
      if (r > 1 && max(abs(dx), max(abs(dy), abs(dz))) != r) return -1;
      bc[0] = c[0] + dx; bc[1] = c[1] + dy; bc[2] = c[2] + dz;
      if (bc[0] < 0 || bc[1] < 0 || bc[2] < 0 || bc[0] >= B.nb[0] || bc[1] >= B.nb[1] || bc[2] >= B.nb[2]) return -1;
      return ((long long)bc[2] * B.nb[1] + bc[1]) * B.nb[0] + bc[0];
    };
    // is this the triangle's own visit: the first bin of its range in the block, and its
    // range did not meet the block of the earlier shells
    auto own_visit = [&](int t, const int bc[3]) {
      const uint2 rg = B.range[t];
      int f[3], g[3];
      range_meets(rg, vl, vh, f);
      if (f[0] != bc[0] || f[1] != bc[1] || f[2] != bc[2]) return false;
      return r == 1 || !range_meets(rg, pl, ph, g);
    };
    // the distance to a centroid bounds the distance to its triangle (relative margin for
    // the float arithmetic)
    float cb = 3.4e38f;
    for (long long q = lane; q < ncube; q += 32) {
      int bc[3];
      const long long bin = shell_bin(q, bc);
      if (bin < 0) continue;
      for (long long e = B.off[bin]; e < B.off[bin + 1]; ++e) {
        const float4 cc = a.cen[B.tri[e]];
        const float dx = cc.x - Pf[0], dy = cc.y - Pf[1], dz = cc.z - Pf[2];
        cb = fminf(cb, dx * dx + dy * dy + dz * dz);
      }
    }
    for (int o = 16; o > 0; o >>= 1) cb = fminf(cb, __shfl_xor_sync(0xffffffffu, cb, o));
    if (cb < 3.4e38f) thr = fmin(thr, sqrt((double)cb) * (1.0 + 1e-5) + 4e-6);
    const double thr2 = thr * thr;
    // chunks of 32 bins: candidates into the list (a lane whose share does not fit
    // evaluates the rest itself), then the list over the lanes
    for (long long q0 = 0; q0 < ncube; q0 += 32) {
      const long long q = q0 + lane;
      int bc[3];
      const long long bin = q < ncube ? shell_bin(q, bc) : -1;
      int n = 0;
      if (bin >= 0)
        for (long long e = B.off[bin]; e < B.off[bin + 1]; ++e) {
          const int t = B.tri[e];
          if ((double)box_dist2(Pf, a.blo[t], a.bhi[t]) <= thr2 && own_visit(t, bc)) ++n;
        }
      int pre = n;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
      }
      const int total = __shfl_sync(0xffffffffu, pre, 31);
      pre -= n;
      if (n > 0) {
        int k = pre;
        for (long long e = B.off[bin]; e < B.off[bin + 1]; ++e) {
          const int t = B.tri[e];
          if ((double)box_dist2(Pf, a.blo[t], a.bhi[t]) > thr2 || !own_visit(t, bc)) continue;
          if (k < CAND_MAX) cq[k] = t;
          else consider(t);
          ++k;
        }
      }
      __syncwarp();
      for (int k = lane; k < min(total, CAND_MAX); k += 32) consider(cq[k]);
      __syncwarp();
    }
    best = lb;
    bidx = lt;
    float unused = 0.f;
    warp_argmin(best, bidx, unused);
    thr = sqrt(best) + 4e-6;
    // distance from P to the bins outside the visited cube
    double lv = 1e300;
    bool more = false;
    for (int d = 0; d < 3; ++d) {
      if (c[d] - r - 1 >= 0) { more = true; lv = fmin(lv, P[d] - (B.lo[d] + (c[d] - r) * B.h)); }
      if (c[d] + r + 1 < B.nb[d]) { more = true; lv = fmin(lv, (B.lo[d] + (c[d] + r + 1) * B.h) - P[d]); }
    }
    if (!more || lv > thr) break;
  }
  // the closest point from a lane that evaluated the winning triangle (same arithmetic on
  // every lane, so any of them)
  const unsigned own = __ballot_sync(0xffffffffu, lt == bidx && lb == best);
  const int src = own ? __ffs(own) - 1 : 0;
  for (int d = 0; d < 3; ++d) Q[d] = __shfl_sync(0xffffffffu, lq[d], src);
}

// Neumann coefficient of a row (moving-boundary datum): g = p(IP) - l q with l = |IP - GC|
// and q the derivative along (IP - GC) / l, so g - sum w v = kappa q, kappa = -l, divided by
// 1 - w_self when the row's own weight was moved to the left-hand side
__device__ __forceinline__ double row_kappa(const double P[3], const double IP[3], bool moved, double wself) {
  const double ex = IP[0] - P[0], ey = IP[1] - P[1], ez = IP[2] - P[2];
  const double l = sqrt((ex * ex + ey * ey) + ez * ez);
  return moved ? -l / (1.0 - wself) : -l;
}

// a nearest-neighbour fallback row: l = |centre(nb) - GC| (0 without a neighbour)
__device__ __forceinline__ double fallback_kappa(const GhostArgs &a, const double P[3], long long nb) {
  if (nb < 0) return 0.0;
  const int i = (int)(nb % a.nx), j = (int)((nb / a.nx) % a.ny), k = (int)(nb / ((long long)a.nx * a.ny));
  const double fx = a.xc[i] - P[0], fy = a.yc[j] - P[1], fz = a.zc[k] - P[2];
  return -sqrt((fx * fx + fy * fy) + fz * fz);
}

__global__ void __launch_bounds__(TABLE_THREADS) k_ghost_tables(GhostArgs a) {
  __shared__ int cand[TABLE_THREADS / 32][CAND_MAX];
  const int lane = threadIdx.x & 31;
  long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (g >= a.ng) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  long long lin = a.gcell[g];
  int gi = (int)(lin % nx);
  int gj = (int)((lin / nx) % ny);
  int gk = (int)(lin / ((long long)nx * ny));
  double P[3] = {a.xc[gi], a.yc[gj], a.zc[gk]};
  double best, BQ[3];
  int bidx;
  find_closest(a, P, lane, best, bidx, BQ, cand[threadIdx.x >> 5]);
  if (lane != 0) return;
  double IP[3];
  for (int d = 0; d < 3; ++d) {
    IP[d] = (BQ[d] + BQ[d]) - P[d];
    a.bi[3 * g + d] = BQ[d];
    a.ip[3 * g + d] = IP[d];
  }
  int i0, j0, k0;
  double tx, ty, tz;
  base_t(a.xc, nx, IP[0], i0, tx);
  base_t(a.yc, ny, IP[1], j0, ty);
  base_t(a.zc, nz, IP[2], k0, tz);
  a.base[3 * g + 0] = i0; a.base[3 * g + 1] = j0; a.base[3 * g + 2] = k0;
  double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
  double w[8];
  long long rf[8];
  unsigned valid = 0;
  for (int c = 0; c < 8; ++c) {
    int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    long long l = ((long long)(k0 + bz) * ny + (j0 + by)) * nx + (i0 + bx);
    rf[c] = l;
    w[c] = (wx[bx] * wy[by]) * wz[bz];
    if (a.ib[l] != 1) valid |= 1u << c;
  }
  double s = 0.0;
  for (int c = 0; c < 8; ++c)
    if (valid & (1u << c)) s = s + w[c];
  bool fallback = s < WEIGHT_SUM_MIN;
  double wn[8];
  bool moved = false;    // the row's own weight moved to the left-hand side
  double wself = 0.0;
  if (!fallback) {
    for (int c = 0; c < 8; ++c) wn[c] = (valid & (1u << c)) ? w[c] / s : 0.0;
    int selfc = -1;
    for (int c = 0; c < 8; ++c)
      if ((valid & (1u << c)) && rf[c] == lin) { selfc = c; break; }
    if (selfc >= 0) {
      double ws = wn[selfc];
      if (ws >= SELF_WEIGHT_MAX) {
        fallback = true;
      } else {
        for (int c = 0; c < 8; ++c) wn[c] = wn[c] / (1.0 - ws);
        wn[selfc] = 0.0;
        moved = true;
        wself = ws;
      }
    }
  }
  int flags = 0;
  a.tri[g] = bidx;
  a.wself[g] = (moved && !fallback) ? wself : 0.0;
  if (!fallback) a.kappa[g] = row_kappa(P, IP, moved, wself);
  if (fallback) {
    flags |= 1;
    long long bestl = -1;
    double bd = 0.0;
    const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
    for (int q = 0; q < 6; ++q) {
      int ii = gi + di[q], jj = gj + dj[q], kk = gk + dk[q];
      if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
      long long l = ((long long)kk * ny + jj) * nx + ii;
      if (a.ib[l] != 0) continue;
      double ex = IP[0] - a.xc[ii], ey = IP[1] - a.yc[jj], ez = IP[2] - a.zc[kk];
      double d2 = (ex * ex + ey * ey) + ez * ez;
      if (bestl < 0 || d2 < bd) { bestl = l; bd = d2; }
    }
    for (int c = 0; c < 8; ++c) { a.w[8 * g + c] = 0.0; a.ref[8 * g + c] = -1; }
    a.w[8 * g] = 1.0;
    a.ref[8 * g] = bestl;
    a.kappa[g] = fallback_kappa(a, P, bestl);
  } else {
    flags |= (int)(valid << 8);
    for (int c = 0; c < 8; ++c) {
      a.w[8 * g + c] = wn[c];
      a.ref[8 * g + c] = wn[c] != 0.0 ? rf[c] : -1;
    }
  }
  a.flags[g] = flags;
  // row scale: coefficients of the fluid rows that reference this ghost
  double sc = 0.0;
  long long sy = nx, sz = (long long)nx * ny;
  if (gi > 0 && a.ib[lin - 1] == 0) sc = sc + a.cxp[gi - 1];
  if (gi < nx - 1 && a.ib[lin + 1] == 0) sc = sc + a.cxm[gi + 1];
  if (gj > 0 && a.ib[lin - sy] == 0) sc = sc + a.cyp[gj - 1];
  if (gj < ny - 1 && a.ib[lin + sy] == 0) sc = sc + a.cym[gj + 1];
  if (gk > 0 && a.ib[lin - sz] == 0) sc = sc + a.czp[gk - 1];
  if (gk < nz - 1 && a.ib[lin + sz] == 0) sc = sc + a.czm[gk + 1];
  a.scale[g] = sc;
}

// triangle boxes (outward-rounded to float) and centroids, for the pruned search
__global__ void k_tri_boxes(const double *tv, int ntri, float4 *blo, float4 *bhi, float4 *cen) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  const double *v = tv + 9 * t;
  float lo[3], hi[3], c[3];
  for (int d = 0; d < 3; ++d) {
    double l = fmin(v[d], fmin(v[3 + d], v[6 + d])), h = fmax(v[d], fmax(v[3 + d], v[6 + d]));
    lo[d] = __double2float_rd(l);
    hi[d] = __double2float_ru(h);
    c[d] = (float)((v[d] + v[3 + d] + v[6 + d]) / 3.0);
  }
  blo[t] = make_float4(lo[0], lo[1], lo[2], 0.f);
  bhi[t] = make_float4(hi[0], hi[1], hi[2], 0.f);
  cen[t] = make_float4(c[0], c[1], c[2], 0.f);
}

__global__ void k_gather_tris(const double *verts, const int *tris, int ntri, double *tv) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  for (int q = 0; q < 3; ++q)
    for (int d = 0; d < 3; ++d) tv[9 * t + 3 * q + d] = verts[3 * tris[3 * t + q] + d];
}

// -------------------------------------------------------------------------- membranes

// Zero-thickness membranes (closed = 0): every cell is a fluid row; links between
// face-neighbours that a membrane triangle crosses are cut, and each cut link i -> j gives
// the ghost entry (j, side of i).  Exact predicates on the snapped lattice, as the
// closed-body test: a link along axis a is cut when a triangle covers its line in the
// projection onto the next two axes (cyclic order, counter-clockwise, top-left rule) and
// the crossing coordinate N / D lies strictly between the two centres; when several
// triangles cross a link the lowest index decides; side = sign of orient3d(A, B, C, centre)
// with the vertices in mesh order.

__device__ __forceinline__ __int128 orient3d_i128(const long long a[3], const long long b[3], const long long c[3],
                                                  const long long d[3]) {
  const long long abx = b[0] - a[0], aby = b[1] - a[1], abz = b[2] - a[2];
  const long long acx = c[0] - a[0], acy = c[1] - a[1], acz = c[2] - a[2];
  const __int128 nx = (__int128)aby * acz - (__int128)abz * acy;
  const __int128 ny = (__int128)abz * acx - (__int128)abx * acz;
  const __int128 nz = (__int128)abx * acy - (__int128)aby * acx;
  return nx * (d[0] - a[0]) + ny * (d[1] - a[1]) + nz * (d[2] - a[2]);
}

__device__ __forceinline__ void snap_tri(const double *tv, int t, long long v[3][3]) {
  for (int q = 0; q < 3; ++q)
    for (int d = 0; d < 3; ++d) v[q][d] = snapd(tv[9 * t + 3 * q + d]);
}

// "no crossing triangle" in the per-link minimum: the value a byte memset of 0x7f leaves,
// above every triangle index (the triangle count is below 2^31 / 8)
constexpr int NO_TRI = 0x7f7f7f7f;

// one (triangle, axis) record of the cut-link search
struct MTri {
  long long pu[3], pv[3], pa[3];   // projected vertices (counter-clockwise) and axis coordinates
  long long area;                  // twice the projected area (> 0)
  int iu0, iu1, iv0, iv1;          // covered centre lines (half-open) in u and v
};

struct Axes {
  const long long *C[3];   // snapped centres per axis
  int n[3];
};

__global__ void k_mem_setup(const double *tv, int ntri, Axes ax, MTri *out, long long *count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= 3 * ntri) return;
  const int a = p / ntri, t = p - a * ntri, u = (a + 1) % 3, w = (a + 2) % 3;
  long long v[3][3];
  snap_tri(tv, t, v);
  const long long D = orient2d(v[0][u], v[0][w], v[1][u], v[1][w], v[2][u], v[2][w]);
  MTri M;
  long long cnt = 0;
  const int ord[2][3] = {{0, 1, 2}, {0, 2, 1}};
  const int *o = ord[D > 0 ? 0 : 1];
  for (int q = 0; q < 3; ++q) { M.pu[q] = v[o[q]][u]; M.pv[q] = v[o[q]][w]; M.pa[q] = v[o[q]][a]; }
  M.area = D > 0 ? D : -D;
  const long long ul = min(M.pu[0], min(M.pu[1], M.pu[2])), uh = max(M.pu[0], max(M.pu[1], M.pu[2]));
  const long long vl = min(M.pv[0], min(M.pv[1], M.pv[2])), vh = max(M.pv[0], max(M.pv[1], M.pv[2]));
  M.iu0 = lower_bound_dev(ax.C[u], ax.n[u], ul); M.iu1 = upper_bound_dev(ax.C[u], ax.n[u], uh);
  M.iv0 = lower_bound_dev(ax.C[w], ax.n[w], vl); M.iv1 = upper_bound_dev(ax.C[w], ax.n[w], vh);
  if (D != 0 && M.iu1 > M.iu0 && M.iv1 > M.iv0) cnt = (long long)(M.iu1 - M.iu0) * (M.iv1 - M.iv0);
  out[p] = M;
  count[p] = cnt;
}

// every (record, line) pair: covering test, crossing, lowest crossing triangle per link
// (linktri[a * ncell + lower cell])
__global__ void k_mem_pairs(const MTri *recs, const long long *off, int nrec, long long total, int ntri, Axes ax,
                            long long ncell, int *linktri) {
  const int nx = ax.n[0], ny = ax.n[1];
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int r = upper_bound_dev(off, nrec + 1, p) - 1;
    const MTri &M = recs[r];
    const int a = r / ntri, t = r - a * ntri, u = (a + 1) % 3, w = (a + 2) % 3;
    const long long local = p - off[r];
    const int niu = M.iu1 - M.iu0;
    const int iu = M.iu0 + (int)(local % niu), iv = M.iv0 + (int)(local / niu);
    const long long qu = ax.C[u][iu], qv = ax.C[w][iv];
    const long long wa = orient2d(M.pu[1], M.pv[1], M.pu[2], M.pv[2], qu, qv);
    const long long wb = orient2d(M.pu[2], M.pv[2], M.pu[0], M.pv[0], qu, qv);
    const long long wc = orient2d(M.pu[0], M.pv[0], M.pu[1], M.pv[1], qu, qv);
    const bool cov = (wa > 0 || (wa == 0 && top_left(M.pu[1], M.pv[1], M.pu[2], M.pv[2]))) &&
                     (wb > 0 || (wb == 0 && top_left(M.pu[2], M.pv[2], M.pu[0], M.pv[0]))) &&
                     (wc > 0 || (wc == 0 && top_left(M.pu[0], M.pv[0], M.pu[1], M.pv[1])));
    if (!cov) continue;
    const __int128 N = (__int128)wa * M.pa[0] + (__int128)wb * M.pa[1] + (__int128)wc * M.pa[2];
    const __int128 D = (__int128)M.area;
    __int128 q = N / D;
    const __int128 rem = N - q * D;
    if (rem != 0 && N < 0) q -= 1;          // floor division (D > 0)
    const long long qa = (long long)q;
    const long long *Ca = ax.C[a];
    const int na = ax.n[a];
    const int m = (rem != 0) ? upper_bound_dev(Ca, na, qa) : lower_bound_dev(Ca, na, qa);   // centres < N/D
    const int lo = m - 1;
    if (lo < 0 || lo + 1 >= na || !(Ca[lo + 1] > qa)) continue;
    int ijk[3];
    ijk[a] = lo; ijk[u] = iu; ijk[w] = iv;
    const long long lin = ((long long)ijk[2] * ny + ijk[1]) * nx + ijk[0];
    atomicMin(&linktri[a * ncell + lin], t);
  }
}

// cut and side bytes of every cell from its six links
__global__ void k_mem_cut(const int *linktri, long long ncell, Axes ax, const double *tv, uint8_t *cut,
                          uint8_t *side) {
  const int nx = ax.n[0], ny = ax.n[1], nz = ax.n[2];
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < ncell;
       l += (long long)gridDim.x * blockDim.x) {
    const int idx[3] = {(int)(l % nx), (int)((l / nx) % ny), (int)(l / ((long long)nx * ny))};
    const long long step[3] = {1, nx, (long long)nx * ny};
    const long long P[3] = {ax.C[0][idx[0]], ax.C[1][idx[1]], ax.C[2][idx[2]]};
    uint8_t c = 0, sd = 0;
    for (int a = 0; a < 3; ++a) {
      for (int dir = 0; dir < 2; ++dir) {       // dir 0: -a (link from the lower cell), 1: +a
        int t;
        if (dir == 1) t = idx[a] + 1 < ax.n[a] ? linktri[a * ncell + l] : NO_TRI;
        else t = idx[a] > 0 ? linktri[a * ncell + l - step[a]] : NO_TRI;
        if (t == NO_TRI) continue;
        long long v[3][3];
        snap_tri(tv, t, v);
        const int bit = 2 * a + dir;
        c |= (uint8_t)(1u << bit);
        if (orient3d_i128(v[0], v[1], v[2], P) > 0) sd |= (uint8_t)(1u << bit);
      }
    }
    (void)nz;
    cut[l] = c;
    side[l] = sd;
  }
}

// entries of cell l: one per side from which a cut link reaches it (bit s of the result)
__device__ __forceinline__ unsigned entry_sides(uint8_t c, uint8_t sd) {
  unsigned e = 0;
  for (int d = 0; d < 6; ++d)
    if ((c >> d) & 1u) e |= 1u << (1u - ((sd >> d) & 1u));
  return e;
}

__global__ void k_mem_count(const uint8_t *cut, const uint8_t *side, long long ncell, long long *bcount) {
  __shared__ int s[GM_THREADS];
  const long long base = (long long)blockIdx.x * GM_THREADS * GM_PER + (long long)threadIdx.x * GM_PER;
  int c = 0;
  for (int q = 0; q < GM_PER; ++q) {
    const long long l = base + q;
    if (l < ncell && cut[l]) c += __popc(entry_sides(cut[l], side[l]));
  }
  s[threadIdx.x] = c;
  __syncthreads();
  for (int st = GM_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) bcount[blockIdx.x] = s[0];
}

// entries in (cell, side) order: cell, side and the sort key 2 cell + side
__global__ void k_mem_scatter(const uint8_t *cut, const uint8_t *side, long long ncell, const long long *boff,
                              long long *gcell, uint8_t *gside, long long *keys) {
  __shared__ int s[GM_THREADS];
  const long long base = (long long)blockIdx.x * GM_THREADS * GM_PER + (long long)threadIdx.x * GM_PER;
  int c = 0;
  for (int q = 0; q < GM_PER; ++q) {
    const long long l = base + q;
    if (l < ncell && cut[l]) c += __popc(entry_sides(cut[l], side[l]));
  }
  s[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < GM_THREADS; ++t) { int v = s[t]; s[t] = run; run += v; }
  }
  __syncthreads();
  long long o = boff[blockIdx.x] + s[threadIdx.x];
  for (int q = 0; q < GM_PER; ++q) {
    const long long l = base + q;
    if (l >= ncell || !cut[l]) continue;
    const unsigned e = entry_sides(cut[l], side[l]);
    for (unsigned sd = 0; sd < 2; ++sd)
      if ((e >> sd) & 1u) { gcell[o] = l; gside[o] = (uint8_t)sd; keys[o] = 2 * l + sd; ++o; }
  }
}

struct MemArgs {
  long long ncell;
  const long long *keys;       // 2 cell + side of every entry, ascending
  const uint8_t *gside, *cut, *side;
  const long long *Xs, *Ys, *Zs;
  int ntri;
};

// is the segment P-Q (snapped) cut by triangle t: endpoints strictly on opposite sides of its
// plane, and the segment's line through the closed triangle
__device__ __forceinline__ bool seg_cut_tri(const long long P[3], const long long Q[3], const long long v[3][3]) {
  const __int128 sp = orient3d_i128(v[0], v[1], v[2], P), sq = orient3d_i128(v[0], v[1], v[2], Q);
  if (sp == 0 || sq == 0 || (sp > 0) == (sq > 0)) return false;
  const __int128 e1 = orient3d_i128(P, Q, v[0], v[1]);
  const __int128 e2 = orient3d_i128(P, Q, v[1], v[2]);
  const __int128 e3 = orient3d_i128(P, Q, v[2], v[0]);
  return (e1 >= 0 && e2 >= 0 && e3 >= 0) || (e1 <= 0 && e2 <= 0 && e3 <= 0);
}

// one warp per entry: boundary intercept and image point (as for closed bodies), corners
// blocked by the membrane (exact segment tests), same-side entries for blocked corners,
// weights, fallback and row scale
__global__ void __launch_bounds__(TABLE_THREADS) k_mem_tables(GhostArgs a, MemArgs m) {
  __shared__ int cand[TABLE_THREADS / 32][CAND_MAX];
  const int lane = threadIdx.x & 31;
  const long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (g >= a.ng) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long lin = a.gcell[g];
  const unsigned gs = m.gside[g];
  const int gi = (int)(lin % nx), gj = (int)((lin / nx) % ny), gk = (int)(lin / ((long long)nx * ny));
  double P[3] = {a.xc[gi], a.yc[gj], a.zc[gk]};
  double best, BQ[3];
  int bidx;
  find_closest(a, P, lane, best, bidx, BQ, cand[threadIdx.x >> 5]);
  double IP[3];
  for (int d = 0; d < 3; ++d) IP[d] = (BQ[d] + BQ[d]) - P[d];
  int i0, j0, k0;
  double tx, ty, tz;
  base_t(a.xc, nx, IP[0], i0, tx);
  base_t(a.yc, ny, IP[1], j0, ty);
  base_t(a.zc, nz, IP[2], k0, tz);
  // blocked corners: lanes split the (corner, triangle) pairs whose boxes overlap
  const long long SIP[3] = {snapd(IP[0]), snapd(IP[1]), snapd(IP[2])};
  unsigned blocked = 0;
  for (int c = 0; c < 8; ++c) {
    const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    const long long Q[3] = {m.Xs[i0 + bx], m.Ys[j0 + by], m.Zs[k0 + bz]};
    // segment box, widened past the snapping distance (2^-25) and FP32 rounding, so the box
    // filter never drops a triangle the exact test would count
    float lo[3], hi[3];
    double dlo[3], dhi[3];
    for (int d = 0; d < 3; ++d) {
      dlo[d] = (double)min(SIP[d], Q[d]) / SNAP_SCALE - 1e-6;
      dhi[d] = (double)max(SIP[d], Q[d]) / SNAP_SCALE + 1e-6;
      lo[d] = __double2float_rd(dlo[d]);
      hi[d] = __double2float_ru(dhi[d]);
    }
    // a triangle that crosses the segment meets its box, so it is listed in a bin the box
    // meets; lanes split each bin's list (a triangle listed in several bins is tested again)
    int b0[3], b1[3];
    box_bin_range(dlo, dhi, a.bins, b0, b1);
    bool hit = false;
    for (int bz = b0[2]; bz <= b1[2]; ++bz)
      for (int by = b0[1]; by <= b1[1]; ++by)
        for (int bx = b0[0]; bx <= b1[0]; ++bx) {
          const long long bin = ((long long)bz * a.bins.nb[1] + by) * a.bins.nb[0] + bx;
          for (long long e = a.bins.off[bin] + lane; e < a.bins.off[bin + 1] && !hit; e += 32) {
            const int t = a.bins.tri[e];
            int f[3];   // test each triangle once: in the first bin of its range inside the box
            range_meets(a.bins.range[t], b0, b1, f);
            if (f[0] != bx || f[1] != by || f[2] != bz) continue;
            const float4 bl = a.blo[t], bh = a.bhi[t];
            if (bl.x > hi[0] || bh.x < lo[0] || bl.y > hi[1] || bh.y < lo[1] || bl.z > hi[2] || bh.z < lo[2]) continue;
            long long v[3][3];
            snap_tri(a.tv, t, v);
            if (seg_cut_tri(SIP, Q, v)) hit = true;
          }
        }
    if (__any_sync(0xffffffffu, hit)) blocked |= 1u << c;
  }
  if (lane != 0) return;
  for (int d = 0; d < 3; ++d) {
    a.bi[3 * g + d] = BQ[d];
    a.ip[3 * g + d] = IP[d];
  }
  a.base[3 * g + 0] = i0; a.base[3 * g + 1] = j0; a.base[3 * g + 2] = k0;
  double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty}, wz[2] = {1.0 - tz, tz};
  double w[8];
  long long rf[8];
  unsigned valid = 0;
  for (int c = 0; c < 8; ++c) {
    const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    const long long l = ((long long)(k0 + bz) * ny + (j0 + by)) * nx + (i0 + bx);
    w[c] = (wx[bx] * wy[by]) * wz[bz];
    if (!((blocked >> c) & 1u)) {
      rf[c] = l;
      valid |= 1u << c;
    } else {
      const long long key = 2 * l + gs;
      const int e = lower_bound_dev(m.keys, (int)a.ng, key);
      if (e < a.ng && m.keys[e] == key) {
        rf[c] = m.ncell + e;
        valid |= 1u << c;
      } else {
        rf[c] = -1;
      }
    }
  }
  double s = 0.0;
  for (int c = 0; c < 8; ++c)
    if (valid & (1u << c)) s = s + w[c];
  bool fallback = s < WEIGHT_SUM_MIN;
  double wn[8];
  bool moved = false;    // the row's own weight moved to the left-hand side
  double wself = 0.0;
  if (!fallback) {
    for (int c = 0; c < 8; ++c) wn[c] = (valid & (1u << c)) ? w[c] / s : 0.0;
    int selfc = -1;
    for (int c = 0; c < 8; ++c)
      if ((valid & (1u << c)) && rf[c] == m.ncell + g) { selfc = c; break; }
    if (selfc >= 0) {
      const double ws = wn[selfc];
      if (ws >= SELF_WEIGHT_MAX) {
        fallback = true;
      } else {
        for (int c = 0; c < 8; ++c) wn[c] = wn[c] / (1.0 - ws);
        wn[selfc] = 0.0;
        moved = true;
        wself = ws;
      }
    }
  }
  a.tri[g] = bidx;
  a.wself[g] = (moved && !fallback) ? wself : 0.0;
  // the cells that use the entry: face-neighbours n of the cell cut from side gs (the
  // cell's own side bit of that link is the other side)
  const uint8_t cc = m.cut[lin], cs = m.side[lin];
  const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
  const double *coef[6] = {a.cxp, a.cxm, a.cyp, a.cym, a.czp, a.czm};
  int flags = 0;
  double sc = 0.0;
  long long bestl = -1;
  double bd = 0.0;
  for (int d = 0; d < 6; ++d) {
    if (!((cc >> d) & 1u) || ((cs >> d) & 1u) == gs) continue;
    const int ii = gi + di[d], jj = gj + dj[d], kk = gk + dk[d];
    const int ax_idx = d < 2 ? ii : (d < 4 ? jj : kk);
    sc = sc + coef[d][ax_idx];
    const double ex = IP[0] - a.xc[ii], ey = IP[1] - a.yc[jj], ez = IP[2] - a.zc[kk];
    const double d2 = (ex * ex + ey * ey) + ez * ez;
    if (bestl < 0 || d2 < bd) { bestl = ((long long)kk * ny + jj) * nx + ii; bd = d2; }
  }
  if (fallback) {
    flags |= 1;
    for (int c = 0; c < 8; ++c) { a.w[8 * g + c] = 0.0; a.ref[8 * g + c] = -1; }
    a.w[8 * g] = 1.0;
    a.ref[8 * g] = bestl;
    a.kappa[g] = fallback_kappa(a, P, bestl);
  } else {
    a.kappa[g] = row_kappa(P, IP, moved, wself);
    flags |= (int)(valid << 8);
    for (int c = 0; c < 8; ++c) {
      a.w[8 * g + c] = wn[c];
      a.ref[8 * g + c] = wn[c] != 0.0 ? rf[c] : -1;
    }
  }
  a.flags[g] = flags;
  a.scale[g] = sc;
}

// Device scratch of one tables object.  Allocations are bump pointers into a block the
// tables keep between classifications; a call that needs more than the block holds takes
// extra blocks, and when it ends the tables' block is regrown to the whole amount, so
// repeated classifications of similar geometry allocate nothing.
struct Scratch {
  ibm_tables *t;
  size_t used = 0, extra_bytes = 0;
  std::vector<void *> extra;
  explicit Scratch(ibm_tables *tt) : t(tt) {}
  template <typename T>
  cudaError_t get(T **p, size_t n) {
    const size_t bytes = ((n ? n : 1) * sizeof(T) + 255) & ~(size_t)255;
    if (used + bytes <= t->scratch_cap) {
      *p = reinterpret_cast<T *>(t->scratch + used);
      used += bytes;
      return cudaSuccess;
    }
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e == cudaSuccess) { extra.push_back(*p); extra_bytes += bytes; }
    return e;
  }
  // call after the stream has drained: release the extra blocks, regrow the kept one
  cudaError_t finish() {
    for (void *q : extra) cudaFree(q);
    extra.clear();
    if (extra_bytes == 0) return cudaSuccess;
    const size_t want = used + extra_bytes;
    extra_bytes = 0;
    if (t->scratch) cudaFree(t->scratch);
    t->scratch = nullptr;
    t->scratch_cap = 0;
    cudaError_t e = cudaMalloc((void **)&t->scratch, want);
    if (e == cudaSuccess) t->scratch_cap = want;
    return e;
  }
  ~Scratch() { for (void *q : extra) cudaFree(q); }
};

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// bounding box and total area of the meshes' triangles (host arrays)
struct TriStats {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  double area = 0.0;
  void add(const ibm_mesh &m) {
    for (long long t = 0; t < m.ntris; ++t) {
      const double *v[3];
      for (int q = 0; q < 3; ++q) {
        v[q] = m.verts + 3LL * m.tris[3 * t + q];
        for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], v[q][d]); hi[d] = std::max(hi[d], v[q][d]); }
      }
      const double u[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
      const double w[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
      const double c[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
      area += 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
  }
};

// Bins for the closest-triangle search: edge twice the square root of the mean triangle
// area (a few triangles per bin near the surface), at most 256 bins per axis (the per-
// triangle ranges are stored as bytes) and 2^20 in total.  One readback (the number of
// entries) sizes the index list.
cudaError_t build_bins(Scratch &S, const double *tv, int ntri, const TriStats &ts, cudaStream_t st, TriBins &B) {
  double ext = 0.0;
  for (int d = 0; d < 3; ++d) ext = std::max(ext, ts.hi[d] - ts.lo[d]);
  double h = 2.0 * std::sqrt(ts.area / std::max(1, ntri));
  h = std::max({h, ext / 255.0, 1e-12});   // <= 256 bins per axis: bin indices fit in a byte
  auto nbins = [&](double hh) {
    long long n = 1;
    for (int d = 0; d < 3; ++d) n *= (long long)std::floor((ts.hi[d] - ts.lo[d]) / hh) + 1;
    return n;
  };
  while (nbins(h) > (1LL << 20)) h *= 1.25;
  for (int d = 0; d < 3; ++d) {
    B.lo[d] = ts.lo[d];
    B.nb[d] = (int)std::floor((ts.hi[d] - ts.lo[d]) / h) + 1;
  }
  B.h = h;
  B.inv = 1.0 / h;
  const long long nb = (long long)B.nb[0] * B.nb[1] * B.nb[2];
  long long *cnt = nullptr, *off = nullptr;
  int *tri = nullptr;
  cudaError_t e;
  if ((e = S.get(&cnt, nb)) != cudaSuccess || (e = S.get(&off, nb + 1)) != cudaSuccess) return e;
  uint2 *range = nullptr;
  if ((e = S.get(&range, ntri)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(long long) * nb, st)) != cudaSuccess) return e;
  k_bin_count<<<nblk(ntri, 128), 128, 0, st>>>(tv, ntri, B, cnt, range);
  k_scan_single<<<1, 1024, 0, st>>>(cnt, off, (int)nb);
  long long total = 0;
  if ((e = cudaMemcpyAsync(&total, off + nb, sizeof(long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  if ((e = S.get(&tri, total)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(long long) * nb, st)) != cudaSuccess) return e;
  k_bin_fill<<<nblk(ntri, 128), 128, 0, st>>>(tv, ntri, B, off, cnt, tri);
  B.off = off;
  B.tri = tri;
  B.range = range;
  return cudaGetLastError();
}

ibm_status check_meshes(const ibm_mesh *meshes, int nmesh, long long &totverts, long long &tottris) {
  if (nmesh < 0 || (nmesh > 0 && !meshes)) return IBM_ERR_INVALID_ARG;
  totverts = tottris = 0;
  int nclosed = 0;
  for (int m = 0; m < nmesh; ++m) {
    const ibm_mesh &M = meshes[m];
    if (M.nverts < 0 || M.ntris < 0 || (M.ntris > 0 && (!M.verts || !M.tris))) return IBM_ERR_INVALID_ARG;
    if (M.closed != 0 && M.closed != 1) return IBM_ERR_INVALID_ARG;
    nclosed += M.closed;
    for (long long q = 0; q < 3LL * M.nverts; ++q)
      if (!(std::fabs(M.verts[q]) <= COORD_LIMIT)) return IBM_ERR_INVALID_ARG;
    for (long long q = 0; q < 3LL * M.ntris; ++q)
      if (M.tris[q] < 0 || M.tris[q] >= M.nverts) return IBM_ERR_INVALID_ARG;
    totverts += M.nverts;
    tottris += M.ntris;
  }
  if (nclosed != 0 && nclosed != nmesh) return IBM_ERR_NOT_IMPLEMENTED;   // membranes with closed bodies
  return IBM_OK;
}

// grow the per-ghost arrays of the tables to hold ng entries (contents are rewritten)
cudaError_t ensure_ghost_capacity(ibm_tables *T, long long ng) {
  if (ng <= T->gcap && T->gcell) return cudaSuccess;
  const long long cap = std::max<long long>(std::max<long long>(ng + ng / 4, 1024), T->gcap);
  void *ps[] = {T->gcell, T->gbi,   T->gip,  T->gw,     T->gscale, T->gbase, T->gflags,
                T->gref,  T->gside, T->gkeys, T->gkappa, T->gd,     T->gtri,   T->gwself};
  for (void *q : ps) if (q) cudaFree(q);
  T->gcell = nullptr; T->gbi = T->gip = T->gw = T->gscale = nullptr; T->gbase = T->gflags = nullptr; T->gref = nullptr;
  T->gside = nullptr; T->gkeys = nullptr; T->gkappa = T->gd = nullptr; T->gtri = nullptr; T->gwself = nullptr;
  T->gcap = 0;
  cudaError_t e = cudaMalloc(&T->gcell, cap * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&T->gbi, cap * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T->gip, cap * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T->gw, cap * 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T->gscale, cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T->gbase, cap * 3 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&T->gflags, cap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&T->gref, cap * 8 * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&T->gside, cap);
  if (e == cudaSuccess) e = cudaMalloc(&T->gkeys, cap * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&T->gkappa, cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T->gd, cap * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&T->gtri, cap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&T->gwself, cap * sizeof(double));
  if (e == cudaSuccess) T->gcap = cap;
  return e;
}

// Membrane classification (all meshes closed = 0): cut links, ghost entries and their rows.
ibm_status membrane_into(ibm_tables *T, const ibm_mesh *meshes, int nmesh, long long totverts, long long tottris,
                         cudaStream_t st, Scratch &S, double *const dc[3], double *const dcm[3],
                         double *const dcp[3], long long *const ds[3]) {
  const int nx = T->nx, ny = T->ny, nz = T->nz;
  const long long ncell = T->ncell;
  ibm_ctx *ctx = T->ctx;
#define MTRY(call)                                                  \
  do {                                                              \
    cudaError_t e__ = (call);                                       \
    if (e__ != cudaSuccess) return ibm::check(e__, #call);          \
  } while (0)
  if (!T->cut) MTRY(cudaMalloc(&T->cut, ncell));
  if (!T->cside) MTRY(cudaMalloc(&T->cside, ncell));
  T->nfluid = ncell;
  T->nsolid = 0;
  // all membrane triangles, concatenated in mesh order (global triangle index)
  double *dverts = nullptr, *tv = nullptr;
  int *dtris = nullptr;
  MTRY(S.get(&dverts, 3 * totverts));
  MTRY(S.get(&dtris, 3 * tottris));
  MTRY(S.get(&tv, 9 * tottris));
  TriStats ts;
  long long vo = 0, to = 0;
  for (int m = 0; m < nmesh; ++m) {
    const int nt = meshes[m].ntris;
    if (meshes[m].nverts)
      MTRY(cudaMemcpyAsync(dverts + 3 * vo, meshes[m].verts, 3 * sizeof(double) * meshes[m].nverts,
                           cudaMemcpyHostToDevice, st));
    if (nt) {
      MTRY(cudaMemcpyAsync(dtris + 3 * to, meshes[m].tris, 3 * sizeof(int) * nt, cudaMemcpyHostToDevice, st));
      k_gather_tris<<<nblk(nt, 128), 128, 0, st>>>(dverts + 3 * vo, dtris + 3 * to, nt, tv + 9 * to);
      ts.add(meshes[m]);
    }
    vo += meshes[m].nverts;
    to += nt;
  }
  if (tottris >= NO_TRI) return IBM_ERR_INVALID_ARG;
  const int ntri = (int)tottris;
  Axes ax;
  ax.C[0] = ds[0]; ax.C[1] = ds[1]; ax.C[2] = ds[2];
  ax.n[0] = nx; ax.n[1] = ny; ax.n[2] = nz;
  // cut links: lowest crossing triangle per link, then the cells' cut and side bytes
  int *linktri = nullptr;
  MTRY(S.get(&linktri, 3 * ncell));
  MTRY(cudaMemsetAsync(linktri, 0x7f, sizeof(int) * 3 * ncell, st));   // every link: NO_TRI
  if (ntri > 0) {
    MTri *recs = nullptr;
    long long *cnt = nullptr, *off = nullptr;
    MTRY(S.get(&recs, 3 * (size_t)ntri));
    MTRY(S.get(&cnt, 3 * (size_t)ntri));
    MTRY(S.get(&off, 3 * (size_t)ntri + 1));
    k_mem_setup<<<nblk(3 * ntri, 128), 128, 0, st>>>(tv, ntri, ax, recs, cnt);
    k_scan_single<<<1, 1024, 0, st>>>(cnt, off, 3 * ntri);
    long long total = 0;
    MTRY(cudaMemcpyAsync(&total, off + 3 * ntri, sizeof(long long), cudaMemcpyDeviceToHost, st));
    MTRY(cudaStreamSynchronize(st));
    if (total > 0) {
      const unsigned blocks = (unsigned)std::min<long long>(nblk(total, 256), 4LL * ctx->wave);
      k_mem_pairs<<<blocks, 256, 0, st>>>(recs, off, 3 * ntri, total, ntri, ax, ncell, linktri);
    }
  }
  k_mem_cut<<<ctx->wave, 256, 0, st>>>(linktri, ncell, ax, tv, T->cut, T->cside);
  MTRY(cudaGetLastError());
  // ghost entries in (cell, side) order
  const long long chunk = (long long)GM_THREADS * GM_PER;
  const unsigned nb = (unsigned)((ncell + chunk - 1) / chunk);
  long long *bc = nullptr, *bo = nullptr;
  MTRY(S.get(&bc, nb));
  MTRY(S.get(&bo, nb + 1));
  k_mem_count<<<nb, GM_THREADS, 0, st>>>(T->cut, T->cside, ncell, bc);
  k_scan_single<<<1, 1024, 0, st>>>(bc, bo, (int)nb);
  long long ng = 0;
  MTRY(cudaMemcpyAsync(&ng, bo + nb, sizeof(long long), cudaMemcpyDeviceToHost, st));
  MTRY(cudaStreamSynchronize(st));
  T->nghost = ng;
  MTRY(ensure_ghost_capacity(T, ng));
  if (ng > 0) {
    k_mem_scatter<<<nb, GM_THREADS, 0, st>>>(T->cut, T->cside, ncell, bo, T->gcell, T->gside, T->gkeys);
    float4 *blo = nullptr, *bhi = nullptr, *cen = nullptr;
    MTRY(S.get(&blo, ntri)); MTRY(S.get(&bhi, ntri)); MTRY(S.get(&cen, ntri));
    k_tri_boxes<<<nblk(ntri, 128), 128, 0, st>>>(tv, ntri, blo, bhi, cen);
    GhostArgs ga;
    MTRY(build_bins(S, tv, ntri, ts, st, ga.bins));
    ga.nx = nx; ga.ny = ny; ga.nz = nz;
    ga.xc = dc[0]; ga.yc = dc[1]; ga.zc = dc[2];
    ga.cxm = dcm[0]; ga.cxp = dcp[0]; ga.cym = dcm[1]; ga.cyp = dcp[1]; ga.czm = dcm[2]; ga.czp = dcp[2];
    ga.ib = T->iblank;
    ga.tv = tv; ga.blo = blo; ga.bhi = bhi; ga.cen = cen;
    ga.ng = ng; ga.gcell = T->gcell;
    ga.bi = T->gbi; ga.ip = T->gip; ga.w = T->gw; ga.scale = T->gscale;
    ga.base = T->gbase; ga.flags = T->gflags; ga.ref = T->gref;
    ga.kappa = T->gkappa; ga.tri = T->gtri; ga.wself = T->gwself;
    MemArgs ma;
    ma.ncell = ncell; ma.keys = T->gkeys; ma.gside = T->gside; ma.cut = T->cut; ma.side = T->cside;
    ma.Xs = ds[0]; ma.Ys = ds[1]; ma.Zs = ds[2]; ma.ntri = ntri;
    k_mem_tables<<<nblk(32 * ng, TABLE_THREADS), TABLE_THREADS, 0, st>>>(ga, ma);
    MTRY(cudaGetLastError());
  }
  MTRY(cudaStreamSynchronize(st));
  ctx->launches += 4 + (ntri > 0 ? 3 : 0) + (ng > 0 ? 6 : 0);   // bins: count, scan, fill
#undef MTRY
  return IBM_OK;
}

// Classification of the meshes on the tables' grid, into the tables' own arrays.
ibm_status classify_into(ibm_tables *T, const ibm_mesh *meshes, int nmesh, long long totverts, long long tottris,
                         cudaStream_t st) {
  const int nx = T->nx, ny = T->ny, nz = T->nz;
  const long long ncell = T->ncell;
  ibm_ctx *ctx = T->ctx;
  Scratch S(T);
#define CTRY(call)                                                  \
  do {                                                              \
    cudaError_t e__ = (call);                                       \
    if (e__ != cudaSuccess) return ibm::check(e__, #call);          \
  } while (0)
  // axes (grid only, once per tables): faces, centres, snapped centres, widths, coefficients
  const int ns[3] = {nx, ny, nz};
  const std::vector<double> *fs[3] = {&T->xf, &T->yf, &T->zf};
  if (!T->axis) {
    size_t words = 0;
    for (int a = 0; a < 3; ++a) words += 6 * (size_t)ns[a] + 1;
    CTRY(cudaMalloc((void **)&T->axis, words * sizeof(double)));
    size_t o = 0;
    for (int a = 0; a < 3; ++a) {
      double *base = T->axis + o;
      double *df = base, *dc = df + ns[a] + 1, *dw = dc + ns[a], *dcm = dw + ns[a], *dcp = dcm + ns[a];
      long long *ds = reinterpret_cast<long long *>(dcp + ns[a]);
      CTRY(cudaMemcpyAsync(df, fs[a]->data(), (ns[a] + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
      k_axis<<<nblk(ns[a], 128), 128, 0, st>>>(df, ns[a], dc, ds, dw, dcm, dcp);
      o += 6 * (size_t)ns[a] + 1;
    }
    CTRY(cudaGetLastError());
    ctx->launches += 3;
  }
  double *dc[3], *dcm[3], *dcp[3];
  long long *ds[3];
  {
    size_t o = 0;
    for (int a = 0; a < 3; ++a) {
      double *base = T->axis + o;
      dc[a] = base + ns[a] + 1;
      dcm[a] = dc[a] + 2 * ns[a];
      dcp[a] = dcm[a] + ns[a];
      ds[a] = reinterpret_cast<long long *>(dcp[a] + ns[a]);
      o += 6 * (size_t)ns[a] + 1;
    }
  }
  if (!T->iblank) CTRY(cudaMalloc(&T->iblank, ncell));
  CTRY(cudaMemsetAsync(T->iblank, 0, ncell, st));
  T->membrane = nmesh > 0 && meshes[0].closed == 0;
  // a new classification clears the moving-boundary datum; the meshes' triangle ranges serve
  // ibm_neumann_rigid
  T->has_datum = false;
  T->mesh_tri_off.assign(1, 0);
  for (int m = 0; m < nmesh; ++m) T->mesh_tri_off.push_back(T->mesh_tri_off.back() + meshes[m].ntris);
  if (T->membrane) {
    ibm_status ms = membrane_into(T, meshes, nmesh, totverts, tottris, st, S, dc, dcm, dcp, ds);
    if (ms != IBM_OK) return ms;
    CTRY(S.finish());
    T->geom_version += 1;
    return IBM_OK;
  }

  // inside test per closed mesh
  double *dverts = nullptr;
  int *dtris = nullptr;
  CTRY(S.get(&dverts, 3 * totverts));
  CTRY(S.get(&dtris, 3 * tottris));
  std::vector<int> vbase(nmesh), tbase(nmesh);
  {
    long long vo = 0, to = 0;
    for (int m = 0; m < nmesh; ++m) {
      vbase[m] = (int)vo; tbase[m] = (int)to;
      if (meshes[m].nverts)
        CTRY(cudaMemcpyAsync(dverts + 3 * vo, meshes[m].verts, 3 * sizeof(double) * meshes[m].nverts,
                             cudaMemcpyHostToDevice, st));
      if (meshes[m].ntris)
        CTRY(cudaMemcpyAsync(dtris + 3 * to, meshes[m].tris, 3 * sizeof(int) * meshes[m].ntris,
                             cudaMemcpyHostToDevice, st));
      vo += meshes[m].nverts;
      to += meshes[m].ntris;
    }
  }
  const int words = (nz + 1 + 31) / 32;
  unsigned *leak = nullptr;   // set by k_parity: some column crosses a closed mesh an odd number of times
  CTRY(S.get(&leak, 1));
  CTRY(cudaMemsetAsync(leak, 0, sizeof(unsigned), st));
  if (tottris > 0) {
    unsigned *tog = nullptr, *ons = nullptr;
    CTRY(S.get(&tog, (size_t)nx * ny * words));
    CTRY(S.get(&ons, (size_t)nx * ny * words));
    CTRY(cudaMemsetAsync(tog, 0, (size_t)nx * ny * words * 4, st));
    CTRY(cudaMemsetAsync(ons, 0, (size_t)nx * ny * words * 4, st));
    for (int m = 0; m < nmesh; ++m) {
      const int nt = meshes[m].ntris;
      if (nt == 0) continue;
      Tri *tr = nullptr;
      long long *cnt = nullptr, *off = nullptr;
      CTRY(S.get(&tr, nt)); CTRY(S.get(&cnt, nt)); CTRY(S.get(&off, nt + 1));
      k_tri_setup<<<nblk(nt, 128), 128, 0, st>>>(dverts + 3LL * vbase[m], dtris + 3LL * tbase[m], nt, ds[0], nx,
                                                  ds[1], ny, ds[2], nz, tr, cnt);
      k_scan_single<<<1, 1024, 0, st>>>(cnt, off, nt);
      long long total = 0;
      CTRY(cudaMemcpyAsync(&total, off + nt, sizeof(long long), cudaMemcpyDeviceToHost, st));
      CTRY(cudaStreamSynchronize(st));
      if (total > 0) {
        unsigned blocks = (unsigned)std::min<long long>(nblk(total, 256), 4LL * ctx->wave);
        k_tri_pairs<<<blocks, 256, 0, st>>>(tr, off, nt, total, ds[0], ds[1], ds[2], nx, ny, nz, words, tog, ons);
      }
      // columns of the mesh's xy box
      double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
      for (long long q = 0; q < meshes[m].nverts; ++q)
        for (int d = 0; d < 2; ++d) {
          lo[d] = std::min(lo[d], meshes[m].verts[3 * q + d]);
          hi[d] = std::max(hi[d], meshes[m].verts[3 * q + d]);
        }
      int i0 = (int)(std::lower_bound(T->xf.begin(), T->xf.end(), lo[0]) - T->xf.begin()) - 1;
      int i1 = (int)(std::upper_bound(T->xf.begin(), T->xf.end(), hi[0]) - T->xf.begin());
      int j0 = (int)(std::lower_bound(T->yf.begin(), T->yf.end(), lo[1]) - T->yf.begin()) - 1;
      int j1 = (int)(std::upper_bound(T->yf.begin(), T->yf.end(), hi[1]) - T->yf.begin());
      i0 = std::max(0, i0 - 1); j0 = std::max(0, j0 - 1);
      i1 = std::min(nx, i1 + 1); j1 = std::min(ny, j1 + 1);
      if (i1 > i0 && j1 > j0) {
        dim3 gp(nblk(i1 - i0, 128), j1 - j0);
        k_parity<<<gp, 128, 0, st>>>(tog, ons, words, nx, ny, nz, i0, i1, j0, j1, T->iblank, leak);
      }
      CTRY(cudaGetLastError());
    }
  }

  // ghost marking + sorted compaction
  const long long chunk = (long long)GM_THREADS * GM_PER;
  const unsigned nb = (unsigned)((ncell + chunk - 1) / chunk);
  unsigned long long *cellcnt = nullptr;
  {
    long long *bc = nullptr, *bo = nullptr;
    CTRY(S.get(&bc, nb)); CTRY(S.get(&bo, nb + 1));
    CTRY(S.get(&cellcnt, 2));
    CTRY(cudaMemsetAsync(cellcnt, 0, 16, st));
    k_ghost_count<<<nb, GM_THREADS, 0, st>>>(T->iblank, nx, ny, nz, ncell, bc);
    k_scan_single<<<1, 1024, 0, st>>>(bc, bo, (int)nb);
    long long ng = 0;
    CTRY(cudaMemcpyAsync(&ng, bo + nb, sizeof(long long), cudaMemcpyDeviceToHost, st));
    CTRY(cudaStreamSynchronize(st));
    T->nghost = ng;
    CTRY(ensure_ghost_capacity(T, ng));
    if (ng) {
      k_ghost_scatter<<<nb, GM_THREADS, 0, st>>>(T->iblank, nx, ny, nz, ncell, bo, T->gcell);
      k_ghost_bits<<<nblk(ng, 256), 256, 0, st>>>(T->iblank, T->gcell, ng);
    }
    k_count_cells<<<ctx->wave, 256, 0, st>>>(T->iblank, ncell, cellcnt);
    CTRY(cudaGetLastError());
  }
  const long long ng = T->nghost;
  if (ng > 0) {
    // all closed-mesh triangles, concatenated in mesh order (global triangle index)
    double *tv = nullptr;
    float4 *blo = nullptr, *bhi = nullptr, *cen = nullptr;
    CTRY(S.get(&tv, 9 * tottris));
    CTRY(S.get(&blo, tottris)); CTRY(S.get(&bhi, tottris)); CTRY(S.get(&cen, tottris));
    TriStats ts;
    for (int m = 0; m < nmesh; ++m) {
      const int nt = meshes[m].ntris;
      if (nt == 0) continue;
      k_gather_tris<<<nblk(nt, 128), 128, 0, st>>>(dverts + 3LL * vbase[m], dtris + 3LL * tbase[m], nt,
                                                    tv + 9LL * tbase[m]);
      ts.add(meshes[m]);
    }
    k_tri_boxes<<<nblk(tottris, 128), 128, 0, st>>>(tv, (int)tottris, blo, bhi, cen);
    GhostArgs ga;
    CTRY(build_bins(S, tv, (int)tottris, ts, st, ga.bins));
    ga.nx = nx; ga.ny = ny; ga.nz = nz;
    ga.xc = dc[0]; ga.yc = dc[1]; ga.zc = dc[2];
    ga.cxm = dcm[0]; ga.cxp = dcp[0]; ga.cym = dcm[1]; ga.cyp = dcp[1]; ga.czm = dcm[2]; ga.czp = dcp[2];
    ga.ib = T->iblank;
    ga.tv = tv; ga.blo = blo; ga.bhi = bhi; ga.cen = cen;
    ga.ng = ng; ga.gcell = T->gcell;
    ga.bi = T->gbi; ga.ip = T->gip; ga.w = T->gw; ga.scale = T->gscale;
    ga.base = T->gbase; ga.flags = T->gflags; ga.ref = T->gref;
    ga.kappa = T->gkappa; ga.tri = T->gtri; ga.wself = T->gwself;
    k_ghost_tables<<<nblk(32 * ng, TABLE_THREADS), TABLE_THREADS, 0, st>>>(ga);
    CTRY(cudaGetLastError());
  }
  unsigned long long hc[2];
  unsigned hleak = 0;
  CTRY(cudaMemcpyAsync(hc, cellcnt, 16, cudaMemcpyDeviceToHost, st));
  CTRY(cudaMemcpyAsync(&hleak, leak, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CTRY(cudaStreamSynchronize(st));
  T->nfluid = (long long)hc[0];
  T->nsolid = (long long)hc[1];
  CTRY(S.finish());
  T->geom_version += 1;
  ctx->launches += 2 + 2 * (long long)nmesh * 3 + 5 + (T->nghost > 0 ? 5 + (long long)nmesh : 0);
#undef CTRY
  if (hleak) return IBM_ERR_MESH_NOT_CLOSED;
  return T->nfluid == 0 ? IBM_ERR_NO_FLUID : IBM_OK;
}

}  // namespace

// Host orchestration of ibm_classify (see include/ibm_poisson.h).
ibm_status classify_impl(ibm_ctx *ctx, const ibm_grid *grid, const ibm_mesh *meshes, int nmesh, ibm_tables **out,
                         cudaStream_t st) {
  if (!ctx || !grid || !out) return IBM_ERR_INVALID_ARG;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  if (nx < 2 || ny < 2 || nz < 2 || !grid->xf || !grid->yf || !grid->zf) return IBM_ERR_INVALID_ARG;
  const double *fs[3] = {grid->xf, grid->yf, grid->zf};
  const int ns[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i <= ns[a]; ++i) {
      double v = fs[a][i];
      if (!(std::fabs(v) <= COORD_LIMIT) || (i > 0 && !(v > fs[a][i - 1]))) return IBM_ERR_INVALID_ARG;
    }
  long long totverts = 0, tottris = 0;
  ibm_status s = check_meshes(meshes, nmesh, totverts, tottris);
  if (s != IBM_OK) return s;
  IBM_TRY(cudaSetDevice(ctx->device));
  ibm_tables *T = new ibm_tables();
  T->ctx = ctx;
  T->nx = nx; T->ny = ny; T->nz = nz;
  T->xf.assign(grid->xf, grid->xf + nx + 1);
  T->yf.assign(grid->yf, grid->yf + ny + 1);
  T->zf.assign(grid->zf, grid->zf + nz + 1);
  T->ncell = (long long)nx * ny * nz;
  s = classify_into(T, meshes, nmesh, totverts, tottris, st);
  if (s != IBM_OK) {
    ibm_tables_destroy(T);
    return s;
  }
  *out = T;
  return IBM_OK;
}

// Host orchestration of ibm_reclassify: same grid, new body positions, the tables' memory.
ibm_status reclassify_impl(ibm_ctx *ctx, ibm_tables *T, const ibm_mesh *meshes, int nmesh, cudaStream_t st) {
  if (!ctx || !T || T->ctx != ctx) return IBM_ERR_INVALID_ARG;
  long long totverts = 0, tottris = 0;
  ibm_status s = check_meshes(meshes, nmesh, totverts, tottris);
  if (s != IBM_OK) return s;
  IBM_TRY(cudaSetDevice(ctx->device));
  return classify_into(T, meshes, nmesh, totverts, tottris, st);
}

// ---------------------------------------------------------------------- Neumann datum
//
// The moving-boundary pressure condition dp/dn = -rho Du_b/Dt . n (the fractional-step
// projection at a body moving with acceleration a): ghost row g - sum w v = kappa q with q
// the derivative along the row's direction (towards IP, or towards a fallback neighbour).

namespace {

__global__ void k_set_datum(const double *kappa, const double *q, long long ng, double *d) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g < ng) d[g] = kappa[g] * q[g];
}

constexpr int MAX_RIGID = 32;
struct RigidMotions {
  int n;
  int off[MAX_RIGID + 1];   // first global triangle index of each mesh, and the total
  double m[MAX_RIGID][12];  // per mesh: a0 (3), angular acceleration (3), angular velocity (3), centre (3)
};

// q = -a(BI) . n (rho = 1), a(x) = a0 + alpha x r + omega x (omega x r), r = x - centre, for
// the mesh holding the ghost's closest triangle; n the unit direction of the row; d = kappa q
__global__ void k_rigid_datum(const double *kappa, const double *bi, const double *ip, const long long *gcell,
                              const int *flags, const long long *ref, const int *tri, long long ng, const double *xc,
                              const double *yc, const double *zc, int nx, int ny, RigidMotions M, double *d) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ng) return;
  int lo = 0, hi = M.n;   // the mesh: largest m with off[m] <= tri
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (M.off[mid] <= tri[g]) lo = mid; else hi = mid;
  }
  const double *mm = M.m[lo];
  const long long c = gcell[g];
  const double G[3] = {xc[c % nx], yc[(c / nx) % ny], zc[c / ((long long)nx * ny)]};
  double t[3];
  if (flags[g] & 1) {
    const long long nb = ref[8 * g];
    t[0] = xc[nb % nx] - G[0]; t[1] = yc[(nb / nx) % ny] - G[1]; t[2] = zc[nb / ((long long)nx * ny)] - G[2];
  } else {
    for (int q = 0; q < 3; ++q) t[q] = ip[3 * g + q] - G[q];
  }
  const double len = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  const double r[3] = {bi[3 * g] - mm[9], bi[3 * g + 1] - mm[10], bi[3 * g + 2] - mm[11]};
  const double *al = mm + 3, *om = mm + 6;
  const double wr[3] = {om[1] * r[2] - om[2] * r[1], om[2] * r[0] - om[0] * r[2], om[0] * r[1] - om[1] * r[0]};
  double a[3];
  a[0] = mm[0] + (al[1] * r[2] - al[2] * r[1]) + (om[1] * wr[2] - om[2] * wr[1]);
  a[1] = mm[1] + (al[2] * r[0] - al[0] * r[2]) + (om[2] * wr[0] - om[0] * wr[2]);
  a[2] = mm[2] + (al[0] * r[1] - al[1] * r[0]) + (om[0] * wr[1] - om[1] * wr[0]);
  const double q = len > 0.0 ? -(a[0] * t[0] + a[1] * t[1] + a[2] * t[2]) / len : 0.0;
  d[g] = kappa[g] * q;
}

// device pointers to the cell centres of each axis in the tables' axis block
void axis_centres(const ibm_tables *T, const double *c[3]) {
  const int ns[3] = {T->nx, T->ny, T->nz};
  size_t o = 0;
  for (int a = 0; a < 3; ++a) {
    c[a] = T->axis + o + ns[a] + 1;
    o += 6 * (size_t)ns[a] + 1;
  }
}

}  // namespace

ibm_status neumann_set_impl(ibm_tables *T, const double *q, cudaStream_t st) {
  if (!q) { T->has_datum = false; return IBM_OK; }
  const long long ng = T->nghost;
  if (ng > 0) k_set_datum<<<nblk(ng, 256), 256, 0, st>>>(T->gkappa, q, ng, T->gd);
  IBM_TRY(cudaGetLastError());
  T->has_datum = ng > 0;
  T->ctx->launches += ng > 0 ? 1 : 0;
  return IBM_OK;
}

ibm_status neumann_rigid_impl(ibm_tables *T, const double *motions, int nmesh, cudaStream_t st) {
  if (nmesh < 1 || nmesh + 1 != (int)T->mesh_tri_off.size() || !motions) return IBM_ERR_INVALID_ARG;
  if (nmesh > MAX_RIGID) return IBM_ERR_CAPACITY;
  RigidMotions M;
  M.n = nmesh;
  for (int m = 0; m <= nmesh; ++m) M.off[m] = T->mesh_tri_off[m];
  for (int m = 0; m < nmesh; ++m)
    for (int q = 0; q < 12; ++q) M.m[m][q] = motions[12 * m + q];
  const long long ng = T->nghost;
  if (ng > 0) {
    const double *c[3];
    axis_centres(T, c);
    k_rigid_datum<<<nblk(ng, 256), 256, 0, st>>>(T->gkappa, T->gbi, T->gip, T->gcell, T->gflags, T->gref, T->gtri, ng,
                                                 c[0], c[1], c[2], T->nx, T->ny, M, T->gd);
    T->ctx->launches += 1;
  }
  IBM_TRY(cudaGetLastError());
  T->has_datum = ng > 0;
  return IBM_OK;
}

}  // namespace ibm
