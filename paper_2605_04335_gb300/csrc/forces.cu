// Surface pressure on both sides of the classified meshes' triangles and the nodal pressure
// forces: the pressure part of the external force on the structure's nodes (Sec. "Force
// Formulations": each node receives one third of the traction times the area of every
// triangle that holds it, the traction's pressure part being -dp n).
//
// The paper does not say how dp is read from the cell-centred pressure.  Reading (the probe
// rule of ghost-cell methods with the image-point interpolation of the classification):
//   triangle t: N = (v1 - v0) x (v2 - v0), n = N / |N|, centroid c = ((v0 + v1) + v2) / 3;
//   probe distance d = 1.5 x the diagonal of the cell holding c; side s = +1 / -1 probes at
//   X = c + (s d) n, trilinear weights on the cell-centre lattice (base corner clamped to
//   [0, n-2], t clamped to [0, 1]); a corner is used when it holds fluid on side s (closed
//   bodies: iblank 0; membranes: its centre strictly on side s of the triangle's plane);
//   p_s = (sum w p) / (sum w) - (s d) q, q = dp/dn at c (given per triangle, or -a(c).n from
//   rigid kinematics per mesh, or 0); sum w < 1e-3 leaves p_s = 0 and sets flag bit s.
//   Closed bodies: p_- = 0.  f_t = -(dp (N / 2)), dp = p_+ - p_-; node i: sum over its
//   triangles, in ascending order, of f_t / 3.
// Every FP64 operation is separately rounded (built with -fmad=false) in that order, so the
// results are reproducible bit for bit by a plain implementation of the same definition.
#include <vector>

#include "ibm_internal.cuh"

namespace ibm {

namespace {

constexpr double PROBE_FACTOR = 1.5;
constexpr double SIDE_WEIGHT_MIN = 1e-3;
constexpr int FLAG_ZERO_AREA = 4;
constexpr int MAX_MOTIONS = 32;
constexpr int SCAN_THREADS = 1024;

struct Motions {
  int n;                        // 0: no rigid kinematics
  int off[MAX_MOTIONS + 1];     // first triangle of each mesh, and the total
  double m[MAX_MOTIONS][12];    // per mesh: a0 (3), angular acceleration (3), angular velocity (3), centre (3)
};

struct ForceArgs {
  const double *verts;          // [nvert][3], all meshes
  const int *tris;              // [ntri][3], global vertex indices
  int ntri;
  const double *f[3], *c[3], *w[3];   // per axis: faces, centres, widths
  int n[3];
  const uint8_t *iblank;        // closed bodies
  bool membrane;
  const double *p;              // [nz][ny][nx]
  const double *q;              // per triangle, or null
  double *pside;                // [ntri][2]
  uint8_t *flags;               // [ntri]
  double *share;                // [ntri][3]: f_t / 3
};

// number of entries <= v in the ascending array a[0..n)
__device__ __forceinline__ int count_le(const double *a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void lattice(const double *c, int n, double v, int &i0, double &t) {
  i0 = count_le(c, n, v) - 1;
  i0 = i0 < 0 ? 0 : (i0 > n - 2 ? n - 2 : i0);
  t = (v - c[i0]) / (c[i0 + 1] - c[i0]);
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

__global__ void k_tri_pressure(ForceArgs a, Motions M) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.ntri) return;
  const double *v0 = a.verts + 3LL * a.tris[3 * t], *v1 = a.verts + 3LL * a.tris[3 * t + 1],
               *v2 = a.verts + 3LL * a.tris[3 * t + 2];
  const double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
  const double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
  const double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const double a2 = sqrt((N[0] * N[0] + N[1] * N[1]) + N[2] * N[2]);
  const bool live = a2 > 0.0;
  double n[3];
  for (int d = 0; d < 3; ++d) n[d] = live ? N[d] / a2 : 0.0;
  double c[3];
  for (int d = 0; d < 3; ++d) c[d] = ((v0[d] + v1[d]) + v2[d]) / 3.0;
  double q = 0.0;
  if (a.q) {
    q = a.q[t];
  } else if (M.n > 0) {
    int lo = 0, hi = M.n;   // the mesh: largest m with off[m] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (M.off[mid] <= t) lo = mid; else hi = mid;
    }
    const double *mm = M.m[lo], *al = mm + 3, *om = mm + 6;
    const double r[3] = {c[0] - mm[9], c[1] - mm[10], c[2] - mm[11]};
    const double wr[3] = {om[1] * r[2] - om[2] * r[1], om[2] * r[0] - om[0] * r[2], om[0] * r[1] - om[1] * r[0]};
    const double ax = (mm[0] + (al[1] * r[2] - al[2] * r[1])) + (om[1] * wr[2] - om[2] * wr[1]);
    const double ay = (mm[1] + (al[2] * r[0] - al[0] * r[2])) + (om[2] * wr[0] - om[0] * wr[2]);
    const double az = (mm[2] + (al[0] * r[1] - al[1] * r[0])) + (om[0] * wr[1] - om[1] * wr[0]);
    q = -((ax * n[0] + ay * n[1]) + az * n[2]);
  }
  double h[3];
  for (int d = 0; d < 3; ++d) {
    int i = count_le(a.f[d], a.n[d] + 1, c[d]) - 1;
    i = i < 0 ? 0 : (i > a.n[d] - 1 ? a.n[d] - 1 : i);
    h[d] = a.w[d][i];
  }
  const double dist = PROBE_FACTOR * sqrt((h[0] * h[0] + h[1] * h[1]) + h[2] * h[2]);
  int flags = live ? 0 : FLAG_ZERO_AREA;
  const int nx = a.n[0], ny = a.n[1];
  double ps[2] = {0.0, 0.0};
  const int nside = a.membrane ? 2 : 1;
  for (int slot = 0; slot < nside; ++slot) {
    const double sd = slot == 0 ? dist : -dist;
    int b[3];
    double tw[3];
    for (int d = 0; d < 3; ++d) lattice(a.c[d], a.n[d], c[d] + sd * n[d], b[d], tw[d]);
    const double wx[2] = {1.0 - tw[0], tw[0]}, wy[2] = {1.0 - tw[1], tw[1]}, wz[2] = {1.0 - tw[2], tw[2]};
    double sw = 0.0, v = 0.0;
    for (int cc = 0; cc < 8; ++cc) {
      const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
      const long long lin = ((long long)(b[2] + bz) * ny + (b[1] + by)) * nx + (b[0] + bx);
      const double w = (wx[bx] * wy[by]) * wz[bz];
      bool use;
      if (a.membrane) {
        const double dot = ((a.c[0][b[0] + bx] - c[0]) * n[0] + (a.c[1][b[1] + by] - c[1]) * n[1]) +
                           (a.c[2][b[2] + bz] - c[2]) * n[2];
        use = slot == 0 ? dot > 0.0 : dot < 0.0;
      } else {
        use = a.iblank[lin] == 0;
      }
      if (use) {
        sw = sw + w;
        v = v + w * a.p[lin];
      }
    }
    if (live && sw >= SIDE_WEIGHT_MIN) ps[slot] = v / sw - sd * q;
    else if (live) flags |= 1 << slot;
  }
  a.pside[2 * t] = ps[0];
  a.pside[2 * t + 1] = ps[1];
  a.flags[t] = (uint8_t)flags;
  const double dp = ps[0] - ps[1];
  for (int d = 0; d < 3; ++d) a.share[3 * t + d] = live ? -(dp * (0.5 * N[d])) / 3.0 : 0.0;
}

// vertex -> triangle incidence (CSR): counts, exclusive scan, fill
__global__ void k_inc_count(const int *tris, int ntri, int *cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntri)
    for (int k = 0; k < 3; ++k) atomicAdd(cnt + tris[3 * t + k], 1);
}

// exclusive scan of cnt[0..n) into off[0..n] in one block: per-thread chunks, then a scan of
// the chunk totals
__global__ void __launch_bounds__(SCAN_THREADS) k_inc_scan(const int *cnt, int n, int *off) {
  __shared__ int tot[SCAN_THREADS];
  const int chunk = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  const int b = threadIdx.x * chunk, e = min(n, b + chunk);
  int s = 0;
  for (int i = b; i < e; ++i) s += cnt[i];
  tot[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < SCAN_THREADS; d <<= 1) {
    const int x = threadIdx.x >= d ? tot[threadIdx.x - d] : 0;
    __syncthreads();
    tot[threadIdx.x] += x;
    __syncthreads();
  }
  int run = tot[threadIdx.x] - s;
  for (int i = b; i < e; ++i) {
    off[i] = run;
    run += cnt[i];
  }
  if (threadIdx.x == SCAN_THREADS - 1) off[n] = tot[SCAN_THREADS - 1];
}

__global__ void k_inc_fill(const int *tris, int ntri, const int *off, int *cur, int *list) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntri) return;
  for (int k = 0; k < 3; ++k) {
    const int v = tris[3 * t + k];
    list[off[v] + atomicAdd(cur + v, 1)] = t;
  }
}

// F_i = sum of the shares of node i's triangles in ascending triangle order (the fill order is
// arbitrary: each step takes the smallest triangle index above the last one, with its
// multiplicity)
__global__ void k_node_forces(const int *off, const int *list, const double *share, long long nvert, double *F) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nvert) return;
  const int b = off[i], e = off[i + 1];
  double acc[3] = {0.0, 0.0, 0.0};
  int last = -1;
  for (int done = b; done < e;) {
    int tmin = 0x7fffffff, mult = 0;
    for (int k = b; k < e; ++k) {
      const int t = list[k];
      if (t > last && t < tmin) { tmin = t; mult = 1; }
      else if (t == tmin) ++mult;
    }
    for (int r = 0; r < mult; ++r)
      for (int d = 0; d < 3; ++d) acc[d] = acc[d] + share[3LL * tmin + d];
    last = tmin;
    done += mult;
  }
  for (int d = 0; d < 3; ++d) F[3 * i + d] = acc[d];
}

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

ibm_status surface_forces_impl(ibm_tables *T, const ibm_mesh *meshes, int nmesh, const double *p,
                               const double *q_tri, const double *motions, double *p_side, uint8_t *flags,
                               double *f_node, cudaStream_t st) {
  if (!meshes || nmesh < 1 || !p || !f_node || (q_tri && motions)) return IBM_ERR_INVALID_ARG;
  if (nmesh + 1 != (int)T->mesh_tri_off.size()) return IBM_ERR_INVALID_ARG;
  if (motions && nmesh > MAX_MOTIONS) return IBM_ERR_CAPACITY;
  long long nvert = 0;
  for (int m = 0; m < nmesh; ++m) {
    const ibm_mesh &M = meshes[m];
    if (M.ntris != T->mesh_tri_off[m + 1] - T->mesh_tri_off[m]) return IBM_ERR_INVALID_ARG;
    if ((M.closed == 0) != T->membrane) return IBM_ERR_INVALID_ARG;
    if (M.nverts < 0 || (M.ntris > 0 && (!M.verts || !M.tris))) return IBM_ERR_INVALID_ARG;
    for (long long k = 0; k < 3LL * M.ntris; ++k)
      if (M.tris[k] < 0 || M.tris[k] >= M.nverts) return IBM_ERR_INVALID_ARG;
    nvert += M.nverts;
  }
  const long long ntri = T->mesh_tri_off[nmesh];
  if (nvert > 0x7ffffffeLL || ntri > 0x7ffffffeLL / 3) return IBM_ERR_CAPACITY;
  if (nvert == 0) return IBM_OK;
  // device working set in the tables' force buffer (grown when needed, kept between calls)
  const size_t b_verts = align256(24 * nvert), b_share = align256(24 * (ntri + 1)), b_side = align256(16 * (ntri + 1)),
               b_tris = align256(12 * (ntri + 1)), b_cnt = align256(4 * (nvert + 1)), b_flags = align256(ntri + 1);
  const size_t need = b_verts + b_share + b_side + 2 * b_tris + 3 * b_cnt + b_flags;
  if (need > T->fcap) {
    IBM_TRY(cudaStreamSynchronize(st));
    if (T->fbuf) cudaFree(T->fbuf);
    T->fbuf = nullptr;
    T->fcap = 0;
    IBM_TRY(cudaMalloc((void **)&T->fbuf, need));
    T->fcap = need;
  }
  char *o = T->fbuf;
  double *dverts = (double *)o; o += b_verts;
  double *share = (double *)o; o += b_share;
  double *side_tmp = (double *)o; o += b_side;
  int *dtris = (int *)o; o += b_tris;
  int *list = (int *)o; o += b_tris;
  int *cnt = (int *)o; o += b_cnt;
  int *off = (int *)o; o += b_cnt;
  int *cur = (int *)o; o += b_cnt;
  uint8_t *flags_tmp = (uint8_t *)o;
  // global vertex numbering: mesh after mesh (host staging of the offset triangle indices)
  std::vector<int> htris(3 * (size_t)ntri);
  long long vo = 0, to = 0;
  for (int m = 0; m < nmesh; ++m) {
    const ibm_mesh &M = meshes[m];
    if (M.nverts)
      IBM_TRY(cudaMemcpyAsync(dverts + 3 * vo, M.verts, 24 * (size_t)M.nverts, cudaMemcpyHostToDevice, st));
    for (long long k = 0; k < 3LL * M.ntris; ++k) htris[3 * to + k] = (int)(M.tris[k] + vo);
    vo += M.nverts;
    to += M.ntris;
  }
  if (ntri > 0) IBM_TRY(cudaMemcpyAsync(dtris, htris.data(), 12 * (size_t)ntri, cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemsetAsync(cnt, 0, 4 * (size_t)(nvert + 1), st));
  IBM_TRY(cudaMemsetAsync(cur, 0, 4 * (size_t)(nvert + 1), st));
  Motions Mo;
  Mo.n = motions ? nmesh : 0;
  for (int m = 0; m <= nmesh && m <= MAX_MOTIONS; ++m) Mo.off[m] = T->mesh_tri_off[m];
  if (motions)
    for (int m = 0; m < nmesh; ++m)
      for (int k = 0; k < 12; ++k) Mo.m[m][k] = motions[12 * m + k];
  ForceArgs a;
  a.verts = dverts;
  a.tris = dtris;
  a.ntri = (int)ntri;
  const int ns[3] = {T->nx, T->ny, T->nz};
  size_t ao = 0;
  for (int d = 0; d < 3; ++d) {   // axis block: faces (n+1), centres, widths, coefficients, ...
    a.f[d] = T->axis + ao;
    a.c[d] = a.f[d] + ns[d] + 1;
    a.w[d] = a.c[d] + ns[d];
    a.n[d] = ns[d];
    ao += 6 * (size_t)ns[d] + 1;
  }
  a.iblank = T->iblank;
  a.membrane = T->membrane;
  a.p = p;
  a.q = q_tri;
  a.pside = p_side ? p_side : side_tmp;
  a.flags = flags ? flags : flags_tmp;
  a.share = share;
  long long launches = 2;
  if (ntri > 0) {
    k_tri_pressure<<<nblocks(ntri, 128), 128, 0, st>>>(a, Mo);
    k_inc_count<<<nblocks(ntri, 256), 256, 0, st>>>(dtris, (int)ntri, cnt);
    launches += 2;
  }
  k_inc_scan<<<1, SCAN_THREADS, 0, st>>>(cnt, (int)nvert, off);
  if (ntri > 0) {
    k_inc_fill<<<nblocks(ntri, 256), 256, 0, st>>>(dtris, (int)ntri, off, cur, list);
    ++launches;
  }
  k_node_forces<<<nblocks(nvert, 128), 128, 0, st>>>(off, list, share, nvert, f_node);
  IBM_TRY(cudaGetLastError());
  T->ctx->launches += launches;
  // the staging vector is read by the copy above before it returns (pageable host memory)
  return IBM_OK;
}

}  // namespace ibm
