// Batched solves: many independent pressure Poisson problems of uneven sizes advanced
// together, one persistent launch per V-cycle stage.  Included by mg.cu (uses its level
// views, stencil helpers and per-problem hierarchies).
//
// A stage (one colour of a sweep at level l, ghost rows, restriction l -> l+1, the
// coarsest solves, prolongation l+1 -> l, the FP64 residual, the refinement update) is a
// single kernel over the work items of every problem that has that stage: a grid of a
// few blocks per SM walks a global item index, and a binary search over the per-problem
// item prefix finds the problem of each item.  Problems whose hierarchies are shallower
// simply have no items at the deeper stages; each problem's coarsest level is solved in
// one common launch between the downward and the upward pass.  Items are chunks that
// never straddle two problems, so per-problem sums are written per chunk and added in a
// fixed order (deterministic).  A converged problem's flag turns its items into no-ops,
// so the captured graph of one batched cycle can be replayed unchanged.
#pragma once

namespace ibm {
namespace {

constexpr int BT = 128;          // threads per block of the batched kernels
constexpr int BCHUNK = 256;      // coarse cells (restriction) / rows (residual) per reduction chunk

template <typename T>
struct BLev {                    // one problem at one level
  LV<T> v;
  T *e, *r;
  int present;                   // this level exists and is not the problem's coarsest
  int coarsest;                  // this level is the problem's coarsest
};

struct BProb {
  double *scal;                  // NSCAL device scalars of this problem
  const int *active;             // 1 while the problem iterates
  // finest level, FP64 side
  double *p64, *b64;
  LV<double> v64;
  long long ng;
  const long long *gsrc, *gdst;
  const double *gw;
  const float *gw32;
  const double *gscale;
  double *gtmp;
  // coarsest
  const void *minv;   // element type of the levels
  const int *cidx, *ncoarse;
  long long ntot0;
};

__device__ __forceinline__ int find_prob(const long long *off, int np, long long item) {
  int lo = 0, hi = np;          // largest p with off[p] <= item
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid;
  }
  return lo;
}

// one colour of red-black SOR at level l for every problem: item = (row j,k, x-block)
template <typename T>
__global__ void kb_rbgs(const BLev<T> *L, const BProb *P, const long long *off, int np, int colour, float omega,
                        int shift_slot) {
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    if (!*P[p].active) continue;
    const BLev<T> &B = L[p];
    const LV<T> &v = B.v;
    const long long loc = it - off[p];
    const int xb = (v.nx + 1) / 2, nxb = (xb + BT - 1) / BT;
    const int bx = (int)(loc % nxb);
    const long long row = loc / nxb;
    const int j = (int)(row % v.ny), k = (int)(row / v.ny);
    const int i = 2 * (bx * BT + threadIdx.x) + ((j + k + colour) & 1);
    if (i >= v.nx) continue;
    const long long id = vidx(v, i, j, k);
    if (v.mask[id] != 0) continue;
    T c[6];
    coefs(v, i, j, k, id, c);
    const T D = v.sdx ? (v.sdx[i] + v.sdy[j]) + v.sdz[k] : ((c[0] + c[1]) + (c[2] + c[3])) + (c[4] + c[5]);
    if (D == (T)0) continue;
    const T rhs = B.r[id] - (T)P[p].scal[shift_slot];
    const T res = stencil_sum(v, B.e, id, c) - D * B.e[id] - rhs;
    B.e[id] += (T)__fdividef(omega * (float)res, (float)D);
  }
}

// ghost rows of the finest level (Jacobi: evaluate into gtmp, then store)
template <typename T>
__global__ void kb_ghost_eval(const BLev<T> *L, const BProb *P, const long long *off, int np, int with_rhs) {
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    if (!*P[p].active) continue;
    const long long g = (it - off[p]) * BT + threadIdx.x;
    if (g >= P[p].ng) continue;
    const T *e = L[p].e;
    T s = (T)0;
    for (int c = 0; c < 8; ++c) {
      const long long q = P[p].gsrc[8 * g + c];
      if (q < 0) continue;
      const T w = sizeof(T) == 8 ? (T)P[p].gw[8 * g + c] : (T)P[p].gw32[8 * g + c];
      s += w * e[q & ~GHOST_CORNER];
    }
    if (with_rhs) s += L[p].r[P[p].gdst[g]];
    ((T *)P[p].gtmp)[g] = s;
  }
}

template <typename T>
__global__ void kb_ghost_store(const BLev<T> *L, const BProb *P, const long long *off, int np) {
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    if (!*P[p].active) continue;
    const long long g = (it - off[p]) * BT + threadIdx.x;
    if (g >= P[p].ng) continue;
    L[p].e[P[p].gdst[g]] = ((const T *)P[p].gtmp)[g];
  }
}

// residual of level l restricted to level l+1 (and the coarse correction zeroed);
// item = chunk of BCHUNK coarse cells; partial sum of V_c r_c per chunk
template <typename T>
__global__ void kb_restrict(const BLev<T> *F, const BLev<T> *Cl, const BProb *P, const long long *off, int np,
                            int shift_slot, double *part) {
  __shared__ double sm[BT];
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    double acc_all = 0.0;
    if (*P[p].active) {
      const LV<T> &f = F[p].v, &cv = Cl[p].v;
      const T sh = (T)P[p].scal[shift_slot];
      const long long nc = (long long)cv.nx * cv.ny * cv.nz;
      const long long c0 = (it - off[p]) * BCHUNK;
      for (long long l = c0 + threadIdx.x; l < min(nc, c0 + BCHUNK); l += BT) {
        const int I = (int)(l % cv.nx);
        const long long q = l / cv.nx;
        const int J = (int)(q % cv.ny), K = (int)(q / cv.ny);
        const long long ic = vidx(cv, I, J, K);
        Cl[p].e[ic] = (T)0;
        if (cv.mask[ic] != 0) { Cl[p].r[ic] = (T)0; continue; }
        T acc = (T)0;
        for (int c = 0; c < 8; ++c) {
          const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
          if (i >= f.nx || j >= f.ny || k >= f.nz) continue;
          const long long id = vidx(f, i, j, k);
          if (f.mask[id] != 0) continue;
          T cf[6];
          coefs(f, i, j, k, id, cf);
          const T D = f.sdx ? (f.sdx[i] + f.sdy[j]) + f.sdz[k] : ((cf[0] + cf[1]) + (cf[2] + cf[3])) + (cf[4] + cf[5]);
          const T res = (F[p].r[id] - sh) - (stencil_sum(f, F[p].e, id, cf) - D * F[p].e[id]);
          acc += (f.wx[i] * f.wy[j]) * f.wz[k] * res;
        }
        const T vc = (cv.wx[I] * cv.wy[J]) * cv.wz[K];
        Cl[p].r[ic] = acc / vc;
        acc_all += (double)acc;
      }
    }
    sm[threadIdx.x] = acc_all;
    __syncthreads();
    for (int st = BT / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[it] = sm[0];
    __syncthreads();
  }
}

// per problem: coarse projection shift = sum of its chunk partials / fluid volume
__global__ void kb_finalize_shift(const BProb *P, const long long *off, int np, const double *part,
                                  const double *fluid_vol, int slot) {
  const int p = blockIdx.x;
  if (p >= np || !*P[p].active) return;
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (long long c = off[p]; c < off[p + 1]; ++c) s += part[c];
    P[p].scal[slot] = fluid_vol[p] > 0 ? s / fluid_vol[p] : 0.0;
  }
}

// prolongation l+1 -> l: item = (row, x-block) of the fine level
template <typename T>
__global__ void kb_prolong(const BLev<T> *Cl, const BLev<T> *F, const BProb *P, const long long *off, int np,
                           int8_t *const *poff, float *const *pt) {
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    if (!*P[p].active) continue;
    const LV<T> &f = F[p].v, &cv = Cl[p].v;
    const long long loc = it - off[p];
    const int nxb = (f.nx + BT - 1) / BT;
    const int i = (int)(loc % nxb) * BT + threadIdx.x;
    const long long row = loc / nxb;
    const int j = (int)(row % f.ny), k = (int)(row / f.ny);
    if (i >= f.nx) continue;
    const long long id = vidx(f, i, j, k);
    if (f.mask[id] != 0) continue;
    const int8_t *ox = poff[p], *oy = ox + f.nx, *oz = oy + f.ny;
    const float *tx = pt[p], *ty = tx + f.nx, *tz = ty + f.ny;
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const float wx[2] = {1.0f - tx[i], tx[i]}, wy[2] = {1.0f - ty[j], ty[j]}, wz[2] = {1.0f - tz[k], tz[k]};
    T s = (T)0;
    float ws = 0.0f;
    for (int c = 0; c < 8; ++c) {
      const int a = c & 1, b = (c >> 1) & 1, d = (c >> 2) & 1;
      const float w = (wx[a] * wy[b]) * wz[d];
      if (w == 0.0f) continue;
      const long long ic = vidx(cv, I + a * ox[i], J + b * oy[j], K + d * oz[k]);
      if (cv.mask[ic] != 0) continue;
      s += (T)w * Cl[p].e[ic];
      ws += w;
    }
    if (ws > 0.0f) F[p].e[id] += s * (T)(1.0f / ws);
  }
}

// every problem's coarsest level, one block per problem
template <typename T>
__global__ void kb_coarsest(const BLev<T> *const *Lc, const BProb *P, int np) {
  __shared__ double rs[MAX_COARSE + 1];
  const int p = blockIdx.x;
  if (p >= np || !*P[p].active) return;
  const BLev<T> &B = *Lc[p];
  const int n = *P[p].ncoarse, m = n + 1;
  for (int q = threadIdx.x; q < n; q += blockDim.x) rs[q] = (double)B.r[P[p].cidx[q]];
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    double s = 0.0;
    const T *Mv = static_cast<const T *>(P[p].minv);
    for (int c = 0; c < n; ++c) s += (double)Mv[q * m + c] * rs[c];
    B.e[P[p].cidx[q]] = (T)s;
  }
}

// FP64 fine residual per problem: item = chunk of BCHUNK rows; partials (V r, r, r^2) per chunk
__global__ void kb_residual64(const BProb *P, const long long *off, int np, const float *const *r32, int use_p,
                              double *part) {
  __shared__ double sm[3][BT];
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    double A0 = 0.0, A1 = 0.0, A2 = 0.0;
    if (*P[p].active) {
      const LV<double> &v = P[p].v64;
      const double lam = P[p].scal[S_LAMBDA];
      float *r = r32 ? (float *)r32[p] : nullptr;   // no FP32 copy in FP64 mode
      const long long rows = (long long)v.ny * v.nz;
      const long long r0 = (it - off[p]) * BCHUNK;
      for (long long row = r0; row < min(rows, r0 + BCHUNK); ++row) {
        const int j = (int)(row % v.ny), k = (int)(row / v.ny);
        const double cym = v.cym[j], cyp = v.cyp[j], czm = v.czm[k], czp = v.czp[k];
        const double syz = v.sdy[j] + v.sdz[k];
        const float dydz = (float)(v.dy[j] * v.dz[k]);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int i = threadIdx.x; i < v.nx; i += BT) {
          const long long id = vidx(v, i, j, k);
          if (v.mask[id] != 0) continue;
          double res;
          const double *pp = P[p].p64;
          if (use_p) {
            double s = v.cxm[i] * pp[id - 1];
            s = fma(v.cxp[i], pp[id + 1], s);
            s = fma(cym, pp[id - v.sy], s);
            s = fma(cyp, pp[id + v.sy], s);
            s = fma(czm, pp[id - v.sz], s);
            s = fma(czp, pp[id + v.sz], s);
            s = fma(-(v.sdx[i] + syz), pp[id], s);
            res = (P[p].b64[id] - lam) - s;
          } else {
            res = P[p].b64[id] - lam;
          }
          const float rf = (float)res;
          if (r) r[id] = rf;
          a0 = fmaf((float)v.dx[i] * dydz, rf, a0);
          a1 += rf;
          a2 = fmaf(rf, rf, a2);
        }
        A0 += a0; A1 += a1; A2 += a2;
      }
    }
    sm[0][threadIdx.x] = A0; sm[1][threadIdx.x] = A1; sm[2][threadIdx.x] = A2;
    __syncthreads();
    for (int st = BT / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st)
        for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < 3; ++q) part[3 * it + q] = sm[q][0];
    __syncthreads();
  }
}

// ghost-row residuals per problem: item = chunk of BCHUNK ghosts; partial (s r_G)^2 per chunk
__global__ void kb_ghost_resid64(const BProb *P, const long long *off, int np, const float *const *r32, double *part) {
  __shared__ double sm[BT];
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    double a = 0.0;
    if (*P[p].active) {
      const long long g0 = (it - off[p]) * BCHUNK;
      const double *pp = P[p].p64;
      float *r = r32 ? (float *)r32[p] : nullptr;   // no FP32 copy in FP64 mode
      for (long long g = g0 + threadIdx.x; g < min(P[p].ng, g0 + BCHUNK); g += BT) {
        double s = 0.0;
        for (int c = 0; c < 8; ++c) {
          const long long q = P[p].gsrc[8 * g + c];
          if (q >= 0) s += P[p].gw[8 * g + c] * pp[q & ~GHOST_CORNER];
        }
        const double rg = s - pp[P[p].gdst[g]];
        if (r) r[P[p].gdst[g]] = (float)rg;
        const double sr = P[p].gscale[g] * rg;
        a += sr * sr;
      }
    }
    sm[threadIdx.x] = a;
    __syncthreads();
    for (int st = BT / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[it] = sm[0];
    __syncthreads();
  }
}

__global__ void kb_finalize_resid(const BProb *P, int np, const long long *roff, const double *rpart,
                                  const long long *goff, const double *gpart, int update_lambda) {
  const int p = blockIdx.x;
  if (p >= np || !*P[p].active || threadIdx.x != 0) return;
  double sv = 0, s1 = 0, s2 = 0, sg = 0;
  for (long long c = roff[p]; c < roff[p + 1]; ++c) { sv += rpart[3 * c]; s1 += rpart[3 * c + 1]; s2 += rpart[3 * c + 2]; }
  for (long long c = goff[p]; c < goff[p + 1]; ++c) sg += gpart[c];
  double *scal = P[p].scal;
  const double mu = sv / scal[S_FLUIDVOL];
  const double n2 = s2 - 2.0 * mu * s1 + scal[S_NF] * mu * mu;
  scal[S_MU] = mu;
  scal[S_NORM2] = (n2 > 0.0 ? n2 : 0.0) + sg;
  if (update_lambda) scal[S_LAMBDA] += mu;
}

// p += e (mixed) or e = 0 (start of an inner solve): item = chunk of padded cells
template <typename T>
__global__ void kb_fine_elementwise(const BLev<T> *L0, const BProb *P, const long long *off, int np, int op) {
  const long long total = off[np];
  for (long long it = blockIdx.x; it < total; it += gridDim.x) {
    const int p = find_prob(off, np, it);
    if (!*P[p].active) continue;
    const long long q = (it - off[p]) * BT + threadIdx.x;
    if (q >= P[p].ntot0) continue;
    if (op == 0) L0[p].e[q] = (T)0;
    else P[p].p64[q] += (double)L0[p].e[q];
  }
}

}  // namespace

// ------------------------------------------------------------------ batched driver

namespace {

struct BatchPlan {
  int np = 0, nlev = 0, prec = 0;
  std::vector<Hierarchy *> hs;
  std::vector<ibm_tables *> ts;
  // device tables
  void *d_lev = nullptr;                 // BLev<T>[nlev][np]
  BProb *d_prob = nullptr;
  int *d_active = nullptr;
  double *d_scal = nullptr;              // np * NSCAL
  double *d_fvol = nullptr;              // nlev * np coarse fluid volumes
  const BLev<float> **d_lc32 = nullptr;  // per problem: its coarsest BLev (either type)
  int8_t **d_poff = nullptr;             // nlev * np
  float **d_pt = nullptr;
  float **d_r32 = nullptr;               // np
  long long *d_off = nullptr;            // all prefix arrays, (np+1) each
  double *d_part = nullptr;
  std::vector<long long> off_host;
  // prefix offsets (indices into d_off, in units of np+1)
  std::vector<int> o_rbgs, o_restrict, o_prolong;
  int o_ghost = 0, o_res = 0, o_gres = 0, o_fine = 0;
  std::vector<long long> tot_rbgs, tot_restrict, tot_prolong;
  long long tot_ghost = 0, tot_res = 0, tot_gres = 0, tot_fine = 0;
  void *graph_exec = nullptr;
  long long graph_key = -1, graph_launches = 0;
};

void free_plan(BatchPlan &B) {
  void *ps[] = {B.d_lev, B.d_prob, B.d_active, B.d_scal, B.d_fvol, B.d_lc32, B.d_poff, B.d_pt, B.d_r32, B.d_off, B.d_part};
  for (void *p : ps) if (p) cudaFree(p);
  if (B.graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)B.graph_exec);
}

inline unsigned persistent_grid(ibm_ctx *ctx, long long items) {
  const long long cap = 8LL * (ctx->sm_count > 0 ? ctx->sm_count : 152);
  return (unsigned)std::max<long long>(1, std::min<long long>(items, cap));
}

template <typename T>
ibm_status plan_batch(ibm_ctx *ctx, BatchPlan &B, cudaStream_t st) {
  const int np = B.np;
  int nlev = 0;
  for (Hierarchy *h : B.hs) nlev = std::max(nlev, (int)h->lv.size());
  B.nlev = nlev;
  std::vector<BLev<T>> lev((size_t)nlev * np);
  std::vector<BProb> prob(np);
  std::vector<double> fvol((size_t)nlev * np, 0.0);
  std::vector<int8_t *> poff((size_t)nlev * np, nullptr);
  std::vector<float *> pt((size_t)nlev * np, nullptr);
  std::vector<float *> r32(np, nullptr);
  std::vector<long long> off;
  auto add_prefix = [&](const std::vector<long long> &cnt) {
    int at = (int)(off.size() / (np + 1));
    long long run = 0;
    for (int p = 0; p < np; ++p) { off.push_back(run); run += cnt[p]; }
    off.push_back(run);
    return std::make_pair(at, run);
  };
  for (int p = 0; p < np; ++p) {
    Hierarchy *h = B.hs[p];
    const int L = (int)h->lv.size();
    for (int l = 0; l < nlev; ++l) {
      BLev<T> &b = lev[(size_t)l * np + p];
      std::memset(&b, 0, sizeof(b));
      if (l < L) {
        b.v = view<T>(h->lv[l]);
        b.e = (T *)h->lv[l].e;
        b.r = (T *)h->lv[l].r;
        b.present = l < L - 1;
        b.coarsest = l == L - 1;
        fvol[(size_t)l * np + p] = h->lv[l].fluid_vol;
        poff[(size_t)l * np + p] = h->lv[l].poff;
        pt[(size_t)l * np + p] = h->lv[l].pt;
      }
    }
    if (sizeof(T) == 8) { lev[p].e = (T *)h->p64; lev[p].r = (T *)h->b64; }
    BProb &q = prob[p];
    q.scal = nullptr; q.active = nullptr;
    q.p64 = h->p64; q.b64 = h->b64;
    q.v64 = fine_view64(h);
    q.ng = B.ts[p]->nghost;
    q.gsrc = h->gsrc; q.gdst = h->gdst; q.gw = B.ts[p]->gw; q.gw32 = h->gw32; q.gscale = B.ts[p]->gscale;
    q.gtmp = h->gtmp;
    q.minv = h->minv; q.cidx = h->cidx; q.ncoarse = h->dncoarse;
    q.ntot0 = h->lv[0].g.ntot;
    r32[p] = sizeof(T) == 4 ? (float *)h->lv[0].r : nullptr;
  }
  // work prefixes
  B.o_rbgs.assign(nlev, 0); B.o_restrict.assign(nlev, 0); B.o_prolong.assign(nlev, 0);
  B.tot_rbgs.assign(nlev, 0); B.tot_restrict.assign(nlev, 0); B.tot_prolong.assign(nlev, 0);
  for (int l = 0; l < nlev; ++l) {
    std::vector<long long> c1(np, 0), c2(np, 0), c3(np, 0);
    for (int p = 0; p < np; ++p) {
      Hierarchy *h = B.hs[p];
      const int L = (int)h->lv.size();
      if (l >= L - 1) continue;
      const LevelGeom &g = h->lv[l].g, &gc = h->lv[l + 1].g;
      c1[p] = (long long)(((g.nx + 1) / 2 + BT - 1) / BT) * g.ny * g.nz;
      c2[p] = ((long long)gc.nx * gc.ny * gc.nz + BCHUNK - 1) / BCHUNK;
      c3[p] = (long long)((g.nx + BT - 1) / BT) * g.ny * g.nz;
    }
    auto a = add_prefix(c1); B.o_rbgs[l] = a.first; B.tot_rbgs[l] = a.second;
    auto b = add_prefix(c2); B.o_restrict[l] = b.first; B.tot_restrict[l] = b.second;
    auto c = add_prefix(c3); B.o_prolong[l] = c.first; B.tot_prolong[l] = c.second;
  }
  {
    std::vector<long long> cg(np), cr(np), cgr(np), cf(np);
    for (int p = 0; p < np; ++p) {
      const LevelGeom &g = B.hs[p]->lv[0].g;
      cg[p] = (B.ts[p]->nghost + BT - 1) / BT;
      cr[p] = ((long long)g.ny * g.nz + BCHUNK - 1) / BCHUNK;
      cgr[p] = (B.ts[p]->nghost + BCHUNK - 1) / BCHUNK;
      cf[p] = (g.ntot + BT - 1) / BT;
    }
    auto a = add_prefix(cg); B.o_ghost = a.first; B.tot_ghost = a.second;
    auto b = add_prefix(cr); B.o_res = b.first; B.tot_res = b.second;
    auto c = add_prefix(cgr); B.o_gres = c.first; B.tot_gres = c.second;
    auto d = add_prefix(cf); B.o_fine = d.first; B.tot_fine = d.second;
  }
  long long maxpart = std::max<long long>(3 * B.tot_res + B.tot_gres + 16, 16);
  for (int l = 0; l < nlev; ++l) maxpart = std::max(maxpart, B.tot_restrict[l] + 16);
  IBM_TRY(cudaMalloc(&B.d_lev, sizeof(BLev<T>) * lev.size()));
  IBM_TRY(cudaMalloc((void **)&B.d_prob, sizeof(BProb) * np));
  IBM_TRY(cudaMalloc((void **)&B.d_active, sizeof(int) * np));
  IBM_TRY(cudaMalloc((void **)&B.d_scal, sizeof(double) * NSCAL * np));
  IBM_TRY(cudaMalloc((void **)&B.d_fvol, sizeof(double) * fvol.size()));
  IBM_TRY(cudaMalloc((void **)&B.d_lc32, sizeof(void *) * np));
  IBM_TRY(cudaMalloc((void **)&B.d_poff, sizeof(void *) * poff.size()));
  IBM_TRY(cudaMalloc((void **)&B.d_pt, sizeof(void *) * pt.size()));
  IBM_TRY(cudaMalloc((void **)&B.d_r32, sizeof(void *) * np));
  IBM_TRY(cudaMalloc((void **)&B.d_off, sizeof(long long) * off.size()));
  IBM_TRY(cudaMalloc((void **)&B.d_part, sizeof(double) * (4 * maxpart + 64)));
  for (int p = 0; p < np; ++p) {
    prob[p].scal = B.d_scal + (size_t)p * NSCAL;
    prob[p].active = B.d_active + p;
  }
  std::vector<const void *> lc(np);
  for (int p = 0; p < np; ++p) {
    const int L = (int)B.hs[p]->lv.size();
    lc[p] = (const char *)B.d_lev + sizeof(BLev<T>) * ((size_t)(L - 1) * np + p);
  }
  IBM_TRY(cudaMemcpyAsync(B.d_lev, lev.data(), sizeof(BLev<T>) * lev.size(), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_prob, prob.data(), sizeof(BProb) * np, cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_fvol, fvol.data(), sizeof(double) * fvol.size(), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_lc32, lc.data(), sizeof(void *) * np, cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_poff, poff.data(), sizeof(void *) * poff.size(), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_pt, pt.data(), sizeof(void *) * pt.size(), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_r32, r32.data(), sizeof(void *) * np, cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaMemcpyAsync(B.d_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, st));
  IBM_TRY(cudaStreamSynchronize(st));
  B.off_host = off;
  return IBM_OK;
}

struct BatchRun {
  ibm_ctx *ctx;
  BatchPlan *B;
  cudaStream_t st;
  int nu1, nu2;
  float omega;
};

template <typename T>
void b_ghosts(BatchRun &R, int with_rhs) {
  BatchPlan &B = *R.B;
  if (B.tot_ghost == 0) return;
  const long long *off = B.d_off + (long long)B.o_ghost * (B.np + 1);
  const unsigned g = persistent_grid(R.ctx, B.tot_ghost);
  kb_ghost_eval<T><<<g, BT, 0, R.st>>>((const BLev<T> *)B.d_lev, B.d_prob, off, B.np, with_rhs);
  kb_ghost_store<T><<<g, BT, 0, R.st>>>((const BLev<T> *)B.d_lev, B.d_prob, off, B.np);
  R.ctx->launches += 2;
}

template <typename T>
void b_smooth(BatchRun &R, int l, int sweeps, int shift_slot, int with_rhs) {
  BatchPlan &B = *R.B;
  if (B.tot_rbgs[l] == 0) return;
  const long long *off = B.d_off + (long long)B.o_rbgs[l] * (B.np + 1);
  const BLev<T> *L = (const BLev<T> *)B.d_lev + (size_t)l * B.np;
  const unsigned g = persistent_grid(R.ctx, B.tot_rbgs[l]);
  for (int s = 0; s < sweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour)
      kb_rbgs<T><<<g, BT, 0, R.st>>>(L, B.d_prob, off, B.np, colour, R.omega, shift_slot);
    R.ctx->launches += 2;
    if (l == 0) b_ghosts<T>(R, with_rhs);
  }
}

// one batched V-cycle (all problems, each to its own depth)
template <typename T>
void b_vcycle(BatchRun &R, int fine_shift_slot, int with_rhs) {
  BatchPlan &B = *R.B;
  const int np = B.np;
  for (int l = 0; l + 1 < B.nlev; ++l) {
    const int slot = l == 0 ? fine_shift_slot : S_LEVEL_SHIFT + l;
    b_smooth<T>(R, l, R.nu1, slot, with_rhs);
    if (B.tot_restrict[l] == 0) continue;
    const long long *off = B.d_off + (long long)B.o_restrict[l] * (np + 1);
    const BLev<T> *F = (const BLev<T> *)B.d_lev + (size_t)l * np, *C = F + np;
    kb_restrict<T><<<persistent_grid(R.ctx, B.tot_restrict[l]), BT, 0, R.st>>>(F, C, B.d_prob, off, np, slot, B.d_part);
    kb_finalize_shift<<<np, 32, 0, R.st>>>(B.d_prob, off, np, B.d_part, B.d_fvol + (size_t)(l + 1) * np,
                                          S_LEVEL_SHIFT + l + 1);
    R.ctx->launches += 2;
  }
  kb_coarsest<T><<<np, 128, 0, R.st>>>((const BLev<T> *const *)B.d_lc32, B.d_prob, np);
  R.ctx->launches += 1;
  for (int l = B.nlev - 2; l >= 0; --l) {
    const int slot = l == 0 ? fine_shift_slot : S_LEVEL_SHIFT + l;
    if (B.tot_prolong[l] == 0) continue;
    const long long *off = B.d_off + (long long)B.o_prolong[l] * (np + 1);
    const BLev<T> *F = (const BLev<T> *)B.d_lev + (size_t)l * np, *C = F + np;
    kb_prolong<T><<<persistent_grid(R.ctx, B.tot_prolong[l]), BT, 0, R.st>>>(C, F, B.d_prob, off, np,
                                                                            B.d_poff + (size_t)l * np,
                                                                            B.d_pt + (size_t)l * np);
    R.ctx->launches += 1;
    if (l == 0) b_ghosts<T>(R, with_rhs);
    b_smooth<T>(R, l, R.nu2, slot, with_rhs);
  }
}

void b_residual(BatchRun &R, int use_p, bool mixed, int update_lambda) {
  BatchPlan &B = *R.B;
  const int np = B.np;
  const long long *roff = B.d_off + (long long)B.o_res * (np + 1);
  const long long *goff = B.d_off + (long long)B.o_gres * (np + 1);
  double *rpart = B.d_part, *gpart = B.d_part + 3 * B.tot_res + 8;
  const float *const *r32 = mixed ? (const float *const *)B.d_r32 : nullptr;
  kb_residual64<<<persistent_grid(R.ctx, B.tot_res), BT, 0, R.st>>>(B.d_prob, roff, np, mixed ? r32 : nullptr, use_p,
                                                                     rpart);
  R.ctx->launches += 1;
  if (use_p && B.tot_gres > 0) {
    kb_ghost_resid64<<<persistent_grid(R.ctx, B.tot_gres), BT, 0, R.st>>>(B.d_prob, goff, np, r32, gpart);
    R.ctx->launches += 1;
  }
  kb_finalize_resid<<<np, 32, 0, R.st>>>(B.d_prob, np, roff, rpart, goff, gpart, update_lambda);
  R.ctx->launches += 1;
}

}  // namespace

ibm_status solve_batched_impl(ibm_ctx *ctx, int n, ibm_tables *const *ts, const double *const *rhs, double tol,
                              double *const *p_user, const ibm_solve_opts *opts, ibm_solve_info *infos,
                              cudaStream_t st) {
  const int prec = opts->precision;
  BatchPlan B;
  B.np = n;
  B.prec = prec;
  for (int p = 0; p < n; ++p) {
    ibm_status s = build_hierarchy(ts[p], prec, st);
    if (s != IBM_OK) return s;
    B.ts.push_back(ts[p]);
    B.hs.push_back(ts[p]->hier[prec]);
  }
  struct Guard { BatchPlan &b; ~Guard() { free_plan(b); } } guard{B};
  {
    ibm_status s = prec == 0 ? plan_batch<double>(ctx, B, st) : plan_batch<float>(ctx, B, st);
    if (s != IBM_OK) return s;
  }
  // inputs and per-problem constants
  std::vector<double> hs((size_t)n * NSCAL, 0.0);
  for (int p = 0; p < n; ++p) {
    Hierarchy *h = B.hs[p];
    Level &L0 = h->lv[0];
    const long long n0 = (long long)L0.g.nx * L0.g.ny * L0.g.nz;
    k_pack<<<PACK_BLOCKS, 256, 0, st>>>(rhs[p], L0.g, h->b64, nullptr);
    k_pack<<<PACK_BLOCKS, 256, 0, st>>>(p_user[p], L0.g, h->p64, L0.mask);
    const long long ng = ts[p]->nghost;
    if (ng > 0) {
      k_ghost_eval<double, double><<<nblk(ng, 128), 128, 0, st>>>(h->gsrc, h->gdst, ts[p]->gw, ng, nullptr, h->p64,
                                                                  nullptr,
                                                                  h->gtmp);
      k_ghost_store<double><<<nblk(ng, 128), 128, 0, st>>>(h->gdst, ng, nullptr, h->gtmp, h->p64);
    }
    ctx->launches += ng > 0 ? 5 : 3;
    hs[(size_t)p * NSCAL + S_FLUIDVOL] = L0.fluid_vol;
    hs[(size_t)p * NSCAL + S_NF] = (double)L0.nfluid;
  }
  IBM_TRY(cudaMemcpyAsync(B.d_scal, hs.data(), sizeof(double) * hs.size(), cudaMemcpyHostToDevice, st));
  std::vector<int> act(n, 1);
  IBM_TRY(cudaMemcpyAsync(B.d_active, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  BatchRun R{ctx, &B, st, opts->nu1, opts->nu2, (float)opts->omega};
  const bool mixed = prec == 1;
  // reference norms ||S P b||, then the initial residual
  b_residual(R, 0, false, 0);
  std::vector<double> bn(n), rel(n, 0.0);
  IBM_TRY(cudaMemcpyAsync(hs.data(), B.d_scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  for (int p = 0; p < n; ++p) {
    double v = std::sqrt(hs[(size_t)p * NSCAL + S_NORM2]);
    bn[p] = v > 0 ? v : 1.0;
  }
  b_residual(R, 1, mixed, 1);
  IBM_TRY(cudaMemcpyAsync(hs.data(), B.d_scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  std::vector<int> cycles(n, 0);
  int remaining = 0;
  for (int p = 0; p < n; ++p) {
    rel[p] = std::sqrt(hs[(size_t)p * NSCAL + S_NORM2]) / bn[p];
    act[p] = rel[p] > tol;
    remaining += act[p];
  }
  IBM_TRY(cudaMemcpyAsync(B.d_active, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  auto body = [&](cudaStream_t bs) {
    R.st = bs;
    if (!mixed) {
      b_vcycle<double>(R, S_LAMBDA, 0);
      b_residual(R, 1, false, 1);
    } else {
      const long long *foff = B.d_off + (long long)B.o_fine * (n + 1);
      for (int q = 0; q < std::max(1, opts->inner_cycles); ++q) {
        if (q == 0) {
          kb_fine_elementwise<float><<<persistent_grid(ctx, B.tot_fine), BT, 0, bs>>>(
              (const BLev<float> *)B.d_lev, B.d_prob, foff, n, 0);
          ctx->launches += 1;
        }
        b_vcycle<float>(R, S_MU, 1);
      }
      kb_fine_elementwise<float><<<persistent_grid(ctx, B.tot_fine), BT, 0, bs>>>((const BLev<float> *)B.d_lev,
                                                                                  B.d_prob, foff, n, 1);
      ctx->launches += 1;
      b_residual(R, 1, true, 1);
    }
    R.st = st;
  };
  // capture one batched cycle as a CUDA graph and replay it
  bool graph = opts->use_graph && ctx->cap_stream;
  cudaGraphExec_t ge = nullptr;
  long long per_cycle = 0;
  if (graph) {
    cudaGraph_t g = nullptr;
    const long long l0 = ctx->launches;
    IBM_TRY(cudaStreamSynchronize(st));
    IBM_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    body(ctx->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (ce != cudaSuccess) return check(ce, "batched graph capture");
    ce = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return check(ce, "batched graph instantiate");
    B.graph_exec = ge;
    per_cycle = ctx->launches - l0;
    ctx->launches = l0;
  }
  int it = 0;
  ibm_status result = IBM_OK;
  while (remaining > 0 && it < opts->max_cycles) {
    if (graph) {
      IBM_TRY(cudaGraphLaunch(ge, st));
      ctx->launches += per_cycle;
    } else {
      body(st);
    }
    IBM_TRY(cudaGetLastError());
    IBM_TRY(cudaMemcpyAsync(hs.data(), B.d_scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
    IBM_TRY(cudaStreamSynchronize(st));
    ++it;
    remaining = 0;
    for (int p = 0; p < n; ++p) {
      if (!act[p]) continue;
      ++cycles[p];
      rel[p] = std::sqrt(hs[(size_t)p * NSCAL + S_NORM2]) / bn[p];
      if (infos && infos[p].resid_history && infos[p].history_len < infos[p].history_cap)
        infos[p].resid_history[infos[p].history_len++] = rel[p];
      if (!std::isfinite(rel[p])) { result = IBM_ERR_DIVERGED; act[p] = 0; continue; }
      if (rel[p] <= tol) act[p] = 0;
      remaining += act[p];
    }
    IBM_TRY(cudaMemcpyAsync(B.d_active, act.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  }
  if (remaining > 0 && result == IBM_OK) result = IBM_ERR_NOT_CONVERGED;
  // gauge and unpack every problem
  for (int p = 0; p < n; ++p) {
    Hierarchy *h = B.hs[p];
    Level &L0 = h->lv[0];
    const long long n0 = (long long)L0.g.nx * L0.g.ny * L0.g.nz;
    double *ps = B.d_scal + (size_t)p * NSCAL;
    k_gauge_sum<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, st>>>(fine_view64(h), h->p64, ctx->partials);
    k_gauge_finalize<<<1, 256, 0, st>>>(ctx->partials, REDUCE_BLOCKS, ps);
    k_unpack_gauge<<<PACK_BLOCKS, 256, 0, st>>>(h->p64, L0.mask, L0.g, ps, p_user[p]);
    ctx->launches += 3;
  }
  IBM_TRY(cudaGetLastError());
  IBM_TRY(cudaMemcpyAsync(hs.data(), B.d_scal, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
  IBM_TRY(cudaStreamSynchronize(st));
  if (infos)
    for (int p = 0; p < n; ++p) {
      infos[p].cycles = cycles[p];
      infos[p].rel_resid = rel[p];
      infos[p].lambda = hs[(size_t)p * NSCAL + S_LAMBDA];
    }
  return result;
}

}  // namespace ibm
