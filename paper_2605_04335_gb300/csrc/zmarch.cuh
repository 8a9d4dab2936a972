// Fused two-colour red-black Gauss-Seidel sweep on the finest level: z-march with
// TMA-staged planes in shared memory.
//
// One CTA owns an x-y tile (TX x TY) and a z-range [k0, k1).  Step q of the march
//   1. updates the red cells of plane q on the tile plus the one-cell ring that the tile's
//      black cells read (rows -1 and TY over the tile's x range, columns -1 and TX over its
//      y range; the ring is recomputed by both neighbouring CTAs, in the same operation
//      order, so no inter-CTA exchange is needed), in place in plane q's shared buffer;
//   2. updates the black cells of plane q-1 on the tile and stores plane q-1 of the tile.
// Every value is read from the input array and written to a separate output array, so the
// result is exactly one red half-sweep followed by one black half-sweep (deterministic,
// independent of the tiling).
//
// Each thread owns a fixed strip of 4 consecutive x-cells of the tile and keeps that strip's
// values in planes q-2 .. q+1 in registers, with the rhs, mask and z coefficients of plane
// q-1.  Red results go back to the plane's buffer (their y-neighbours in other warps read
// them in the next step) and stay in the registers (the strip's black update two steps
// later reads its z-1 neighbours there); black results go only to registers and global
// memory, since nothing in the march reads a black value after its update.  x-neighbours across strips move by warp
// shuffle; only the tile edges read the ring from shared memory.  A red update reads only
// black cells and a black update only red ones, so the in-place writes never change a value
// another thread reads in the same step: one barrier per step suffices.
//
// Planes of e (halo 2 in x and y), the right-hand side and the mask (halo 1) arrive by
// cp.async.bulk.tensor into rings of shared-memory buffers DP steps ahead of their use,
// one mbarrier per buffer; the tensor maps zero-fill everything outside the padded arrays.
// Waits are bounded: a wait that gives up sets the error flag, waits (bounded) for the
// copies still in flight and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ibm {
namespace zm {

constexpr int TX = 64;          // tile width (cells); multiple of 16
constexpr int SR = 16;          // rows of one strip set (a multiple of 4)
constexpr int NS = 2;           // interior strips per thread: rows y and y + SR
constexpr int TY = SR * NS;     // tile height
constexpr int BX = TX + 8;      // staged width of e and rhs: x in [-4, TX + 4)
constexpr int BXM = TX + 16;    // staged width of the mask (an 8-bit box row must be 16-byte multiple)
constexpr int EY = TY + 4;      // e rows: y in [-2, TY + 2)
constexpr int RY = TY + 2;      // rhs / mask rows: y in [-1, TY + 1)
constexpr int THREADS = (TX / 4) * SR;       // NS interior strips per thread
constexpr int MIN_CTAS = 65536 / (THREADS * 128);   // resident CTAs per SM at up to 128 registers
constexpr int RING = 2 * (TX / 4);           // ring row strips (rows -1 and TY, x in [0, TX)): warp 0
constexpr int CELL_WARP = 1;                 // the warp of the ring column cells
constexpr int CELLS = TY;                    // ring column cells per plane (the red one of each y pair)
static_assert(RING == 32 && CELLS <= 32 && THREADS >= 64, "ring rows fill warp 0, the columns fit warp 1");
static_assert(SR % 4 == 0 && (NS == 1 || NS == 2), "strips at rows y and y + SR share the colour parity");
constexpr long long WAIT_LIMIT = 1LL << 22;

// prefetch distance in planes; rings hold the planes in use at step q (e: q-1 .. q+1,
// rhs/mask: q) plus the ones in flight
template <typename T> struct Depth { static constexpr int D = sizeof(T) == 4 ? 2 : 1; };
template <typename T> constexpr int NE = 3 + Depth<T>::D;
template <typename T> constexpr int NR = 1 + Depth<T>::D;

constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }

// every TMA destination starts on a 128-byte boundary
template <typename T>
struct Smem {
  alignas(128) T e[NE<T>][pad128(EY * BX * (int)sizeof(T)) / (int)sizeof(T)];
  alignas(128) T r[NR<T>][pad128(RY * BX * (int)sizeof(T)) / (int)sizeof(T)];
  alignas(128) uint8_t m[NR<T>][pad128(RY * BXM)];
  alignas(8) uint64_t bar_e[NE<T>];
  alignas(8) uint64_t bar_r[NR<T>];
};

template <typename T> struct Strip;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try(b, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(saddr(dst)),
      "l"(map), "r"(saddr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <typename T>
struct Args {
  int nx, ny, nz, px;
  long long sy, sz;
  int kz;                 // planes per CTA
  const T *cxm, *cxp, *cym, *cyp, *czm, *czp, *sdx, *sdy, *sdz;
  const double *shift;
  float omega;
  T *out;
  int *err;
};

// four consecutive elements: one 16-byte (float) or two 16-byte (double) accesses
template <typename T>
struct Q4 {
  T v[4];
};

template <typename T>
__device__ __forceinline__ Q4<T> ld4(const T *p) {
  Q4<T> q;
  if constexpr (sizeof(T) == 4) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    q.v[0] = a.x; q.v[1] = a.y; q.v[2] = a.z; q.v[3] = a.w;
  } else {
    double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    q.v[0] = a.x; q.v[1] = a.y; q.v[2] = b.x; q.v[3] = b.y;
  }
  return q;
}

template <typename T>
__device__ __forceinline__ void st4(T *p, const Q4<T> &q) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
  } else {
    reinterpret_cast<double2 *>(p)[0] = make_double2(q.v[0], q.v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(q.v[2], q.v[3]);
  }
}

// a strip of 4 x-cells with its coefficients (registers for the whole march)
template <typename T>
struct Strip {
  int xs, y;          // tile coordinates of the first cell
  unsigned valid;     // bit u: cell xs+u is in the grid and in [xlo, xhi]
  int ie, ir, im;     // offsets of the first cell in an e / rhs / mask plane buffer
  int par;            // (x0 + xs + y0 + y) mod 2
  T cxm[4], cxp[4], sx[4], cym, cyp, sy;
};

template <typename T>
__device__ __forceinline__ void make_strip(Strip<T> &S, const Args<T> &a, int x0, int y0, int xs, int y, int xlo,
                                           int xhi) {
  S.xs = xs; S.y = y; S.valid = 0;
  S.ie = (y + 2) * BX + (xs + 4);
  S.ir = (y + 1) * BX + (xs + 4);
  S.im = (y + 1) * BXM + (xs + 4);
  S.par = (x0 + xs + y0 + y) & 1;
  const int gj = y0 + y;
  const bool jok = gj >= 0 && gj < a.ny;
  for (int u = 0; u < 4; ++u) {
    const int x = xs + u, gi = x0 + x;
    const bool ok = jok && gi >= 0 && gi < a.nx && x >= xlo && x <= xhi;
    if (ok) S.valid |= 1u << u;
    S.cxm[u] = ok ? a.cxm[gi] : (T)0;
    S.cxp[u] = ok ? a.cxp[gi] : (T)0;
    S.sx[u] = ok ? a.sdx[gi] : (T)0;
  }
  S.cym = jok ? a.cym[gj] : (T)0;
  S.cyp = jok ? a.cyp[gj] : (T)0;
  S.sy = jok ? a.sdy[gj] : (T)0;
}

// Relax the cells of colour par ((gi + gj + k) mod 2 == par) of strip S in plane buffer P
// (Pm, Pp: planes k-1, k+1): e += omega (sum_d c_d e_nb - D e - rhs) / D.  The residual is
// formed in T; the relaxation factor and step are FP32 (they do not move the fixed point,
// the exact T-precision solution of the row), keeping FP64 work to the stencil itself.
// C returns the strip's values after the update.
template <typename T>
__device__ __forceinline__ void relax_colour(const Strip<T> &S, T *P, const T *Pm, const T *Pp, const T *R,
                                             const uint8_t *M, int par, int x0, int y0, int k, T czm, T czp, T sz,
                                             T sh, float om, Q4<T> &C) {
  const int ie = S.ie;
  C = ld4(P + ie);
  const unsigned m4 = *reinterpret_cast<const unsigned *>(M + S.im);
  // cells of colour par in the strip: u = ua and ua + 2
  const int ua = (S.par + k + par) & 1;
  unsigned act = 0;
  for (int u = ua; u < 4; u += 2)
    if (((S.valid >> u) & 1u) && ((m4 >> (8 * u)) & 0xffu) == 0u) act |= 1u << u;
  if (!act) return;
  const Q4<T> N = ld4(P + ie - BX), So = ld4(P + ie + BX), B = ld4(Pm + ie), U = ld4(Pp + ie);
  const Q4<T> Rh = ld4(R + S.ir);
  const T L = P[ie - 1], Rr = P[ie + 4];
  const T syz = S.sy + sz;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (!((act >> u) & 1u)) continue;
    const T west = u == 0 ? L : C.v[u - 1];
    const T east = u == 3 ? Rr : C.v[u + 1];
    const T D = S.sx[u] + syz;
    T sum = S.cxm[u] * west;
    sum += S.cxp[u] * east;
    sum += S.cym * N.v[u];
    sum += S.cyp * So.v[u];
    sum += czm * B.v[u];
    sum += czp * U.v[u];
    const T res = (sum - D * C.v[u]) - (Rh.v[u] - sh);
    C.v[u] += (T)__fdividef(om * (float)res, (float)D);
  }
  st4(P + ie, C);
}

// one cell at ie of plane buffer P, in the same operation order as relax_colour / relax_reg
// (so a ring cell gets the bits its owner computes)
template <typename T>
__device__ __forceinline__ void relax_cell(T *P, const T *Pm, const T *Pp, int ie, T rh, T cxm, T cxp, T cym, T cyp,
                                           T sx, T sy, T czm, T czp, T sz, T sh, float om) {
  const T c = P[ie];
  const T syz = sy + sz;
  const T D = sx + syz;
  T sum = cxm * P[ie - 1];
  sum += cxp * P[ie + 1];
  sum += cym * P[ie - BX];
  sum += cyp * P[ie + BX];
  sum += czm * Pm[ie];
  sum += czp * Pp[ie];
  const T res = (sum - D * c) - (rh - sh);
  P[ie] = c + (T)__fdividef(om * (float)res, (float)D);
}

// Interior strip update from registers: cells u = UA and UA + 2 of C (UA warp-uniform: a
// warp's rows share one parity), neighbours N/So (rows y -1 / +1 of the same plane), Zm/Zp
// (the strip in planes k -1 / +1), west/east (the cells left of u = 0 and right of u = 3).
template <int UA, typename T>
__device__ __forceinline__ void relax_reg(const T (&cxm)[4], const T (&cxp)[4], const T (&sx)[4], unsigned valid,
                                          T cym, T cyp, T sy, Q4<T> &C, const Q4<T> &N, const Q4<T> &So,
                                          const Q4<T> &Zm, const Q4<T> &Zp, const Q4<T> &Rh, unsigned m4, T west,
                                          T east, T czm, T czp, T sz, T sh, float om) {
  constexpr int u0 = UA, u1 = UA + 2;
  const bool ok0 = ((valid >> u0) & 1u) && ((m4 >> (8 * u0)) & 0xffu) == 0u;
  const bool ok1 = ((valid >> u1) & 1u) && ((m4 >> (8 * u1)) & 0xffu) == 0u;
  const T syz = sy + sz;
  const T c0 = C.v[u0], c1 = C.v[u1];
  const T D0 = sx[u0] + syz, D1 = sx[u1] + syz;
  T s0 = cxm[u0] * (UA == 0 ? west : C.v[0]);
  s0 += cxp[u0] * C.v[u0 + 1];
  s0 += cym * N.v[u0];
  s0 += cyp * So.v[u0];
  s0 += czm * Zm.v[u0];
  s0 += czp * Zp.v[u0];
  T s1 = cxm[u1] * C.v[u1 - 1];
  s1 += cxp[u1] * (UA == 1 ? east : C.v[3]);
  s1 += cym * N.v[u1];
  s1 += cyp * So.v[u1];
  s1 += czm * Zm.v[u1];
  s1 += czp * Zp.v[u1];
  const T r0 = (s0 - D0 * c0) - (Rh.v[u0] - sh);
  const T r1 = (s1 - D1 * c1) - (Rh.v[u1] - sh);
  if (ok0) C.v[u0] = c0 + (T)__fdividef(om * (float)r0, (float)D0);
  if (ok1) C.v[u1] = c1 + (T)__fdividef(om * (float)r1, (float)D1);
}

// one CTA's march: tile (bx, by) of the grid, planes [bz kz, min(nz, (bz + 1) kz)); the
// tensor maps in parameter or global memory
template <typename T>
__device__ __forceinline__ void sweep_block(const CUtensorMap *tm_e, const CUtensorMap *tm_r, const CUtensorMap *tm_m,
                                            const Args<T> &a, int bx, int by, int bz) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<T> &s = *reinterpret_cast<Smem<T> *>(smem_raw);
  constexpr int NEt = NE<T>, NRt = NR<T>, DP = Depth<T>::D;
  const int tid = threadIdx.x;
  const int x0 = bx * TX, y0 = by * TY;
  const int k0 = bz * a.kz;
  const int k1 = min(a.nz, k0 + a.kz);
  if (k0 >= k1) return;
  if (tid == 0) {
    for (int b = 0; b < NEt; ++b) mbar_init(&s.bar_e[b], 1);
    for (int b = 0; b < NRt; ++b) mbar_init(&s.bar_r[b], 1);
    fence_mbar_init();
  }
  // this thread's interior strips (registers: x coefficients shared, y ones per strip), and
  // the ring strips (red updates of the one-cell ring; shared memory, read only by their
  // owners, once per step)
  __shared__ Strip<T> ring[RING];
  const int l16 = tid & 15;
  // warp w takes rows r and r + 2 (lanes 0-15 and 16-31), r = 4 (w / 2) + (w mod 2), so a
  // warp's strips share one colour parity; strip s lies SR s rows below strip 0 (same parity)
  const int ys = 4 * ((tid >> 5) >> 1) + ((tid >> 5) & 1) + 2 * ((tid & 31) >> 4), xs = 4 * l16;
  const int ie0 = (ys + 2) * BX + (xs + 4), ir0 = (ys + 1) * BX + (xs + 4), im0 = (ys + 1) * BXM + (xs + 4);
  const int par = (x0 + xs + y0 + ys) & 1;
  T cxm[4], cxp[4], sx[4];
  unsigned xvalid = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gi = x0 + xs + u;
    const bool ok = gi < a.nx;
    if (ok) xvalid |= 1u << u;
    cxm[u] = ok ? a.cxm[gi] : (T)0;
    cxp[u] = ok ? a.cxp[gi] : (T)0;
    sx[u] = ok ? a.sdx[gi] : (T)0;
  }
  T cym[NS], cyp[NS], sy[NS];
  unsigned valid[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int gj = y0 + ys + SR * q;
    const bool jok = gj < a.ny;
    valid[q] = jok ? xvalid : 0u;
    cym[q] = jok ? a.cym[gj] : (T)0;
    cyp[q] = jok ? a.cyp[gj] : (T)0;
    sy[q] = jok ? a.sdy[gj] : (T)0;
  }
  const bool has_ring = tid < RING;
  if (has_ring) make_strip(ring[tid], a, x0, y0, 4 * (tid & 15), tid < 16 ? -1 : TY, 0, TX - 1);
  const bool has_cell = (tid >> 5) == CELL_WARP && (tid & 31) < CELLS;
  __syncthreads();
  const unsigned ebytes = EY * BX * sizeof(T), rbytes = RY * BX * sizeof(T) + RY * BXM;
  // buffer slots: plane p lives in e slot (p + 2 NE) mod NE and rhs/mask slot (p + 2 NR) mod
  // NR; the march advances the slots by one (wrapping) per step
  auto wrap_e = [](int x) { return x >= NEt ? x - NEt : x; };
  auto wrap_r = [](int x) { return x >= NRt ? x - NRt : x; };
  // padded coordinates: cell (i, j, k) at (i + OX, j + 1, k + 1); OX = 4
  auto load_e = [&](int plane, int b) {
    mbar_expect_tx(&s.bar_e[b], ebytes);
    tma_load3(s.e[b], tm_e, &s.bar_e[b], x0, y0 - 1, plane + 1);
  };
  auto load_r = [&](int plane, int b) {
    mbar_expect_tx(&s.bar_r[b], rbytes);
    tma_load3(s.r[b], tm_r, &s.bar_r[b], x0, y0, plane + 1);
    tma_load3(s.m[b], tm_m, &s.bar_r[b], x0, y0, plane + 1);
  };
  unsigned pe = 0, pr = 0;   // bit b: parity of the next completion of buffer b
  bool bad = false;
  auto wait_e = [&](int b) {
    if (!bad && !mbar_wait(&s.bar_e[b], (pe >> b) & 1u)) bad = true;
    pe ^= 1u << b;
  };
  auto wait_r = [&](int b) {
    if (!bad && !mbar_wait(&s.bar_r[b], (pr >> b) & 1u)) bad = true;
    pr ^= 1u << b;
  };
  const int se0 = (k0 - 2 + 2 * NEt) % NEt, sr0 = (k0 - 1 + 2 * NRt) % NRt;   // planes k0 - 2 / k0 - 1
  // prologue: e planes k0-2 .. k0-1+DP and rhs/mask planes k0-1 .. k0-2+DP.  Step q waits
  // for e plane q+1 and rhs/mask plane q and, after the step's barrier (so no thread still
  // reads the buffers being refilled), prefetches e plane q+1+DP (into the buffer of plane
  // q-2, last read in step q-1) and rhs/mask plane q+DP (buffer of plane q-1).  Every load
  // is issued once and waited for once.
  if (tid == 0) {
    for (int pl = k0 - 2, b = se0; pl <= min(k0 - 1 + DP, k1 + 1); ++pl, b = wrap_e(b + 1)) load_e(pl, b);
    for (int pl = k0 - 1, b = sr0; pl <= min(k0 - 2 + DP, k1); ++pl, b = wrap_r(b + 1)) load_r(pl, b);
  }
  int sq = wrap_e(se0 + 1), rq = sr0;   // slots of plane q (e, rhs/mask)
  wait_e(se0);
  wait_e(sq);
  // registers: each strip in planes q-2 (Cm2; its red cells are final once plane q-2's red
  // pass is done), q-1 (Cm1) and q (C0); its rhs and mask in plane q-1; the z coefficients
  // of plane q-1
  Q4<T> Cm2[NS], Cm1[NS], C0[NS], Rb[NS];
  unsigned Mb[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    Cm1[q] = ld4(s.e[se0] + ie0 + SR * q * BX);
    C0[q] = ld4(s.e[sq] + ie0 + SR * q * BX);
    Cm2[q] = Cm1[q];
    Rb[q] = Cm1[q];
    Mb[q] = 0u;
  }
  T czm_b = (T)0, czp_b = (T)0, sz_b = (T)0;
  const T sh = a.shift ? (T)(*a.shift) : (T)0;
  const float om = a.omega;
  T *const dst0 = a.out + (long long)(y0 + ys + 1) * a.px + (x0 + xs + 4);
  // unrolled by 3: the strips' register rotation (planes q-2, q-1, q) becomes renaming
#pragma unroll 3
  for (int q = k0 - 1; q <= k1; ++q) {
    const int sp1 = wrap_e(sq + 1), sm1 = sq == 0 ? NEt - 1 : sq - 1;
    wait_e(sp1);
    wait_r(rq);
    if (__syncthreads_or(bad)) break;
    if (tid == 0) {
      fence_proxy_async();
      if (q + 1 + DP <= k1 + 1) load_e(q + 1 + DP, wrap_e(sp1 + DP));
      if (q + DP <= k1) load_r(q + DP, wrap_r(rq + DP));
    }
    T *P = s.e[sq], *Pm = s.e[sm1];
    const T *Pp = s.e[sp1];
    const T *R = s.r[rq];
    const uint8_t *M = s.m[rq];
    Q4<T> U[NS];
    T wr[NS], er[NS], wb[NS], eb[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int ie = ie0 + SR * t * BX;
      U[t] = ld4(Pp + ie);
      // x-edges: the cell west of u = 0 and east of u = 3, from the adjacent lanes (same
      // row), or from the ring in shared memory at the tile edges; all lanes take part
      wr[t] = __shfl_up_sync(0xffffffffu, C0[t].v[3], 1, 16);
      er[t] = __shfl_down_sync(0xffffffffu, C0[t].v[0], 1, 16);
      wb[t] = __shfl_up_sync(0xffffffffu, Cm1[t].v[3], 1, 16);
      eb[t] = __shfl_down_sync(0xffffffffu, Cm1[t].v[0], 1, 16);
      if (l16 == 0) { wr[t] = P[ie - 1]; wb[t] = Pm[ie - 1]; }
      if (l16 == 15) { er[t] = P[ie + 4]; eb[t] = Pm[ie + 4]; }
    }
    // red cells of plane q on the tile (from registers) and the ring (from shared memory)
    T czm = (T)0, czp = (T)0, sz = (T)0;
    Q4<T> R0[NS];
    unsigned M0[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) { R0[t] = Rb[t]; M0[t] = 0u; }
    if (q >= 0 && q < a.nz) {
      czm = a.czm[q]; czp = a.czp[q]; sz = a.sdz[q];
      const bool ua0 = ((par + q) & 1) == 0;
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        const int ie = ie0 + SR * t * BX;
        const Q4<T> N = ld4(P + ie - BX), So = ld4(P + ie + BX);
        R0[t] = ld4(R + ir0 + SR * t * BX);
        M0[t] = *reinterpret_cast<const unsigned *>(M + im0 + SR * t * BXM);
        if (ua0)
          relax_reg<0, T>(cxm, cxp, sx, valid[t], cym[t], cyp[t], sy[t], C0[t], N, So, Cm1[t], U[t], R0[t], M0[t],
                          wr[t], er[t], czm, czp, sz, sh, om);
        else
          relax_reg<1, T>(cxm, cxp, sx, valid[t], cym[t], cyp[t], sy[t], C0[t], N, So, Cm1[t], U[t], R0[t], M0[t],
                          wr[t], er[t], czm, czp, sz, sh, om);
        st4(P + ie, C0[t]);
      }
      if (has_ring && ring[tid].valid) {
        Q4<T> Cr;
        relax_colour<T>(ring[tid], P, Pm, Pp, R, M, 0, x0, y0, q, czm, czp, sz, sh, om, Cr);
      }
      // ring column cell of this lane (warp CELL_WARP, lanes < CELLS): x = -1 or TX, y the
      // red one of (2i, 2i + 1)
      const int cl = tid & 31, cx = (cl >= CELLS / 2) ? TX : -1, cya = 2 * (cl % (CELLS / 2)), cgi = x0 + cx;
      if (has_cell && cgi >= 0 && cgi < a.nx) {
        const int cy = cya + ((cgi + y0 + cya + q) & 1), cgj = y0 + cy;
        const int ie = (cy + 2) * BX + (cx + 4);
        if (cgj < a.ny && M[(cy + 1) * BXM + (cx + 4)] == 0)
          relax_cell<T>(P, Pm, Pp, ie, R[(cy + 1) * BX + (cx + 4)], a.cxm[cgi], a.cxp[cgi], a.cym[cgj], a.cyp[cgj],
                        a.sdx[cgi], a.sdy[cgj], czm, czp, sz, sh, om);
      }
    }
    // black cells of plane q-1 on the tile: neighbours all red, updated by now (in-plane ones
    // in shared memory, the z-neighbours in Cm2 and C0); store the strips from registers
    const int kb = q - 1;
    if (kb >= k0 && kb < k1) {
      const bool ua0 = ((par + kb + 1) & 1) == 0;
      T *const dk = dst0 + (long long)(kb + 1) * a.sz;
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        const int ie = ie0 + SR * t * BX;
        const Q4<T> N = ld4(Pm + ie - BX), So = ld4(Pm + ie + BX);
        if (ua0)
          relax_reg<0, T>(cxm, cxp, sx, valid[t], cym[t], cyp[t], sy[t], Cm1[t], N, So, Cm2[t], C0[t], Rb[t], Mb[t],
                          wb[t], eb[t], czm_b, czp_b, sz_b, sh, om);
        else
          relax_reg<1, T>(cxm, cxp, sx, valid[t], cym[t], cyp[t], sy[t], Cm1[t], N, So, Cm2[t], C0[t], Rb[t], Mb[t],
                          wb[t], eb[t], czm_b, czp_b, sz_b, sh, om);
        if (valid[t]) {
          T *dst = dk + (long long)(SR * t) * a.px;
          if (valid[t] == 0xfu) {
            st4(dst, Cm1[t]);
          } else {
            for (int u = 0; u < 4; ++u)
              if ((valid[t] >> u) & 1u) dst[u] = Cm1[t].v[u];
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      Cm2[t] = Cm1[t];
      Cm1[t] = C0[t];
      C0[t] = U[t];
      Rb[t] = R0[t];
      Mb[t] = M0[t];
    }
    czm_b = czm; czp_b = czp; sz_b = sz;
    sq = sp1;
    rq = wrap_r(rq + 1);
  }
  if (bad) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      // let copies still in flight land before the block's shared memory is released
      for (int b = 0; b < NEt; ++b) mbar_wait(&s.bar_e[b], (pe >> b) & 1u);
      for (int b = 0; b < NRt; ++b) mbar_wait(&s.bar_r[b], (pr >> b) & 1u);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(THREADS, MIN_CTAS) k_sweep_zmarch(const __grid_constant__ CUtensorMap tm_e,
                                                         const __grid_constant__ CUtensorMap tm_r,
                                                         const __grid_constant__ CUtensorMap tm_m, Args<T> a) {
  sweep_block<T>(&tm_e, &tm_r, &tm_m, a, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace zm
}  // namespace ibm
