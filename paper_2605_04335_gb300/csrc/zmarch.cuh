// Fused two-colour red-black Gauss-Seidel sweep of one multigrid level: z-march with
// TMA-staged planes in shared memory, persistent CTAs over (x-y tile, z-chunk) items.  FP32
// (the mixed solves' multigrid, two CTAs per SM) and FP64 (the FP64 solve's smoother on p,
// one CTA per SM: its buffers take 190 KB of shared memory) share the code, for the finest
// level and (FP32) the coarse levels of at least 2^18 cells; a coarse level may store its e
// and r in BF16 (S = bf16: staged as BF16, widened exactly on load, rounded on store).  A
// batched form (k_sweep_zmarch_batch) sweeps the same level of several problems in one launch.
//
// One item is an x-y tile (TX x TY) and a z-range [k0, k1).  Step q of its march
//   1. updates the red cells of plane q on the tile, and the one-cell ring that the tile's
//      black cells read (rows -1 and TY over the tile's x range, columns -1 and TX over its
//      y range; the ring is recomputed by both neighbouring items with the same arithmetic,
//      so no inter-CTA exchange is needed), in place in plane q's shared buffer;
//   2. updates the black cells of plane q-1 on the tile and stores plane q-1 of the tile.
// Every value is read from the input array and written to a separate output array, so the
// result is exactly one red half-sweep followed by one black half-sweep (deterministic,
// independent of the tiling).
//
// Warps 0..6 own the tile, one row per warp and strip set: each thread keeps two strips of 4
// consecutive x-cells (rows y and y + SR) in registers for planes q-2 .. q+1 (the rhs and
// mask are read from shared memory by each pass).  Red
// results go back to the plane's buffer (their y-neighbours in other warps read them in the
// next step) and stay in the registers (the strip's black update two steps later reads its
// z-1 neighbours there); black results go only to registers and global memory.
// x-neighbours across strips move by warp shuffle; the two edge lanes of a row read the
// ring from shared memory at a per-lane address, so the update is branch-free.  Warp 7 owns
// the ring -- its two rows of 32 strips and its 14 red column cells per plane (coefficients
// from a shared table) -- and issues the copies; its work per step is below a tile warp's,
// so no warp of the tile waits for it at the barrier.  A red update reads only black cells and
// a black update only red ones, so the in-place writes never change a value another thread
// reads in the same step: one barrier per step suffices.
//
// Coarse levels (COARSE = true) carry face fractions (the area fraction of open fine faces)
// in their coefficients.  Their mask here is the z-march mask: 0 for a regular fluid cell
// (every face with a coefficient fully open, so the rediscretised coefficients and the
// separable diagonal apply), 8 for an irregular fluid cell (near a body; its update reads the
// six fractions from global memory and forms the diagonal as their weighted sum), anything
// else for a cell that is not updated.  Tiles crossing a body therefore cost more, and coarse
// launches hand their items out from a counter (dynamic schedule) rather than in a fixed order.
//
// Planes of e (halo 2 in x and y), the right-hand side and the mask (halo 1) arrive by
// cp.async.bulk.tensor into rings of shared-memory buffers DP steps ahead of their use,
// one mbarrier per buffer; the tensor maps zero-fill everything outside the padded arrays.
// Waits are bounded: a wait that gives up sets the error flag; the issuing thread then
// waits (bounded) for every copy it issued that has not been seen to land, and the CTA
// returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dfloat.cuh"
#include "storage.cuh"

namespace ibm {
namespace zm {

constexpr int TX = 128;         // tile width (cells): 32 lanes x 4 cells
constexpr int SR = 7;           // rows of one strip set: one per tile warp
constexpr int NS = 2;           // interior strips per thread: rows y and y + SR
constexpr int TY = SR * NS;     // tile height
constexpr int BX = TX + 8;      // staged width of e and rhs: x in [-4, TX + 4)
constexpr int BXM = TX + 16;    // staged width of the mask (an 8-bit box row must be 16-byte multiple)
constexpr int EY = TY + 4;      // e rows: y in [-2, TY + 2)
constexpr int RY = TY + 2;      // rhs / mask rows: y in [-1, TY + 1)
constexpr int TILE_WARPS = SR;                 // one row of strips each
constexpr int RING_WARP = TILE_WARPS;          // the ring and the copies
constexpr int THREADS = (TILE_WARPS + 1) * 32;
constexpr int MIN_CTAS = 2;
constexpr int COL_LANES = TY;                  // ring warp lanes with a column cell (pairs of rows)
static_assert(TX == 128 && THREADS == 256 && TY % 2 == 0 && COL_LANES <= 32,
              "a warp's 32 lanes cover one row of the tile; the ring warp's lanes its column cells");
static_assert(NS == 2 && SR % 2 == 1, "strip 1 lies an odd number of rows below strip 0: the other colour");
constexpr int WAIT_LIMIT = 1 << 22;
constexpr int KZ_MAX = 256;     // planes per item at most (the z-coefficient table)

// prefetch distance in planes; rings hold the planes in use at step q (e: q-1 .. q+1,
// rhs/mask: q-1 and q) plus the ones in flight
constexpr int DP = 2;
constexpr int NE = 3 + DP;
constexpr int NR = 2 + DP;

constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }
template <typename T> constexpr int esz() { return pad128(EY * BX * (int)sizeof(T)) / (int)sizeof(T); }  // per e buffer
template <typename T> constexpr int rsz() { return pad128(RY * BX * (int)sizeof(T)) / (int)sizeof(T); }  // per rhs buffer
constexpr int MSZ = pad128(RY * BXM);          // bytes per mask buffer

// four consecutive cells of a strip (16 bytes in FP32, 32 in FP64)
struct alignas(32) dbl4 {
  double x, y, z, w;
};
template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = dbl4; };
template <typename T> using vec4 = typename V4<T>::type;

// z coefficients of one plane
template <typename T>
struct ZC {
  T m, p, s, pad;   // czm, czp, czm + czp
};

// every TMA destination starts on a 128-byte boundary; e and r staged in their storage type S
template <typename T, typename S = T>
struct Smem {
  alignas(128) S e[NE][esz<S>()];
  alignas(128) S r[NR][rsz<S>()];
  alignas(128) uint8_t m[NR][MSZ];
  alignas(32) ZC<T> zc[KZ_MAX + 4];   // planes k0 - 2 .. k1 + 1
  alignas(16) T cc[32][16];           // ring warp lanes' coefficients (ring rows, column cell)
  alignas(16) unsigned ccu[32][4];    // ... their invalid-cell bytes and row flags
  alignas(8) uint64_t bar_e[NE];
  alignas(8) uint64_t bar_r[NR];
  int next;                           // the CTA's next item (dynamic schedule)
};

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

// waits for the completion of the phase with the given parity, at most `limit` tries
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it)
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
  int kz;                 // planes per item
  int tiles_x, tiles_y;   // item i: tile (i mod tiles_x, (i / tiles_x) mod tiles_y), chunk i / tiles
  int items;
  int *counter;           // dynamic schedule: items after the first gridDim.x are taken from this
                          // counter (zeroed before the launch); null: item i + k gridDim.x
  int first_wait;         // tries of each item's first wait (WAIT_LIMIT; less only to test the
                          // error path)
  const T *cxm, *cxp, *cym, *cyp, *czm, *czp, *sdx, *sdy, *sdz;
  const T *fx, *fy, *fz;  // coarse levels: face fractions (padded level arrays); else unused
  const double *shift;
  float omega;
  void *out;              // the output e, of the storage type
  int *err;
};

template <typename T>
__device__ __forceinline__ vec4<T> ld4(const T *p) { return *reinterpret_cast<const vec4<T> *>(p); }
template <typename T>
__device__ __forceinline__ void st4(T *p, const vec4<T> &v) { *reinterpret_cast<vec4<T> *>(p) = v; }
// a strip in its storage type <-> the arithmetic type
__device__ __forceinline__ float4 lds4(const float *p) { return ld4<float>(p); }
__device__ __forceinline__ dbl4 lds4(const double *p) { return ld4<double>(p); }
__device__ __forceinline__ float4 lds4(const bf16 *p) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  return make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
}
__device__ __forceinline__ void sts4(float *p, const float4 &v) { st4<float>(p, v); }
__device__ __forceinline__ void sts4(double *p, const dbl4 &v) { st4<double>(p, v); }
__device__ __forceinline__ void sts4(bf16 *p, const float4 &v) {
  *reinterpret_cast<uint2 *>(p) = make_uint2(bf16_pack(v.x, v.y), bf16_pack(v.z, v.w));
}
// a strip's values as they read back after a store of type S
template <typename S, typename V>
__device__ __forceinline__ V stored4(V v) {
  v.x = as_stored<S>(v.x); v.y = as_stored<S>(v.y); v.z = as_stored<S>(v.z); v.w = as_stored<S>(v.w);
  return v;
}

template <typename T>
__device__ __forceinline__ vec4<T> make4(T a, T b, T c, T d) {
  vec4<T> v;
  v.x = a; v.y = b; v.z = c; v.w = d;
  return v;
}

// One cell: e + omega (sum_d c_d e_d - D e - (rhs - sh)) / D.  The residual is formed in FP32
// in a fixed order; the relaxation factor omega / D uses an approximate reciprocal (it does
// not move the fixed point, the exact FP32 solution of the row).  Every path (tile strips,
// ring strips, ring columns) calls this, so a ring cell gets the bits its owner computes.
__device__ __forceinline__ float relax1(float c, float w, float ea, float n, float s, float zm, float zp, float cxm,
                                       float cxp, float cym, float cyp, float czm, float czp, float D, float rsh,
                                       float om) {
  float acc = fmaf(-D, c, -rsh);
  acc = fmaf(cxm, w, acc);
  acc = fmaf(cxp, ea, acc);
  acc = fmaf(cym, n, acc);
  acc = fmaf(cyp, s, acc);
  acc = fmaf(czm, zm, acc);
  acc = fmaf(czp, zp, acc);
  return fmaf(acc, __fdividef(om, D), c);
}

// The same cell in FP64 (the FP64 solve's smoother): the residual in FP64 in the same order; the
// relaxation factor omega / D in FP32 from D rounded toward zero, widened exactly (both
// conversions by bit manipulation, off the FP64 pipe).  As in FP32, the factor does not move
// the fixed point.
__device__ __forceinline__ double relax1(double c, double w, double ea, double n, double s, double zm, double zp,
                                        double cxm, double cxp, double cym, double cyp, double czm, double czp,
                                        double D, double rsh, float om) {
  double acc = fma(-D, c, -rsh);
  acc = fma(cxm, w, acc);
  acc = fma(cxp, ea, acc);
  acc = fma(cym, n, acc);
  acc = fma(cyp, s, acc);
  acc = fma(czm, zm, acc);
  acc = fma(czp, zp, acc);
  return fma(acc, dfl::widen(__fdividef(om, dfl::narrow_trunc(D))), c);
}

// z-march mask byte of an irregular coarse cell
constexpr unsigned IRREGULAR = 8u;

// An irregular coarse cell: each coefficient scaled by its face's open fraction, the diagonal
// their sum (in the order of the two-pass coarse kernels); a cell with no open face keeps
// its value.
template <typename T>
__device__ __forceinline__ float relax_frac(const Args<T> &a, long long id, float c, float w, float ea, float n,
                                           float s, float zm, float zp, float cxm, float cxp, float cym, float cyp,
                                           float czm, float czp, float rsh, float om) {
  // products rounded on their own (never fused into the diagonal's sums), so every kernel that
  // compiles this sweep gives the same bits
  const float c0 = __fmul_rn(cxm, a.fx[id - 1]), c1 = __fmul_rn(cxp, a.fx[id]), c2 = __fmul_rn(cym, a.fy[id - a.sy]),
              c3 = __fmul_rn(cyp, a.fy[id]), c4 = __fmul_rn(czm, a.fz[id - a.sz]), c5 = __fmul_rn(czp, a.fz[id]);
  const float D = ((c0 + c1) + (c2 + c3)) + (c4 + c5);
  return D > 0.f ? relax1(c, w, ea, n, s, zm, zp, c0, c1, c2, c3, c4, c5, D, rsh, om) : c;
}

using U0 = std::integral_constant<int, 0>;   // a strip's colour: u of its first cell to relax
using U1 = std::integral_constant<int, 1>;

// x coefficients of a strip's four cells
template <typename T>
struct XCoef {
  vec4<T> m, p, s;   // cxm, cxp, cxm + cxp
};

// Relax the cells u = UA and UA + 2 of strip C (a warp's strips share UA): west/east are the
// cells left of u = 0 and right of u = 3, N/S the strip in rows y -1 / +1, Zm/Zp in planes
// k -1 / +1, R the rhs, mm the mask bytes (nonzero: not updated, except IRREGULAR on coarse
// levels; invalid cells carry 0xff); gid the padded index of the strip's first cell (coarse
// levels' fractions).  Called by all 32 lanes of a warp.
template <int UA, bool COARSE, typename T>
__device__ __forceinline__ void relax_strip(vec4<T> &C, T west, T east, const vec4<T> &N, const vec4<T> &S,
                                            const vec4<T> &Zm, const vec4<T> &Zp, const vec4<T> &R, unsigned mm,
                                            const XCoef<T> &X, T cym, T cyp, T syz, T czm, T czp, T sh, float om,
                                            const Args<T> &a, long long gid) {
  const T c0 = UA == 0 ? C.x : C.y, c1 = UA == 0 ? C.z : C.w;
  const T w0 = UA == 0 ? west : C.x, e0 = UA == 0 ? C.y : C.z;
  const T w1 = UA == 0 ? C.y : C.z, e1 = UA == 0 ? C.w : east;
  const T n0 = UA == 0 ? N.x : N.y, n1 = UA == 0 ? N.z : N.w, s0 = UA == 0 ? S.x : S.y, s1 = UA == 0 ? S.z : S.w;
  const T zm0 = UA == 0 ? Zm.x : Zm.y, zm1 = UA == 0 ? Zm.z : Zm.w;
  const T zp0 = UA == 0 ? Zp.x : Zp.y, zp1 = UA == 0 ? Zp.z : Zp.w;
  const T r0 = (UA == 0 ? R.x : R.y) - sh, r1 = (UA == 0 ? R.z : R.w) - sh;
  const T xm0 = UA == 0 ? X.m.x : X.m.y, xm1 = UA == 0 ? X.m.z : X.m.w;
  const T xp0 = UA == 0 ? X.p.x : X.p.y, xp1 = UA == 0 ? X.p.z : X.p.w;
  const T xs0 = UA == 0 ? X.s.x : X.s.y, xs1 = UA == 0 ? X.s.z : X.s.w;
  T v0 = relax1(c0, w0, e0, n0, s0, zm0, zp0, xm0, xp0, cym, cyp, czm, czp, xs0 + syz, r0, om);
  T v1 = relax1(c1, w1, e1, n1, s1, zm1, zp1, xm1, xp1, cym, cyp, czm, czp, xs1 + syz, r1, om);
  unsigned b0 = (mm >> (8 * UA)) & 0xffu, b1 = (mm >> (8 * (UA + 2))) & 0xffu;
  if constexpr (COARSE) {
    if (__any_sync(0xffffffffu, b0 == IRREGULAR || b1 == IRREGULAR)) {
      if (b0 == IRREGULAR) {
        v0 = relax_frac(a, gid + UA, c0, w0, e0, n0, s0, zm0, zp0, xm0, xp0, cym, cyp, czm, czp, r0, om);
        b0 = 0u;
      }
      if (b1 == IRREGULAR) {
        v1 = relax_frac(a, gid + UA + 2, c1, w1, e1, n1, s1, zm1, zp1, xm1, xp1, cym, cyp, czm, czp, r1, om);
        b1 = 0u;
      }
    }
  }
  v0 = b0 ? c0 : v0;
  v1 = b1 ? c1 : v1;
  if constexpr (UA == 0) {
    C.x = v0;
    C.z = v1;
  } else {
    C.y = v0;
    C.w = v1;
  }
}

template <typename T>
__device__ __forceinline__ XCoef<T> load_x(const Args<T> &a, int gi0) {
  XCoef<T> X;
  T m[4], p[4], s[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gi = gi0 + u;
    const bool ok = gi >= 0 && gi < a.nx;
    m[u] = ok ? a.cxm[gi] : (T)0;
    p[u] = ok ? a.cxp[gi] : (T)0;
    s[u] = ok ? a.sdx[gi] : (T)0;
  }
  X.m = make4<T>(m[0], m[1], m[2], m[3]);
  X.p = make4<T>(p[0], p[1], p[2], p[3]);
  X.s = make4<T>(s[0], s[1], s[2], s[3]);
  return X;
}

// mask bytes 0xff for strip cells outside the grid (x) or outside the update range
__device__ __forceinline__ unsigned invalid_bytes(int gi0, int nx, bool jok) {
  unsigned v = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (!jok || gi0 + u < 0 || gi0 + u >= nx) v |= 0xffu << (8 * u);
  return v;
}

// resident CTAs per SM: two in FP32; one in FP64, whose buffers take most of the shared memory
template <typename T>
constexpr int min_ctas() { return sizeof(T) == 4 ? MIN_CTAS : 1; }

// One item's march: tile origin (x0, y0), planes [k0, k1) of the level that a, tm_e, tm_r and
// tm_m describe, shift sh and relaxation factor om.  The mbarrier parities and in-flight
// copies (pe, pr, pend_e, pend_r) carry over from item to item; bad is set when a wait gives up.
template <typename T, bool COARSE, typename S>
__device__ __forceinline__ void march_item(Smem<T, S> &s, const Args<T> &a, const CUtensorMap *tm_e,
                                           const CUtensorMap *tm_r, const CUtensorMap *tm_m, int x0, int y0, int k0,
                                           int k1, T sh, float om, int first_wait, unsigned &pe, unsigned &pr,
                                           unsigned &pend_e, unsigned &pend_r, bool &bad) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ring = warp == RING_WARP;
  const bool issuer = ring && lane == 0;
  const unsigned ebytes = EY * BX * sizeof(S), rbytes = RY * BX * sizeof(S) + RY * BXM;
  // this thread's strips: tile warp w takes row w (strip 0) and row w + SR (strip 1), lane l
  // the cells 4 l .. 4 l + 3, so the lanes of a warp share each strip's colour parity.  The
  // ring warp's lanes take the ring strips at x = 4 l of rows -1 and TY, and lanes
  // l < COL_LANES the column cell x = -1 (l < TY / 2) or TX (the rest), the red one of the
  // pair of rows 2 (l mod TY / 2), 2 (l mod TY / 2) + 1.
  const int xs = 4 * lane;
  const int ys = ring ? 0 : warp;
  const int ie0 = (ys + 2) * BX + (xs + 4), ir0 = (ys + 1) * BX + (xs + 4), im0 = (ys + 1) * BXM + (xs + 4);
  const int eoff = lane == 0 ? -1 : 4;   // edge lanes: the ring cell beside the strip
  // coefficients of this thread's strips (registers for the item's whole march)
  const XCoef<T> X = load_x(a, x0 + xs);
  T cym[NS], cyp[NS], sy[NS];
  unsigned inval[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int gj = y0 + ys + SR * t;
    const bool jok = gj < a.ny;
    inval[t] = invalid_bytes(x0 + xs, a.nx, jok);
    cym[t] = jok ? a.cym[gj] : (T)0;
    cyp[t] = jok ? a.cyp[gj] : (T)0;
    sy[t] = jok ? a.sdy[gj] : (T)0;
  }
  // ring warp: its ring strips' row coefficients (slots 0-2: row -1, 3-5: row TY; cym, cyp,
  // sdy) and invalid bytes (ccu 0, 1), then its column cell's (slots 6-14): cxm, cxp, sdx,
  // then cym, cyp, sdy of the pair's two rows, and which rows are in the grid (ccu 2)
  if (ring) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gj = y0 + (h == 0 ? -1 : TY);
      const bool jok = gj >= 0 && gj < a.ny;
      T *cc = s.cc[lane] + 3 * h;
      cc[0] = jok ? a.cym[gj] : (T)0;
      cc[1] = jok ? a.cyp[gj] : (T)0;
      cc[2] = jok ? a.sdy[gj] : (T)0;
      s.ccu[lane][h] = invalid_bytes(x0 + xs, a.nx, jok);
    }
    const int pr_ = lane % (TY / 2);
    const int cgi = x0 + (lane < TY / 2 ? -1 : TX), gj0 = y0 + 2 * pr_;
    const bool cxok = lane < COL_LANES && cgi >= 0 && cgi < a.nx;
    const bool ok0 = cxok && gj0 < a.ny, ok1 = cxok && gj0 + 1 < a.ny;
    T *cc = s.cc[lane] + 6;
    cc[0] = cxok ? a.cxm[cgi] : (T)0;
    cc[1] = cxok ? a.cxp[cgi] : (T)0;
    cc[2] = cxok ? a.sdx[cgi] : (T)0;
    cc[3] = ok0 ? a.cym[gj0] : (T)0;
    cc[4] = ok1 ? a.cym[gj0 + 1] : (T)0;
    cc[5] = ok0 ? a.cyp[gj0] : (T)0;
    cc[6] = ok1 ? a.cyp[gj0 + 1] : (T)0;
    cc[7] = ok0 ? a.sdy[gj0] : (T)0;
    cc[8] = ok1 ? a.sdy[gj0 + 1] : (T)0;
    s.ccu[lane][2] = (ok0 ? 1u : 0u) | (ok1 ? 2u : 0u);
  }
  // the item's z coefficients, read from shared memory by every step (planes k0 - 2 .. k1 + 1)
  for (int pl = k0 - 2 + tid; pl <= k1 + 1; pl += THREADS) {
    const bool ok = pl >= 0 && pl < a.nz;
    ZC<T> z;
    z.m = ok ? a.czm[pl] : (T)0;
    z.p = ok ? a.czp[pl] : (T)0;
    z.s = ok ? a.sdz[pl] : (T)0;
    z.pad = (T)0;
    s.zc[pl - (k0 - 2)] = z;
  }
  // slots: plane p lives in e slot (p + 2 NE) mod NE and rhs/mask slot (p + 2 NR) mod NR
  auto wrap_e = [](int x) { return x >= NE ? x - NE : x; };
  auto wrap_r = [](int x) { return x >= NR ? x - NR : x; };
  // padded coordinates: cell (i, j, k) at (i + OX, j + 1, k + 1); OX = 4
  auto load_e = [&](int plane, int b) {
    mbar_expect_tx(&s.bar_e[b], ebytes);
    tma_load3(s.e[b], tm_e, &s.bar_e[b], x0, y0 - 1, plane + 1);
    pend_e |= 1u << b;
  };
  auto load_r = [&](int plane, int b) {
    mbar_expect_tx(&s.bar_r[b], rbytes);
    tma_load3(s.r[b], tm_r, &s.bar_r[b], x0, y0, plane + 1);
    tma_load3(s.m[b], tm_m, &s.bar_r[b], x0, y0, plane + 1);
    pend_r |= 1u << b;
  };
  auto wait_e = [&](int b, int lim) {
    if (bad) return;
    if (mbar_wait(&s.bar_e[b], (pe >> b) & 1u, lim)) { pe ^= 1u << b; pend_e &= ~(1u << b); }
    else bad = true;
  };
  auto wait_r = [&](int b) {
    if (bad) return;
    if (mbar_wait(&s.bar_r[b], (pr >> b) & 1u, WAIT_LIMIT)) { pr ^= 1u << b; pend_r &= ~(1u << b); }
    else bad = true;
  };
  const int se0 = (k0 - 2 + 2 * NE) % NE, sr0 = (k0 - 1 + 2 * NR) % NR;   // planes k0 - 2 / k0 - 1
  // prologue: e planes k0-2 .. k0-1+DP and rhs/mask planes k0-1 .. k0-2+DP.  Step q waits
  // for e plane q+1 and rhs/mask plane q and, after the step's barrier (so no thread still
  // reads the buffers being refilled), prefetches e plane q+1+DP (into the buffer of plane
  // q-2, last read in step q-1) and rhs/mask plane q+DP (buffer of plane q-2, last read by
  // the black pass of step q-1).  Every load is issued once and waited for once.
  if (issuer) {
    fence_proxy_async();
    for (int pl = k0 - 2, b = se0; pl <= min(k0 - 1 + DP, k1 + 1); ++pl, b = wrap_e(b + 1)) load_e(pl, b);
    for (int pl = k0 - 1, b = sr0; pl <= min(k0 - 2 + DP, k1); ++pl, b = wrap_r(b + 1)) load_r(pl, b);
  }
  int sq = wrap_e(se0 + 1), rq = sr0;   // slots of plane q (e, rhs/mask)
  wait_e(se0, first_wait);
  wait_e(sq, WAIT_LIMIT);
  // registers: each strip in planes q-2 (Cm2; its red cells are final once plane q-2's red
  // pass is done), q-1 (Cm1) and q (C0)
  vec4<T> Cm2[NS], Cm1[NS], C0[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    Cm1[t] = lds4(s.e[se0] + ie0 + SR * t * BX);
    C0[t] = lds4(s.e[sq] + ie0 + SR * t * BX);
    Cm2[t] = Cm1[t];
  }
  S *const dst0 = static_cast<S *>(a.out) + (long long)(y0 + ys + 1) * a.px + (x0 + xs + 4);
  // not unrolled: with the coarse levels' irregular-cell path, three copies of the step
  // overflow the instruction cache (measured: most stalls waiting for instructions), and the
  // strips' rotation by register moves costs the FP32 kernel nothing measurable
#pragma unroll 1
  for (int q = k0 - 1; q <= k1; ++q) {
    const int sp1 = wrap_e(sq + 1), sm1 = sq == 0 ? NE - 1 : sq - 1;
    wait_e(sp1, WAIT_LIMIT);
    wait_r(rq);
    if (__syncthreads_or(bad)) {   // every thread leaves the march together
      bad = true;
      break;
    }
    if (issuer) {
      fence_proxy_async();
      if (q + 1 + DP <= k1 + 1) load_e(q + 1 + DP, wrap_e(sp1 + DP));
      if (q + DP <= k1) load_r(q + DP, wrap_r(rq + DP));
    }
    S *P = s.e[sq], *Pm = s.e[sm1];
    const S *Pp = s.e[sp1];
    const int rqm = rq == 0 ? NR - 1 : rq - 1;   // rhs/mask slot of plane q-1
    const S *R = s.r[rq], *Rm = s.r[rqm];
    const uint8_t *M = s.m[rq], *Mm = s.m[rqm];
    // z coefficients of planes q (red pass) and q-1 (black pass)
    const ZC<T> zq = s.zc[q - (k0 - 2)], zb = s.zc[q - 1 - (k0 - 2)];
    const T zmr = zq.m, zpr = zq.p, szr = zq.s, zmb = zb.m, zpb = zb.p, szb = zb.s;
    const bool red = q >= 0 && q < a.nz;
    // x0 + xs is even: strip t relaxes u = (y0 + ys + SR t + q) & 1 (SR is odd, so strip 1 has
    // the other colour of strip 0)
    const bool parq = ((y0 + ys + q) & 1) == 0;
    vec4<T> U[NS];   // the strips in plane q+1
#pragma unroll
    for (int t = 0; t < NS; ++t) U[t] = lds4(Pp + ie0 + SR * t * BX);
    // red cells of strip t of plane q (ua: its colour's u, a compile-time constant):
    // x-edges from the adjacent lanes, or the ring at the edges
    // In FP32 a pass gathers both strips' inputs (x-edges, the rows above and below, rhs,
    // mask) before relaxing either, so the shared-memory loads of the two strips overlap (the
    // kernel's main stall is their latency); the FP64 form, bound by the FP64 pipe and short
    // of registers, takes one strip at a time.
    struct In {
      T w, e;
      vec4<T> N, So, Rr;
      unsigned mm;
    };
    auto red_load = [&](const int t) {
      const int ie = ie0 + SR * t * BX;
      In in;
      const T ep = ld1(P + ie + eoff);
      T w = __shfl_up_sync(0xffffffffu, C0[t].w, 1);
      T e = __shfl_down_sync(0xffffffffu, C0[t].x, 1);
      in.w = lane == 0 ? ep : w;
      in.e = lane == 31 ? ep : e;
      in.N = lds4(P + ie - BX);
      in.So = lds4(P + ie + BX);
      in.Rr = lds4(R + ir0 + SR * t * BX);
      in.mm = *reinterpret_cast<const unsigned *>(M + im0 + SR * t * BXM) | inval[t];
      return in;
    };
    auto red_do = [&](auto ua, const int t, const In &in) {
      const int ie = ie0 + SR * t * BX;
      const long long gid = (long long)(q + 1) * a.sz + (long long)(y0 + ys + SR * t + 1) * a.sy + (x0 + xs + 4);
      relax_strip<decltype(ua)::value, COARSE>(C0[t], in.w, in.e, in.N, in.So, Cm1[t], U[t], in.Rr, in.mm, X, cym[t],
                                               cyp[t], sy[t] + szr, zmr, zpr, sh, om, a, gid);
      C0[t] = stored4<S>(C0[t]);   // the registers hold what every reader of the buffer sees
      sts4(P + ie, C0[t]);
    };
    if (!ring && red) {
      if constexpr (sizeof(T) == 4) {
        const In i0 = red_load(0), i1 = red_load(1);
        if (parq) {
          red_do(U0{}, 0, i0);
          red_do(U1{}, 1, i1);
        } else {
          red_do(U1{}, 0, i0);
          red_do(U0{}, 1, i1);
        }
      } else {
        if (parq) {
          red_do(U0{}, 0, red_load(0));
          red_do(U1{}, 1, red_load(1));
        } else {
          red_do(U1{}, 0, red_load(0));
          red_do(U0{}, 1, red_load(1));
        }
      }
    }
    if (ring && red) {
      // ring row strips (rows -1 and TY, this lane's x): red cells of plane q, in place
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const T *cc = s.cc[lane] + 3 * h;
        const int yr = h == 0 ? -1 : TY;
        const int iq0 = (yr + 2) * BX + (xs + 4), irq0 = (yr + 1) * BX + (xs + 4), imq0 = (yr + 1) * BXM + (xs + 4);
        vec4<T> C = lds4(P + iq0);
        const vec4<T> N = lds4(P + iq0 - BX), So = lds4(P + iq0 + BX), Zm = lds4(Pm + iq0), Zp = lds4(Pp + iq0);
        const vec4<T> Rr = lds4(R + irq0);
        const unsigned mm = *reinterpret_cast<const unsigned *>(M + imq0) | s.ccu[lane][h];
        const T ep = ld1(P + iq0 + eoff);
        T w = __shfl_up_sync(0xffffffffu, C.w, 1);
        T e = __shfl_down_sync(0xffffffffu, C.x, 1);
        w = lane == 0 ? ep : w;
        e = lane == 31 ? ep : e;
        const long long gid = (long long)(q + 1) * a.sz + (long long)(y0 + yr + 1) * a.sy + (x0 + xs + 4);
        if (((y0 + yr + q) & 1) == 0)
          relax_strip<0, COARSE>(C, w, e, N, So, Zm, Zp, Rr, mm, X, cc[0], cc[1], cc[2] + szr, zmr, zpr, sh, om,
                                 a, gid);
        else
          relax_strip<1, COARSE>(C, w, e, N, So, Zm, Zp, Rr, mm, X, cc[0], cc[1], cc[2] + szr, zmr, zpr, sh, om,
                                 a, gid);
        sts4(P + iq0, C);
      }
      // ring column cell (x = -1 or TX): the red one of the lane's pair of rows
      if (lane < COL_LANES) {
        const int pr_ = lane % (TY / 2);
        const int cxl = lane < TY / 2 ? -1 : TX;
        const int h = (x0 + cxl + y0 + 2 * pr_ + q) & 1, cy = 2 * pr_ + h;
        const int ic = (cy + 2) * BX + (cxl + 4);
        const int icr = (cy + 1) * BX + (cxl + 4), icm = (cy + 1) * BXM + (cxl + 4);
        const T *cf = s.cc[lane] + 6;
        const T cc0 = ld1(P + ic), cw = ld1(P + ic - 1), ce = ld1(P + ic + 1), cn = ld1(P + ic - BX),
                cs = ld1(P + ic + BX), czmv = ld1(Pm + ic), czpv = ld1(Pp + ic), crs = ld1(R + icr) - sh;
        T v = relax1(cc0, cw, ce, cn, cs, czmv, czpv, cf[0], cf[1], cf[3 + h], cf[5 + h], zmr, zpr,
                     cf[2] + (cf[7 + h] + szr), crs, om);
        unsigned mb = M[icm];
        if constexpr (COARSE) {
          if (mb == IRREGULAR) {
            const long long id = (long long)(q + 1) * a.sz + (long long)(y0 + cy + 1) * a.sy + (x0 + cxl + 4);
            v = relax_frac(a, id, cc0, cw, ce, cn, cs, czmv, czpv, cf[0], cf[1], cf[3 + h], cf[5 + h], zmr, zpr,
                           crs, om);
            mb = 0u;
          }
        }
        if (((s.ccu[lane][2] >> h) & 1u) && mb == 0u) st1(P + ic, v);
      }
    }
    // black cells of plane q-1: neighbours all red, updated by now (in-plane ones in
    // shared memory, the z-neighbours in Cm2 and C0); store the strips from registers
    const int kb = q - 1;
    // black cells of strip t of plane q-1 (they sit at the same u as the red cells of plane q)
    auto black_load = [&](const int t) {
      const int ie = ie0 + SR * t * BX;
      In in;
      const T ep = ld1(Pm + ie + eoff);
      T w = __shfl_up_sync(0xffffffffu, Cm1[t].w, 1);
      T e = __shfl_down_sync(0xffffffffu, Cm1[t].x, 1);
      in.w = lane == 0 ? ep : w;
      in.e = lane == 31 ? ep : e;
      in.N = lds4(Pm + ie - BX);
      in.So = lds4(Pm + ie + BX);
      in.Rr = lds4(Rm + ir0 + SR * t * BX);
      in.mm = *reinterpret_cast<const unsigned *>(Mm + im0 + SR * t * BXM) | inval[t];
      return in;
    };
    auto black_do = [&](auto ua, const int t, const In &in, S *const dk) {
      const long long gid = (long long)q * a.sz + (long long)(y0 + ys + SR * t + 1) * a.sy + (x0 + xs + 4);
      relax_strip<decltype(ua)::value, COARSE>(Cm1[t], in.w, in.e, in.N, in.So, Cm2[t], C0[t], in.Rr, in.mm, X,
                                               cym[t], cyp[t], sy[t] + szb, zmb, zpb, sh, om, a, gid);
      if ((inval[t] & 0xffu) == 0u) {   // the strip's row is in the grid
        S *dst = dk + (long long)(SR * t) * a.px;
        if (inval[t] == 0u) {
          sts4(dst, Cm1[t]);
        } else {
          if (!(inval[t] & 0xff00u)) st1(dst + 1, Cm1[t].y);
          if (!(inval[t] & 0xff0000u)) st1(dst + 2, Cm1[t].z);
          if (!(inval[t] & 0xff000000u)) st1(dst + 3, Cm1[t].w);
          st1(dst, Cm1[t].x);
        }
      }
    };
    if (!ring && kb >= k0 && kb < k1) {
      S *const dk = dst0 + (long long)(kb + 1) * a.sz;
      if constexpr (sizeof(T) == 4) {
        const In i0 = black_load(0), i1 = black_load(1);
        if (parq) {
          black_do(U0{}, 0, i0, dk);
          black_do(U1{}, 1, i1, dk);
        } else {
          black_do(U1{}, 0, i0, dk);
          black_do(U0{}, 1, i1, dk);
        }
      } else {
        if (parq) {
          black_do(U0{}, 0, black_load(0), dk);
          black_do(U1{}, 1, black_load(1), dk);
        } else {
          black_do(U1{}, 0, black_load(0), dk);
          black_do(U0{}, 1, black_load(1), dk);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      Cm2[t] = Cm1[t];
      Cm1[t] = C0[t];
      C0[t] = U[t];
    }
    sq = sp1;
    rq = wrap_r(rq + 1);
  }
}

// a wait gave up: flag it and let copies still in flight land before the block's shared
// memory is released (the issuing thread; every thread then leaves)
template <typename T, typename S>
__device__ __forceinline__ void march_abort(Smem<T, S> &s, int *err, unsigned pe, unsigned pr, unsigned pend_e,
                                            unsigned pend_r) {
  if (threadIdx.x == RING_WARP * 32) {
    atomicExch(err, 1);
    for (int b = 0; b < NE; ++b)
      if ((pend_e >> b) & 1u) mbar_wait(&s.bar_e[b], (pe >> b) & 1u, WAIT_LIMIT);
    for (int b = 0; b < NR; ++b)
      if ((pend_r >> b) & 1u) mbar_wait(&s.bar_r[b], (pr >> b) & 1u, WAIT_LIMIT);
  }
  __syncthreads();
}

template <typename T, typename S>
__device__ __forceinline__ Smem<T, S> &march_smem() {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<T, S> &s = *reinterpret_cast<Smem<T, S> *>(smem_raw);
  if (threadIdx.x == 0) {
    for (int b = 0; b < NE; ++b) mbar_init(&s.bar_e[b], 1);
    for (int b = 0; b < NR; ++b) mbar_init(&s.bar_r[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  return s;
}

template <typename T, bool COARSE, typename S = T>
__global__ void __launch_bounds__(THREADS, min_ctas<T>()) k_sweep_zmarch(const __grid_constant__ CUtensorMap tm_e,
                                                                         const __grid_constant__ CUtensorMap tm_r,
                                                                         const __grid_constant__ CUtensorMap tm_m,
                                                                         Args<T> a) {
  static_assert(sizeof(T) == 4 || !COARSE, "coarse levels are swept in FP32");
  static_assert(std::is_same<typename Arith<S>::type, T>::value, "storage of the arithmetic type, or BF16 for FP32");
  Smem<T, S> &s = march_smem<T, S>();
  const int tid = threadIdx.x;
  const float om = a.omega;
  const T sh = a.shift ? (T)(*a.shift) : (T)0;
  // per slot: parity of its next completion (toggled when a wait sees it land); the issuer
  // also keeps which slots have a copy in flight that it has not yet seen land
  unsigned pe = 0, pr = 0, pend_e = 0, pend_r = 0;
  bool bad = false;
  const int first_wait = a.first_wait;
  const int tiles = a.tiles_x * a.tiles_y;
  for (int item = blockIdx.x; item < a.items;) {
    // the next item: fetched by one thread now, read by all after this item's barriers
    if (a.counter && tid == 0) s.next = (int)gridDim.x + atomicAdd(a.counter, 1);
    const int bx = item % a.tiles_x, by = (item / a.tiles_x) % a.tiles_y, bz = item / tiles;
    const int x0 = bx * TX, y0 = by * TY;
    const int k0 = bz * a.kz, k1 = min(a.nz, k0 + a.kz);
    if (k0 >= k1) {   // an empty chunk (not produced by the host's chunking)
      __syncthreads();
      const int nxt = a.counter ? s.next : item + (int)gridDim.x;
      __syncthreads();
      item = nxt;
      continue;
    }
    march_item<T, COARSE, S>(s, a, &tm_e, &tm_r, &tm_m, x0, y0, k0, k1, sh, om, first_wait, pe, pr, pend_e, pend_r,
                             bad);
    if (bad) {
      march_abort(s, a.err, pe, pr, pend_e, pend_r);
      return;
    }
    const int nxt = a.counter ? s.next : item + (int)gridDim.x;
    __syncthreads();   // the next item's prologue refills buffers this item's last step read
    item = nxt;
  }
}

// Several problems' sweeps of one level in one launch (FP32, storage FP32): problem q's items
// are items item0[q] .. item0[q + 1] - 1 of the launch, each with that problem's arguments and
// tensor maps (kernel parameters, indexed by q).  Items are taken in turn from counter (zeroed
// before the launch), or item + k gridDim.x when counter is null.
constexpr int BATCH_MAX = 48;   // problems per batched launch (kernel parameters of at most 32 KB)

template <typename T>
struct Batch {
  CUtensorMap tm[BATCH_MAX][3];   // e (the input buffer), r, mask
  Args<T> a[BATCH_MAX];
  int item0[BATCH_MAX + 1];
  int n;
  int *counter;
  int *err;
};
static_assert(sizeof(Batch<float>) <= 32764, "kernel parameters are limited to 32764 bytes");

template <typename T, bool COARSE>
__global__ void __launch_bounds__(THREADS, min_ctas<T>()) k_sweep_zmarch_batch(const __grid_constant__ Batch<T> B) {
  static_assert(sizeof(T) == 4, "batched sweeps are FP32");
  Smem<T, T> &s = march_smem<T, T>();
  const int tid = threadIdx.x;
  unsigned pe = 0, pr = 0, pend_e = 0, pend_r = 0;
  bool bad = false;
  const int items = B.item0[B.n];
  for (int item = blockIdx.x; item < items;) {
    if (B.counter && tid == 0) s.next = (int)gridDim.x + atomicAdd(B.counter, 1);
    int q = 0, hi = B.n - 1;   // the problem: the last q with item0[q] <= item
    while (q < hi) {
      const int mid = (q + hi + 1) >> 1;
      if (B.item0[mid] <= item) q = mid;
      else hi = mid - 1;
    }
    const Args<T> &a = B.a[q];
    const int li = item - B.item0[q];
    const int bx = li % a.tiles_x, by = (li / a.tiles_x) % a.tiles_y, bz = li / (a.tiles_x * a.tiles_y);
    const int k0 = bz * a.kz, k1 = min(a.nz, k0 + a.kz);
    if (k0 < k1) {
      const T sh = a.shift ? (T)(*a.shift) : (T)0;
      march_item<T, COARSE, T>(s, a, &B.tm[q][0], &B.tm[q][1], &B.tm[q][2], bx * TX, by * TY, k0, k1, sh, a.omega,
                               a.first_wait, pe, pr, pend_e, pend_r, bad);
      if (bad) {
        march_abort(s, B.err, pe, pr, pend_e, pend_r);
        return;
      }
    } else {
      __syncthreads();
    }
    const int nxt = B.counter ? s.next : item + (int)gridDim.x;
    __syncthreads();
    item = nxt;
  }
}

}  // namespace zm
}  // namespace ibm
