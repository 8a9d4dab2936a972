// Fused two-colour red-black Gauss-Seidel sweep on the finest level: z-march with
// TMA-staged planes in shared memory.
//
// One CTA owns an x-y tile (TX x TY) and a z-range [k0, k1).  Step q of the march
//   1. updates the red cells of plane q on the tile plus a one-cell ring (the ring is
//      recomputed by both neighbouring CTAs, so no inter-CTA exchange is needed),
//   2. updates the black cells of plane q-1 on the tile (its red neighbours in planes
//      q-2, q-1, q are all new by then),
//   3. stores plane q-1 of the tile to the output array.
// Every value is read from the input array and written to a separate output array, so the
// result is exactly one red half-sweep followed by one black half-sweep (deterministic,
// independent of the tiling).  Planes of e (halo 2 in x and y), the right-hand side and
// the mask (halo 1) arrive by cp.async.bulk.tensor into rings of shared-memory buffers two
// steps ahead of their use, with one mbarrier per buffer; the tensor maps zero-fill
// everything outside the padded arrays.  Waits are bounded: a wait that gives up sets
// the error flag, waits (bounded) for the copies still in flight and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ibm {
namespace zm {

constexpr int TX = 64;          // tile width (cells); multiple of 16
constexpr int TY = 16;          // tile height
constexpr int BX = TX + 8;      // staged width of e and rhs: x in [-4, TX + 4)
constexpr int BXM = TX + 16;    // staged width of the mask (an 8-bit box row must be 16-byte multiple)
constexpr int EY = TY + 4;      // e rows: y in [-2, TY + 2)
constexpr int RY = TY + 2;      // rhs / mask rows: y in [-1, TY + 1)
constexpr int THREADS = 256;
// prefetch distance in planes (bytes in flight per SM hide the DRAM latency); rings hold
// the planes in use (e: q-2 .. q+1, rhs/mask: q-1 .. q) plus the ones in flight
template <typename T> struct Depth { static constexpr int D = sizeof(T) == 4 ? 3 : 2; };
template <typename T> constexpr int NE = 4 + Depth<T>::D;
template <typename T> constexpr int NR = 2 + Depth<T>::D;
constexpr long long WAIT_LIMIT = 1LL << 22;

constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }

// every TMA destination starts on a 128-byte boundary
template <typename T>
struct Smem {
  alignas(128) T e[NE<T>][pad128(EY * BX * (int)sizeof(T)) / (int)sizeof(T)];
  alignas(128) T r[NR<T>][pad128(RY * BX * (int)sizeof(T)) / (int)sizeof(T)];
  alignas(128) uint8_t m[NR<T>][pad128(RY * BXM)];
  alignas(8) uint64_t bar_e[NE<T>];
  alignas(8) uint64_t bar_r[NR<T>];
  T cx[2][TX + 2], cy[2][TY + 2], sx[TX + 2], sy[TY + 2];
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

// one colour update of cell (x, y) of plane buffer P (planes pm, pp below/above):
// e += omega (sum_d c_d e_nb - D e - rhs) / D.  The residual is formed in T; the relaxation
// factor 1/D and the step are FP32 (they do not move the fixed point, which is the exact
// T-precision solution of the row), keeping FP64 work to the stencil in the FP64 variant.
template <typename T>
__device__ __forceinline__ void relax(const Smem<T> &s, T *P, const T *pm, const T *pp, const T *R, const uint8_t *M,
                                      int x, int y, T czm, T czp, T syz, T sh, float omega) {
  const int ie = (y + 2) * BX + (x + 4);
  const int ir = (y + 1) * BX + (x + 4);
  if (M[(y + 1) * BXM + (x + 4)] != 0) return;
  const T D = s.sx[x + 1] + syz;
  T sum = s.cx[0][x + 1] * P[ie - 1];
  sum += s.cx[1][x + 1] * P[ie + 1];
  sum += s.cy[0][y + 1] * P[ie - BX];
  sum += s.cy[1][y + 1] * P[ie + BX];
  sum += czm * pm[ie];
  sum += czp * pp[ie];
  const T pc = P[ie];
  const T res = (sum - D * pc) - (R[ir] - sh);
  const float step = omega * (float)res * __frcp_rn((float)D);
  P[ie] = pc + (T)step;
}

template <typename T>
__global__ void __launch_bounds__(THREADS) k_sweep_zmarch(const __grid_constant__ CUtensorMap tm_e,
                                                         const __grid_constant__ CUtensorMap tm_r,
                                                         const __grid_constant__ CUtensorMap tm_m, Args<T> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem<T> &s = *reinterpret_cast<Smem<T> *>(smem_raw);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * a.kz;
  const int k1 = min(a.nz, k0 + a.kz);
  if (k0 >= k1) return;
  // 1-D coefficients of the tile (halo 1); zero outside the grid
  for (int q = tid; q < TX + 2; q += THREADS) {
    int i = x0 + q - 1;
    bool ok = i >= 0 && i < a.nx;
    s.cx[0][q] = ok ? a.cxm[i] : (T)0;
    s.cx[1][q] = ok ? a.cxp[i] : (T)0;
    s.sx[q] = ok ? a.sdx[i] : (T)0;
  }
  for (int q = tid; q < TY + 2; q += THREADS) {
    int j = y0 + q - 1;
    bool ok = j >= 0 && j < a.ny;
    s.cy[0][q] = ok ? a.cym[j] : (T)0;
    s.cy[1][q] = ok ? a.cyp[j] : (T)0;
    s.sy[q] = ok ? a.sdy[j] : (T)0;
  }
  constexpr int NEt = NE<T>, NRt = NR<T>, DP = Depth<T>::D;
  if (tid == 0) {
    for (int b = 0; b < NEt; ++b) mbar_init(&s.bar_e[b], 1);
    for (int b = 0; b < NRt; ++b) mbar_init(&s.bar_r[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned ebytes = EY * BX * sizeof(T), rbytes = RY * BX * sizeof(T) + RY * BXM;
  // padded coordinates: cell (i, j, k) at (i + OX, j + 1, k + 1); OX = 4
  auto load_e = [&](int plane) {   // plane in [k0-2, k1+2]
    int b = (plane + 2 * NEt) % NEt;
    mbar_expect_tx(&s.bar_e[b], ebytes);
    tma_load3(s.e[b], &tm_e, &s.bar_e[b], x0, y0 - 1, plane + 1);
  };
  auto load_r = [&](int plane) {
    int b = (plane + 2 * NRt) % NRt;
    mbar_expect_tx(&s.bar_r[b], rbytes);
    tma_load3(s.r[b], &tm_r, &s.bar_r[b], x0, y0, plane + 1);
    tma_load3(s.m[b], &tm_m, &s.bar_r[b], x0, y0, plane + 1);
  };
  // phase bit per buffer: number of completed loads of that buffer, mod 2
  unsigned pe = 0, pr = 0;   // bit b = parity expected for buffer b
  // prologue: e planes k0-2 .. k0-1+DP and rhs/mask planes k0-1 .. k0-2+DP; step q then
  // prefetches e plane q+1+DP and rhs/mask plane q+DP and waits for e plane q+1 and
  // rhs/mask plane q, so every load is issued once and waited for once
  if (tid == 0) {
    for (int pl = k0 - 2; pl <= min(k0 - 1 + DP, k1 + 1); ++pl) load_e(pl);
    for (int pl = k0 - 1; pl <= min(k0 - 2 + DP, k1); ++pl) load_r(pl);
  }
  bool bad = false;
  auto wait_e = [&](int plane) {
    int b = (plane + 2 * NEt) % NEt;
    if (!bad && !mbar_wait(&s.bar_e[b], (pe >> b) & 1u)) bad = true;
    pe ^= 1u << b;
  };
  auto wait_r = [&](int plane) {
    int b = (plane + 2 * NRt) % NRt;
    if (!bad && !mbar_wait(&s.bar_r[b], (pr >> b) & 1u)) bad = true;
    pr ^= 1u << b;
  };
  wait_e(k0 - 2);
  wait_e(k0 - 1);
  const T sh = a.shift ? (T)(*a.shift) : (T)0;
  const float om = a.omega;
  for (int q = k0 - 1; q <= k1; ++q) {
    // prefetch: e plane q+1+DP (its buffer held plane q-3), rhs/mask plane q+DP (held q-2);
    // both were last read in the black phase of step q-1, which ended at a barrier
    if (tid == 0) {
      fence_proxy_async();
      if (q + 1 + DP <= k1 + 1) load_e(q + 1 + DP);
      if (q + DP <= k1) load_r(q + DP);
    }
    wait_e(q + 1);
    wait_r(q);
    if (__syncthreads_or(bad)) break;
    T *Pm = s.e[(q - 1 + 2 * NEt) % NEt], *P = s.e[(q + 2 * NEt) % NEt], *Pp = s.e[(q + 1 + 2 * NEt) % NEt];
    // red cells of plane q on the tile plus the ring
    if (q >= 0 && q < a.nz) {
      const T czm = a.czm[q], czp = a.czp[q], szk = a.sdz[q];
      const T *R = s.r[(q + 2 * NRt) % NRt];
      const uint8_t *M = s.m[(q + 2 * NRt) % NRt];
      const int rowred = (TX + 2) / 2;
      for (int c = tid; c < rowred * (TY + 2); c += THREADS) {
        int y = c / rowred - 1;
        int gj = y0 + y;
        int x = ((gj + q) & 1 ? -1 : 0) + 2 * (c % rowred);
        int gi = x0 + x;
        if (gi < 0 || gi >= a.nx || gj < 0 || gj >= a.ny) continue;
        relax<T>(s, P, Pm, Pp, R, M, x, y, czm, czp, s.sy[y + 1] + szk, sh, om);
      }
    }
    __syncthreads();
    // black cells of plane q-1 on the tile, then store plane q-1
    const int kb = q - 1;
    if (kb >= k0 && kb < k1) {
      T *Bm = s.e[(kb - 1 + 2 * NEt) % NEt], *B = s.e[(kb + 2 * NEt) % NEt], *Bp = P;
      const T czm = a.czm[kb], czp = a.czp[kb], szk = a.sdz[kb];
      const T *R = s.r[(kb + 2 * NRt) % NRt];
      const uint8_t *M = s.m[(kb + 2 * NRt) % NRt];
      for (int c = tid; c < (TX / 2) * TY; c += THREADS) {
        int y = c / (TX / 2);
        int gj = y0 + y;
        int x = ((gj + kb + 1) & 1) + 2 * (c % (TX / 2));
        int gi = x0 + x;
        if (gi >= a.nx || gj >= a.ny) continue;
        relax<T>(s, B, Bm, Bp, R, M, x, y, czm, czp, s.sy[y + 1] + szk, sh, om);
      }
      __syncthreads();
      // store the tile of plane kb (every cell: updated fluid values, copied others)
      constexpr int V = 4;
      for (int c = tid; c < (TX / V) * TY; c += THREADS) {
        int y = c / (TX / V), x = V * (c % (TX / V));
        int gj = y0 + y, gi = x0 + x;
        if (gj >= a.ny || gi >= a.nx) continue;
        const T *src = &B[(y + 2) * BX + (x + 4)];
        T *dst = a.out + ((long long)(kb + 1) * (a.ny + 2) + (gj + 1)) * a.px + (gi + 4);
        if (gi + V <= a.nx) {
          if (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(src);
          } else {
            reinterpret_cast<double2 *>(dst)[0] = reinterpret_cast<const double2 *>(src)[0];
            reinterpret_cast<double2 *>(dst)[1] = reinterpret_cast<const double2 *>(src)[1];
          }
        } else {
          for (int u = 0; u < V && gi + u < a.nx; ++u) dst[u] = src[u];
        }
      }
    }
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

}  // namespace zm
}  // namespace ibm
