// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ibm_poisson.h"

namespace ibm {

// Padded cell arrays: one halo layer in every direction; element i = 0 of a row sits at
// offset OX so rows start 32-byte aligned for float and double.
constexpr int OX = 4;
// Fixed reduction width: block partials are summed in a fixed order, so every reduction (and
// with it every result) is the same on any device, whatever its SM count.
constexpr int REDUCE_BLOCKS = 608;
// a second fixed width (grid-stride kernels over ghost rows, fluid statistics, cut-cell flags):
// the same partial-sum layout, hence the same bits, on any number of SMs
constexpr int FIXED_BLOCKS = 152;
constexpr int REDUCE_THREADS = 256;
constexpr int NSCAL = 32;            // device scalars per context

// Device scalar slots (ctx->scal).
enum Scal {
  S_LAMBDA = 0,   // compatibility constant of the fine system
  S_MU = 1,       // fluid mean of the last fine residual
  S_NORM2 = 2,    // ||S P r||^2 of the last fine residual
  S_FLUIDVOL = 3, // sum of fluid volumes (fine)
  S_NF = 4,       // number of fluid cells (fine)
  S_MEANP = 5,    // fluid mean of p (gauge)
  S_PNZ = 6,      // the packed initial p has a nonzero value (an integer flag in the slot's bits)
  S_LEVEL_SHIFT = 8  // S_LEVEL_SHIFT + l: projection shift of coarse level l
};

struct LevelGeom {
  int nx, ny, nz, px;
  long long sy, sz, ntot;  // strides and padded size
};

inline LevelGeom make_geom(int nx, int ny, int nz) {
  LevelGeom g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.px = ((nx + OX + 1 + 15) / 16) * 16;   // 16-byte row pitch even for the 8-bit mask (TMA)
  g.sy = g.px;
  g.sz = (long long)g.px * (ny + 2);
  g.ntot = g.sz * (nz + 2);
  return g;
}

__host__ __device__ inline long long pidx(const LevelGeom &g, int i, int j, int k) {
  return ((long long)(k + 1) * (g.ny + 2) + (j + 1)) * g.px + (i + OX);
}

constexpr long long GHOST_CORNER = 1LL << 62;   // flag on a ghost-row source that is itself a ghost
// finest-level mask value of a fluid cell with a cut membrane link: a fluid row whose stencil
// reads ghost entries, updated by the cut-cell kernels instead of the regular ones
constexpr uint8_t MASK_CUT = 4;
__host__ __device__ __forceinline__ bool fluid_row(uint8_t m) { return m == 0 || m == MASK_CUT; }

// One multigrid level; arrays are device memory owned by the hierarchy.
struct Level {
  LevelGeom g;
  uint8_t *mask = nullptr;                  // padded; 0 = active fluid row
  uint8_t *inner = nullptr;                 // levels >= 1, padded: 1 where the cell and its 26
                                            // neighbours are all fluid
  void *e = nullptr, *r = nullptr;          // padded, element type of the hierarchy
  void *fx = nullptr, *fy = nullptr, *fz = nullptr;   // face fractions (levels >= 1)
  void *c1d = nullptr;                      // cxm cxp cym cyp czm czp (n each, element type)
  double *w1d = nullptr;                    // widths dx dy dz
  double *cen = nullptr;                    // centres xc yc zc
  int8_t *poff = nullptr;                   // prolongation: neighbour offset per fine index (x,y,z)
  float *pt = nullptr;                      // prolongation: weight of the neighbour (x,y,z)
  void *wT = nullptr;                       // widths dx dy dz in the element type
  void *sdiag = nullptr;                    // finest level: cxm+cxp, cym+cyp, czm+czp (element type)
  double fluid_vol = 0.0;
  long long nfluid = 0;
  // levels >= 1 swept by the fused z-march (large enough FP32 levels)
  bool zm = false;
  uint8_t *zmask = nullptr;                 // padded: 0 regular fluid, 8 irregular fluid, 1 other
  void *ealt = nullptr;                     // second e buffer (ping-pong of the fused sweep)
  void *zsd = nullptr;                      // cxm+cxp, cym+cyp, czm+czp (element type)
  CUtensorMap ztm_e[2], ztm_r, ztm_m;       // tensor maps of e (both buffers), r and zmask
  bool bf16 = false;                        // e, r and ealt stored in BF16 (a z-march level of a
                                            // hierarchy built with BF16 coarse storage)
};

struct Hierarchy {
  int elem = 8;                             // bytes per element of levels (4 or 8)
  std::vector<Level> lv;
  // fine-level outer arrays p and b: FP64, or in double-FP32 mode the same bytes as two
  // float arrays each (hi: first ntot floats, lo: next ntot)
  double *p64 = nullptr, *b64 = nullptr;
  // coarsest dense bordered inverse
  int ncoarse = 0;                          // unknowns of the coarsest level (fluid cells)
  void *minv = nullptr;                     // (MAX_COARSE+1)^2, element type of the levels
  void *gj = nullptr;                       // Gauss-Jordan work matrix (global fallback)
  int *cidx = nullptr;                      // padded index of each coarsest unknown
  int *dncoarse = nullptr;                  // device copy of ncoarse
  double *c64 = nullptr;                    // FP64 fine coefficients cxm cxp cym cyp czm czp
  float *cdf = nullptr;                     // fine coefficients, diagonal parts and widths split
                                            // into hi (4n floats) and lo (4n) parts
  // solver-side ghost rows: padded source indices (-1 unused), weights (double and float)
  long long *gsrc = nullptr;
  long long *gdst = nullptr;
  double *gw64 = nullptr;
  float *gw32 = nullptr;
  double *gtmp = nullptr;                   // new ghost values (Jacobi)
  long long geom_version = -1;              // classification the geometry-dependent parts match
  long long gcap = 0;                       // capacity of the solver-side ghost arrays
  double *d_fvol = nullptr;                 // fluid volume per level (device)
  long long *d_ng = nullptr;                // ghost count (device)
  void *graph_exec = nullptr;               // one captured cycle (see solve_impl)
  long long graph_key = 0;
  long long graph_launches = 0;             // kernels in the captured cycle
  // finest level ping-pong for the fused z-march sweep: the second buffer of the
  // level-0 unknown (p64 in FP64 mode, lv[0].e in mixed mode) and TMA tensor maps
  void *e_alt = nullptr;
  int grid_blocks[1] = {1216};              // resident blocks of the restriction
  long long slotcap = 0;                    // membranes: ghost-entry slots after the finest cells
  long long nslot = 0;                      // elements of the finest arrays (cells + slots); in
                                            // double-FP32 mode the hi/lo split point of p and b
  // membranes: cut cells (fluid rows with a cut link), red ones first, each half ascending
  long long cutcap = 0, parcap = 0;
  long long *cut_id = nullptr;              // padded index
  long long *cut_nb = nullptr;              // 6 per cut cell: index of the value each link reads
  int *cut_ijk = nullptr;                   // 3 per cut cell
  long long *par_id = nullptr;              // coarse parents of cut cells (padded index, ascending)
  long long *d_cnt = nullptr;               // device: red cut cells, all cut cells, parents
  long long hcnt[3] = {0, 0, 0};            // host copy
  uint8_t *par_flag = nullptr;              // level-1 scratch flags (kept zero between uses)
  void *bicg_buf = nullptr;                 // workspace of the paper's solver (BiCGStab + SRJ)
  long long bicg_n = 0;
  void *helm_buf = nullptr;                 // workspace of the advection-diffusion solve
  long long helm_n = 0;
  int helm_layout = -1;                     // its u and f arrays hold FP64 (0) or FP32 pairs (1)
  int gcr_m = 0;                            // Krylov directions allocated
  void *gcr_buf = nullptr;                  // 2 gcr_m arrays of nslot elements of T (Z then Q)
  void *gcr_state = nullptr;                // device state of the Krylov acceleration
  double *gcr_part = nullptr;               // its block partial sums
  long long *scan_buf = nullptr;            // compaction scratch: block counts and offsets
  long long scan_cap = 0;
  int tail_level = -1;                      // first level of the one-block coarse tail (-1: none)
  bool zmarch = false;
  int zm_per_sm = 1;                        // resident CTAs per SM of the fused sweep
  int zmc_per_sm = 1;                       // the same for its coarse-level form
  bool coarse_bf16 = false;                 // z-march coarse levels store e and r in BF16
  int *zcount = nullptr;                    // per level: the coarse sweep's item counter
  CUtensorMap tm_e[2], tm_r, tm_m;
  void *tm_base[2] = {nullptr, nullptr};    // which buffer each tm_e describes
  const void *tm_rbase = nullptr;           // the right-hand side tm_r describes
};

}  // namespace ibm

struct ibm_ctx {
  int device = 0;
  double *partials = nullptr;   // REDUCE_BLOCKS * 8 doubles
  double *scal = nullptr;       // NSCAL device scalars
  double *hscal = nullptr;      // pinned host mirror of scal
  int sm_count = 0;
  int wave = 1216;              // 256-thread blocks of one full wave: 8 per SM x sm_count
                                // (launch shape of the grid-stride element-wise kernels)
  long long launches = 0;       // kernels launched by this context (all calls)
  int *errflag = nullptr;       // device flag: a bounded device-side wait gave up
  int sweep_first_wait = -1;    // tries of the fused sweep's first wait per item (-1: the
                                // normal limit; set only to test the timeout path)
  std::string tune_cache;       // autotuner cache file (empty: none)
  cudaStream_t cap_stream = nullptr;   // private stream used only to capture CUDA graphs
  // batched solves: the streams the problems' step graphs run on, fork/join events, and
  // per-problem scalars (device and pinned host) and block partials
  static constexpr int NBSTREAM = 8;
  cudaStream_t bstream[NBSTREAM] = {};
  cudaEvent_t bevent[NBSTREAM + 1] = {};
  double *bscal = nullptr, *bhscal = nullptr, *bpart = nullptr;
  int bcap = 0;                        // problems the batch buffers hold
  // lockstep batches: dynamic-schedule counters of one step's batched sweeps, and the
  // problems' coarse-tail arguments (device copies)
  int *lk_count = nullptr;
  void *lk_tail = nullptr;
  int lk_tail_cap = 0;
};

struct ibm_tables {
  ibm_ctx *ctx = nullptr;
  int nx = 0, ny = 0, nz = 0;
  std::vector<double> xf, yf, zf;   // host copies of the faces
  long long ncell = 0, nfluid = 0, nghost = 0, nsolid = 0;
  // classification (device)
  uint8_t *iblank = nullptr;
  long long *gcell = nullptr;
  double *gbi = nullptr, *gip = nullptr, *gw = nullptr, *gscale = nullptr;
  int *gbase = nullptr, *gflags = nullptr;
  long long *gref = nullptr;
  long long gcap = 0;                // capacity of the per-ghost arrays (entries)
  bool membrane = false;             // classified against membranes (closed = 0): all cells fluid,
                                     // ghost entries are (cell, side) pairs of cut links
  uint8_t *cut = nullptr, *cside = nullptr;   // membranes: per cell, bit d = link in direction d
                                              // (-x +x -y +y -z +z) cut / this cell's side of it
  uint8_t *gside = nullptr;          // membranes: side of each ghost entry
  long long *gkeys = nullptr;        // membranes: 2 cell + side of each entry (ascending)
  // moving-boundary Neumann datum: ghost row g - sum w v = kappa q (q the pressure's normal
  // derivative along the row's direction); d = kappa q is set by ibm_set_neumann or
  // ibm_neumann_rigid and cleared by every classification
  double *gkappa = nullptr, *gd = nullptr;
  int *gtri = nullptr;               // closest triangle of each ghost (global index)
  double *gwself = nullptr;          // each row's own weight moved to the left-hand side (else 0):
                                     // the Dirichlet rows of the velocity systems need it
  bool has_datum = false;
  std::vector<int> mesh_tri_off;     // first global triangle index of each mesh, and the total
  long long geom_version = 0;        // incremented by every classification of these tables
  double *axis = nullptr;            // per-axis faces, centres, widths, coefficients, snapped centres
  char *scratch = nullptr;           // classification scratch kept between classifications
  size_t scratch_cap = 0;
  char *fbuf = nullptr;              // surface-force working set (meshes, incidence, shares)
  size_t fcap = 0;
  // solver hierarchies by precision mode (lazy)
  // one hierarchy per precision (0, 1, 2), then precisions 1 and 2 with BF16 coarse storage
  ibm::Hierarchy *hier[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace ibm {

void set_cuda_error(cudaError_t e, const char *where);
ibm_status check(cudaError_t e, const char *where);
void free_hierarchy(Hierarchy *h);

}  // namespace ibm

#define IBM_TRY(call)                                                   \
  do {                                                                  \
    cudaError_t e__ = (call);                                           \
    if (e__ != cudaSuccess) return ibm::check(e__, #call);              \
  } while (0)
