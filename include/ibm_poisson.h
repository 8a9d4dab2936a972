/*
 * ibm_poisson.h -- C ABI of the GB300 ghost-cell immersed-boundary pressure Poisson library.
 *
 * The library implements the per-time-step pressure Poisson solve of a sharp-interface
 * ghost-cell immersed-boundary method on a stretched cell-centred Cartesian grid
 * (arxiv 2605.04335, Sec. "Governing Equations and Numerical Methods": fractional-step
 * projection, second-order finite differences; Sec. "GPU Porting": iblanking, ghost-cell
 * modules and sparse linear solvers).  Two operations follow the paper's statement of the
 * problem: classify the grid against a triangulated body (iblank, ghost cells, image
 * points), then solve the pressure Poisson equation on the classified grid.
 *
 * Conventions for every function:
 *   - Return an ibm_status; 0 (IBM_OK) is success.  Nothing throws, nothing exits, and a
 *     failed call leaves caller-owned memory in an unspecified but valid state.
 *   - Cell arrays are [k][j][i] with i fastest (x contiguous), nx*ny*nz elements, indexed
 *     by the 64-bit linear index l = (k*ny + j)*nx + i.
 *   - "_dev" pointers are CUDA device pointers on the context's device; everything else is
 *     host memory.  The caller owns every pointer it passes; the library copies what it
 *     keeps.
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default stream.  All
 *     device work of a call is ordered on that stream.  Calls that report results to the
 *     host (counts, convergence) synchronise that stream before returning.
 *   - A context serves one host thread at a time.
 */
#ifndef IBM_POISSON_H
#define IBM_POISSON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IBM_OK = 0,
  IBM_ERR_INVALID_ARG = 1,   /* a pointer, size or option is out of range            */
  IBM_ERR_OOM = 2,           /* device allocation failed                             */
  IBM_ERR_CUDA = 3,          /* a CUDA runtime call failed (see ibm_last_cuda_error) */
  IBM_ERR_NO_FLUID = 4,      /* every cell is solid                                  */
  IBM_ERR_NOT_CONVERGED = 5, /* max cycles reached; the last iterate is returned     */
  IBM_ERR_DIVERGED = 6,      /* residual became non-finite or grew by > 1e6          */
  IBM_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                   */
  IBM_ERR_NOT_IMPLEMENTED = 8,
  IBM_ERR_CAPACITY = 9,      /* a fixed-size internal buffer is too small            */
  IBM_ERR_MESH_NOT_CLOSED = 10 /* a closed mesh is crossed an odd number of times by a
                                  grid column (a hole in the surface on that line)     */
} ibm_status;

typedef struct ibm_ctx ibm_ctx;       /* opaque: device, scratch, reduction buffers      */
typedef struct ibm_tables ibm_tables; /* opaque: classified grid + multigrid hierarchy   */

/* Grid: nx, ny, nz cells (each >= 2); nx+1, ny+1, nz+1 strictly increasing face
 * coordinates (host, float64).  Coordinates must lie in [-4, 4] (the exact inside test
 * works on the integer lattice 2^-24 of that range).  Walls are homogeneous Neumann. */
typedef struct {
  int32_t nx, ny, nz;
  const double *xf, *yf, *zf;
} ibm_grid;

/* Triangulated surface (host).  verts: nverts x 3 float64; tris: ntris x 3 int32 vertex
 * indices, counter-clockwise seen from outside.  closed = 1: a watertight solid body
 * (cells whose centre is inside are solid); closed = 0: a zero-thickness membrane (every
 * cell stays fluid; links between face-neighbours that the membrane crosses are cut, and
 * the cell across a cut link is replaced by a ghost entry of the near side).  Closed meshes
 * must not overlap; membranes and closed bodies are not mixed in one classification
 * (IBM_ERR_NOT_IMPLEMENTED). */
typedef struct {
  int32_t nverts, ntris;
  const double *verts;
  const int32_t *tris;
  int32_t closed;
} ibm_mesh;

/* Solver options; ibm_solve_opts_default fills the defaults shown. */
typedef struct {
  int32_t precision;    /* 0: FP64 throughout; 1: FP32 multigrid inside FP64 iterative
                           refinement (FP64 fine residual, update, gauge, coarsest);
                           2: as 1, but the refinement loop (accumulated p, b, the fine
                           residual, update and gauge) in double-FP32: each value an
                           unevaluated sum of two floats (48-bit significand), residual by
                           error-free transformations on the FP32 pipe.  Mode 2 is this
                           library's choice for hardware with a slow FP64 pipe; the paper
                           states FP64 for the outer loop (mode 1).                     [0] */
  int32_t nu1, nu2;     /* pre-/post-smoothing red-black Gauss-Seidel sweeps        [2,2] */
  int32_t max_cycles;   /* V-cycles (precision 0) or refinement steps (1, 2)        [100] */
  int32_t inner_cycles; /* FP32 V-cycles per refinement step (precision 1, 2)         [2] */
  int32_t use_graph;    /* capture one cycle as a CUDA graph and replay it            [1] */
  double omega;         /* Gauss-Seidel over-relaxation factor, in (0, 2)           [1.3] */
  int32_t krylov;       /* 0: plain refinement (precision 1, 2) or V-cycle iteration
                           (precision 0); 1..8: GCR acceleration with that many
                           directions, restarted, each step's V-cycle correction (FP32
                           in modes 1 and 2, FP64 in mode 0, which then runs in
                           correction form) as preconditioner; -1 automatic: 8 for
                           membrane tables, 0 otherwise.                            [-1] */
  int32_t method;       /* 0: geometric multigrid (this library's solver); 1: BiCGStab
                           preconditioned with scheduled relaxed Jacobi, the paper's
                           pressure solver (precision 0 only, not batched): each
                           preconditioner application is srj_steps Jacobi sweeps with the
                           relaxation factors 1 / Chebyshev nodes of [2/K^2, 2] (K =
                           srj_steps); max_cycles counts BiCGStab iterations.            [0] */
  int32_t srj_steps;    /* Jacobi sweeps per preconditioner application, 1..64            [8] */
  int32_t coarse_bf16;  /* 1: the coarse levels swept by the fused z-march (levels >= 1 of at
                           least 2^18 cells) store their error and right-hand side in BF16,
                           arithmetic in FP32 (loads widen exactly, stores round to nearest
                           even); precision 1 or 2, closed bodies (IBM_ERR_INVALID_ARG
                           otherwise).  A storage experiment of this library; the paper runs
                           FP64 throughout.  The hierarchy is kept beside the FP32 one.     [0] */
  int32_t sweep_chunk;  /* planes per z-chunk of the finest level's fused sweep (the z extent
                           of its tiles; each x-y tile is 128 x 14 cells); 0: chosen by the
                           sweep's cost model (the fewest plane steps for one wave of resident
                           blocks), else 1..256 (IBM_ERR_INVALID_ARG outside).  Searched by
                           ibm_autotune.                                                  [0] */
  int32_t batch_schedule; /* poisson_solve_batched only: 0 = lockstep when every problem allows
                           it (precision 1 or 2, closed bodies, krylov 0 or automatic, FP32
                           coarse storage): each V-cycle stage is one launch over all problems
                           still iterating, else the stream pool; 1 = the stream pool: each
                           problem's step as its own CUDA graph, the problems' graphs running
                           concurrently on the context's streams.  Both give every problem the
                           result of its own poisson_solve.  IBM_ERR_INVALID_ARG outside 0..1.
                                                                                           [0] */
} ibm_solve_opts;

/* Solve report.  resid_history (host, optional) receives the relative residual after
 * every cycle, up to history_cap entries. */
typedef struct {
  int32_t cycles;       /* V-cycles (precision 0) or refinement steps (precision 1, 2)  */
  int32_t history_len;
  double rel_resid;     /* ||S P r|| / ||S P b|| of the returned p (see poisson_solve)  */
  double lambda;        /* the compatibility constant of the bordered system            */
  double ms_total;      /* wall time of the call (host clock, after the final sync)     */
  double *resid_history;
  int32_t history_cap;
} ibm_solve_info;

const char *ibm_status_str(ibm_status s);
/* Text of the last CUDA error seen by this host thread (empty if none). */
const char *ibm_last_cuda_error(void);

/* Create a context on CUDA device `device` (allocates reduction scratch).
 * tune_cache_path (host string, nullable): a JSON file where ibm_autotune keeps the schedules
 * it found (created on the first tuning; see ibm_autotune). */
ibm_status ibm_ctx_create(ibm_ctx **out, int32_t device, const char *tune_cache_path);
ibm_status ibm_ctx_destroy(ibm_ctx *ctx);

/* Iblanking and ghost-cell tables (paper Sec. "GPU Porting", items 1 and 2).
 * Closed meshes: classifies every cell centre (solid iff strictly inside a mesh by the
 * exact lattice parity test with half-open tie rules; a centre on the surface is fluid),
 * marks ghost cells (solid with a fluid face-neighbour), and for each ghost computes the
 * boundary intercept BI (closest surface point), the image point IP = 2 BI - GC and its
 * trilinear interpolation row.  Membranes (closed = 0): every cell is fluid; a link between
 * face-neighbours is cut when a triangle crosses it (exact lattice test, lowest crossing
 * triangle decides), and every cut link i -> j gives the ghost entry (j, side of i), side =
 * sign of orient3d of the crossing triangle and centre i; entries are ordered by cell, then
 * side; the IP's corners count only on the entry's side (exact segment tests), blocked
 * corners through the same-side entry of that cell.  nmesh may be 0 (no body).  On
 * success *out owns device memory until ibm_tables_destroy.  A closed mesh that some grid
 * column (the vertical line through cell centres (x_i, y_j)) crosses an odd number of times
 * has a hole on that line: the call returns IBM_ERR_MESH_NOT_CLOSED and *out is not set
 * (holes that no column passes through leave the classification unchanged and are not
 * reported). */
ibm_status ibm_classify(ibm_ctx *ctx, const ibm_grid *grid, const ibm_mesh *meshes,
                        int32_t nmesh, ibm_tables **out, void *stream);
ibm_status ibm_tables_destroy(ibm_tables *t);

/* Reclassify existing tables for new body positions on the same grid (a moving body, one
 * call per time step).  Same classification as ibm_classify with these meshes, written
 * into the tables' own device memory: its arrays are reused (the per-ghost arrays grow
 * when the ghost count exceeds their capacity, never shrink), and the solver work arrays
 * of every precision keep their grid-only data; their geometry-dependent parts (masks,
 * face fractions, fluid volumes, coarsest inverse, ghost rows) are recomputed by the next
 * solve, which replays its captured cycle when the ghost capacity did not change.
 * Device arrays obtained earlier from ibm_tables_export are not updated.  Synchronises
 * `stream`.  On IBM_ERR_NO_FLUID the tables hold the new (fluid-free) classification and
 * cannot be solved; other errors leave them unusable except for ibm_tables_destroy. */
ibm_status ibm_reclassify(ibm_ctx *ctx, ibm_tables *t, const ibm_mesh *meshes, int32_t nmesh,
                          void *stream);

/* Sizes of a classified grid: cells, fluid cells, ghost entries, solid cells. */
ibm_status ibm_tables_counts(const ibm_tables *t, int64_t *ncell, int64_t *nfluid,
                             int64_t *nghost, int64_t *nsolid);

/* Copy the classification out to caller-owned device arrays (any may be NULL):
 *   iblank_dev  uint8[ncell]   0 fluid, 1 solid, 3 ghost (solid | 2); membranes: all 0
 *   cell_dev    int64[nghost]  linear cell index of each ghost, ascending (membranes: of
 *                              each entry, ascending, side 0 before side 1)
 *   bi_dev      double[nghost*3], ip_dev double[nghost*3]   (x,y,z)
 *   base_dev    int32[nghost*3]  base corner (i0,j0,k0) of the IP's cell-centre box
 *   flags_dev   int32[nghost]    bit 0: nearest-neighbour fallback; bits 8-15: valid corners
 *   ref_dev     int64[nghost*8]  linear cell index of each interpolation source, -1 unused
 *                              (membranes: ncell + e refers to ghost entry e)
 *   w_dev       double[nghost*8] weights (sum 1; own weight moved to the left-hand side)
 *   scale_dev   double[nghost]   residual scale of the ghost row
 * Corner slot c = bx + 2 by + 4 bz addresses cell (i0+bx, j0+by, k0+bz). */
ibm_status ibm_tables_export(const ibm_tables *t, uint8_t *iblank_dev, int64_t *cell_dev,
                             double *bi_dev, double *ip_dev, int32_t *base_dev,
                             int32_t *flags_dev, int64_t *ref_dev, double *w_dev,
                             double *scale_dev, void *stream);

/* Membrane tables only (IBM_ERR_INVALID_ARG otherwise): copy out, to caller-owned device
 * arrays (any may be NULL), per cell uint8[ncell] cut_dev (bit d set: the link in direction
 * d = -x, +x, -y, +y, -z, +z is cut) and side_dev (bit d: the cell's side of that link,
 * 1 = positive orient3d), and per entry uint8[nghost] gside_dev.  Synchronises `stream`. */
ibm_status ibm_tables_export_membrane(const ibm_tables *t, uint8_t *cut_dev, uint8_t *side_dev,
                                      uint8_t *gside_dev, void *stream);

/* Moving-boundary Neumann datum (paper Sec. "Governing Equations and Numerical Methods": the
 * pressure condition of the projection at a moving body, dp/dn = -rho Du_b/Dt . n).  Ghost
 * row G reads  g_G - sum_k w_k v_k = kappa_G q_G, where q_G is the pressure's derivative
 * along the row's unit direction: from the ghost cell's centre GC towards its image point
 * (the body's outward normal at BI), or towards its neighbour on a nearest-neighbour
 * fallback row.  kappa_G = -|IP - GC| (fallback: -|centre - GC|), divided by 1 - w_self
 * when the row's own interpolation weight was moved to the left-hand side.  Every
 * classification (ibm_classify, ibm_reclassify) clears the datum (q = 0, a fixed body).
 *
 * ibm_set_neumann: q_dev double[nghost] (device, in ghost order) sets the data; NULL clears
 *   them.  Stream-ordered; q_dev may be released once `stream` has passed the call.
 * ibm_neumann_rigid: q from rigid-body kinematics, rho = 1: for the mesh holding each ghost's
 *   closest triangle, q = -a(BI) . n with a(x) = a0 + alpha x (x - c) + omega x (omega x
 *   (x - c)).  motions (host) double[nmesh * 12]: per mesh in classification order a0 (3),
 *   alpha (3), omega (3), c (3).  nmesh must equal the classification's mesh count (at most
 *   32; IBM_ERR_CAPACITY beyond).
 * ibm_tables_export_neumann: copy out kappa_dev double[nghost], tri_dev int32[nghost] (the
 *   closest triangle's global index, meshes concatenated in order) and d_dev double[nghost]
 *   (kappa q, 0 without data); any may be NULL.  Synchronises `stream`. */
ibm_status ibm_set_neumann(ibm_tables *t, const double *q_dev, void *stream);
ibm_status ibm_neumann_rigid(ibm_tables *t, const double *motions, int32_t nmesh, void *stream);
ibm_status ibm_tables_export_neumann(const ibm_tables *t, double *kappa_dev, int32_t *tri_dev,
                                     double *d_dev, void *stream);

/* ibm_tables_export_self_weight: copy out wself_dev double[nghost], each ghost row's own
 * interpolation weight w_s where it was moved to the left-hand side (0 otherwise; the stored
 * weights are divided by 1 - w_s).  Synchronises `stream`. */
ibm_status ibm_tables_export_self_weight(const ibm_tables *t, double *wself_dev, void *stream);

/* Advection-diffusion (Helmholtz-type) velocity solve of the fractional step with no-slip
 * ghost rows (paper Sec. "Governing Equations and Numerical Methods": the momentum equation's
 * advection-diffusion step, solved with scheduled relaxed Jacobi; Sec. "GPU Porting" item 2:
 * no-slip on the immersed surface).  One velocity component u solves
 *   fluid row i:  (1 + alpha sum_d c_{i,d}) u_i - alpha sum_d c_{i,d} v_nb = f_i
 *   ghost row G:  (1 + w_s) u_G + (1 - w_s) sum_k w_k v_k = 2 u_b,G
 * with the pressure system's coefficients c (zero across the outer walls), neighbours v_nb
 * as in poisson_solve, and the image-point rows of the tables (w_s: see
 * ibm_tables_export_self_weight); the ghost row sets the value at BI, the midpoint of the
 * ghost centre and its image point, to u_b.  alpha = dt nu / 2 for Crank-Nicolson diffusion.
 * Iteration: cycles of srj_steps Jacobi sweeps with the relaxation factors 1 / (Chebyshev
 * nodes of [1 - rho, 1 + rho]), rho = alpha S / (1 + alpha S), S the largest coefficient sum
 * of a cell, the ghost rows re-evaluated after every sweep; precisions 1 and 2 run each cycle
 * in FP32 on the correction equation inside iterative refinement.  Convergence:
 * ||S r|| / ||S b|| <= tol over fluid and ghost rows, S = alpha s_G on ghost rows (s_G the
 * row scale of the pressure system), 1 on fluid rows.
 *   f_dev    double[ncell]   right-hand side on fluid cells (others ignored); not modified.
 *   ub_dev   double[nghost]  boundary values per ghost entry in ghost order, or NULL (0).
 *   u_dev    double[ncell]   in: initial guess on fluid and ghost cells; out: u on fluid
 *                            cells, the ghost value on ghost cells, 0 on other solid cells
 *                            (membranes: every cell is fluid; entry values are internal).
 * Uses the tables' FP64 multigrid hierarchy for its layout (built on first use).  Returns
 * IBM_ERR_NOT_CONVERGED after max_cycles cycles (u = last iterate), IBM_ERR_DIVERGED if the
 * residual grows a millionfold or is not finite; IBM_ERR_INVALID_ARG for NULL arrays,
 * alpha < 0, tol <= 0 or options out of range; IBM_ERR_CAPACITY for ny or nz above 65535.  Synchronises `stream` once per cycle to read the residual. */
typedef struct {
  int32_t precision;    /* 0: FP64 cycles; 1: FP32 cycles inside FP64 refinement; 2: as 1
                           with the refinement loop (u, f, residual, update) in
                           double-FP32 pairs and error-free transformations on the FP32
                           pipe, as precision 2 of poisson_solve                      [2] */
  int32_t srj_steps;    /* Jacobi sweeps (relaxation factors) per cycle, 1..64            [8] */
  int32_t max_cycles;   /* cycles (precision 0) or refinement steps (precision 1)       [100] */
} ibm_helmholtz_opts;

void ibm_helmholtz_opts_default(ibm_helmholtz_opts *opts);
ibm_status ibm_helmholtz_solve(ibm_ctx *ctx, ibm_tables *t, double alpha, const double *f_dev,
                               const double *ub_dev, double tol, double *u_dev,
                               const ibm_helmholtz_opts *opts, ibm_solve_info *info, void *stream);

/* Measurement: nsweeps (1..4096) launches of the Helmholtz solve's fine-level Jacobi sweep
 * kernel alone (precision 0: FP64 on u; 1: FP32 on the correction), after the solve's setup
 * with f_dev and u_dev (as for ibm_helmholtz_solve; u_dev is not written), each launch
 * bracketed by CUDA events on `stream`; *kernel_ms = the mean launch duration.  Synchronises
 * `stream`. */
ibm_status ibm_helmholtz_sweeps_timed(ibm_ctx *ctx, ibm_tables *t, double alpha, int32_t precision,
                                      int32_t nsweeps, const double *f_dev, double *u_dev, void *stream,
                                      double *kernel_ms);

/* Rigid-body boundary velocity of every ghost entry: u_b = v0 + omega x (BI - c) for the mesh
 * holding the entry's closest triangle.  motions (host) double[nmesh * 9]: per mesh in
 * classification order v0 (3), omega (3), c (3); nmesh must equal the classification's mesh
 * count (at most 32; IBM_ERR_CAPACITY beyond).  ub_dev double[3][nghost] out (device),
 * component-major.  Stream-ordered. */
ibm_status ibm_boundary_velocity_rigid(ibm_tables *t, const double *motions, int32_t nmesh,
                                       double *ub_dev, void *stream);

/* Surface pressure and nodal pressure forces (paper Sec. "Force Formulations": the external
 * force on a structure node is one third of the traction times the area, summed over the
 * node's triangles; here the pressure part, -dp n A).  The shear part is not computed.
 *
 * Per triangle t of the classified meshes (N = (v1 - v0) x (v2 - v0), n = N / |N|, centroid
 * c): the pressure on side s = +1 (the side n points to) and s = -1 is read at the probe
 * X = c + s d n, d = 1.5 x the diagonal of the cell holding c, by trilinear interpolation of
 * the cell pressures that hold fluid on side s (closed bodies: fluid cells; membranes: cells
 * whose centre lies strictly on side s of the triangle's plane), renormalised, minus s d q
 * with q = dp/dn at c.  A side whose usable weights sum below 1e-3 reads 0 and sets flag bit
 * s (bit 0 for +, bit 1 for -); a zero-area triangle sets bit 2 and has no force.  Closed
 * bodies have no fluid on the - side (outward normals): p_- = 0.  The triangle's force
 * f = -(p_+ - p_-) N / 2 goes in equal thirds to its three nodes; node sums run over
 * triangles in ascending order, so results are deterministic.
 *   meshes, nmesh   the meshes of the last classification of t, same order and triangle
 *                   counts (vertex positions may have moved since, topology not), host.
 *                   Vertices and triangles are numbered mesh after mesh.
 *   p_dev           double[ncell] cell pressures (poisson_solve's output), device.
 *   q_tri_dev       double[ntri] dp/dn per triangle (device), or NULL;
 *   motions         or rigid kinematics per mesh as for ibm_neumann_rigid (host), q = -a(c).n;
 *                   at most one of the two; neither means q = 0 (a fixed body).
 *   p_side_dev      double[ntri][2] (p_+, p_-) out, device, or NULL.
 *   flags_dev       uint8[ntri] out, device, or NULL.
 *   f_node_dev      double[nvert][3] nodal forces out, device.
 * Stream-ordered; the host arrays may be released when the call returns.  The tables keep a
 * device working set that grows with the mesh (reallocation synchronises `stream`).
 * Errors: IBM_ERR_INVALID_ARG for NULL p_dev / f_node_dev, both q_tri_dev and motions, or
 * meshes that do not match the classification; IBM_ERR_CAPACITY beyond 2^31 - 2 vertices
 * or 32 meshes with motions. */
ibm_status ibm_surface_forces(ibm_tables *t, const ibm_mesh *meshes, int32_t nmesh, const double *p_dev,
                              const double *q_tri_dev, const double *motions, double *p_side_dev,
                              uint8_t *flags_dev, double *f_node_dev, void *stream);

void ibm_solve_opts_default(ibm_solve_opts *opts);

/* Pressure Poisson solve (paper Sec. "Governing Equations and Numerical Methods") on a
 * classified grid, by geometric-multigrid V-cycles with red-black Gauss-Seidel smoothing
 * and the ghost-cell image-point rows updated after every sweep.
 *
 * Solves, for p on fluid cells and g on ghost cells and the scalar lambda,
 *   fluid row i: sum_d c_{i,d} (v_nb - p_i) = b_i - lambda   (v_nb: p, or g at a ghost)
 *   ghost row G: g_G - sum_k w_k v_k = kappa_G q_G           (dp/dn at BI; 0 unless a
 *                                                              datum is set, see above)
 * with c_{i,+x} = 1/(dx_i (x_{i+1} - x_i)) etc., zero across walls, and returns p gauged
 * to zero volume-weighted mean over fluid cells.  Convergence: the relative projected
 * residual ||S P r|| / ||S P b|| <= tol (P removes the volume-weighted fluid mean of r,
 * S scales ghost rows by the sum of the coefficients that reference them).
 *   rhs_dev  double[ncell]  b on fluid cells (other cells ignored); not modified.
 *   p_dev    double[ncell]  in: initial guess on fluid and ghost cells; out: p on fluid
 *                           cells, g on ghost cells, 0 on other solid cells.
 * Returns IBM_ERR_NOT_CONVERGED (p = last iterate) if max_cycles is reached;
 * IBM_ERR_DIVERGED before any cycle when rhs or the initial guess holds a NaN or an Inf on
 * a fluid row (or in a value a ghost row reads), and during the iteration when the residual
 * becomes non-finite or grows a millionfold. */
ibm_status poisson_solve(ibm_ctx *ctx, const ibm_tables *t, const double *rhs_dev, double tol,
                         double *p_dev, const ibm_solve_opts *opts, ibm_solve_info *info,
                         void *stream);

/* Batched pressure Poisson solves: n independent problems (each its own classified grid, of
 * any size; closed bodies or membranes; every precision mode and Krylov setting) advanced
 * together, each with its own device scalars and partial sums, with one read-back per step
 * for all of them.  Schedule (opts->batch_schedule): lockstep, where each V-cycle stage and
 * each kernel of the outer step is one launch over every problem still iterating (mixed
 * precision, closed bodies, no Krylov acceleration, FP32 coarse storage); or each problem's
 * step captured once as a CUDA graph, the graphs of the problems still iterating launched on
 * a small pool of streams owned by the context (forked from and joined back into `stream`).
 * Either way each problem gets the bits of its own poisson_solve.  Same equations, options
 * and outputs as poisson_solve, per problem:
 *   tables[p], rhs_dev[p], p_dev[p] as in poisson_solve (p_dev[p] is in/out);
 *   infos (optional, n entries) receives each problem's report; ms_total is the batch's.
 * The tables must be distinct (each problem owns its work arrays); the context's batch
 * buffers grow to the largest n seen.  Returns IBM_ERR_NOT_CONVERGED if some problem did not
 * reach tol in max_cycles (its last iterate is returned). */
ibm_status poisson_solve_batched(ibm_ctx *ctx, int32_t n, const ibm_tables *const *tables,
                                 const double *const *rhs_dev, double tol, double *const *p_dev,
                                 const ibm_solve_opts *opts, ibm_solve_info *infos, void *stream);

/* Autotuner: times complete solves of the given problem (rhs_dev, tol) with candidate
 * smoother schedules -- over-relaxation 1.2/1.3/1.4, sweeps (1,1)/(2,1)/(2,2) and, for
 * precision 1 or 2, 1/2/3 FP32 V-cycles per refinement step; Krylov acceleration none or
 * GCR(2), and GCR(8) on membrane tables -- then, for the fastest, the z extent of the fused
 * sweep's tiles (sweep_chunk: the cost model's choice, 128, 64, 32 planes), and returns the
 * fastest in *best (its time in *best_ms, optional).  p_work_dev (double[ncell], device) is overwritten.
 * Use the result for poisson_solve / poisson_solve_batched of similar problems.
 * With a tune cache (ibm_ctx_create), the cache is read first: an entry for the same grid
 * (cell counts and a hash of the face coordinates), precision and body kind (closed or
 * membrane) is returned as it is, with its recorded time, and nothing is launched.  Otherwise
 * the search runs and its result is added to the file (one JSON object per line, rewritten
 * through a temporary file and a rename); IBM_ERR_INVALID_ARG if the file cannot be
 * written (*best is filled all the same). */
ibm_status ibm_autotune(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, const double *rhs_dev,
                        double *p_work_dev, double tol, ibm_solve_opts *best, double *best_ms,
                        void *stream);

/* Measurement: run `nsweeps` smoother sweeps (red, black, ghost rows) on the finest level
 * of the hierarchy of the given precision, exactly as inside a V-cycle, on whatever the
 * solver's work arrays hold (call after a poisson_solve of that precision).  No result;
 * used to time the smoother in isolation.  Asynchronous on `stream`. */
ibm_status ibm_smoother_sweeps(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, int32_t nsweeps,
                               void *stream);

/* Measurement: as ibm_smoother_sweeps (nsweeps >= 1), with CUDA events recorded on `stream`
 * immediately before and after each sweep's kernel(s) -- the fused sweep in FP32, the two
 * colour passes in FP64 -- so the ghost-row refresh between sweeps is excluded.  Waits for
 * the stream and returns the mean duration of one sweep's kernels in *kernel_ms.  The paper
 * has no counterpart; it serves roofline measurements. */
ibm_status ibm_smoother_sweeps_timed(ibm_ctx *ctx, const ibm_tables *t, int32_t precision,
                                     int32_t nsweeps, void *stream, double *kernel_ms);

/* Test hook: the finest level's smoother applied to caller data.  e_dev and r_dev
 * (double[ncell], [k][j][i], device, read only) are loaded into the finest level of the
 * hierarchy of the given precision (built when missing), rounded to its type (FP32 for
 * precision 1 and 2), and nsweeps sweeps with over-relaxation omega run exactly as inside a
 * V-cycle: each fluid cell of one colour, red ((i + j + k) even) then black, takes
 *   e_i += omega ((A e)_i - (r_i - mu)) / D_i,   D_i = -A_ii
 * (A the fluid rows of the pressure operator, Sec. "Governing Equations and Numerical
 * Methods"; a row's neighbours include ghost values), the cut cells of membranes follow, and
 * the ghost rows are refreshed, Jacobi among ghosts: e_G = sum_k w_k e_k + r_G.  e_out_dev
 * (double[ncell], device, caller-owned) receives the finest level's e; other cells keep
 * their loaded values.  The solver's work arrays are overwritten (each solve initialises
 * them again).  Waits for the stream.  IBM_ERR_INVALID_ARG for a null pointer, omega outside
 * (0, 2), nsweeps < 0 or a non-finite mu; IBM_ERR_TIMEOUT if a bounded wait of the fused
 * sweep gave up.  The paper has no counterpart: it checks the smoother against a direct
 * restatement of Gauss-Seidel. */
ibm_status ibm_smoother_apply(ibm_ctx *ctx, const ibm_tables *t, int32_t precision, int32_t nsweeps,
                              double omega, const double *e_dev, const double *r_dev, double mu,
                              double *e_out_dev, void *stream);

/* Measurement: the device's FP64 fused multiply-add rate (FMAs per second, *dfma_per_s),
 * from a kernel of independent dependent chains filling every SM, best of three timed
 * launches after one warm-up.  The paper has no counterpart; it is the roofline denominator
 * of the FP64 smoother, whose work is FP64 arithmetic rather than memory traffic.  Waits for
 * the stream. */
ibm_status ibm_measure_fp64_rate(ibm_ctx *ctx, double *dfma_per_s, void *stream);

/* Number of CUDA kernels this context has launched so far (all calls). */
ibm_status ibm_ctx_launch_count(const ibm_ctx *ctx, int64_t *count);

/* Test hook (no counterpart in the paper): the number of tries of the first bounded
 * shared-memory wait of every item of the fused FP32 sweep.  0 makes that wait give up at
 * once: the sweep sets the context's error flag, waits (with the normal bound) for every copy
 * it has in flight, and returns, so the next synchronising call (poisson_solve) reports
 * IBM_ERR_TIMEOUT and the context stays usable.  tries < 0 restores the normal limit.
 * Solves captured as CUDA graphs are recaptured when the setting changes. */
ibm_status ibm_ctx_set_sweep_wait_limit(ibm_ctx *ctx, int32_t tries);

/* Relative projected residual of a pressure field, with NO device allocation.  The paper
 * has no counterpart: this exists for callers that cannot allocate device memory after
 * start-up -- e.g. a flow solver that owns a fixed device arena, where cudaMalloc/cudaFree
 * would synchronise the whole device (breaking compute/communication overlap) or could
 * fail in the middle of a time-step loop.  It needs no context and no tables object: the
 * caller passes the grid (host faces), the classification of CLOSED bodies as exported by
 * ibm_tables_export (iblank, ghost cells, interpolation sources, weights, row scales), the
 * optional ghost-row data d = kappa q as ibm_tables_export_neumann writes it (NULL: zero),
 * the right-hand side and the pressure (user layout, ghost values at ghost cells, as
 * poisson_solve returns it), all on the current CUDA device.
 *   result (host, 3 doubles): ||S P r|| / ||S P b||, ||S P r||, ||S P b||, with the same
 *   definitions as poisson_solve: fluid rows r = b - A p, the volume-weighted fluid mean
 *   removed (P), ghost rows r_G = d_G - (g_G - sum w v) scaled by the row scale (S).  The
 *   means are taken in a first pass and the squared deviations in a second, so a right-hand
 *   side with a large fluid mean does not cancel the result away.
 * Membrane tables are rejected with IBM_ERR_INVALID_ARG: any ghost row whose cell is not a
 * closed body's ghost cell (iblank 3), or whose cell or source index is outside the
 * nx*ny*nz cells, sets an error word in the scratch; p is never read at such an index.
 * Scratch: one fixed device array of about 0.2 MB inside this library, held by every GPU
 * that loads it until the process exits.  Grids with more than 2048 cells along any axis
 * are rejected with IBM_ERR_CAPACITY.  The first call on a device (and the first after a
 * new CUDA context replaces the device's old one) looks up that array's device address:
 * make that first call before any stream capture.  Every call reuses the same array:
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Synchronises `stream` before returning. */
ibm_status ibm_residual_norm_noalloc(const ibm_grid *grid, const uint8_t *iblank_dev, int64_t nghost,
                                     const int64_t *ghost_cell_dev, const int64_t *ghost_ref_dev,
                                     const double *ghost_w_dev, const double *ghost_scale_dev,
                                     const double *ghost_d_dev, const double *rhs_dev, const double *p_dev,
                                     double *result, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IBM_POISSON_H */
