/*
 * dg_atmo.h -- C ABI of a GB300 (sm_103a) matrix-free DG solver for the
 * compressible Euler equations on 2:1 non-conforming terrain-following meshes,
 * advanced in time by a second-order IMEX Runge-Kutta scheme.
 *
 * Method (arXiv 2408.08129):
 *   Eq. (1), Sec. 2  compressible Euler with gravity, ideal gas, g = 9.81, R = 287;
 *   Sec. 2           DG on non-conforming meshes (no hanging nodes), IMEX-RK2 with
 *                    continuity explicit and momentum/energy coupled implicitly;
 *   Sec. 3.1         orography, constant-N background atmosphere, wall bottom;
 *   Sec. 3.2         matrix-free operator action; pressure fixed-point loop with
 *                    GMRES for the non-symmetric linear system.
 * Discretisation details the paper leaves to earlier work are readings:
 * collocated Gauss-Lobatto-Legendre nodal basis, Rusanov flux (advective
 * speed only for the IMEX-explicit terms), subface evaluation on 2:1 faces,
 * strong-form gradient / weak-form divergence with centred traces for the
 * pressure Helmholtz problem, ARK2(2,3,2) tableau.
 *
 * Conventions shared by every call:
 *  - Return value: a dg_status (0 = DG_OK, negative = error).  No call throws,
 *    aborts or exits.  dg_last_error() gives a message for the calling thread.
 *  - Device arrays are caller-owned CUDA device pointers (for example the
 *    data_ptr() of a contiguous torch tensor), aligned to 16 bytes, laid out
 *    structure-of-arrays: variable-major, then cell, then node inside the cell
 *    ([var][cell][node]); a node's index inside its cell is
 *    i0 + n*i1 (+ n*n*i2), n = degree+1, axis 0 = x, the last axis vertical.
 *    Variables: rho, momentum components (vertical last), rho*E.
 *  - Host arrays are plain host pointers, only read during the call.
 *  - Every device call is enqueued on the given CUDA stream (NULL = legacy
 *    default stream) and returns without waiting, unless documented.  Calls on
 *    one mesh share that mesh's scratch buffers, so they must be ordered on one
 *    stream (or otherwise serialised by the caller).
 *  - Precision: DG_FP64 arrays are double; DG_FP32 arrays are float and hold
 *    the PERTURBATION about the hydrostatic background for state inputs
 *    (rho - rho_bar, momentum, rho*E - p_bar/(gamma-1)); the FP64 background is
 *    added inside the kernels.
 */
#ifndef DG_ATMO_H
#define DG_ATMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;
typedef struct dg_mesh dg_mesh;
typedef struct dg_state dg_state;

typedef enum {
  DG_OK = 0,
  DG_EINVAL = -1,      /* bad argument                                       */
  DG_ENOMEM = -2,      /* device or host allocation failed                   */
  DG_ECUDA = -3,       /* a CUDA runtime call failed (message has the code)  */
  DG_ENOTCONV = -4,    /* Krylov / fixed-point loop did not converge         */
  DG_ENONFINITE = -5,  /* NaN or Inf detected in a result                    */
  DG_EUNBALANCED = -6, /* mesh is not 2:1 balanced or not watertight         */
  DG_EBUDGET = -7,     /* request exceeds the serving memory budget          */
  DG_ETIMEOUT = -8     /* a bounded wait ran out                             */
} dg_status;

typedef enum { DG_FP64 = 0, DG_FP32 = 1 } dg_precision;
typedef enum {
  DG_KRYLOV_AUTO = -1,
  DG_KRYLOV_GMRES = 0,
  DG_KRYLOV_CG = 1,
  DG_KRYLOV_GMRES_CGS2 = 2,
  DG_KRYLOV_CHEBYSHEV = 3
} dg_krylov;
typedef enum { DG_TERMS_FULL = 0, DG_TERMS_IMEX_EXPLICIT = 1 } dg_terms;
typedef enum { DG_HILL_NONE = 0, DG_HILL_GAUSS = 1, DG_HILL_BELL = 2, DG_HILL_PARABOLA = 3 } dg_hill_kind;
typedef enum { DG_ATM_NONE = 0, DG_ATM_ISOTHERMAL = 1, DG_ATM_STRATIFIED = 2 } dg_atm_kind;
typedef enum { DG_INIT_REST = 0, DG_INIT_BUBBLE = 1, DG_INIT_INFLOW = 2 } dg_init_kind;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  *out receives the handle. */
int dg_ctx_create(int device, dg_ctx** out);
int dg_ctx_destroy(dg_ctx* ctx);
/* Message of the last non-OK status returned on the calling thread ("" if none). */
const char* dg_last_error(void);
/* Library version string. */
const char* dg_version(void);

/* Optional timing of the operator classes with CUDA events (the per-block
 * time breakdown of Sec. 3.2, Fig. 5).  Categories: */
typedef enum {
  DG_PROF_EXPLICIT = 0,  /* explicit DG operator applies                    */
  DG_PROF_HELMHOLTZ = 1, /* Helmholtz mat-vecs inside GMRES                 */
  DG_PROF_GRAD = 2,      /* DG gradients                                    */
  DG_PROF_DIV = 3,       /* DG divergences                                  */
  DG_PROF_KRYLOV = 4,    /* GMRES orthogonalisation and updates (BLAS-1)    */
  DG_PROF_GMRES = 5,     /* whole fused GMRES solves (persistent kernel)    */
  DG_PROF_STEP = 6,      /* whole IMEX-RK2 steps                            */
  DG_PROF_N = 8
} dg_prof_category;
/* Turn event timing on (1) or off (0) for every call made with this context.
 * Events are recorded on the stream of each call; the overhead is one event
 * pair per operator launch.  on = 2 also turns on the clocks inside the
 * persistent solves (dg_profile_read_gmres_phases, dg_profile_read_cta_passes),
 * which cost a little time of their own. */
int dg_profile_enable(dg_ctx* ctx, int on);
/* Synchronise the device, then copy the accumulated milliseconds and call
 * counts per category into ms[DG_PROF_N] and counts[DG_PROF_N] (host arrays). */
int dg_profile_read(dg_ctx* ctx, double* ms, long long* counts);
int dg_profile_reset(dg_ctx* ctx);
/* Nanoseconds spent in each phase of the fused GMRES solves while profiling
 * was on at level 2, as seen by block 0 (a phase that ends at a grid barrier includes the
 * wait for the slowest block), into ns[16]: 1 gradient (one cell pass with its
 * face terms), 3 divergence (the same), 4 wait at the barrier after the
 * Gram-Schmidt dots, 5 wait at the barrier after the basis update, 6 second
 * Gram-Schmidt pass (classical form), 7 FP64 residual, 8 solution update,
 * 9 Gram-Schmidt dots (work), 10 sums of the block partials, 11 Hessenberg
 * column and Givens rotation, 12 update coefficients, 13 basis update (work);
 * ns[14] = second passes, ns[15] = GMRES iterations.  Synchronises the device. */
int dg_profile_read_gmres_phases(dg_ctx* ctx, double* ns);
/* Per-CTA clocks of the Chebyshev solves while profiling was on at level 2: for CTA i <
 * max_ctas (at most 512) of the persistent launch, the nanoseconds of its own
 * gradient passes (grad_ns[i]) and divergence passes (div_ns[i]), summed over
 * the steps and solves, each from the end of the CTA's wait for the grid
 * barrier inside the pass to the pass's end (the barriers' own time is not
 * counted); coarse[i] = 1 if its cell batch holds the coarse side of a 2:1
 * face.  Host arrays.  Synchronises the device. */
int dg_profile_read_cta_passes(dg_ctx* ctx, double* grad_ns, double* div_ns, int* coarse, int max_ctas);
/* Self-test of the library's own FP64 math on the device (no counterpart in
 * the paper): op 0 writes y[i] = 1/sqrt(x[i]) as computed by the Newton
 * iteration the solvers use (FP32 seed, two Newton steps), for device arrays
 * x, y of n doubles, x[i] > 0 and within the FP32 range.  Enqueued on stream.
 * DG_EINVAL for another op or null arrays. */
int dg_math_selftest(int op, const double* x, double* y, int64_t n, void* stream);
/* Test hook for the bounded barrier of batched launches (dg_batch_step and
 * batch plans captured afterwards; no counterpart in the paper).  Every wait
 * at a member's barrier inside a batched launch gives up after
 * barrier_limit_s seconds (2 s by default; accepted range 1e-3 .. 10), raises
 * the launch's error flag and lets every later barrier of the launch return
 * at once, so the step returns DG_ETIMEOUT instead of hanging.  With
 * missing_cta_member >= 0, the member at that position in each batched
 * launch's member list is told it has one CTA more than the launch gives it,
 * so its first barrier can never complete and its wait runs out (nothing
 * faults: the kernel only returns early); -1 turns this off.  Host-side
 * setting of the context, read when a batched launch is enqueued. */
int dg_batch_barrier_test(dg_ctx* ctx, double barrier_limit_s, int missing_cta_member);
/* Arithmetic-throughput probe (no counterpart in the paper; the ALU peaks the
 * operator kernels are reported against): enqueue on `stream` one kernel of
 * `blocks` CTAs x 256 threads, each thread running 16 independent fused
 * multiply-add chains for `iters` steps in DG_FP64 or DG_FP32; `out` is a
 * device array of blocks*256 elements of that type (receives the chains'
 * sums).  *flops receives the floating-point operations the kernel performs
 * (2 per FMA); the caller times the launch, e.g. with CUDA events. */
int dg_peak_fma(int precision, int64_t iters, int blocks, void* out, void* stream, double* flops);
/* Number of CUDA kernels the library has launched through this context so far. */
int dg_launch_count(const dg_ctx* ctx, long long* out);

/* ---------------------------------------------------------------- mesh
 * Sec. 3.1 meshes: a forest of quad/oct-trees over a base grid of
 * base[0] x base[1] (x base[2]) cells covering [0, extent[a]] per axis, each
 * leaf refined 0..7 times, neighbours differing by at most one level (2:1).
 * The physical mesh is the terrain-following map z = zeta + h(x,y)(1 - zeta/H)
 * (H = extent of the vertical axis), isoparametric of degree `degree` on base
 * cells; refined cells take their nodes from their base cell's polynomial.
 */
typedef struct {
  int dim;                /* 2 (x-z) or 3 (x-y-z)                               */
  int degree;             /* polynomial degree r, 1..5; n = r+1 GLL nodes/axis  */
  int64_t n_cells;        /* number of leaves                                   */
  const uint8_t* level;   /* host [n_cells]: refinement level of each leaf      */
  const int32_t* ijk;     /* host [n_cells*dim]: integer coords at own level    */
  int base[3];            /* base grid cells per axis                           */
  double extent[3];       /* domain length per axis (m)                         */
  int periodic[3];        /* 1 = periodic axis, 0 = slip walls at both ends     */
  int hill_kind;          /* dg_hill_kind: orography h(x[,y]) (Sec. 3.1)        */
  double hill_hc;         /* hill height (m)                                    */
  double hill_half_width; /* Gaussian: h(half_width) = hc/2; bell: a_c          */
  double hill_xc, hill_yc;/* hill centre (m)                                    */
  int atm_kind;           /* dg_atm_kind: hydrostatic background (Sec. 3.1)     */
  double atm_T;           /* isothermal T0, or stratified T_ref (K)             */
  double atm_N;           /* buoyancy frequency of the stratified case (1/s)    */
  double atm_p_ref;       /* surface pressure (Pa)                              */
  double gravity;         /* g (9.81 in Eq. (1)); 0 turns gravity off           */
  /* Rayleigh damping layer below the top boundary (absorbs upward-going waves;
   * the paper's non-reflecting boundaries are described elsewhere, this is a
   * reading): in the top sponge_depth metres of physical height the time step
   * adds -tau(z) (U - U_ref) to the explicit tendency, with
   * tau(z) = sponge_rate sin^2(pi/2 (z - z_d)/sponge_depth) for z > z_d =
   * H - sponge_depth (0 below) and U_ref the hydrostatic background with the
   * uniform x-velocity sponge_u0 (rho_bar, rho_bar u0, 0, p_bar/(gamma-1) +
   * rho_bar u0^2/2).  sponge_depth = 0 turns it off.  Explicit treatment:
   * keep sponge_rate dt <= 1. */
  double sponge_depth;    /* (m), 0..H                                          */
  double sponge_rate;     /* tau at the top (1/s), >= 0                         */
  double sponge_u0;       /* reference x-velocity (m/s)                         */
  /* Lateral absorbing layers (the lateral boundaries of the paper's runs are
   * non-reflecting too; this is the same reading as the top layer): within
   * sponge_lateral_width metres of a lateral domain boundary (x = 0, x = Lx,
   * and in 3D y = 0, y = Ly), tau_lat = sponge_lateral_rate sin^2(pi/2 (w - d)/w),
   * d the distance to the nearest of them, w the width; a node is damped at
   * max(tau_top, tau_lat) towards the same U_ref.  Width 0 turns it off. */
  double sponge_lateral_width; /* (m), 0 .. half the smallest lateral extent    */
  double sponge_lateral_rate;  /* tau at the lateral boundaries (1/s), >= 0     */
  /* Optional caller-built geometry and topology (for meshes generated
   * elsewhere, as the paper's are).  Each may be NULL / 0: then it is built
   * from the tree and the terrain map above.  Host arrays, read during the
   * call only, in the layouts dg_mesh_get_coords / dg_mesh_get_faces export:
   *  - node_xyz [dim][n_cells][nodes_per_cell]: the nodal physical
   *    coordinates (GLL nodes of each cell, node index as above).  Checked:
   *    J > 0 at every node (DG_EINVAL), and watertight faces -- the two sides
   *    of a conforming face, and a fine face against its coarse face's
   *    polynomial, agree to 1e-9 of the domain size (DG_EUNBALANCED).
   *  - the three face tables, given together (all or none): conforming
   *    [n_conforming*4] (minus cell, minus local face, plus cell, plus local
   *    face), subfaces [n_subfaces*4] (fine cell, fine local face, coarse
   *    cell, subface position), walls [n_walls*2] (cell, local face).
   *    Checked against level/ijk (DG_EUNBALANCED): every cell face listed
   *    exactly once, opposite local faces, neighbours adjacent (periodic axes
   *    wrap) at the same level on conforming faces and one level apart on 2:1
   *    faces (position s matching), walls on non-periodic domain boundaries,
   *    the 2^(dim-1) subfaces of each coarse face complete. */
  const double* node_xyz;
  int64_t n_conforming;
  const int32_t* conforming;
  int64_t n_subfaces;
  const int32_t* subfaces;
  int64_t n_walls;
  const int32_t* walls;
} dg_mesh_desc;

typedef struct {
  int dim, degree, n_vars, nodes_per_cell;
  int64_t n_cells, n_nodes, n_dof;      /* n_dof = n_vars * n_nodes           */
  int64_t n_conforming, n_subfaces, n_walls;
  int max_level;
  double min_edge;                      /* smallest computational cell edge   */
  size_t device_bytes;                  /* device memory held by the mesh     */
  int solver_form[2];                   /* autotuned Helmholtz solver for FP64 */
                                        /* [0] and FP32 [1]: 0 GMRES one launch */
                                        /* per kernel, 1 GMRES persistent, 2    */
                                        /* Chebyshev persistent; -1 not tuned   */
  float solver_ms[2][3];                /* the timed solves [precision][form]   */
                                        /* (0 where a form was not timed)       */
  int n_batches[2];                     /* cell batches of the implicit passes: */
                                        /* [0] CPB consecutive cells each, [1]  */
                                        /* balanced (0 if not built)            */
  int solver_partition[2];              /* autotuned partition per precision    */
  float solver_ms_balanced[2][3];       /* the timed solves on partition 1      */
} dg_mesh_info;

/* Build connectivity (conforming faces, 2:1 subfaces, walls), check the 2:1
 * balance (DG_EUNBALANCED) and J > 0 (DG_EINVAL), compute the geometry and
 * background on the host in FP64 and upload everything to the device.  The
 * descriptor's arrays are copied; the caller may free them afterwards. */
int dg_mesh_create(dg_ctx* ctx, const dg_mesh_desc* desc, dg_mesh** out);
int dg_mesh_destroy(dg_mesh* mesh);
int dg_mesh_get_info(const dg_mesh* mesh, dg_mesh_info* info);
/* Choose the cell partition of the implicit cell passes (gradient,
 * divergence, Helmholtz, the persistent solves): 0 = batches of CPB
 * consecutive cells (CPB = 256 / nodes per cell), 1 = balanced for the
 * persistent solves (two CTAs per SM): on meshes with no more uniform batches
 * than CTAs, cost-balanced batches of at most CPB consecutive cells, one per
 * CTA, cut so that the largest batch's work (nodes plus 2:1 face points) is as
 * small as the greedy cut allows; on larger meshes, the uniform batches in an
 * order that gives every CTA about the same work.  The operators' values do
 * not depend on it (each node's
 * arithmetic is the same); only the launch shapes do.  Steps use the
 * partition chosen last, here or by the autotuner: the first step with
 * krylov = DG_KRYLOV_AUTO times both (dg_mesh_info.solver_partition).
 * DG_EINVAL if partition k was not built. */
int dg_mesh_set_partition(dg_mesh* mesh, int k);
/* Host copies of the face tables, for inspection.  Each pointer may be NULL.
 * conforming [n_conforming*4]: minus cell, minus local face, plus cell, plus
 *   local face (local face = 2*axis + side, side 1 = upper end of the axis);
 * subfaces   [n_subfaces*4]: fine cell, fine local face, coarse cell, packed
 *   subface position s = s_t1 + 2 s_t2 over the face's tangential axes;
 * walls      [n_walls*2]: cell, local face. */
int dg_mesh_get_faces(const dg_mesh* mesh, int32_t* conforming, int32_t* subfaces, int32_t* walls);
/* Host copy of the nodal physical coordinates, [dim][n_cells][nodes_per_cell]. */
int dg_mesh_get_coords(const dg_mesh* mesh, double* xyz);
/* Write the hydrostatic background state U_bg (FP64, [n_vars][cells][nodes])
 * into the device array Ubg. */
int dg_background(dg_ctx* ctx, const dg_mesh* mesh, double* Ubg, void* stream);
/* Initial state on the device (FP64, full variables): rest, the warm bubble
 * (params: amp K, radius m, xc, zc[, yc] m; Delta theta = amp cos^2(pi r/(2R)),
 * at constant pressure) or a uniform inflow (params: u0 m/s). */
int dg_init_state(dg_ctx* ctx, const dg_mesh* mesh, int kind, const double* params, int n_params,
                  double* U, void* stream);

/* ---------------------------------------------------------------- operators */

/* Explicit DG operator (Eq. (1) discretised, Sec. 2): R = M^-1 [volume - faces] + S.
 * terms = DG_TERMS_FULL: all of Eq. (1), Rusanov with |u.n| + c.
 * terms = DG_TERMS_IMEX_EXPLICIT: the terms the IMEX split keeps explicit
 *   (div(rho u), div(rho u u), div(k rho u), energy source -g rho w),
 *   Rusanov with |u.n|.
 * U, R: device [n_vars][cells][nodes]; FP64: U full state; FP32: U perturbation. */
int dg_apply_explicit(dg_ctx* ctx, const dg_mesh* mesh, const void* U, void* R, int precision, int terms,
                      void* stream);
/* Nodal gradient grad_h p = M^-1 G p (strong form, centred traces, p- on
 * walls), optionally multiplied node by node by h (h may be NULL).
 * p: [cells][nodes]; g: [dim][cells][nodes]. */
int dg_apply_grad(dg_ctx* ctx, const dg_mesh* mesh, const void* p, const void* h, void* g, int precision,
                  void* stream);
/* Nodal divergence div_h f = M^-1 D f (weak form, centred traces, zero normal
 * flux on walls).  f: [dim][cells][nodes]; out: [cells][nodes]. */
int dg_apply_div(dg_ctx* ctx, const dg_mesh* mesh, const void* f, void* out, int precision, void* stream);
/* Pressure Helmholtz operator of the implicit stage (Sec. 3.2 linear system):
 *   Ap = p/(gamma-1) - alpha div_h(h grad_h p),  alpha = (a_ii dt)^2.
 * h, p, Ap: [cells][nodes].  M*A is symmetric positive definite; A is not
 * symmetric, hence GMRES. */
int dg_apply_implicit(dg_ctx* ctx, const dg_mesh* mesh, const void* h, const void* p, void* Ap, double alpha,
                      int precision, void* stream);
/* The Helmholtz operator of dg_apply_implicit, for callers that cannot
 * allocate device memory (no cudaMalloc, no allocating library routine):
 * same arguments and result, bit for bit, but the one scratch buffer the
 * operator needs (the h-scaled gradient between its two launches) comes from
 * a fixed 4 MiB array compiled into the library, held by every GPU that loads
 * the library until the process exits.  The paper has no counterpart; this
 * is a deployment aid.
 *  - Meshes whose scratch, dim*n_nodes elements (8 bytes each for DG_FP64, 4
 *    for DG_FP32), exceeds 4 MiB are rejected with DG_EINVAL and a message
 *    giving the bytes needed.
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.  Calls
 *    outside a capture look the address up again (a device reset reloads the
 *    library's module and moves the array); calls during a capture use the
 *    address found before it.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; each call writes every scratch element before reading it, so no
 *    clearing is needed.  Calls whose executions overlap on the GPU (other
 *    streams, other threads) race on the array: serialise them. */
int dg_apply_implicit_noalloc(dg_ctx* ctx, const dg_mesh* mesh, const void* h, const void* p, void* Ap,
                              double alpha, int precision, void* stream);
/* Total mass and total energy, sum over nodes of w J rho and w J rho E, in
 * FP64 with a fixed reduction order (bitwise reproducible).  U: FP64 full
 * state on the device; out: 2 doubles on the device. */
int dg_conservation(dg_ctx* ctx, const dg_mesh* mesh, const double* U, double* out, void* stream);

/* ---------------------------------------------------------------- time stepping */

typedef struct {
  int picard;          /* fixed-point iterations per implicit stage (3)          */
  int restart;         /* GMRES restart length m (30, at most 64)                */
  int max_iters;       /* GMRES iteration cap per solve (2000)                   */
  double tol;          /* relative residual target ||b - A x|| / ||b|| (1e-12)   */
  int precision;       /* DG_FP64, or DG_FP32 = FP32 applies + inner GMRES      */
                       /*   inside FP64 iterative refinement                    */
  double inner_tol;    /* DG_FP32: relative tolerance of each inner solve (1e-6) */
  int max_refine;      /* DG_FP32: outer refinement steps cap (20)              */
  int fused;           /* 1: each GMRES solve is one persistent cooperative     */
                       /*    kernel; 0: one launch per Krylov kernel; -1       */
                       /*    (default): autotuned per mesh and precision by     */
                       /*    timing both forms on the first solve               */
  int krylov;          /* DG_KRYLOV_AUTO (default): the first solve of a mesh  */
                       /*    and precision is timed as GMRES (both forms) and   */
                       /*    as Chebyshev, and the fastest is kept; in batched  */
                       /*    steps (no timing) the mesh's tuned persistent form */
                       /*    is used, else Chebyshev.                           */
                       /*  DG_KRYLOV_GMRES (Sec. 3.2): persistent form with one */
                       /*    reduction per Arnoldi step (second Gram-Schmidt    */
                       /*    pass delayed into the next step); with fused = -1 */
                       /*    the persistent and one-launch-per-kernel forms are */
                       /*    timed and the faster kept.                         */
                       /*  DG_KRYLOV_GMRES_CGS2: classical Gram-Schmidt twice   */
                       /*    per step (two or three reductions).                */
                       /*  DG_KRYLOV_CG: conjugate gradients in the w J inner   */
                       /*    product, in which the Helmholtz operator is        */
                       /*    self-adjoint and positive (persistent form only).  */
                       /*  DG_KRYLOV_CHEBYSHEV: Chebyshev iteration on the      */
                       /*    spectral interval [1/(gamma-1), lmax], lmax from   */
                       /*    power iteration on the first solve, kept per state */
                       /*    (persistent form only; no inner products, two grid */
                       /*    barriers per step; falls back to GMRES if the      */
                       /*    residual grows).                                   */
                       /*  The one-launch-per-kernel form (fused = 0) runs      */
                       /*  GMRES with classical Gram-Schmidt twice.             */
} dg_solver_opts;

typedef struct {
  int gmres_iters;     /* total inner GMRES iterations in the step              */
  int solves;          /* linear solves (stages x Picard iterations)            */
  int refine_steps;    /* FP64 outer corrections (DG_FP32 only)                 */
  double max_rel_residual; /* worst final FP64 relative residual of the solves  */
} dg_step_stats;

/* Fill opts with the defaults listed above. */
void dg_solver_opts_default(dg_solver_opts* opts);

/* Device-resident solution and workspaces for one mesh (library-owned). */
int dg_state_create(dg_ctx* ctx, const dg_mesh* mesh, const dg_solver_opts* opts, dg_state** out);
int dg_state_destroy(dg_state* state);
/* Device pointer to the FP64 state [n_vars][cells][nodes] (owned by the state). */
double* dg_state_data(dg_state* state);
/* Host <-> device copies of the state (host array of n_dof doubles), on the
 * state's stream; both wait for completion. */
int dg_state_upload(dg_state* state, const double* host_U);
int dg_state_download(dg_state* state, double* host_U);
/* Upper spectral bound the state's DG_KRYLOV_CHEBYSHEV solves use, with the
 * alpha = (a_ii dt)^2 it belongs to: get[2] (host, may be NULL) receives the
 * current pair ({0, 0} before the first Chebyshev solve); set[2] (host, may
 * be NULL) replaces it -- a caller who knows the spectrum can skip the power
 * iteration; a bound with set[0] <= 1/(gamma-1) is cleared (re-estimated on the
 * next solve).  A bound that is too low is detected and repaired by the solve
 * (GMRES fallback, re-estimate).  Synchronises the device first. */
int dg_state_chebyshev_bound(dg_state* state, double* get, const double* set);

/* One IMEX-RK2 step U^n -> U^{n+1} of size dt (Sec. 2 scheme; readings: ARK2
 * tableau, Picard loop on the pressure with lagged enthalpy and kinetic
 * energy, GMRES(m) on the Helmholtz problem).  Enqueued on `stream`; returns
 * after the step has finished (the Krylov loops read residuals on the host).
 * Returns DG_ENOTCONV if a solve missed its tolerance within max_iters (the
 * state then holds the unconverged step), DG_ENONFINITE if the new state has
 * a NaN/Inf. `stats` may be NULL. */
int imex_rk2_step(dg_ctx* ctx, const dg_mesh* mesh, dg_state* state, double dt, const dg_solver_opts* opts,
                  dg_step_stats* stats, void* stream);

/* Ensemble step (batching of many uneven members, one persistent kernel per
 * stage): advance n independent members -- each with its own mesh and state,
 * any mix of dimensions and degrees, the same solver options -- by one IMEX-RK2
 * step each, member i with step dt[i].  Each phase of the step is enqueued for
 * every member before the next phase; the Helmholtz solves of one Picard
 * iteration of all members run in ONE cooperative launch per (dimension,
 * degree, precision) group, each member on its own share of the CTAs (in
 * proportion to its node count) with its own barrier, so members progress and
 * converge independently inside the launch.  Each member's result equals the
 * result of imex_rk2_step on that member alone (same kernels, same order).
 * Two members may not share a mesh (DG_EINVAL).  stats[n] and statuses[n] may
 * be NULL; returns the first non-OK member status, DG_ETIMEOUT if a barrier
 * wait of the batched launch ran out (bounded at 2 s; never expected). */
int dg_batch_step(dg_ctx* ctx, int n, const dg_mesh* const* meshes, dg_state* const* states, const double* dt,
                  const dg_solver_opts* opts, dg_step_stats* stats, int* statuses, void* stream);

/* Batch plan: the ensemble step of dg_batch_step captured once as a CUDA graph
 * and replayed for every later step (the paper's ensemble has no counterpart;
 * this is the batching form of the step, Sec. 2 scheme per member).  In the
 * graph, each member's per-phase kernels sit on one of up to 16 parallel
 * branches, joined before each batched Helmholtz launch (one cooperative node
 * per (dimension, degree, precision) group and Picard iteration), and the
 * solve results and flags are copied to pinned host memory at the end.
 * dg_batch_plan_create captures (runs nothing on the device); the members'
 * meshes and states, and dt[i], are fixed for the plan's lifetime: meshes and
 * states must outlive the plan and may not be used by another call while a
 * plan step runs.  Needs the persistent solve (opts->fused != 0, or CG);
 * DG_EINVAL otherwise or if two members share a mesh.  Each replay computes
 * exactly what dg_batch_step computes on the same members (same kernels,
 * same launch shapes, same per-member order).
 * dg_batch_plan_step launches the graph on `stream`, waits for it, and fills
 * stats[n] / statuses[n] (either may be NULL) like dg_batch_step. */
typedef struct dg_batch_plan dg_batch_plan;
int dg_batch_plan_create(dg_ctx* ctx, int n, const dg_mesh* const* meshes, dg_state* const* states,
                         const double* dt, const dg_solver_opts* opts, dg_batch_plan** out);
int dg_batch_plan_step(dg_batch_plan* plan, dg_step_stats* stats, int* statuses, void* stream);
int dg_batch_plan_destroy(dg_batch_plan* plan);

/* ---------------------------------------------------------------- serving
 * A request loop for simulation requests of different mesh sizes, degrees,
 * orographies and precisions.  Requests are queued on submit; a worker thread
 * (its own context and stream, on the device of the creating context) admits
 * them first come first served while their device-memory footprint fits the
 * budget and a slot is free, keeps every admitted member's state resident,
 * and advances all resident members one IMEX-RK2 step per tick with
 * dg_batch_step (continuous batching: members join and leave between ticks,
 * their work overlaps in the batched launches).  A member's result equals the
 * result of stepping it alone to the Krylov tolerance.  The paper has no
 * serving layer; this is the deployment form of the same path. */
typedef struct dg_server dg_server;

typedef struct {
  size_t hbm_budget_bytes; /* admission budget for resident members (bytes)      */
  int max_members;         /* resident slots; 0 = limited by the budget only     */
} dg_serve_opts;

typedef struct {
  dg_mesh_desc mesh;       /* copied on submit (level and ijk arrays too)        */
  int init_kind;           /* dg_init_kind                                       */
  double init_params[8];   /* see dg_init_state                                  */
  int n_init_params;
  double dt;               /* step size (s)                                      */
  int steps;               /* IMEX-RK2 steps to run                              */
  dg_solver_opts solver;   /* precision and Krylov settings                      */
} dg_request;

typedef enum { DG_REQ_QUEUED = 0, DG_REQ_RUNNING = 1, DG_REQ_DONE = 2, DG_REQ_FAILED = 3 } dg_request_state;

typedef struct {
  int state;               /* dg_request_state                                   */
  int status;              /* DG_OK, or why the request failed                   */
  int steps_done;
  long long gmres_iters;   /* inner GMRES iterations so far                      */
  double t_submit, t_admit, t_finish; /* seconds since the server was created    */
  size_t footprint_bytes;  /* device bytes reserved while resident (estimate)    */
  int64_t n_dof;
} dg_request_info;

typedef struct {
  int queued, running;
  size_t used_bytes;
  long long ticks;
  double elapsed_s;
} dg_serve_info;

int dg_serve_create(dg_ctx* ctx, const dg_serve_opts* opts, dg_server** out);
/* Queue a request; *id identifies it.  DG_EINVAL for a malformed request,
 * DG_EBUDGET if its footprint exceeds the whole budget (it could never be
 * admitted); neither disturbs resident members. */
int dg_serve_submit(dg_server* server, const dg_request* req, uint64_t* id);
/* Non-blocking status; host_U (may be NULL) receives the final state
 * ([n_vars][cells][nodes] doubles) once the request is done. */
int dg_serve_poll(dg_server* server, uint64_t id, dg_request_info* info, double* host_U);
/* Wait until the request is done or failed, at most timeout_s seconds
 * (DG_ETIMEOUT otherwise). */
int dg_serve_wait(dg_server* server, uint64_t id, double timeout_s);
/* Forget a finished request and free its stored result. */
int dg_serve_release(dg_server* server, uint64_t id);
int dg_serve_stats(dg_server* server, dg_serve_info* info);
/* Stop the worker: resident members are freed, queued ones fail. */
int dg_serve_destroy(dg_server* server);

#ifdef __cplusplus
}
#endif

#endif /* DG_ATMO_H */
