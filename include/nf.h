/*
 * nf.h — C ABI of the B300 differentiable cut-cell fluid step library (libnf).
 *
 * One time step on a 3D MAC grid (Sec. 2.3.1 of arXiv 2405.14903): RK2
 * semi-Lagrangian advection (Eq. advection_matrix; Appendix B, Eqs.
 * advection_1/advection_2), rasterisation of a parametric solid into per-face
 * fluid fractions alpha (Sec. 2.3.1, Projection), and the cut-cell pressure
 * projection (Eq. projection_matrix, Eq. u_next_matrix) solved by a
 * matrix-free multigrid-preconditioned conjugate gradient; plus the adjoint
 * of the step (Sec. 2.3.2 and 2.3.3) for back-propagation through a rollout.
 *
 * Conventions shared by every call:
 *  - Status: every call returns an int status (NF_OK = 0 or an NF_E_* code);
 *    nothing throws across the ABI and no kernel traps. nf_status_string()
 *    names a code; nf_last_error() gives the calling thread's last message.
 *  - Layout: a grid has nx*ny*nz cells of edge dx. Face arrays are separate
 *    per component, x fastest: ux is [nz][ny][nx+1], uy [nz][ny+1][nx],
 *    uz [nz+1][ny][nx]; cell arrays are [nz][ny][nx]. Pointers given in a
 *    3-array are (x, y, z) components.
 *  - Memory: `mem` selects NF_MEM_DEVICE (device pointers on the context's
 *    device, e.g. torch data_ptr()) or NF_MEM_HOST (host pointers; the
 *    library copies them, pinned memory is faster). Caller buffers are
 *    borrowed for the duration of the call only; nothing is retained.
 *  - Ownership: the library owns all episode state (velocity, pressure,
 *    fractions, the multigrid hierarchy, the checkpoint tape) in device
 *    memory, freed by nf_episode_destroy / nf_destroy.
 *  - Streams: all device work of a context is ordered on its stream. Calls
 *    return once their results are in the destination (they synchronise the
 *    stream when they must read solver status on the host).
 *  - Threads: a context is not thread safe; use one context per host thread.
 */
#ifndef NF_H
#define NF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define NF_OK 0
#define NF_E_INVALID 1       /* bad argument, unknown episode id, bad size  */
#define NF_E_OOM 2           /* HBM budget exceeded or device alloc failed */
#define NF_E_NOT_CONVERGED 3 /* iteration cap hit; stats hold iters, resid */
#define NF_E_DIVERGED 4      /* NaN or Inf met in a residual               */
#define NF_E_TIMEOUT 5       /* a bounded device wait expired              */
#define NF_E_CUDA 6          /* a CUDA runtime call failed                 */
#define NF_E_STATE 7         /* call invalid in the episode's state        */
#define NF_E_CANCELED 8      /* a served request dropped by NF_REQ_CANCEL   */

/* ----------------------------------------------------------------- enums */
#define NF_PREC_FP64 0   /* FP64 fields, vectors and multigrid            */
#define NF_PREC_FP32 1   /* FP32 fields, vectors and multigrid            */
#define NF_PREC_MIXED 2  /* FP32 fields; FP32 PCG with BF16 coarse-level
                            coefficients; FP64 dots and FP64 iterative
                            refinement of r = b - A x                     */
#define NF_SOLVER_CG 0    /* unpreconditioned conjugate gradient           */
#define NF_SOLVER_MGPCG 1 /* geometric multigrid V-cycle preconditioned CG */

#define NF_F32 0
#define NF_F64 1
#define NF_MEM_DEVICE 0
#define NF_MEM_HOST 1

#define NF_SCENE_NONE 0    /* no solid                                      */
#define NF_SCENE_SPHERE 1  /* sphere translating with velocity theta[0..2]  */
#define NF_SCENE_CHAMBER 2 /* ellipsoid chamber, radius modulated by 8
                              Fourier coefficients theta, union a duct    */
#define NF_SCENE_PLATE 3   /* plate rotating about z, 4 angle knots theta   */
#define NF_SCENE_SPHERES 4 /* static spheres, no parameters                */
#define NF_SCENE_EXTRUDED 5 /* polar-Bezier shapes extruded along z, CSG
                               union (App. A, Sec. 2.2; the heart of Sec. 3
                               as a union of four): table in nf_scene      */

#define NF_LOSS_KINETIC 0 /* J = 1/2 sum_faces u^2 dx^3                     */
#define NF_LOSS_OUTFLOW 1 /* J = sum over outlet faces of u_x dx^2         */

#define NF_MAX_PARAMS 8

/* ------------------------------------------------------------- structures */
typedef struct nf_ctx nf_ctx;

typedef struct nf_config {
  int device;             /* CUDA device ordinal                              */
  void *stream;           /* cudaStream_t to order work on; NULL: the library
                             creates its own stream. Pass cudaStreamLegacy
                             ((void *)1) for the legacy default stream.       */
  int precision;          /* NF_PREC_*                                        */
  int solver;             /* NF_SOLVER_*                                      */
  double tol;             /* stop when ||b - A P||_2 / ||b||_2 <= tol (FP64) */
  int max_iters;          /* cap on preconditioned iterations per solve       */
  double inner_tol;       /* MIXED: residual reduction per FP32 inner solve   */
  int mg_smooth;          /* red-black Gauss-Seidel sweeps before and after   */
  int mg_coarsest;        /* stop coarsening at this many cells per edge      */
  int advect_order;       /* 2 = RK2 midpoint backtrace, 1 = forward Euler    */
  int checkpoint_every;   /* rollout checkpoint interval C (steps)            */
  size_t hbm_budget;      /* admission budget for episode state; 0 = none     */
  double cfl_max;         /* 0: nf_step advances steps of dt. > 0: nf_step
                             advances frames of dt, each split into
                             m = ceil(max|U| dt / (dx cfl_max)) equal substeps
                             (velocity at the frame start)                   */
  int mg_coarsest_sweeps; /* symmetric red-black sweep pairs on the coarsest
                             multigrid level (0: the default, 8)             */
  int mg_band_sweeps;     /* extra red-black sweeps on the finest level's
                             boundary band (cells with a cut face and their
                             neighbours) before pre- and after post-smoothing */
  int mg_transfer;        /* 0: trilinear prolongation, restriction P^T / 4;
                             1: piecewise-constant prolongation, restriction
                             by the mean of the eight children (the coarse
                             operators are then Galerkin)                    */
  double mg_coarse_weight; /* scale w of every coarse-grid correction, in
                             (0, 2) (0: 1); applied as sqrt(w) on restriction
                             and prolongation so the V-cycle stays symmetric.
                             w near 2 offsets the weak piecewise-constant
                             coarse space (over-correction)                 */
  int mg_smooth_coarse;   /* sweeps on the levels below the finest (0: as
                             mg_smooth)                                      */
  int tape_fractions;     /* 1: the rollout tape keeps every step's face
                             fractions (one face triple per step), so the
                             backward pass copies them instead of
                             rasterising again; 0: recompute them           */
  int mg_persistent;      /* 1: the coarse levels of at most 64^3 cells above
                             the one-block chain run, with the chain, as the
                             phases of one cooperative kernel (constant
                             transfer only); 0: one launch per phase (inside
                             the solver's device-side CG loop these launches
                             cost no more than the cooperative kernel's grid
                             barriers). Same arithmetic either way           */
  int mg_cluster;         /* 1: the coarse levels just above an 8^3-or-smaller
                             local chain (planes splitting evenly over 8
                             CTAs, FP32 data, constant transfer; 32^3 and
                             16^3 at 128^3) run as z-slabs on one 8-CTA
                             thread-block cluster with the chain on its CTA
                             0 (distributed shared memory, cluster barriers);
                             0: one launch per phase (inside the device-side
                             CG loop these cost about as much, and the local
                             chain's serial part dominates either way).
                             Same arithmetic                                  */
  int residual_fp64;      /* MIXED refinement residual r = b - A x (x, b FP64):
                             1: FP64 arithmetic; 0: split-float arithmetic
                             (each FP64 value as a float pair, error-free
                             float transforms: ~48 significant bits, error
                             about 2^-44 max|x|), free of FP64 instructions,
                             which run at 1/64 of the FP32 rate here         */
  int mg_fused;           /* 1: each red-black sweep pair of the finest level
                             (red then black before the coarse correction,
                             black then red after it) is one launch over
                             shared-memory tiles, reading x, b and the
                             fractions once per pair (constant transfer, no
                             band sweeps); 2: the same on every grid level
                             above the one-block chain; 0: one launch per
                             half sweep. Same arithmetic, same bits          */
  int recompute_overlap;  /* 1: during nf_backward (and the serving adjoint),
                             the next checkpoint segment is recomputed on a
                             second stream by a helper thread while the
                             current one is reverted (the same kernels on the
                             same data: the same results); 0: sequential.
                             Costs one more segment of tape, a solver
                             hierarchy and a host thread per episode          */
} nf_config;

typedef struct nf_grid {
  int nx, ny, nz;         /* cells per axis: nx, ny >= 4; nz >= 4, or nz = 1
                             for the 2D variant of App. D as a one-cell slab
                             between closed z walls (its multigrid has one
                             level: the preconditioner is symmetric
                             Gauss-Seidel)                                  */
  double dx;              /* cell edge                                        */
  double dt;              /* time step                                        */
  double rho;             /* density (1 in every shipped scene)               */
  int outlet;             /* 0: closed box; 1: open patch on the high-x wall  */
  int outlet_j0, outlet_k0, outlet_w, outlet_h; /* patch cells in y and z   */
  /* kinematic viscosity (>= 0; 0 = inviscid). With nu > 0 every step applies
     explicit viscosity (Sec. 2.3.1, Eq. viscosity_matrix) between advection
     and projection: U^ = (I - nu h / dx^2 G^T G) U~ for each component on
     its own face lattice, G the difference across each edge between two
     neighbouring lattice points inside the box (none past the walls), h the
     step length. Explicit Euler is stable for nu h / dx^2 <= 1/6; larger
     values are accepted and computed as written. Costs one extra face
     field per episode and one stencil pass each way per step.            */
  double nu;
  /* face fraction rule: NF_FRACTIONS_SUPERSAMPLE (0) = the fluid share of the
     face's dx^3 control volume from 4x4x4 ramp subsamples; NF_FRACTIONS_CORNER
     (1) = the paper's rule (Sec. 2.3.1, Projection): the fluid share of the
     face's area, from phi at its four corners, zero crossings on its edges
     by linear interpolation, and the area of the polygon through the fluid
     corners (phi >= 0) and the crossings in walking order (connected fluid
     where only two diagonal corners are fluid).                          */
  int fractions;
  /* inflow patch (0: none): wall faces of an x wall (inlet_side -1: x = 0,
     +1: x = nx) over cells j0 .. j0 + w - 1, k0 .. k0 + h - 1 whose normal
     velocity is held at inlet_speed (along +x). They are wall faces
     (alpha = 0) whose solid velocity is the inflow: the blended update
     holds them at it and the right-hand side G^T (I - S) U_s carries the
     inflow into the projection (the inlets of Sec. 3's heart scene; the
     inflow boundary of App. D). On the high-x wall it must not overlap the
     outlet patch.                                                         */
  int inlet, inlet_side, inlet_j0, inlet_k0, inlet_w, inlet_h;
  double inlet_speed;
} nf_grid;

#define NF_FRACTIONS_SUPERSAMPLE 0
#define NF_FRACTIONS_CORNER 1

typedef struct nf_scene {
  int kind;               /* NF_SCENE_*                                       */
  int K;                  /* parameters in theta (0..NF_MAX_PARAMS)           */
  double theta[NF_MAX_PARAMS];
  /* kind constants: SPHERE: centre[0..2], radius[3]. CHAMBER: centre[0..2],
     axes[3..5], period[6], duct_x0[7], duct_half[8]. PLATE: centre[0..2],
     half extents[3..5], period[6] (knots at 0, T/3, 2T/3, T).             */
  double consts[16];
  const double *spheres;  /* SPHERES: nspheres x (cx, cy, cz, r), host memory */
  int nspheres;
  /* EXTRUDED: consts[0] shapes (1..4), consts[1] fluid inside the union (1)
     or outside it (0), consts[2] theta mode: 0 = every radius of the table
     in table order (K = their count <= NF_MAX_PARAMS; the table's own radii
     are ignored), 1 = the 4 knots (at t = 0, T/3, 2T/3, T) of a piecewise-
     linear contraction k(t) scaling the radii of shape consts[3], period
     T = consts[4] (its wall moves with the contraction's velocity about the
     cross-section centre), 2 = no parameters. `shapes` is a host table of
     `nshape_values` doubles, copied at creation: per shape
       n keys (1..4), N segments (1..8), z0 < z1, has frame (0/1),
       frame origin (3), frame axes (9, row r = the shape's local axis r in
       world coordinates, orthonormal),
     then per key: centre (x, y) in the local frame, radii rho1_0, rho2_0,
     rho1_1, ... (2N). Key sections are evenly spaced in z0..z1.          */
  const double *shapes;
  int nshape_values;
} nf_scene;

typedef struct nf_step_stats {
  int steps;              /* time steps performed by the call                 */
  int solves;             /* linear solves performed                          */
  int iters;              /* preconditioned iterations, summed over solves    */
  int max_iters;          /* most iterations of a single solve                */
  int outer;              /* FP64 refinement passes, summed over solves       */
  double rel_residual;    /* worst final FP64 relative residual of the call   */
} nf_step_stats;

/* ------------------------------------------------------------- lifecycle */

/* Fill *cfg with defaults: device 0, own stream, MIXED, MGPCG, tol 1e-6,
   max_iters 500, inner_tol 1e-3, mg_smooth 2, mg_coarsest 4, RK2,
   checkpoint_every 10, no budget, cfl_max 0 (no sub-stepping),
   mg_coarsest_sweeps 8, mg_band_sweeps 0, mg_transfer 1 (constant),
   mg_coarse_weight 1.9, mg_smooth_coarse 0, tape_fractions 0,
   mg_persistent 0, mg_cluster 0, residual_fp64 1, mg_fused 0,
   recompute_overlap 1. */
int nf_config_default(nf_config *cfg);

/* Create a context on cfg->device. *out receives the handle. */
int nf_create(nf_ctx **out, const nf_config *cfg);

/* Free every episode and the context. */
int nf_destroy(nf_ctx *ctx);

/* The calling thread's last error message (valid until its next call). */
const char *nf_last_error(nf_ctx *ctx);
const char *nf_status_string(int status);

/* Wait for all work of the context's stream. */
int nf_synchronize(nf_ctx *ctx);

/* ---------------------------------------------------------------- episode */

/* Create an episode: a grid, a scene with parameters theta, zero velocity,
   step counter 0. NF_E_INVALID for a grid with fewer than 4 cells in x or y,
   nz not 1 or >= 4, dx, dt <= 0, nu < 0 or not finite, an unknown fraction rule, or an
   outlet patch off the high-x wall. Admission: NF_E_OOM when its device state would exceed the
   context's HBM budget. Geometry is evaluated analytically at
   t_{n+1} = (n + 1) dt in every step (Sec. 2.3.1, Projection). */
int nf_episode_create(nf_ctx *ctx, const nf_grid *g, const nf_scene *s,
                      int64_t *id);
int nf_episode_destroy(nf_ctx *ctx, int64_t id);

/* Device bytes held by the episode (fields, hierarchy, tape so far). */
int nf_episode_bytes(nf_ctx *ctx, int64_t id, size_t *bytes);

/* Replace the scene parameters theta (K values, host memory). Clears the tape. */
int nf_set_params(nf_ctx *ctx, int64_t id, const double *theta, int K);

/* Set the velocity u (3 face arrays of dtype NF_F32/NF_F64 in `mem`), reset
   the step counter to 0 and clear the tape. With project != 0 the field is
   first made divergence free with the t = 0 cut-cell system (projection
   only, no advection); that projection is recorded and is part of the
   adjoint computed by nf_backward. */
int nf_set_velocity(nf_ctx *ctx, int64_t id, const void *const u[3],
                    int dtype, int mem, int project, nf_step_stats *st);

/* Advance nsteps time steps (or frames, when cfl_max > 0: each frame of dt
   is split into substeps by the CFL rule; the rule of Table 1's caption).
   One step of length h from t to t + h: rasterise alpha and u_s at t + h,
   advect (Eq. advection_matrix), apply viscosity when nu > 0 (Eq.
   viscosity_matrix), solve Eq. projection_matrix, apply the
   blended update U = S (U^ - c G P) + (I - S) U_s with c = h / (rho dx).
   On fluid components that touch no open face the right-hand side is
   projected to zero mean and the pressure is returned with zero mean.
   Records checkpoints every checkpoint_every steps for nf_backward; st->steps
   counts the steps taken. Returns NF_E_NOT_CONVERGED if a solve hit
   max_iters (the step is still applied). */
int nf_step(nf_ctx *ctx, int64_t id, int nsteps, nf_step_stats *st);

/* Loss of the current velocity: J (host double) and optionally dJ/dU into
   gU (device or host arrays, may be NULL). */
int nf_loss(nf_ctx *ctx, int64_t id, int loss_kind, double *J,
            void *const gU[3], int dtype, int mem);

/* Back-propagate through the most recent unreverted step (Sec. 2.3.2,
   2.3.3): from dJ/dU^{n+1} (gU_next) compute dJ/dU^n (gU_prev, may alias
   gU_next) and add that step's dJ/dtheta into g_theta (K host doubles).
   Recomputes the step's segment from its checkpoint when needed. After the
   last time step it reverts the initial projection, if one was recorded.
   NF_E_STATE when nothing is left to revert. */
int nf_backward_step(nf_ctx *ctx, int64_t id, const void *const gU_next[3],
                     void *const gU_prev[3], int dtype, int mem,
                     double *g_theta, nf_step_stats *st);

/* Back-propagate through the whole recorded rollout: gU_final = dJ/dU^T,
   gU0 (may be NULL) receives dJ/dU^0 of the velocity given to
   nf_set_velocity, g_theta (K host doubles) is overwritten with dJ/dtheta.
   Uses checkpoints and per-segment recomputation. */
int nf_backward(nf_ctx *ctx, int64_t id, const void *const gU_final[3],
                void *const gU0[3], int dtype, int mem, double *g_theta,
                nf_step_stats *st);

/* ---------------------------------------------------------------- queries */
int nf_get_velocity(nf_ctx *ctx, int64_t id, void *const u[3], int dtype,
                    int mem);
/* Pressure of the last solve (cell array). */
int nf_get_pressure(nf_ctx *ctx, int64_t id, void *p, int dtype, int mem);
/* Face fractions alpha of the last step (3 face arrays). */
int nf_get_fractions(nf_ctx *ctx, int64_t id, void *const a[3], int dtype,
                     int mem);
/* Velocity U^ of the last step before projection: advected, then viscous
   when nu > 0 (3 face arrays). */
int nf_get_advected(nf_ctx *ctx, int64_t id, void *const u[3], int dtype,
                    int mem);
/* Advance n episodes (distinct ids, 1 <= n <= 64) of this context by
   nframes frames each (nf_step), solving every substep's projections as
   one stacked system: the members' boxes stacked along z with their closed
   z walls between them, so the stacked operator is block diagonal and each
   solver launch (smoothing, restriction, coarse chain, CG updates, dots,
   FP64 residual) serves every member. Members must share nx, ny, nz and
   their multigrid depth (NF_E_INVALID otherwise); scenes, dt, viscosity,
   fraction rule and openings may differ. With CFL sub-stepping each member
   takes its own substeps; a substep's batch holds the members that have
   it. Each member's right-hand side enters the stack scaled by a power of
   two to norm in [1/2, 2) (undone on its pressure, exactly), and the
   stacked solve stops when ||r|| <= tol min_e ||b_e||, which keeps every
   member's relative residual within tol; a member's result differs
   from its solve alone within that tolerance (one Krylov process serves all
   members). st (n entries, may be NULL) receives each member's statistics
   (the shared solves counted for each) and status (n entries, may be NULL)
   each member's status: a member whose right-hand side turns non-finite
   leaves the batch with NF_E_DIVERGED while the others go on. The call
   returns the worst member status. The tape of each member is
   recorded as by nf_step, so nf_backward works per member afterwards. The
   stacked solver's device memory is cached in the context per (cells,
   members) and is not counted in the HBM budget. */
int nf_step_batch(nf_ctx *ctx, const int64_t *ids, int n, int nframes, nf_step_stats *st,
                  int *status);

/* Resume: the episode's state (velocity, frame clock, theta) as host bytes.
   nf_episode_export with buf = NULL sets *bytes to the size needed; with a
   host buffer of *bytes >= that size it writes the state and sets *bytes.
   nf_episode_import loads such bytes into an episode of the same grid,
   scene kind and precision (NF_E_INVALID otherwise, or for a buffer that is
   not an exported state): velocity, theta and the frame clock are restored,
   so the next nf_step continues the rollout at the saved time; the tape
   starts anew (nf_backward reaches back to the import, as after
   nf_set_velocity). Both synchronise the context's stream. Not a step of
   the method: a service for checkpointing and resuming served episodes. */
int nf_episode_export(nf_ctx *ctx, int64_t id, void *buf, size_t *bytes);
int nf_episode_import(nf_ctx *ctx, int64_t id, const void *buf, size_t bytes);

/* Step counter n (the velocity is U^n). */
int nf_get_step(nf_ctx *ctx, int64_t id, int *n);

/* Diagnostic: *out = sum_i a[i] b[i] over n entries of two device arrays
   (dtype NF_F32 or NF_F64) of the context's device, computed by the
   solver's own dot arithmetic (the CG inner products of Eq.
   projection_matrix's solve): FP32 entries give exact products and
   compensated per-thread sums, then FP64 block and grid sums in fixed order.
   Synchronises the context's stream. */
int nf_dot(nf_ctx *ctx, const void *a, const void *b, int64_t n, int dtype,
           double *out);

/* Diagnostic: the face kernels widen FP32 values to FP64 and round FP64
   values to FP32 by integer operations on the bits (the conversion
   instructions issue on the FP64 pipe, at 1/64 of the FP32 rate on this
   part). This runs those routines on the n host values in[] (copied to the
   context's device and back) beside the conversion instructions:
   out_f[i] = the integer FP64 -> FP32 rounding of in[i], out_d[i] = the
   integer FP32 -> FP64 widening of (float)in[i], and *mismatches = the
   number of i where either differs from the instruction's result (bitwise;
   NaN against NaN counts as equal). Host arrays of n entries, owned by the
   caller; n in [0, 2^24]. Synchronises the context's stream. */
int nf_check_conversions(nf_ctx *ctx, const double *in, int64_t n, float *out_f,
                         double *out_d, int64_t *mismatches);

/* Kernel launches issued by this context since creation (a counter of the
   library's own kernels, used to report launches per timed region). */
int nf_launch_count(nf_ctx *ctx, int64_t *count);

/* ------------------------------------------------------------- profiling */
/* Environment: NF_GRAPHS=0 makes the solver launch every kernel directly
   instead of replaying CUDA graphs of its iteration batches (for profilers
   that cannot follow stream capture). Kernels and results are unchanged.
   NF_TEST_STALL_WAITS=1 (test hook, read when an episode is created) makes
   the solver's bounded device waits wait for something that never comes,
   so that they expire (after about a second) and the solve returns
   NF_E_TIMEOUT; the context stays usable. */
/* Kernel classes that nf_profile can time (CUDA events on the context's
   stream bracketing every launch of the class). */
#define NF_K_RASTERIZE 0
#define NF_K_ADVECT 1
#define NF_K_RHS 2
#define NF_K_UPDATE 3
#define NF_K_LOSS 4
#define NF_K_ADJ_GP 5
#define NF_K_ADJ_FACE 6
#define NF_K_ADJ_ADVECT 7
#define NF_K_RESIDUAL64 8
#define NF_K_AXPY64 9
#define NF_K_CG_INIT 10
#define NF_K_APPLY_DOT 11
#define NF_K_CG_XR 12
#define NF_K_CG_RZ 13
#define NF_K_CG_D 14
#define NF_K_MG_COARSEN 15
#define NF_K_MG_SMOOTH 16     /* coarse levels */
#define NF_K_MG_RESIDUAL 17
#define NF_K_MG_RESTRICT 18
#define NF_K_MG_PROLONG 19
#define NF_K_MG_CHAIN 20
#define NF_K_CAST 21
#define NF_K_MG_SMOOTH0 22    /* finest level  */
#define NF_K_GAUGE 23
#define NF_K_MG_MID 24        /* coarse levels + chain, one cooperative kernel */
#define NF_K_VISCOSITY 25     /* explicit viscosity, forward and adjoint */
#define NF_K_COUNT 26

/* Start timing launches of kernel class `kclass` (NF_K_*), or of every class
   with kclass = -1; kclass = -2 stops. Resets the accumulated totals. */
int nf_profile(nf_ctx *ctx, int kclass);
/* Accumulated launches and device milliseconds of one class since
   nf_profile (synchronises the stream). */
int nf_profile_read(nf_ctx *ctx, int kclass, int64_t *launches, double *ms);

/* ----------------------------------------------------------- serving ---
   A request loop over many concurrent gym-style episodes (one simulated
   environment each, Sec. 3's environments behind a reset / step protocol),
   for the pattern of serving many environments from one GPU: episodes stay
   resident on the device, are admitted under an HBM budget, and their
   requests run on `slots` worker streams at once, so a request that arrives
   while others are on the GPU starts as soon as a slot and memory allow and
   its kernels overlap theirs (continuous batching). Requests of one episode
   run in submission order on the slot that opened it; its forward results
   do not depend on what else is in flight (bitwise: the forward kernels are
   deterministic), its gradients only to rounding (the advection adjoint
   scatters with float atomics).

   Kinds:
     NF_REQ_OPEN          create episode `episode` (a client-chosen key) from
                          `grid` and `scene`, velocity at rest. Waits, queued,
                          while the budget cannot hold it.
     NF_REQ_STEP          advance `frames` frames (nf_step).
     NF_REQ_STEP_ADJOINT  advance `frames` frames, then the loss `loss_kind`
                          of the final velocity and dJ/dtheta by BPTT over
                          the episode's whole rollout (nf_backward).
     NF_REQ_CLOSE         destroy the episode; its memory returns to the
                          budget and admits waiting OPENs (FIFO).
     NF_REQ_CANCEL        cancel the episode at once: its requests that have
                          not started complete with NF_E_CANCELED, the one
                          running (if any) completes normally, then the
                          episode closes (the cancel's own result reports
                          NF_REQ_CLOSE once it has); an episode never
                          created is dropped with its reservation, and the
                          cancel completes at once with NF_OK.
   Budget: an OPEN reserves episode_estimate = the episode's base state plus
   its rollout tape for checkpoint_every steps; after every request the
   reservation follows the episode's actual bytes where they are larger.
   Errors are per request (nf_result.status); a request for an unknown or
   failed episode completes with NF_E_INVALID / NF_E_STATE. */
typedef struct nf_server nf_server;

#define NF_REQ_OPEN 0
#define NF_REQ_STEP 1
#define NF_REQ_STEP_ADJOINT 2
#define NF_REQ_CLOSE 3
#define NF_REQ_CANCEL 4

typedef struct nf_request {
  int kind;               /* NF_REQ_*                                         */
  int64_t episode;        /* client key of the episode                        */
  nf_grid grid;           /* OPEN                                             */
  nf_scene scene;         /* OPEN (spheres: host array, copied at submit)     */
  int frames;             /* STEP, STEP_ADJOINT                               */
  int loss_kind;          /* STEP_ADJOINT: NF_LOSS_*                          */
} nf_request;

typedef struct nf_result {
  int status;             /* NF_OK or the request's error                     */
  int kind;
  int64_t episode;
  double loss;            /* STEP_ADJOINT                                     */
  double g_theta[NF_MAX_PARAMS]; /* STEP_ADJOINT: dJ/dtheta                   */
  nf_step_stats fwd, bwd; /* solver statistics of the step and the adjoint    */
  double submit_ms, start_ms, end_ms; /* server clock, ms since creation     */
  size_t episode_bytes;   /* device bytes of the episode after the request    */
} nf_result;

typedef struct nf_server_stats {
  int64_t submitted, completed, open_waiting, episodes;
  size_t bytes_reserved, bytes_peak, budget;
  int slots;
  int64_t batches;          /* batched steps run (2 or more members)        */
  int64_t batched_requests; /* requests served inside those batches         */
} nf_server_stats;

/* cfg: precision, solver and tolerances of every episode (its device and
   stream fields are ignored: each slot creates its own stream on
   cfg->device). slots >= 1. hbm_budget: bytes of episode state (0: no
   limit). */
int nf_server_create(const nf_config *cfg, int slots, size_t hbm_budget,
                     nf_server **out);
/* Queue a request; *ticket identifies its result. Never blocks on the GPU. */
int nf_server_submit(nf_server *srv, const nf_request *req, int64_t *ticket);
/* Wait up to wait_ms (0: do not wait, < 0: forever) for a ticket's result;
   NF_OK and the result (then forgotten by the server), or NF_E_TIMEOUT. */
int nf_server_poll(nf_server *srv, int64_t ticket, int wait_ms, nf_result *out);
/* Wait until every submitted request has completed (wait_ms as in poll). */
int nf_server_drain(nf_server *srv, int wait_ms);
int nf_server_stats_get(nf_server *srv, nf_server_stats *out);
/* Batching: a slot that takes a STEP or STEP_ADJOINT request also takes
   the queued step requests of other episodes of the same slot with the same
   cell counts and frame count (each the oldest queued request of its
   episode), up to max_members in all, and runs their forward frames with
   nf_step_batch (every projection of a substep solved for all of them in
   one stacked solve); STEP_ADJOINT members then run their backward pass
   alone. Admission places an episode on a slot that already holds
   episodes of its cell counts when that slot is within two requests of the
   least loaded. Results: each member's forward differs from its solve alone
   within the solver tolerance. Only episodes of at most max_cells cells
   batch (and get the slot preference): small grids, whose solver launches
   are latency-bound, gain from sharing launches, while large ones fill the
   device alone and lose concurrency to the lockstep. max_members 1 turns
   batching off, the default: on this GPU the slots' concurrent streams
   already overlap small episodes' launches, and the batch's lockstep
   (slot affinity, the slowest member's substeps and iterations) measured
   slower in the serving mixes; batching pays where few streams serve many
   small episodes. */
int nf_server_set_batching(nf_server *srv, int max_members, int64_t max_cells);
/* Stops the workers after their current request, destroys all episodes. */
int nf_server_destroy(nf_server *srv);

/* ---------------------------------------------------------- no-alloc ---
   nf_loss_noalloc: the loss of nf_loss (kinetic energy 1/2 sum u^2 dx^3, or
   the net flux sum u_x dx^2 through the outlet patch) and optionally dJ/dU,
   for a caller's face-velocity triple, with no context, no episode and no
   allocation of any kind. The paper has no counterpart: this is a service
   entry point of this library, not a step of the method.

   Who needs it: callers that must not allocate device memory at this point,
   e.g. a reward or loss evaluation inside an environment loop whose device
   memory is held by another allocator (a framework's caching pool, or a
   serving process admitted under a fixed HBM budget), or any loop where the
   device-wide synchronisation of cudaMalloc/cudaFree would stall other work.

   g       grid (nx, ny, nz >= 1, dx > 0; the outlet fields for the outflow
           loss; dt and rho are ignored).
   u       three DEVICE arrays of the current device, component d of shape
           [nz + (d==2)][ny + (d==1)][nx + (d==0)], x fastest, dtype NF_F32
           or NF_F64. Host pointers, and device pointers of another device,
           are rejected with NF_E_INVALID. The call cannot check the arrays'
           sizes: they must hold the grid's face shapes (the Python binding
           checks shapes and dtypes before the call).
   gU      NULL, or three device arrays of the same shapes and dtype that
           receive dJ/dU.
   J       host double that receives the loss.
   stream  cudaStream_t to run on (NULL: the legacy default stream). The call
           returns after synchronising this stream.

   Scratch: a file-scope device array of NF_NOALLOC_SCRATCH_BYTES (8 KiB:
   block partials, a ticket counter and the result of the deterministic
   fixed-order reduction) used by every call on a device. Maximum size: each
   face component may hold at most NF_NOALLOC_MAX_FACES entries (32-bit index
   decode); larger grids are rejected with NF_E_INVALID before any device
   work. The ticket is cleared (cudaMemsetAsync on `stream`) at every call.
   The first call on each device looks up the array's device address
   (cudaGetSymbolAddress with that device current, checked: NF_E_CUDA on
   failure) and caches it.
   Calls that overlap in time on one device (other streams, other threads)
   share the scratch and race: serialise them. Results equal nf_loss's for
   the same velocity (same kernel, same summation order). */
#define NF_NOALLOC_SCRATCH_BYTES 8192
#define NF_NOALLOC_MAX_FACES 2147483647LL
int nf_loss_noalloc(const nf_grid *g, int loss_kind, const void *const u[3],
                    void *const gU[3], int dtype, double *J, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NF_H */
