/*
 * mpm.h -- C-ABI of the GB300 stabilized implicit u-p material point method.
 *
 * The method is the one of Zhao & Choo, "Stabilized material point methods for
 * coupled large deformation and fluid flow in porous materials" (arXiv
 * 1905.00671): a fully implicit MPM for a fluid-saturated mixture with nodal
 * unknowns [u, p] (equal-order linear interpolation, Sec. 3.1), stabilized by
 * polynomial pressure projection (PPP, Sec. 4.2) and solved by Newton (Sec.
 * 3.4).  Everything behind these calls runs as CUDA kernels on one GPU.
 *
 * The calls follow the paper's statement of the problem (Sec. 2.4): given the
 * Dirichlet data u^, p^, the Neumann data t^, q^ and the initial fields u0 = 0,
 * p0, find u and p.  mpm_create takes the material points (the initial
 * configuration), the material and the permeability; mpm_step advances one
 * load step (Stages 1-4 of Sec. 3.1) with the current loads and boundary
 * conditions; mpm_read returns the material point state.
 *
 * Conventions (all calls)
 *   - SI units.  Tension positive, pore pressure positive in compression
 *     (Eq. darcy-law and the effective stress of Sec. 2.2).
 *   - dim = 2 is plane strain, dim = 3 is 3D.  Per-point vectors are stored
 *     point-major: x[i*dim + k].  Tensors are row-major dim x dim.
 *   - Grid nodes are numbered i + (nx+1)*(j + (ny+1)*k) with nx = ncell[0], ...
 *     Nodal unknowns are interleaved [u_x, u_y, (u_z), p] per node.
 *   - Every pointer argument is a HOST pointer unless stated otherwise; the
 *     library copies what it needs and never keeps a caller pointer.
 *   - Return value: MPM_OK (0) or a negative MPM_ERR_* code.  After an error
 *     mpm_last_error(ctx) describes it; after a failed mpm_create or
 *     mpm_create_batch (no context), mpm_last_error(NULL) does.  A failed mpm_step leaves the state at
 *     the last completed step.  No call throws.
 *   - A context is used by one host thread at a time.
 */
#ifndef UPMPM_MPM_H
#define UPMPM_MPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MPM_OK = 0,
  MPM_ERR_BAD_ARG = -1,          /* invalid argument or size */
  MPM_ERR_OUT_OF_GRID = -2,      /* a material point centre left the background grid */
  MPM_ERR_NEGATIVE_J = -3,       /* det F <= 0 at some material point */
  MPM_ERR_NONFINITE = -4,        /* NaN / Inf in the residual */
  MPM_ERR_NEWTON_DIVERGED = -5,  /* Newton hit its iteration cap */
  MPM_ERR_KRYLOV_STAGNATED = -6, /* the Krylov solver hit its iteration cap */
  MPM_ERR_TIMEOUT = -7,          /* reserved for bounded device-side waits */
  MPM_ERR_CUDA = -8,             /* a CUDA runtime call failed */
  MPM_ERR_NO_MEMORY = -9,        /* device allocation failed */
  MPM_ERR_TOO_LARGE = -10        /* size beyond the fixed scratch of mpm_bin_noalloc */
};

enum { MPM_SHAPE_ORIG = 0, MPM_SHAPE_GIMP = 1 };     /* Sec. 3.1: FE basis or GIMP basis */
enum { MPM_QUASISTATIC = 0, MPM_NEWMARK = 1 };       /* Sec. 3.2: implicit Euler or Newmark */
enum { MPM_FP64 = 0, MPM_MIXED = 1 };

/* Expression of the PPP stabilization parameter tau (Sec. 4.3), evaluated per
 * point and step from the point's Lame constants lambda, G and mobility
 * kappa = k / mu_f, with M = lambda + 2 G (the P-wave modulus K + 4G/3),
 * c_v = M kappa, the step dt and the grid spacing h:
 *   WHITE    (Eq. tau-white)     tau = 1 / (2 G)
 *   SUN      (Eq. tau-sun)       tau = (1 - 3 c_v dt / h^2)
 *                                      (1 + tanh(2 - 12 c_v dt / h^2)) / M
 *   MONFORTE (Eq. tau-monforte)  tau = max(2 / M - (beta / gamma) 12 kappa dt / h^2, 0)
 *                                (2 kappa / c_v written as 2 / M, its value for
 *                                kappa > 0 and its limit at kappa = 0); Newmark
 *                                steps only (it uses beta and gamma).
 * The chosen expression is multiplied by mpm_options.tau_scale. */
enum { MPM_TAU_WHITE = 0, MPM_TAU_SUN = 1, MPM_TAU_MONFORTE = 2 };

/* Permeability of a point: CONSTANT (the given k), or KOZENY_CARMAN
 * (Eq. kozeny-carman): k = k0 (1 - phi0)^2 / phi0^3 * phi^3 / (1 - phi)^2 with
 * the given k as k0, mpm_material.phi0 and the current porosity
 * phi = 1 - (1 - phi0) / J (incompressible constituents); k = 0 once
 * phi <= 0.  The Jacobian carries its derivative with respect to J. */
enum { MPM_PERM_CONSTANT = 0, MPM_PERM_KOZENY_CARMAN = 1 };

/* Stage-1 mapping of the point fields to the nodes (Sec. 3.1): LUMPED,
 * f_i = sum_mp S m f / M_i (Eq. map-from-particles-to-nodes), or CONSISTENT,
 * sum_j M_ij f_j = sum_mp S_i m f with the consistent mass M_ij = sum_mp S_i S_j m
 * (Eq. map-from-particles-to-nodes-consistent; the paper's choice for cyclic
 * loading), solved for the active nodes (those of the Newton system; the
 * others keep the lumped values) by Jacobi-preconditioned CG to a relative
 * residual of 1e-14; a step whose mass matrix CG cannot solve to that
 * tolerance within 1000 iterations fails with MPM_ERR_KRYLOV_STAGNATED. */
enum { MPM_P2G_LUMPED = 0, MPM_P2G_CONSISTENT = 1 };

/* Hyperelastic model of the solid skeleton: NEOHOOKE, tau' = G (b - 1) +
 * lambda ln J 1 (the default), or HENCKY (Sec. 2.2: Psi = lambda/2 (ln J)^2 +
 * G tr((ln b / 2)^2), tau' = lambda ln J 1 + G ln b), with its spectral
 * tangent in the Jacobian and in the Kelvin stress; in precision MPM_MIXED
 * the FP32 Jacobian of HENCKY stages that tangent per (point, node) (the
 * per-term form is neo-Hookean only). */
enum { MPM_MODEL_NEOHOOKE = 0, MPM_MODEL_HENCKY = 1 };

/* Preconditioner of the FGMRES solve of the Newton system: node-block Jacobi,
 * or the Schur-complement block preconditioner of Sec. 3.4 with geometric
 * multigrid V-cycles for the displacement block and the pressure Schur
 * complement (default). */
enum { MPM_PRECOND_BLOCK_JACOBI = 0, MPM_PRECOND_SCHUR_MG = 1 };

/* Approximation of the pressure Schur complement S = C - B2 A^{-1} B1 inside
 * the Schur preconditioner.  DIAG_A: C - B2 diag(A)^{-1} B1 kept on the
 * Jacobian's sparsity (fill lumped to the diagonal); good when A is dominated
 * by the Newmark mass term.  FIXED_STRESS: C plus the lumped pressure mass
 * sum_p S_ip b2_p vol_p / (cs_p K_p) on the diagonal, K = lambda + 2 (G -
 * lambda ln J) / dim the drained bulk modulus (the volumetric part of A
 * replaced by its bulk stiffness); robust in the quasi-static, near-undrained
 * limit.  AUTO (default): FIXED_STRESS for quasi-static steps, DIAG_A for
 * Newmark. */
enum { MPM_SCHUR_AUTO = 0, MPM_SCHUR_DIAG_A = 1, MPM_SCHUR_FIXED_STRESS = 2 };

/* Order of the two sub-solves of the Schur preconditioner.  LOWER (default):
 * the block lower-triangular [A 0; B2 S]^{-1}, z_u = A^-1 v_u then
 * z_p = S^-1 (v_p - B2 z_u).  UPPER: the block upper-triangular
 * [A B1; 0 S]^{-1}, z_p = S^-1 v_p then z_u = A^-1 (v_u - B1 z_p).  Same work
 * per application (two V-cycles and one sparse product with a coupling
 * block); LOWER took 8% fewer FGMRES iterations on the 2D footing. */
enum { MPM_SCHUR_LOWER = 0, MPM_SCHUR_UPPER = 1 };

/* Kernel classes that mpm_options.profile can time with CUDA events (bit k of
 * the mask selects class k; mpm_stats.prof_ms[k] / prof_launches[k]). */
enum {
  MPM_PROF_SPMV = 0,      /* block-CSR SpMV inside the Krylov solver */
  MPM_PROF_JACOBIAN = 1,  /* Jacobian block assembly */
  MPM_PROF_RESIDUAL = 2,  /* residual assembly */
  MPM_PROF_POINT = 3,     /* per-point kinematics / stress / flux evaluation */
  MPM_PROF_ORTH = 4,      /* Gram-Schmidt kernels of FGMRES */
  MPM_PROF_P2G = 5,       /* Stage-1 P2G */
  MPM_PROF_G2P = 6,       /* Stages 3-4 update */
  MPM_PROF_PRECOND = 7,   /* preconditioner application */
  MPM_PROF_SETUP = 8,     /* preconditioner set-up (Schur complement, multigrid
                             hierarchy, coarsest inverse) and system scaling */
  MPM_PROF_PREP = 9,      /* step preparation outside Stage-1 P2G: binning,
                             shape functions, sparsity pattern, initial guess */
  MPM_PROF_COUNT = 10
};

typedef struct mpm_ctx mpm_ctx;

/* Structured background grid, fixed for the whole run (Sec. 3.5: "fixed
 * background mesh").  Square (cubic) cells of size h. */
typedef struct {
  int32_t dim;        /* 2 or 3 */
  int32_t ncell[3];   /* cells per axis; ncell[2] ignored for dim = 2 */
  double origin[3];
  double h;
} mpm_grid;

/* Material points at t = 0 (u0 = 0 there).  n points; arrays of length n or
 * n*dim.  lp are the half lengths of the GIMP domains (Eq. gimp-basis); they
 * also place the surface points of Neumann data (x + lp.n).  surf_id maps a
 * point to its entry in the load arrays of mpm_loads (-1: interior point). */
typedef struct {
  int64_t n;
  const double *x;            /* n*dim positions */
  const double *vol;          /* n volumes */
  const double *lp;           /* n*dim GIMP half lengths (0 < lp < h) */
  const double *p0;           /* n initial pore pressures, NULL = 0 */
  const double *v0;           /* n*dim initial velocities (Newmark), NULL = 0 */
  const int32_t *surf_id;     /* n, -1 = interior; NULL = no surface points */
  const double *surf_normal;  /* n*dim outward unit normals (surface points) */
  const double *surf_area;    /* n boundary measure carried by each surface point */
  int32_t n_surf;             /* number of surface entries */
} mpm_particles;

/* Mixture of incompressible constituents (Sec. 2.1), compressible
 * neo-Hookean skeleton (Kirchhoff effective stress G(b - 1) + lambda ln J 1),
 * Kelvin viscous stress (Sec. 2.2, Newmark only), Darcy flow with mobility
 * k / mu_f (Eq. darcy-law). */
typedef struct {
  const double *E;            /* n Young's moduli */
  const double *nu;           /* n Poisson ratios */
  double rho_s, rho_f;        /* intrinsic densities */
  double phi0;                /* initial porosity */
  double mu_f;                /* fluid dynamic viscosity */
  double alpha_vis;           /* Kelvin damping parameter */
  double g[3];                /* gravity */
} mpm_material;

typedef struct {
  int32_t shape;              /* MPM_SHAPE_ORIG / MPM_SHAPE_GIMP */
  int32_t scheme;             /* MPM_QUASISTATIC / MPM_NEWMARK */
  double beta, gamma;         /* Newmark parameters (Sec. 3.2: 0.3025, 0.6) */
  int32_t stabilize;          /* PPP on (1) / off (0), Eq. stab-term-ppp */
  double tau_scale;           /* tau = tau_scale x the expression of tau_kind */
  int32_t precision;          /* MPM_FP64, or MPM_MIXED: Jacobian values, scaling,
                                 preconditioner and Krylov vectors in FP32 inside the
                                 FP64 Newton loop (residual, kinematics, det F,
                                 ln J and point updates stay FP64); the Krylov
                                 solve then stops at max(krylov_rtol, 1e-6) or its
                                 cap, as an inexact Newton step */
  double newton_rtol;         /* ||R^k|| / ||R^0|| test of Eq. newton-tolerance */
  int32_t newton_max;         /* Newton iteration cap */
  double newton_stag;         /* > 0: accept the round-off floor once
                                 ||R^{k-1}|| <= newton_stag ||R^0|| and R^k fails
                                 to halve it; 0 disables */
  double krylov_rtol;         /* linear solve to rtol of the scaled residual */
  int32_t krylov_restart;     /* FGMRES restart length (<= 128) */
  int32_t krylov_max;         /* total Krylov iterations per Newton iteration */
  int32_t precond;            /* MPM_PRECOND_* */
  double min_volume_fraction; /* a node is active iff sum_p S_ip V_p / h^dim exceeds
                                 this (default 1e-4; 0 = any positive volume).  An
                                 inactive node is removed from the bases of the
                                 points whose support holds it, and those bases
                                 are renormalised over their other nodes. */
  int32_t profile;            /* bit mask of MPM_PROF_* classes timed with CUDA
                                 events on the work stream (0 = none) */
  int32_t precond_lag;        /* Newton iterations of a step served by one set-up of
                                 the Schur/multigrid preconditioner (default 2; 1 =
                                 rebuilt for every Newton iteration; k > 1: rebuilt
                                 at iterations 0, k, 2k, ... of each step and reused
                                 in between, with the current diagonal scaling).
                                 Changes Krylov iteration counts only: the Newton
                                 test is on the exact residual. */
  int32_t schur_approx;       /* MPM_SCHUR_* (default AUTO) */
  void *stream;               /* cudaStream_t for all work; NULL = default stream */
  int32_t tau_kind;           /* MPM_TAU_* (default WHITE) */
  int32_t permeability;       /* MPM_PERM_* (default CONSTANT) */
  int32_t p2g_mass;           /* MPM_P2G_* (default LUMPED) */
  int32_t model;              /* MPM_MODEL_* (default NEOHOOKE) */
  int32_t schur_order;        /* MPM_SCHUR_LOWER (default) / MPM_SCHUR_UPPER */
  int32_t mg_sweeps;          /* smoothing sweeps before and after the coarse
                                 correction on every multigrid level, V(k, k),
                                 k in 1..3 (0 = default 1) */
  double mg_omega;            /* damping of the block-Jacobi smoother, in (0, 1]
                                 (0 = default: 0.7 in 2D, 0.5 in 3D) */
  int32_t autotune;           /* 1: at the first Jacobian assembly of each precision,
                                 time every candidate kernel configuration (FP32:
                                 per-term or staged per-(point, node) vectors; both:
                                 64, 128 or 256 threads per block) on the context's
                                 own data and keep the fastest (reported in
                                 mpm_stats.jac_config; FP32 Hencky: staged only);
                                 0 (default): fixed configuration (FP64 staged,
                                 FP32 per-term (Hencky: staged), 128) */
  int32_t precond_reuse;      /* steps served by one Galerkin product of the multigrid
                                 hierarchies' coarse levels (0 or 1, default: rebuilt
                                 at every step's first set-up; k > 1: rebuilt at every
                                 k-th step, the other steps refreshing only the finest
                                 levels' values and block-Jacobi inverses).  Changes
                                 Krylov iteration counts only. */
} mpm_options;

/* Neumann data of one step: traction t^ per surface entry (n_surf*dim), and
 * optionally the normal flux q^ (n_surf).  traction == NULL keeps the traction
 * uploaded by the previous step; the applied traction is scale * traction. */
typedef struct {
  const double *traction;
  const double *flux;
  double scale;
} mpm_loads;

/* Dirichlet data per grid node (Sec. 2.4).  u_fixed/u_value are nnodes*dim,
 * p_fixed/p_value are nnodes.  u_value is the prescribed displacement
 * increment over the step (the grid is reset every step), p_value the
 * prescribed pore pressure at t_{n+1}.  bcs == NULL keeps the previous data. */
typedef struct {
  const uint8_t *u_fixed;
  const double *u_value;
  const uint8_t *p_fixed;
  const double *p_value;
} mpm_bcs;

/* Caller-owned host buffers, in the caller's original point order; any
 * pointer may be NULL to skip that field. */
typedef struct {
  double *x, *u, *p;          /* n*dim, n*dim, n */
  double *v, *a;              /* n*dim (Newmark state) */
  double *F;                  /* n*dim*dim */
  double *V;                  /* n current volumes */
  double *lp;                 /* n*dim GIMP half lengths */
  double *pd, *pdd;           /* n, dp/dt and d2p/dt2 (Newmark) */
} mpm_particles_out;

#define MPM_MAX_NEWTON 64

typedef struct {
  int32_t newton_iters;                    /* of the last step */
  int32_t krylov_iters[MPM_MAX_NEWTON];    /* per Newton iteration of the last step */
  double res_norm[MPM_MAX_NEWTON + 1];     /* ||R^k|| of the last step */
  int32_t krylov_total;                    /* sum over the last step */
  int64_t steps;                           /* completed steps */
  double t;                                /* time reached */
  int64_t nnzb;                            /* blocks of the last Jacobian */
  int64_t kernel_launches;                 /* kernels launched by the last step */
  double prof_ms[MPM_PROF_COUNT];          /* device time of the profiled classes, last step */
  int64_t prof_launches[MPM_PROF_COUNT];   /* launches of the profiled classes, last step */
  int64_t jac_terms;        /* (point, a, b) terms of one Jacobian assembly of the last step:
                               sum over points of n_p^2, n_p = active nodes of the point's support */
  int64_t jac_point_nodes;  /* sum over points of n_p */
  int32_t jac_config[2];    /* Jacobian kernel in use, [0] FP64 and [1] FP32:
                               threads per block + 1000 if staged (0 = not run yet) */
  int32_t jac_tuned[2];     /* 1 if that configuration was chosen by mpm_options.autotune */
  float jac_tune_ms[2][6];  /* the timings of the candidates: per-term then staged,
                               each for 64, 128, 256 threads (0 = not a candidate) */
} mpm_stats;

/* Fills *o with the defaults: GIMP, quasi-static, beta 0.3025, gamma 0.6,
 * PPP on with tau_W, FP64, Newton rtol 1e-8 (Eq. newton-tolerance), 25
 * iterations, Krylov rtol 1e-8, restart 120, 3000 iterations, Schur-complement
 * multigrid preconditioner set up once per two Newton iterations. */
void mpm_default_options(mpm_options *o);

/* Creates a context and uploads the problem (Sec. 2.4 "given u0, p0"): the
 * points, per-point E, nu and intrinsic permeability k (permeability, n
 * values, m^2).  Allocates all device memory the run needs except what
 * depends on the evolving sparsity and supports (the block matrix, the
 * preconditioner's coupling blocks and the Jacobian's staged per-(point,
 * node) vectors), which a step grows when it needs more.  *out receives the context, or NULL on
 * error (the code says why).  Rejected with MPM_ERR_BAD_ARG before any device
 * call: a non-finite position, a volume that is not positive and finite, an E
 * that is not positive and finite, nu outside (-1, 1/2), a negative or
 * non-finite permeability.  A non-finite p0, load or boundary value is not
 * checked here; the step that meets it fails with MPM_ERR_NONFINITE. */
int mpm_create(const mpm_grid *grid, const mpm_particles *particles, const mpm_material *material,
               const double *permeability, const mpm_options *options, mpm_ctx **out);

/* One load step t_n -> t_n + dt (Sec. 3.1 Stages 1-4): bin the points, map
 * their state to the nodes (Eq. map-from-particles-to-nodes), Newton on the
 * stabilized system (Eq. jacobian-system-stabilized-ppp) with the FGMRES
 * linear solver, then update and convect the points (Sec. 3.5).  loads and
 * bcs may be NULL (keep the previous ones).  Blocks until the step is done. */
int mpm_step(mpm_ctx *ctx, double dt, const mpm_loads *loads, const mpm_bcs *bcs);

/* Copies the point state into caller-owned host buffers (original order). */
int mpm_read(const mpm_ctx *ctx, mpm_particles_out *out);

/* Checkpoint / resume.  All state that persists between steps lives on the
 * material points (the grid is reset every step, Sec. 3.5), so a checkpoint
 * is mpm_read of every field of mpm_particles_out.  mpm_restore writes such a
 * state (caller's original point order) back into a context created with the
 * same initial configuration, and sets its time and step count; stepping on
 * with the same loads and boundary conditions then repeats the original run.
 * NULL fields are left as they are. */
int mpm_restore(mpm_ctx *ctx, const mpm_particles_out *state, double t, int64_t steps);

int mpm_get_stats(const mpm_ctx *ctx, mpm_stats *stats);

/* Human-readable description of the last error on ctx (never NULL).  With
 * ctx == NULL: why the calling thread's last mpm_create / mpm_create_batch
 * failed ("null context" if its last create succeeded or none was made). */
const char *mpm_last_error(const mpm_ctx *ctx);

/* Frees the context and all its device memory.  NULL is a no-op. */
void mpm_destroy(mpm_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched instances.  The paper steps one problem at a time; these calls step
 * many independent problems together (same dim, cell size h, options, time
 * step and material constants rho_s, rho_f, phi0, mu_f, alpha_vis, g; each
 * with its own grid, points, per-point E, nu and permeability, loads and
 * boundary conditions).  The instance grids are laid out on one background
 * grid of the context, at least MPM_BATCH_GAP empty cells apart, so every
 * kernel of a step runs once over all instances.  Each point keeps the
 * coordinates of its own grid and its GIMP domain is clipped by its own grid
 * (Sec. 3.1 as for a single problem), so no support reaches another instance:
 * the instances never couple through the discrete equations.  Newton
 * continues until every instance meets the residual test of
 * Eq. newton-tolerance on its own residual; the FGMRES solve and its
 * preconditioner act on all instances at once.
 * ---------------------------------------------------------------------- */
#define MPM_BATCH_GAP 2

/* Layout of count instance grids on one background grid (no GPU needed):
 * offsets[3*i + k] = cell offset of instance i along axis k (the instance's
 * node (a, b, c) becomes node (a, b, c) + offset); ncell = cells per axis of
 * the background grid.  Instances are placed on shelves of width about
 * sqrt(total area), tallest first; all grids must share dim and h. */
int mpm_batch_pack(int32_t count, const mpm_grid *grids, int32_t *offsets, int32_t *ncell);

/* Creates a context holding count instances (arrays of count entries;
 * permeability[i] has particles[i].n values).  mpm_read then returns the
 * points of all instances in order (instance 0's points first, each in its
 * instance's original order and coordinates); mpm_get_stats reports the
 * whole batch. */
int mpm_create_batch(int32_t count, const mpm_grid *grids, const mpm_particles *particles,
                     const mpm_material *materials, const double *const *permeability,
                     const mpm_options *options, mpm_ctx **out);

/* One load step of every instance.  loads / bcs: count entries each (or NULL
 * to keep all previous data); inside an entry, a NULL array keeps that
 * instance's previous values.  Node arrays of bcs[i] refer to instance i's own
 * grid numbering. */
int mpm_step_batch(mpm_ctx *ctx, double dt, const mpm_loads *loads, const mpm_bcs *bcs);

/* ------------------------------------------------------------------------
 * Inspection entry points.  They expose the intermediate results of one step
 * so that each stage can be compared with an independent implementation.
 * ---------------------------------------------------------------------- */

/* Cell of every point (original order) and the cell-sorted order (original
 * point ids sorted by (cell, id)) of the current state.  cell: n int32,
 * order: n int64. */
int mpm_debug_bin(mpm_ctx *ctx, int32_t *cell, int64_t *order);

/* Runs Stage 1 and the sparsity build for a step of size dt from the current
 * state, without solving; the inspection calls below then refer to it. */
int mpm_debug_prepare(mpm_ctx *ctx, double dt, const mpm_loads *loads, const mpm_bcs *bcs);

/* Block-CSR sparsity of the prepared step: nnodes+1 row pointers, then the
 * block column indices (ascending per row).  Returns the number of blocks, or
 * a negative code; with col_idx == NULL only the count is returned. */
int64_t mpm_debug_pattern(mpm_ctx *ctx, int64_t *row_ptr, int32_t *col_idx, int64_t cap);

/* Lumped nodal mass M, Stage-1 nodal pressure P_n and nodal volume fraction
 * phi = sum_p S_ip V_p / h^dim (each nnodes; any may be NULL) of the prepared
 * step. */
int mpm_debug_nodal(mpm_ctx *ctx, double *M, double *Pn, double *phi);

/* Residual R(X) (nnodes*(dim+1)) and the Jacobian block values (nnzb blocks of
 * (dim+1)^2, row-major, in the pattern's order) at the nodal unknowns X
 * (nnodes*(dim+1), node-interleaved [dU, P]) for the prepared step, exactly as
 * the residual/Jacobian kernels produce them before Dirichlet elimination
 * (apply_bc = 0) or after it (apply_bc = 1).  Jv may be NULL. */
int mpm_debug_eval(mpm_ctx *ctx, const double *X, double *R, double *Jv, int32_t apply_bc);

/* z = M^{-1} v for the preconditioner the Krylov solver would use at the
 * iterate X of the prepared step: the Jacobian (after Dirichlet elimination)
 * is assembled at X, scaled symmetrically by D = |diag J|^{-1/2}, and M^{-1}
 * is the preconditioner of that scaled system.  X, v, z: nnodes*(dim+1). */
int mpm_debug_precond(mpm_ctx *ctx, const double *X, const double *v, double *z);

/* The FP32 Jacobian of the mixed mode (Eq. jacobian-system-stabilized-ppp
 * evaluated in FP32 from FP32 copies of the point records, as the mixed
 * Newton step assembles it) at the nodal unknowns X (FP64, as in
 * mpm_debug_eval) of the prepared step, assembled by one given kernel
 * configuration: form 0 per-term, 1 staged per-(point, node) vectors; tpb 64,
 * 128 or 256 threads per block (the candidates of mpm_options.autotune).  Jv: nnzb blocks of
 * (dim+1)^2 floats in the pattern's order, before (apply_bc = 0) or after
 * (apply_bc = 1) Dirichlet elimination.  MPM_ERR_BAD_ARG for a context that
 * is not mixed-precision, a form or block size outside these sets, form 0 in
 * a Hencky context, or no prepared step. */
int mpm_debug_jacobian32(mpm_ctx *ctx, const double *X, int32_t form, int32_t tpb, float *Jv,
                         int32_t apply_bc);

/* ------------------------------------------------------------------------
 * Allocation-free binning.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory where they bin points
 * (a solver inside a host application that owns all device memory through its
 * own pool, or a latency-critical loop that cannot afford the implicit device
 * synchronisation of cudaMalloc / cudaFree).
 *
 * Computes, like the binning inside mpm_step, the cell of every point
 * (floor((x - origin) / h) per axis, linear id x-fastest) and the points
 * ordered by (cell, index), without allocating: x_dev (n*dim doubles,
 * point-major), cell_dev (n int32) and order_dev (n int64) are DEVICE pointers
 * owned by the caller; stream is a cudaStream_t (NULL = default stream).  The
 * per-cell counters live in a fixed device array of this library (about 3 MiB
 * on every GPU that loads it, held until exit), so the grid may have at most
 * 262,144 cells (also per axis, checked before the cell count is formed);
 * larger grids return MPM_ERR_TOO_LARGE.  A point outside the
 * grid returns MPM_ERR_OUT_OF_GRID (cell_dev then holds -1 for it and
 * order_dev is not written).  Every call copies an error word to the host
 * and waits for `stream`, so it returns when the work is done.  The first call
 * on a device also looks up the array's device address and should come before
 * any stream capture.  All calls on a device share the array and the
 * call clears what it needs at zero; calls that overlap on the GPU race on it
 * and must be ordered by the caller. */
int mpm_bin_noalloc(const mpm_grid *grid, int64_t n, const double *x_dev, int32_t *cell_dev,
                    int64_t *order_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* UPMPM_MPM_H */
