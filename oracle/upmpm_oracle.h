/*
 * upmpm_oracle.h -- plain FP64 CPU oracle of the stabilized implicit u-p
 * material point method (Zhao & Choo, "Stabilized material point methods for
 * coupled large deformation and fluid flow in porous materials").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no header, helper, table or kernel with the CUDA path.
 *
 * The oracle is stateless: every function takes the arrays it reads and the
 * arrays it writes.  The Newton loop, the Dirichlet elimination and the
 * direct linear solve live in oracle/oracle.py.
 *
 * Conventions
 *   dim d = 2 (plane strain) or 3; nb = d + 1 unknowns per node, ordered
 *   [u_x, u_y, (u_z), p].  Node (i,j,k) has linear index i + nn0*(j + nn1*k)
 *   with nn = ncell + 1.  Cell (i,j,k) likewise with ncell.
 *   Per particle and axis the support is `count` consecutive nodes starting at
 *   `first`; the 1D basis values S, dS/dx, S0 are stored in 4 slots per axis
 *   (slot s <-> node first+s).  Tensors are row-major d x d.
 */
#ifndef UPMPM_ORACLE_H
#define UPMPM_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_ERR_BAD_ARG (-1)
#define ORC_ERR_OUT_OF_GRID (-2)
#define ORC_ERR_NEGATIVE_J (-3)

typedef struct {
  int32_t dim;      /* 2 or 3 */
  int32_t shape;    /* 0 = original MPM (FE basis), 1 = GIMP */
  int32_t ncell[3]; /* cells per axis (ncell[2] ignored when dim = 2) */
  double origin[3];
  double h;         /* square / cubic cells */
} orc_grid;

typedef struct {
  int64_t n;
  const double *x;      /* n*d, positions at t_n */
  const double *lp;     /* n*d, GIMP half lengths at t_n */
  const double *F;      /* n*d*d, deformation gradient at t_n */
  const double *V;      /* n, volume at t_n */
  const double *m;      /* n, mixture mass for this step */
  const double *lam;    /* n, Lame lambda */
  const double *G;      /* n, shear modulus */
  const double *kappa;  /* n, mobility k / mu_f */
  const double *tau;    /* n, stabilization parameter (0 = unstabilized) */
  const int32_t *surf;  /* n, surface entry index or -1 */
  const double *surf_n; /* n*d, outward unit normal of surface particles */
  const double *surf_A; /* n, boundary measure carried by the particle */
} orc_particles;

typedef struct {
  double dt;
  int32_t dynamic;   /* 0 = quasi-static implicit Euler, 1 = Newmark */
  double beta, gamma;
  double rho_f;      /* intrinsic fluid density */
  double alpha_vis;  /* Kelvin damping parameter (dynamic only) */
  double g[3];       /* gravity */
  int32_t kozeny;    /* 1: permeability from porosity, Eq. kozeny-carman (kappa given = kappa_0) */
  double phi0;       /* initial porosity (Kozeny-Carman) */
  int32_t hencky;    /* 1: Hencky elasticity (Sec. 2.2), else compressible neo-Hookean */
} orc_step;

typedef struct {
  const double *P;    /* nnodes, nodal pressure at t_n (Stage 1) */
  const double *v;    /* nnodes*d, nodal velocity at t_n (dynamic) */
  const double *a;    /* nnodes*d, nodal acceleration at t_n (dynamic) */
  const double *pd;   /* nnodes, nodal dp/dt at t_n (dynamic) */
  const double *pdd;  /* nnodes, nodal d2p/dt2 at t_n (dynamic) */
} orc_nodal;

int64_t orc_nnodes(const orc_grid *g);
int64_t orc_ncells(const orc_grid *g);

/* 1D basis of one axis (exposed for the shape-function pins); dx = x - origin. */
int orc_shape_1d(int32_t shape, double dx, double lp, double h, int32_t ncell,
                 int32_t *first, int32_t *count, double *S, double *dS, double *S0);

int orc_shape(const orc_grid *g, int64_t n, const double *x, const double *lp,
              int32_t *first, int32_t *count, double *S, double *dS, double *S0);

int orc_bin(const orc_grid *g, int64_t n, const double *x, int32_t *cell, int64_t *order);

int64_t orc_pattern(const orc_grid *g, int64_t n, const int32_t *first, const int32_t *count,
                    int64_t *row_ptr, int32_t *col_idx, int64_t cap);

int orc_p2g(const orc_grid *g, int64_t n, const int32_t *first, const int32_t *count,
            const double *S, const double *m, int32_t nf, const double *fld,
            double *M, double *out);

/* Consistent mass matrix of Eq. map-from-particles-to-nodes-consistent,
 * M_ij = sum_mp S_i S_j m, accumulated into the values mc (nnz) of the node
 * pattern (row_ptr, col_idx) of orc_pattern. */
int orc_consistent_mass(const orc_grid *g, int64_t n, const int32_t *first, const int32_t *count,
                        const double *S, const double *m, const int64_t *row_ptr, const int32_t *col_idx,
                        double *mc);

/* Basis of point p over its support box (node ids, S, t_n gradient d per
 * node, S0), with the inactive nodes removed and the rest renormalised as in
 * orc_eval (active may be NULL).  Returns the node count (<= 4^d). */
int orc_point_basis(const orc_grid *g, int64_t p, const int32_t *first, const int32_t *count,
                    const double *S, const double *dS, const double *S0, const uint8_t *active,
                    int64_t *node, double *Sv, double *Gv, double *S0v);

/* active (nnodes, may be NULL): nodes with active == 0 are removed from the
 * bases of the points whose support box holds them, which are renormalised. */
int orc_eval(const orc_grid *g, const orc_step *sp, const orc_particles *pp,
             const int32_t *first, const int32_t *count, const double *S, const double *dS,
             const double *S0, const uint8_t *active, const orc_nodal *nd, const double *trac,
             const double *flux, const double *X, const int64_t *row_ptr, const int32_t *col_idx,
             double *R, double *Jv);

/* The residual of orc_eval with the terms it leaves unlinearized frozen at
 * the iterate Xf (the Kelvin stress's geometry and mu' or Hencky tangent,
 * Darcy's acceleration; the nodal velocities still from X): its derivative at
 * X = Xf is the analytic Jacobian of orc_eval (Sec. 3.4: some inertia and
 * damping terms are not linearized).  R only. */
int orc_eval_frozen(const orc_grid *g, const orc_step *sp, const orc_particles *pp,
                    const int32_t *first, const int32_t *count, const double *S, const double *dS,
                    const double *S0, const uint8_t *active, const orc_nodal *nd, const double *trac,
                    const double *flux, const double *X, const double *Xf, double *R);

int orc_g2p(const orc_grid *g, const orc_step *sp, int64_t n, const int32_t *first,
            const int32_t *count, const double *S, const double *dS, const double *S0,
            const uint8_t *active, const orc_nodal *nd, const double *X, double *x, double *u,
            double *F, double *V, double *lp, const double *lp0, double *p, double *v, double *a,
            double *pd, double *pdd);

/* Right stretch U = (F^T F)^{1/2} diagonal by Jacobi eigen-iteration. */
void orc_stretch_diag(int32_t d, const double *F, double *Udiag);

#endif
