// mpm_internal.cuh -- data layout, context and device helpers shared by the
// CUDA translation units of the u-p MPM library (not part of the public ABI).
//
// Layout in HBM (all structure-of-arrays, field-major, so that a warp reading
// one field of 32 consecutive material points issues one coalesced load):
//   particles  pf[PF_*][n]   FP64 state, cell-sorted at the start of each step
//   shape      sh_first[k][n], sh_cnt[n] (packed per-axis node counts),
//              sh_S/sh_dS/sh_S0[k*4+s][n]  1D basis values per axis and slot
//   records    rec[RC_*][n]  per-point quantities of the current Newton
//                            iterate (kinematics, stress, flux, stabilization)
//   nodes      nodal fields [field][nnodes]; unknowns X node-interleaved
//              [dU_x, dU_y, (dU_z), P] per node, like the block-CSR blocks
//   matrix     block-CSR: row_ptr[nnodes+1], col[nnzb], val[nnzb][nb][nb]
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mpm.h"

namespace upmpm {

template <typename T>
struct MGHier;

// The scaled Newton system D J D y = -D R and its solver workspace in the
// precision T of the Krylov solve (FP64, or FP32 in the mixed mode).
template <typename T>
struct LinSys {
  T *val = nullptr;            // nnzb_cap * nb * nb block values (scaled in place)
  int64_t cap = 0;             // blocks val can hold
  T *dscale = nullptr;         // nb * nnodes, D = |diag J|^{-1/2}
  T *dscinv = nullptr;         // nb * nnodes, D^{-1} = |diag J|^{1/2} (multiplied, not divided by D)
  T *dinv = nullptr;           // nnodes * nb * nb block-Jacobi inverse
  T *rhs = nullptr, *x = nullptr, *w = nullptr;  // N each
  T *V = nullptr, *Z = nullptr;                  // (m + 1) * N and m * N
  // Schur-complement multigrid preconditioner (mpm_mg.cu)
  MGHier<T> *mgA = nullptr, *mgS = nullptr;
  T *Aval = nullptr, *Sval = nullptr, *DAinv = nullptr, *B1c = nullptr;
  T *W = nullptr;      // B2_ac diag(A)_c^{-1} per block (d values), Schur set-up
  T *B1rs = nullptr;   // per node: sum over its row of the B1 blocks (d values)
  T *vu = nullptr;
  T *B2c = nullptr;    // compact B2 (d values per block), lower-triangular order only
  T *vp = nullptr;     // unscaled v_p, lower-triangular order only
  int64_t sub_cap = 0;
  bool coarse_built = false;  // the hierarchies' coarse levels hold a Galerkin product
  int64_t coarse_step = -1;   // the step (Ctx::steps) of that product
  // The multigrid part of the preconditioner application (both V-cycles and
  // the B1 update between them) captured as a CUDA graph; valid while the
  // matrix buffers it reads stay in place.  The graph reads the S-cycle's
  // level-0 rhs and first iterate of the first sub-solve (the S-cycle in the
  // upper-triangular order, the A-cycle in the lower one) from the buffers the
  // split kernel fills, g_x0 being that first iterate, and leaves the results
  // in g_zp / g_zu (the hierarchies' vector buffers at capture time).
  cudaGraphExec_t gexec = nullptr;
  T *g_x0 = nullptr, *g_zp = nullptr, *g_zu = nullptr;
  int g_lower = 0;     // order the graph was captured for
  const void *gkey_col = nullptr, *gkey_val = nullptr;
  int64_t gkernels = 0;
};

// 64-bit words of the per-node coupling mask of the block sparsity: bit
// (o0 + 3) + 7 (o1 + 3) + 49 (o2 + 3) is set iff node a + o couples with a.
constexpr int PATTERN_MASK_WORDS = 6;

constexpr int MAXS = 4;  // nodes per axis in one support (GIMP half length < h)
// Jacobian staging: per point, one record per node of its support box (at
// most MAXS^d) and one for the point's own coefficients (PnLay below; the
// values are written by k_point_nodes); pn_nslot bounds the records of a
// point.
__host__ __device__ constexpr int pn_nslot(int d) { return (d == 2 ? MAXS * MAXS : MAXS * MAXS * MAXS) + 1; }

// Field offsets of a staged (point, node) record of WORD-byte values.  The
// fields a pair term reads from both of its nodes come first, padded to 16
// bytes, so that the column node's record is read with about half the loads;
// the fields read for the row node only follow; the record is padded to 16
// bytes.  A point's own record holds grad p at GP.
__host__ __device__ constexpr int pn_bpart(int d, bool dyn, int word) {
  return (2 * d + 5 + (dyn ? d : 0) + 16 / word - 1) / (16 / word) * (16 / word);
}
__host__ __device__ constexpr int pn_npf(int d, bool dyn, bool hencky, int word) {
  return pn_bpart(d, dyn, word) + 3 * d + 1 + (dyn ? 1 : 0) + (hencky ? d * d * d : 0);
}
__host__ __device__ constexpr int pn_stride(int d, bool dyn, bool hencky, int word) {
  return (pn_npf(d, dyn, hencky, word) + 16 / word - 1) / (16 / word) * (16 / word);
}
template <int D, bool DYN, bool HK, int WORD>
struct PnLay {
  static constexpr int G = 0;                 // g = F^-T grad S (D values)
  static constexpr int S = D;                 // S
  static constexpr int ST = D + 1;            // S - S0
  static constexpr int P2G = D + 2;           // p2 g (D)
  static constexpr int C = 2 * D + 2;         // p6 S + (p7 + J dk/dJ vol) g.w
  static constexpr int E = 2 * D + 3;         // p7 g.w
  static constexpr int P5S = 2 * D + 4;       // p5 S
  static constexpr int GV = 2 * D + 5;        // g.grad v (D, Newmark)
  static constexpr int BPART = pn_bpart(D, DYN, WORD);  // values read for the column node
  static constexpr int P3G = BPART;           // p3 g (D)
  static constexpr int H = BPART + D;         // p0 g^T tau' + p1 g (D)
  static constexpr int P7G = BPART + 2 * D;   // p7 g (D)
  static constexpr int P8ST = BPART + 3 * D;  // p8 (S - S0)
  static constexpr int MS = P8ST + 1;         // m S (Newmark)
  static constexpr int U = MS + (DYN ? 1 : 0);  // Hencky: staged tangent (D^3)
  static constexpr int STRIDE = pn_stride(D, DYN, HK, WORD);
  static constexpr int GP = 0;                // own record: grad p (D)
};

// ---- particle fields ------------------------------------------------------
enum PField {
  PF_X = 0,        // 3
  PF_U = 3,        // 3
  PF_F = 6,        // 9, row-major d x d in the first d*d entries
  PF_V = 15,       // current volume (at t_n)
  PF_LP = 16,      // 3 GIMP half lengths
  PF_LP0 = 19,     // 3 initial half lengths
  PF_P = 22,       // pore pressure
  PF_VEL = 23,     // 3 velocity
  PF_ACC = 26,     // 3 acceleration
  PF_PD = 29,      // dp/dt
  PF_PDD = 30,     // d2p/dt2
  PF_LAM = 31,     // Lame lambda
  PF_G = 32,       // shear modulus
  PF_KAP = 33,     // mobility k / mu_f
  PF_TAU = 34,     // PPP parameter (0 when unstabilized)
  PF_SN = 35,      // 3 surface normal
  PF_SA = 38,      // surface measure
  PF_INST = 39,    // instance of a batched context (0 otherwise)
  PF_COUNT = 40
};

// One problem instance of a context.  Its points keep the coordinates of its
// own grid (origin org, ncell nc); on the context's background grid that grid
// starts at cell / node offset off.  A single-instance context has one entry
// (its own grid, off = 0).
struct InstDev {
  double org[3];
  int off[3];
  int nc[3];
};

// ---- per-point records of one Newton iterate -------------------------------
enum RField {
  RC_FINV = 0,     // 9  dF^{-1}
  RC_TAU = 9,      // 9  Kirchhoff effective stress tau'
  RC_SVIS = 18,    // 9  alpha (lambda trD 1 + 2 mu' D)   (Newmark)
  RC_GV = 27,      // 9  spatial velocity gradient        (Newmark)
  RC_GP = 36,      // 3  grad p
  RC_W = 39,       // 3  grad p - rho_f (g - a)
  RC_FRC = 42,     // 3  m (g - a)
  RC_CS = 45,      // V_n / J_n
  RC_VOL = 46,     // dJ V_n
  RC_PH = 47,      // p^h
  RC_MUP = 48,     // G - lambda ln J
  RC_LAM = 49,     // lambda
  RC_KV = 50,      // kappa * vol
  RC_CST = 51,     // C_stab factor * V_n
  RC_RST = 52,     // tau V_n (pdot - Pi pdot)
  RC_DIVV = 53,    // vol * div v
  RC_B2 = 54,      // B2 divergence coefficient
  RC_MS = 55,      // m (inertia Jacobian)
  RC_DKV = 56,     // J dkappa/dJ * vol (Kozeny-Carman; 0 for a constant permeability)
  RC_HQ = 57,      // 9  Hencky: principal directions of b (columns, d x d)
  RC_HK = 66,      // 3  Hencky: kappa_A = 2G - 2 tau_A (diagonal part of the tangent)
  RC_HT = 69,      // 3  Hencky: theta_AB of the pairs (0,1), (0,2), (1,2)
  RC_F32 = 72,     // fields above have FP32 copies (mixed mode); those below are FP64 only
  RC_RU = 72,      // 9  residual factor -cs (tau' + s_vis) dF^-T + vol p^h dF^-T (rows i, cols k)
  RC_KW = 81,      // 3  residual factor kappa vol dF^-1 w
  RC_COUNT = 84
};

// error bits raised by kernels (read back at synchronisation points)
enum DevErr : int { DE_OUT_OF_GRID = 1, DE_NEG_J = 2, DE_SUPPORT = 4, DE_SINGULAR = 8 };

struct GridP {
  int d;
  int nc[3];   // cells per axis (1 for unused axes)
  int nn[3];   // nodes per axis (1 for unused axes)
  double org[3];
  double h;
  int64_t nnodes, ncells;
};

struct StepP {
  double dt, beta, gamma, rho_f, alpha_vis;
  double g[3];
  double phi0, rho_s;
  double phi_min;  // minimum nodal volume fraction of an active node
  int kozeny;      // permeability from porosity by Eq. kozeny-carman (else constant)
  int hencky;      // Hencky elasticity (Sec. 2.2), else compressible neo-Hookean
};

// all device pointers the kernels need, passed by value
struct DevView {
  int64_t n;
  double *pf;               // PF_COUNT * n
  int64_t *pid;             // original ids
  int32_t *surf;            // surface entry or -1
  int32_t *cell;            // cell of each point (current order)
  int32_t *cell_start;      // ncells + 1
  int32_t *sh_first;        // 3 * n
  int32_t *sh_cnt;          // n, counts packed 4 bits per axis
  int4 *sh_box;             // n: (first node per axis, sh_cnt) of each point in one 16-byte word
  // first-node bins: the points by the first node of their support box
  // (fb_perm, ascending point index within a bin; bin f is fb_perm[fb_start[f]
  // .. fb_start[f + 1])), and the largest box extent per axis of the step
  const int32_t *fb_start, *fb_perm;
  const int *fb_cmax;
  const int32_t *pn_base;   // n + 1: first staged Jacobian record of each point
  double *sh_S, *sh_dS, *sh_S0;  // 12 * n each
  double *m;                // n mixture mass of the step
  double *rec;              // RC_COUNT * n
  // nodes
  double *M, *Pn, *vn, *an, *pdn, *pddn;  // vn/an: d * nnodes (field-major)
  double *phi;              // nodal volume fraction sum_p S V_p / h^d
  uint8_t *act;             // node active (mass > 0 and phi > phi_min)
  double *sh_nrm;           // 5 * n: 1/sum S, grad sum S (3), 1/sum S0 over active box nodes
  // FP32 copies written in the mixed mode for the FP32 Jacobian (else null)
  float *sh_Sf, *sh_dSf, *sh_S0f, *sh_nrmf, *recf;
  uint8_t *fixed;           // nb * nnodes, node-interleaved
  uint8_t *u_fixed;         // d * nnodes node-interleaved
  double *u_value;          // d * nnodes
  uint8_t *p_fixed;         // nnodes
  double *p_value;          // nnodes
  double *trac;             // n_surf * d (already scaled)
  double *flux;             // n_surf or null
  int *err;                 // device error word
  const InstDev *inst;      // instance table
};

// ---- host-side context ----------------------------------------------------
struct Ctx {
  GridP g{};
  StepP s{};
  int d = 2, nb = 3;
  int shape = MPM_SHAPE_GIMP, dyn = 0, stabilize = 1, precision = MPM_FP64;
  double tau_scale = 1.0;
  mpm_options opt{};
  cudaStream_t st = nullptr;
  bool own_stream = false;   // created by the context (no stream was given)
  int nsm = 152;             // SMs of the context's device
  double *fsd = nullptr;     // nnodes: lumped fixed-stress term of the pressure Schur complement
  bool fixed_stress() const {
    return opt.schur_approx == MPM_SCHUR_FIXED_STRESS || (opt.schur_approx == MPM_SCHUR_AUTO && !dyn);
  }
  bool schur_lower() const { return opt.schur_order == MPM_SCHUR_LOWER; }
  // multigrid smoothing: V(mg_sweeps, mg_sweeps) with damping mg_omega (the
  // options' values, or the defaults 1 and 0.7 in 2D / 0.5 in 3D)
  int mg_sweeps() const { return opt.mg_sweeps > 0 ? opt.mg_sweeps : 1; }
  double mg_omega() const { return opt.mg_omega > 0.0 ? opt.mg_omega : (d == 3 ? 0.5 : 0.7); }
  // instances (batched contexts hold several; see mpm_create_batch)
  int ninst = 1;
  InstDev *inst = nullptr;             // device table
  std::vector<InstDev> inst_h;         // host copy
  std::vector<int64_t> inst_n, inst_nsurf;
  // batched contexts: host copies of the combined loads and Dirichlet data,
  // so that an instance whose entry is NULL keeps its previous values
  std::vector<double> b_trac, b_flux, b_uval, b_pval;
  std::vector<uint8_t> b_ufix, b_pfix;
  bool b_has_flux = false;
  double *inorm = nullptr;             // device: per-instance squared residual norms
  double *h_inorm = nullptr;           // pinned copy
  int32_t *node_inst = nullptr;        // device: instance of every node (-1: between instances)
  // batched FGMRES: per-instance Krylov state (ninst x ...), see mpm_solver.cu
  double *bk = nullptr;                // one block of device doubles, carved below
  int32_t *bk_i = nullptr;             // per-instance flags / column counts
  double *h_bk = nullptr;              // pinned: active-instance count
  bool capturing = false;    // a CUDA graph capture is in progress on st
  int64_t n = 0;
  int32_t n_surf = 0;
  double t = 0.0;
  int64_t steps = 0;
  std::string last_error;
  mpm_stats stats{};
  int64_t launches = 0;

  // device buffers
  double *pf = nullptr, *pf_alt = nullptr;
  int64_t *pid = nullptr, *pid_alt = nullptr;
  int32_t *surf = nullptr, *surf_alt = nullptr;
  int32_t *cell = nullptr, *cell_tmp = nullptr, *cell_start = nullptr, *cell_cursor = nullptr;
  int32_t *perm = nullptr;
  int32_t *sh_first = nullptr, *sh_cnt = nullptr;
  int4 *sh_box = nullptr;
  int32_t *fb_key = nullptr, *fb_start = nullptr, *fb_cursor = nullptr, *fb_perm = nullptr;
  int *fb_cmax = nullptr;
  double *sh_S = nullptr, *sh_dS = nullptr, *sh_S0 = nullptr;
  double *m = nullptr, *rec = nullptr;
  double *M = nullptr, *Pn = nullptr, *vn = nullptr, *an = nullptr, *pdn = nullptr, *pddn = nullptr;
  double *phi = nullptr;
  uint8_t *act = nullptr;
  double *sh_nrm = nullptr;
  float *sh_Sf = nullptr, *sh_dSf = nullptr, *sh_S0f = nullptr, *sh_nrmf = nullptr, *recf = nullptr;
  uint8_t *fixed = nullptr, *u_fixed = nullptr, *p_fixed = nullptr;
  double *u_value = nullptr, *p_value = nullptr, *trac = nullptr, *trac_raw = nullptr, *flux = nullptr;
  int has_flux = 0;
  double trac_scale = 1.0;
  int *err = nullptr;
  int *h_err = nullptr;                  // pinned
  double *h_scalar = nullptr;            // pinned scratch for scalars read by the host
  unsigned long long *terms = nullptr;   // device: Jacobian term counts (n_p^2, n_p sums)
  // consistent-mass Stage 1: the mass on the node pattern and the CG workspace
  double *mc = nullptr, *cm_buf = nullptr;
  int64_t mc_cap = 0, cm_cap = 0;
  // per-(point, support node) vectors of the FP64 Jacobian (pn_nslot(d)
  // records of PN_NPF values per point)
  double *pn = nullptr;
  float *pn32 = nullptr;                 // the same in FP32 (the staged FP32 variant)
  // record layout of the staging: point q's records (one per node of its
  // support box, then its own) start at record pn_base[q]; packed in point
  // order (an exclusive scan of n_q + 1) so that a point's records are
  // contiguous and the staged region is only as large as the supports
  int32_t *pn_cnt = nullptr, *pn_base = nullptr;
  int64_t pn_total = 0;                  // records of the current step
  int64_t pn_cap = 0, pn32_cap = 0;      // records pn / pn32 can hold
  unsigned long long *h_terms = nullptr; // pinned copy
  // Jacobian kernel configuration per precision ([0] FP64, [1] FP32): the
  // form (JAC_DIRECT: node vectors recomputed per term; JAC_STAGED:
  // per-(point, node) vectors formed first) and threads per block.  Fixed
  // defaults, or chosen by timing every candidate at the context's first
  // assembly when mpm_options.autotune is set.
  enum { JAC_DIRECT = 0, JAC_STAGED = 1, JAC_FORMS = 2 };
  struct JacCfg {
    int form, tpb, tuned;
  };
  JacCfg jac_cfg[2] = {{JAC_STAGED, 128, 0}, {JAC_DIRECT, 128, 0}};

  // sparsity + matrix
  int32_t *row_nnz = nullptr, *row_ptr = nullptr, *row_of = nullptr, *col = nullptr;
  uint64_t *row_mask = nullptr;          // per node, 6 words (7^d offsets)
  int64_t nnzb = 0, nnzb_cap = 0;

  // Newton vectors (FP64, length nb * nnodes) and read-back staging
  double *X = nullptr, *R = nullptr, *dX = nullptr, *stage = nullptr;
  // Krylov solve: FP64 system always (debug calls, FP64 mode), FP32 system in
  // the mixed mode; Hessenberg / Givens / reduction scratch in FP64
  int m_restart = 30;
  LinSys<double> L64;
  LinSys<float> L32;
  bool have32 = false;
  double *H = nullptr, *gvec = nullptr, *cs = nullptr, *sn = nullptr, *yv = nullptr;
  double *hcol = nullptr, *part = nullptr, *scal = nullptr;

  // scan scratch
  int32_t *scan_tmp = nullptr;
  int64_t scan_cap = 0;

  bool prepared = false;

  // CUDA-event timing of selected kernel classes (opt.profile bit mask)
  std::vector<cudaEvent_t> ev;           // start/stop pairs
  std::vector<int> ev_kind;
  int ev_used = 0;

  DevView view() const;
  int64_t N() const { return (int64_t)nb * g.nnodes; }
};

// ---- launchers (implemented in the .cu files) -----------------------------
// particles: binning, shape, Stage 1, Stage 3/4
int run_binning(Ctx &c);                          // keys, counting sort, (cell, id) order, permute
void run_shape(Ctx &c);
int run_first_bins(Ctx &c);        // the first-node bins (after run_shape)
void run_mass(Ctx &c);
void run_p2g(Ctx &c);
void run_g2p(Ctx &c);
// assembly
int run_pattern(Ctx &c);                          // builds row_ptr / col / row_of
int run_consistent_p2g(Ctx &c);  // Stage-1 fields by the consistent mass (after run_pattern)
int ensure_jacobian_staging(Ctx &c);  // the FP64 Jacobian's staging buffer (allocated by FP64 contexts at create)
int ensure_jacobian_staging32(Ctx &c);  // the FP32 staged Jacobian's buffer (mixed mode; Hencky always, else when chosen)
void run_initial_guess(Ctx &c);   // also sets the active flags
void run_renorm(Ctx &c);          // per-point renormalisation over active box nodes
int run_pn_layout(Ctx &c);        // first staged Jacobian record of each point (pn_base)
void run_count_terms(Ctx &c);     // Jacobian term counts into c.terms (device)
void run_fs_diag(Ctx &c);         // c.fsd = sum_p S_ip b2 vol / (cs K) (current records)
void run_point_eval(Ctx &c, const double *X);
void run_residual(Ctx &c, const double *X, double *R, int apply_bc);
template <typename T>
void run_jacobian(Ctx &c, T *val, int apply_bc);  // block values in precision T
int run_jacobian32_form(Ctx &c, float *val, int apply_bc, int form, int tpb);  // one given FP32 configuration
// linear algebra
template <typename T>
int linsys_alloc(Ctx &c, LinSys<T> &S, bool krylov);  // vectors; matrix on demand
template <typename T>
void linsys_free(LinSys<T> &S);
template <typename T>
int linsys_reserve(Ctx &c, LinSys<T> &S);           // val for nnzb_cap blocks
template <typename T>
void run_scale_system(Ctx &c, LinSys<T> &S, const double *R);  // scales val, rhs = -D R
template <typename T>
void run_block_jacobi(Ctx &c, LinSys<T> &S);
template <typename T>
int run_fgmres(Ctx &c, LinSys<T> &S, double rtol, int maxit, int *iters);  // S.x from S.rhs
template <typename T>
void run_precond(Ctx &c, LinSys<T> &S, const T *v, T *z);  // z = M^{-1} v (scaled system)
template <typename T>
void run_unscale_add(Ctx &c, const LinSys<T> &S, double *X);  // X += D x

double run_norm(Ctx &c, const double *x);          // synchronises

// Schur-complement multigrid preconditioner
template <typename T>
int schur_alloc(Ctx &c, LinSys<T> &S);
template <typename T>
void schur_free(LinSys<T> &S);
template <typename T>
int schur_setup(Ctx &c, LinSys<T> &S, bool coarse = true);  // before run_scale_system (unscaled val);
                                                             // coarse = false: the finest levels only
template <typename T>
void schur_apply(Ctx &c, LinSys<T> &S, const T *v, T *z);  // z = M^{-1} v

// scan: out[i] = sum_{j<i} in[j]; returns the total (synchronises)
int64_t scan_exclusive(Ctx &c, const int32_t *in, int32_t *out, int64_t n);

// helpers
int check_cuda(Ctx &c, cudaError_t e, const char *what);
int read_dev_err(Ctx &c);   // synchronises; returns MPM_ERR_* or 0

#define UPMPM_LAUNCH(ctx) ((ctx).launches++)

// ---- programmatic dependent launch ------------------------------------------
// The Krylov iteration is a chain of small dependent kernels.  A kernel launched
// with launch_pdl may have its blocks scheduled while the kernel before it in
// the stream is still running, so its launch latency hides behind that kernel.
// Every kernel launched this way calls pdl_enter() before its first global
// memory access: it waits until the preceding kernel has completed and its
// writes are visible, and then lets the next kernel in the stream be scheduled
// (so at most one kernel waits ahead).  Launched without the attribute, both
// instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline void launch_pdl(Ctx &c, void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, A... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);  // a failed launch is left in cudaGetLastError
  c.launches++;
}

// Event timing of kernel class `kind` around the launches between begin/end.
void prof_begin(Ctx &c, int kind);
void prof_end(Ctx &c, int kind);
void prof_collect(Ctx &c);   // synchronises; adds elapsed times into stats

// ---- device helpers -------------------------------------------------------
__host__ __device__ inline int unpack_cnt(int packed, int k) { return (packed >> (4 * k)) & 15; }
constexpr int RENORM_BIT = 1 << 15;  // in sh_cnt: the point's basis is renormalised

// Eq. kozeny-carman: k(J) from k0 with phi = 1 - (1 - phi0) / J
// (incompressible constituents); with jdk, also J dk/dJ = k (2 + 3 (1 - phi) / phi).
// Closed pores (phi <= 0): k = 0.
__host__ __device__ inline double kozeny_carman(double k0, double phi0, double J, double *jdk) {
  const double phi = 1.0 - (1.0 - phi0) / J;
  if (!(phi > 0.0)) {
    if (jdk) *jdk = 0.0;
    return 0.0;
  }
  const double k = k0 * ((1.0 - phi0) * (1.0 - phi0) / (phi0 * phi0 * phi0)) * (phi * phi * phi / ((1.0 - phi) * (1.0 - phi)));
  if (jdk) *jdk = k * (2.0 + 3.0 * (1.0 - phi) / phi);
  return k;
}

template <int D>
__device__ inline double det_d(const double *A) {
  if (D == 2) return A[0] * A[3] - A[1] * A[2];
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

template <int D>
__device__ inline void inv_d(const double *A, double *B) {
  const double det = det_d<D>(A);
  if (D == 2) {
    B[0] = A[3] / det;
    B[1] = -A[1] / det;
    B[2] = -A[2] / det;
    B[3] = A[0] / det;
  } else {
    B[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  }
}

// S_a, S0_a and the t_n-gradient Gn_a of box node a (slots off) of point q.
// Nodes that are inactive are removed from the point's basis, which is then
// renormalised over its active box nodes (constants stay exactly reproduced):
//   S' = S / sum S,  Gn' = (Gn - S' grad sum S) / sum S,  S0' = S0 / sum S0.
template <int D>
__device__ inline void basis_at(const DevView &v, int64_t q, const int off[3], int64_t a, double &S,
                                double &S0, double Gn[3]) {
  const int64_t n = v.n;
  double s[3] = {1.0, 1.0, 1.0}, ds[3] = {0.0, 0.0, 0.0}, s0[3] = {1.0, 1.0, 1.0};
  for (int k = 0; k < D; ++k) {
    s[k] = v.sh_S[(k * MAXS + off[k]) * n + q];
    ds[k] = v.sh_dS[(k * MAXS + off[k]) * n + q];
    s0[k] = v.sh_S0[(k * MAXS + off[k]) * n + q];
  }
  S = s[0] * s[1] * s[2];
  S0 = s0[0] * s0[1] * s0[2];
  Gn[0] = ds[0] * s[1] * s[2];
  Gn[1] = s[0] * ds[1] * s[2];
  Gn[2] = s[0] * s[1] * ds[2];
  if (v.sh_cnt[q] & RENORM_BIT) {
    if (!v.act[a]) {
      S = S0 = 0.0;
      Gn[0] = Gn[1] = Gn[2] = 0.0;
      return;
    }
    const double sinv = v.sh_nrm[0 * n + q];
    S *= sinv;
    for (int k = 0; k < D; ++k) Gn[k] = (Gn[k] - S * v.sh_nrm[(1 + k) * n + q]) * sinv;
    S0 *= v.sh_nrm[4 * n + q];
  }
}

// The same basis from arrays of type R (FP64 or the FP32 copies).
template <typename R>
struct BasisArrays {
  int64_t n;
  const int32_t *cnt;
  const uint8_t *act;
  const R *S, *dS, *S0, *nrm;
};

template <int D, typename R>
__device__ inline void basis_at_t(const BasisArrays<R> &B, int64_t q, const int off[3], int64_t a, R &S,
                                  R &S0, R Gn[3]) {
  const int64_t n = B.n;
  R s[3] = {1, 1, 1}, ds[3] = {0, 0, 0}, s0[3] = {1, 1, 1};
  for (int k = 0; k < D; ++k) {
    s[k] = B.S[(k * MAXS + off[k]) * n + q];
    ds[k] = B.dS[(k * MAXS + off[k]) * n + q];
    s0[k] = B.S0[(k * MAXS + off[k]) * n + q];
  }
  S = s[0] * s[1] * s[2];
  S0 = s0[0] * s0[1] * s0[2];
  Gn[0] = ds[0] * s[1] * s[2];
  Gn[1] = s[0] * ds[1] * s[2];
  Gn[2] = s[0] * s[1] * ds[2];
  if (B.cnt[q] & RENORM_BIT) {
    if (!B.act[a]) {
      S = S0 = 0;
      Gn[0] = Gn[1] = Gn[2] = 0;
      return;
    }
    const R sinv = B.nrm[0 * n + q];
    S *= sinv;
    for (int k = 0; k < D; ++k) Gn[k] = (Gn[k] - S * B.nrm[(1 + k) * n + q]) * sinv;
    S0 *= B.nrm[4 * n + q];
  }
}

// node / cell coordinates
__host__ __device__ inline void node_coords(const GridP &g, int64_t a, int c[3]) {
  c[0] = (int)(a % g.nn[0]);
  int64_t r = a / g.nn[0];
  c[1] = (int)(r % g.nn[1]);
  c[2] = (int)(r / g.nn[1]);
}
__host__ __device__ inline int64_t node_index(const GridP &g, const int c[3]) {
  return c[0] + (int64_t)g.nn[0] * (c[1] + (int64_t)g.nn[1] * c[2]);
}
__host__ __device__ inline int64_t cell_index(const GridP &g, int c0, int c1, int c2) {
  return c0 + (int64_t)g.nc[0] * (c1 + (int64_t)g.nc[1] * c2);
}

// Candidate cells holding points whose support may contain node coordinate a
// along one axis: a point in cell c has support within [c-1, c+2] (GIMP,
// half length < h) or [c, c+1] (original MPM).
template <bool GIMP>
__device__ inline void cand_range(int a, int nc, int &lo, int &hi) {
  lo = GIMP ? a - 2 : a - 1;
  hi = GIMP ? a + 1 : a;
  if (lo < 0) lo = 0;
  if (hi > nc - 1) hi = nc - 1;
}

// First-node bins holding every point whose support box contains both nodes
// ac and bc (ac == bc for one node): along each axis the box origin f has
// f <= min(a, b) and f + extent - 1 >= max(a, b) with extent <= cmax, the
// step's largest extent (3 for GIMP domains narrower than a cell, against the
// 4 cells around a node that can hold such a point).
template <int D>
__device__ inline void fb_window(const int *__restrict__ cmax, const int ac[3], const int bc[3], int lo[3],
                                 int hi[3]) {
  for (int k = 0; k < 3; ++k) {
    lo[k] = k < D ? max(max(ac[k], bc[k]) - cmax[k] + 1, 0) : 0;
    hi[k] = k < D ? min(ac[k], bc[k]) : 0;
  }
}

// The points of bins lo0 .. hi0 along x at (f1, f2) are one contiguous run of
// fb_perm (bins are numbered like nodes, x fastest): [b, e).
__device__ inline void fb_run(const GridP &g, const int32_t *__restrict__ fb_start, int lo0, int hi0, int f1,
                              int f2, int32_t &b, int32_t &e) {
  const int64_t r = (int64_t)g.nn[0] * (f1 + (int64_t)g.nn[1] * f2);
  b = fb_start[r + lo0];
  e = fb_start[r + hi0 + 1];
}

}  // namespace upmpm
