// mpm_api.cu -- the C-ABI of include/mpm.h and the host driver of one load
// step (Sec. 3.1 Stages 1-4, Newton of Sec. 3.4).  The host only sequences
// kernel launches and reads back one scalar per Newton / Krylov iteration;
// every arithmetic step of the method runs in the kernels of this library.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include "mpm_internal.cuh"

namespace upmpm {

DevView Ctx::view() const {
  DevView v{};
  v.n = n;
  v.pf = pf;
  v.pid = pid;
  v.surf = surf;
  v.cell = cell;
  v.cell_start = cell_start;
  v.sh_first = sh_first;
  v.sh_cnt = sh_cnt;
  v.sh_box = sh_box;
  v.fb_start = fb_start;
  v.fb_perm = fb_perm;
  v.fb_cmax = fb_cmax;
  v.pn_base = pn_base;
  v.sh_S = sh_S;
  v.sh_dS = sh_dS;
  v.sh_S0 = sh_S0;
  v.m = m;
  v.rec = rec;
  v.M = M;
  v.Pn = Pn;
  v.vn = vn;
  v.an = an;
  v.pdn = pdn;
  v.pddn = pddn;
  v.phi = phi;
  v.act = act;
  v.sh_nrm = sh_nrm;
  v.sh_Sf = sh_Sf;
  v.sh_dSf = sh_dSf;
  v.sh_S0f = sh_S0f;
  v.sh_nrmf = sh_nrmf;
  v.recf = recf;
  v.fixed = fixed;
  v.u_fixed = u_fixed;
  v.u_value = u_value;
  v.p_fixed = p_fixed;
  v.p_value = p_value;
  v.trac = trac;
  v.flux = has_flux ? flux : nullptr;
  v.err = err;
  v.inst = inst;
  return v;
}

int check_cuda(Ctx &c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return MPM_OK;
  c.last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return MPM_ERR_CUDA;
}

int read_dev_err(Ctx &c) {
  cudaMemcpyAsync(c.h_err, c.err, sizeof(int), cudaMemcpyDeviceToHost, c.st);
  cudaError_t e = cudaStreamSynchronize(c.st);
  if (e != cudaSuccess) return check_cuda(c, e, "kernel execution");
  const int f = *c.h_err;
  if (!f) return MPM_OK;
  cudaMemsetAsync(c.err, 0, sizeof(int), c.st);
  if (f & DE_OUT_OF_GRID) {
    c.last_error = "a material point centre left the background grid";
    return MPM_ERR_OUT_OF_GRID;
  }
  if (f & DE_NEG_J) {
    c.last_error = "non-positive Jacobian det F at a material point";
    return MPM_ERR_NEGATIVE_J;
  }
  if (f & DE_SUPPORT) {
    c.last_error = "GIMP half length outside (0, h) or support wider than 4 nodes";
    return MPM_ERR_BAD_ARG;
  }
  if (f & DE_SINGULAR) {
    c.last_error = "singular diagonal block in the block-Jacobi preconditioner";
    return MPM_ERR_NONFINITE;
  }
  c.last_error = "device error flag";
  return MPM_ERR_CUDA;
}

void prof_begin(Ctx &c, int kind) {
  if (!((c.opt.profile >> kind) & 1) || c.capturing) return;
  if ((size_t)(2 * c.ev_used + 2) > c.ev.size()) {
    if (c.ev.size() >= (1u << 15)) prof_collect(c);  // bounded pool: drain it
    while ((size_t)(2 * c.ev_used + 2) > c.ev.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      c.ev.push_back(e);
    }
    c.ev_kind.resize(c.ev.size() / 2);
  }
  cudaEventRecord(c.ev[2 * c.ev_used], c.st);
}

void prof_end(Ctx &c, int kind) {
  if (!((c.opt.profile >> kind) & 1) || c.capturing) return;
  if ((size_t)(2 * c.ev_used + 2) > c.ev.size()) return;
  cudaEventRecord(c.ev[2 * c.ev_used + 1], c.st);
  c.ev_kind[c.ev_used] = kind;
  ++c.ev_used;
}

void prof_collect(Ctx &c) {
  if (c.ev_used == 0) return;
  cudaStreamSynchronize(c.st);
  for (int i = 0; i < c.ev_used; ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c.ev[2 * i], c.ev[2 * i + 1]) == cudaSuccess) {
      c.stats.prof_ms[c.ev_kind[i]] += ms;
      c.stats.prof_launches[c.ev_kind[i]] += 1;
    }
  }
  c.ev_used = 0;
}

namespace {

constexpr int TPB = 256;
inline int nblk(int64_t n) { return (int)((n + TPB - 1) / TPB); }

// Lame constants from (E, nu), mobility, PPP parameter tau_W = 1 / (2 G)
// (Eq. tau-white) scaled by tau_scale, and the initial state of every field.
template <int D>
__global__ void k_init(int64_t n, double *pf, const double *__restrict__ x, const double *__restrict__ vol,
                       const double *__restrict__ lp, const double *__restrict__ p0,
                       const double *__restrict__ v0, const double *__restrict__ E,
                       const double *__restrict__ nu, const double *__restrict__ k,
                       const double *__restrict__ sn, const double *__restrict__ sa, double mu_f,
                       double tau_scale, int stabilize, int64_t *pid, const int32_t *__restrict__ pinst) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  for (int f = 0; f < PF_COUNT; ++f) pf[f * n + p] = 0.0;
  for (int i = 0; i < D; ++i) {
    pf[(PF_X + i) * n + p] = x[p * D + i];
    pf[(PF_LP + i) * n + p] = lp[p * D + i];
    pf[(PF_LP0 + i) * n + p] = lp[p * D + i];
    pf[(PF_F + i * D + i) * n + p] = 1.0;
    if (v0) pf[(PF_VEL + i) * n + p] = v0[p * D + i];
    if (sn) pf[(PF_SN + i) * n + p] = sn[p * D + i];
  }
  pf[PF_V * n + p] = vol[p];
  pf[PF_P * n + p] = p0 ? p0[p] : 0.0;
  const double e = E[p], v = nu[p];
  const double lam = e * v / ((1.0 + v) * (1.0 - 2.0 * v));
  const double G = e / (2.0 * (1.0 + v));
  pf[PF_LAM * n + p] = lam;
  pf[PF_G * n + p] = G;
  pf[PF_KAP * n + p] = k[p] / mu_f;
  pf[PF_TAU * n + p] = stabilize ? tau_scale / (2.0 * G) : 0.0;
  pf[PF_SA * n + p] = sa ? sa[p] : 0.0;
  pf[PF_INST * n + p] = pinst ? (double)pinst[p] : 0.0;
  pid[p] = p;
}

// PPP parameter of every point for a step of length dt (Sec. 4.3): tau_S
// (Eq. tau-sun) or tau_M (Eq. tau-monforte, 2 kappa / c_v written as 2 / M),
// times tau_scale, with M = lambda + 2 G the P-wave modulus and c_v = M kappa.
// (tau_W of Eq. tau-white does not depend on the step: set once by k_init.)
template <int D>
__global__ void k_tau(int64_t n, double *pf, int kind, double tau_scale, double dt, double h, double beta,
                      double gamma, int kozeny, double phi0) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double M = pf[PF_LAM * n + p] + 2.0 * pf[PF_G * n + p];
  double kap = pf[PF_KAP * n + p];
  if (kozeny) {  // the mobility at the start of the step, J_n = det F_n
    double Fn[9];
    for (int i = 0; i < D * D; ++i) Fn[i] = pf[(PF_F + i) * n + p];
    kap = kozeny_carman(kap, phi0, det_d<D>(Fn), nullptr);
  }
  double tau;
  if (kind == MPM_TAU_SUN) {
    const double cv = M * kap, r = cv * dt / (h * h);
    tau = (1.0 - 3.0 * r) * (1.0 + tanh(2.0 - 12.0 * r)) / M;
  } else {
    tau = fmax(2.0 / M - (beta / gamma) * (12.0 * kap * dt / (h * h)), 0.0);
  }
  pf[PF_TAU * n + p] = tau_scale * tau;
}

// Per-instance squared residual norms: block i sums R^2 over the nodes of
// instance i's grid (a fixed order, so the sums are run-to-run identical).
__global__ void k_inst_norm(GridP g, int nb, const InstDev *__restrict__ inst, const double *__restrict__ R,
                            double *__restrict__ out) {
  __shared__ double part[256];
  const InstDev I = inst[blockIdx.x];
  const int64_t m0 = I.nc[0] + 1, m1 = g.d > 1 ? I.nc[1] + 1 : 1, m2 = g.d > 2 ? I.nc[2] + 1 : 1;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < m0 * m1 * m2; t += blockDim.x) {
    const int64_t i0 = t % m0, i1 = (t / m0) % m1, i2 = t / (m0 * m1);
    const int c3[3] = {(int)i0 + I.off[0], (int)i1 + I.off[1], (int)i2 + I.off[2]};
    const int64_t a = node_index(g, c3);
    for (int k = 0; k < nb; ++k) acc += R[a * nb + k] * R[a * nb + k];
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = part[0];
}

__global__ void k_scale_trac(int64_t m, const double *__restrict__ raw, double s, double *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = s * raw[i];
}

// gather field f (comps components) into original point order
__global__ void k_read_field(int64_t n, const double *__restrict__ pf, int f0, int comps,
                             const int64_t *__restrict__ pid, double *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = pid[i];
  for (int c = 0; c < comps; ++c) out[o * comps + c] = pf[(int64_t)(f0 + c) * n + i];
}

// scatter field f (comps components) from original point order
__global__ void k_write_field(int64_t n, double *__restrict__ pf, int f0, int comps,
                              const int64_t *__restrict__ pid, const double *__restrict__ in) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t o = pid[i];
  for (int c = 0; c < comps; ++c) pf[(int64_t)(f0 + c) * n + i] = in[o * comps + c];
}

__global__ void k_read_cells(int64_t n, const int32_t *__restrict__ cell, const int64_t *__restrict__ pid,
                             int32_t *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[pid[i]] = cell[i];
}

template <typename T>
int dalloc(Ctx &c, T **p, int64_t count) {
  if (count <= 0) count = 1;
  if (cudaMalloc((void **)p, sizeof(T) * (size_t)count) != cudaSuccess) {
    c.last_error = "device allocation failed";
    return MPM_ERR_NO_MEMORY;
  }
  return MPM_OK;
}

int upload_loads(Ctx &c, const mpm_loads *L) {
  if (!L) return MPM_OK;
  const int64_t m = (int64_t)c.n_surf * c.d;
  if (L->traction && m > 0)
    if (cudaMemcpyAsync(c.trac_raw, L->traction, sizeof(double) * m, cudaMemcpyHostToDevice, c.st))
      return check_cuda(c, cudaGetLastError(), "upload traction");
  if (L->flux && c.n_surf > 0) {
    cudaMemcpyAsync(c.flux, L->flux, sizeof(double) * c.n_surf, cudaMemcpyHostToDevice, c.st);
    c.has_flux = 1;
  }
  c.trac_scale = L->scale;
  if (m > 0) {
    k_scale_trac<<<nblk(m), TPB, 0, c.st>>>(m, c.trac_raw, c.trac_scale, c.trac);
    UPMPM_LAUNCH(c);
  }
  return check_cuda(c, cudaGetLastError(), "loads");
}

int upload_bcs(Ctx &c, const mpm_bcs *B) {
  if (!B) return MPM_OK;
  const int64_t nn = c.g.nnodes;
  cudaStream_t s = c.st;
  if (B->u_fixed) cudaMemcpyAsync(c.u_fixed, B->u_fixed, nn * c.d, cudaMemcpyHostToDevice, s);
  if (B->u_value) cudaMemcpyAsync(c.u_value, B->u_value, sizeof(double) * nn * c.d, cudaMemcpyHostToDevice, s);
  if (B->p_fixed) cudaMemcpyAsync(c.p_fixed, B->p_fixed, nn, cudaMemcpyHostToDevice, s);
  if (B->p_value) cudaMemcpyAsync(c.p_value, B->p_value, sizeof(double) * nn, cudaMemcpyHostToDevice, s);
  return check_cuda(c, cudaGetLastError(), "bcs");
}

// Stage 1 and everything fixed over the Newton loop of one step.
int prepare_step(Ctx &c, double dt, const mpm_loads *L, const mpm_bcs *B) {
  if (!(dt > 0.0) || !isfinite(dt)) {
    c.last_error = "dt must be positive and finite";
    return MPM_ERR_BAD_ARG;
  }
  int rc = upload_loads(c, L);
  if (!rc) rc = upload_bcs(c, B);
  if (rc) return rc;
  c.s.dt = dt;
  prof_begin(c, MPM_PROF_PREP);
  rc = run_binning(c);
  if (rc) return rc;
  if (c.stabilize && c.opt.tau_kind != MPM_TAU_WHITE) {  // tau_S, tau_M depend on dt
    if (c.d == 2)
      k_tau<2><<<nblk(c.n), TPB, 0, c.st>>>(c.n, c.pf, c.opt.tau_kind, c.tau_scale, dt, c.g.h, c.opt.beta,
                                           c.opt.gamma, c.s.kozeny, c.s.phi0);
    else
      k_tau<3><<<nblk(c.n), TPB, 0, c.st>>>(c.n, c.pf, c.opt.tau_kind, c.tau_scale, dt, c.g.h, c.opt.beta,
                                           c.opt.gamma, c.s.kozeny, c.s.phi0);
    UPMPM_LAUNCH(c);
  }
  run_shape(c);
  run_mass(c);
  rc = read_dev_err(c);
  if (!rc) rc = run_first_bins(c);
  prof_end(c, MPM_PROF_PREP);
  if (rc) return rc;
  run_p2g(c);
  prof_begin(c, MPM_PROF_PREP);
  rc = run_pattern(c);
  if (!rc && c.opt.p2g_mass == MPM_P2G_CONSISTENT) rc = run_consistent_p2g(c);
  if (!rc) rc = linsys_reserve<double>(c, c.L64);
  if (!rc && c.have32) rc = linsys_reserve<float>(c, c.L32);
  if (rc) return rc;
  run_initial_guess(c);
  run_renorm(c);
  rc = run_pn_layout(c);
  if (rc) return rc;
  run_count_terms(c);
  rc = read_dev_err(c);
  prof_end(c, MPM_PROF_PREP);
  if (rc) return rc;
  c.prepared = true;
  return MPM_OK;
}

int eval_residual(Ctx &c, double *rnorm) {
  run_point_eval(c, c.X);
  int rc = read_dev_err(c);
  if (rc) return rc;
  run_residual(c, c.X, c.R, 1);
  if (c.ninst > 1) {  // per-instance norms (h_inorm) for the Newton test
    k_inst_norm<<<c.ninst, 256, 0, c.st>>>(c.g, c.nb, c.inst, c.R, c.inorm);
    UPMPM_LAUNCH(c);
    cudaMemcpyAsync(c.h_inorm, c.inorm, sizeof(double) * c.ninst, cudaMemcpyDeviceToHost, c.st);
  }
  *rnorm = run_norm(c, c.R);  // synchronises
  if (!isfinite(*rnorm)) {
    c.last_error = "non-finite residual";
    return MPM_ERR_NONFINITE;
  }
  return MPM_OK;
}

// One Newton correction: assemble J (precision T), build the preconditioner
// on the unscaled blocks, scale, FGMRES, X += D x.  In the mixed mode a Krylov
// solve that stops at its iteration cap is an inexact Newton step: the FP64
// residual test of the Newton loop decides convergence.
template <typename T>
int newton_correction(Ctx &c, LinSys<T> &S, int k, int *its) {
  int rc;
  if (sizeof(T) == sizeof(double) && (rc = ensure_jacobian_staging(c))) return rc;
  if (sizeof(T) == sizeof(float) && c.s.hencky && (rc = ensure_jacobian_staging32(c))) return rc;
  run_jacobian<T>(c, S.val, 1);
  prof_begin(c, MPM_PROF_SETUP);
  if (c.opt.precond == MPM_PRECOND_SCHUR_MG) {
    const int lag = c.opt.precond_lag > 1 ? c.opt.precond_lag : 1;
    if (k % lag == 0) {
      // a step's first set-up rebuilds the coarse levels once per
      // precond_reuse steps (default: every step)
      const int reuse = c.opt.precond_reuse > 1 ? c.opt.precond_reuse : 1;
      const bool coarse = k > 0 || S.coarse_step < 0 || c.steps - S.coarse_step >= reuse;
      rc = schur_setup<T>(c, S, coarse);  // on the unscaled blocks
      if (rc) return rc;
    }
    run_scale_system<T>(c, S, c.R);
  } else {
    run_scale_system<T>(c, S, c.R);
    run_block_jacobi<T>(c, S);
  }
  prof_end(c, MPM_PROF_SETUP);
  rc = read_dev_err(c);
  if (rc) return rc;
  const bool inexact = sizeof(T) < sizeof(double);
  const double rtol = inexact ? fmax(c.opt.krylov_rtol, 1e-6) : c.opt.krylov_rtol;
  rc = run_fgmres<T>(c, S, rtol, c.opt.krylov_max, its);
  if (rc == MPM_ERR_KRYLOV_STAGNATED && inexact) rc = MPM_OK;
  if (rc) {
    if (rc == MPM_ERR_KRYLOV_STAGNATED) c.last_error = "FGMRES hit its iteration cap";
    else if (rc == MPM_ERR_NONFINITE) c.last_error = "non-finite value in FGMRES";
    return rc;
  }
  run_unscale_add<T>(c, S, c.X);
  return MPM_OK;
}

int newton(Ctx &c) {
  mpm_stats &st = c.stats;
  st.newton_iters = 0;
  st.krylov_total = 0;
  double rk;
  int rc = eval_residual(c, &rk);
  if (rc) return rc;
  const double r0 = rk;
  st.res_norm[0] = r0;
  double prev = r0;
  // batched contexts: every instance meets its own test (on its own norms);
  // an instance that has met it stays accepted while the others iterate
  const int ni = c.ninst;
  std::vector<double> ri0, riprev, ri;
  std::vector<char> accepted;
  if (ni > 1) {
    ri.resize(ni);
    for (int i = 0; i < ni; ++i) ri[i] = sqrt(c.h_inorm[i]);
    ri0 = ri;
    riprev = ri;
    accepted.assign(ni, 0);
  }
  auto done = [&](double r, double rp, double rz, int kk) {
    if (rz == 0.0 || r <= c.opt.newton_rtol * rz) return true;
    return c.opt.newton_stag > 0.0 && kk >= 2 && rp <= c.opt.newton_stag * rz && r > 0.5 * rp;
  };
  int k = 0;
  while (true) {
    if (ni > 1) {
      bool all = true;
      for (int i = 0; i < ni; ++i) {
        if (!accepted[i] && done(ri[i], riprev[i], ri0[i], k)) accepted[i] = 1;
        all = all && accepted[i];
      }
      if (all) break;
    } else if (done(rk, prev, r0, k)) {
      break;
    }
    if (k >= c.opt.newton_max || k >= MPM_MAX_NEWTON) {
      c.last_error = "Newton did not reach the residual tolerance";
      return MPM_ERR_NEWTON_DIVERGED;
    }
    int its = 0;
    rc = c.have32 ? newton_correction<float>(c, c.L32, k, &its) : newton_correction<double>(c, c.L64, k, &its);
    st.krylov_iters[k] = its;
    st.krylov_total += its;
    if (rc) return rc;
    prev = rk;
    rc = eval_residual(c, &rk);
    if (rc) return rc;
    if (ni > 1) {
      riprev = ri;
      for (int i = 0; i < ni; ++i) ri[i] = sqrt(c.h_inorm[i]);
    }
    ++k;
    st.res_norm[k] = rk;
    st.newton_iters = k;
  }
  return MPM_OK;
}

int do_step(Ctx &c, double dt, const mpm_loads *L, const mpm_bcs *B) {
  c.launches = 0;
  c.ev_used = 0;
  for (int k = 0; k < MPM_PROF_COUNT; ++k) {
    c.stats.prof_ms[k] = 0.0;
    c.stats.prof_launches[k] = 0;
  }
  int rc = prepare_step(c, dt, L, B);
  if (rc) return rc;
  rc = newton(c);
  if (rc) return rc;
  run_g2p(c);
  cudaMemcpyAsync(c.h_terms, c.terms, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.st);
  rc = read_dev_err(c);  // synchronises the stream
  if (rc) return rc;
  c.stats.jac_terms = (int64_t)c.h_terms[0];
  c.stats.jac_point_nodes = (int64_t)c.h_terms[1];
  prof_collect(c);
  c.prepared = false;
  c.t += dt;
  c.steps += 1;
  c.stats.steps = c.steps;
  c.stats.t = c.t;
  c.stats.nnzb = c.nnzb;
  c.stats.kernel_launches = c.launches;
  return MPM_OK;
}

void free_all(Ctx &c) {
  for (cudaEvent_t e : c.ev) cudaEventDestroy(e);
  c.ev.clear();
  linsys_free<double>(c.L64);
  linsys_free<float>(c.L32);
  float *fptrs[] = {c.sh_Sf, c.sh_dSf, c.sh_S0f, c.sh_nrmf, c.recf, c.pn32};
  for (float *p : fptrs)
    if (p) cudaFree(p);
  void *ptrs[] = {c.pf, c.pf_alt, c.pid, c.pid_alt, c.surf, c.surf_alt, c.cell, c.cell_tmp,
                  c.cell_start, c.cell_cursor, c.perm, c.sh_first, c.sh_cnt, c.sh_box, c.fb_key, c.fb_start, c.fb_cursor, c.fb_perm, c.fb_cmax, c.pn_cnt, c.pn_base, c.sh_S, c.sh_dS,
                  c.sh_S0, c.m, c.rec, c.pn, c.M, c.Pn, c.vn, c.an, c.pdn, c.pddn, c.phi, c.act, c.fsd, c.sh_nrm, c.fixed, c.u_fixed,
                  c.p_fixed, c.u_value, c.p_value, c.trac, c.trac_raw, c.flux, c.err, c.row_nnz,
                  c.row_ptr, c.row_of, c.col, c.row_mask, c.X, c.R, c.dX, c.stage, c.H, c.gvec,
                  c.cs, c.sn, c.yv, c.hcol, c.part, c.scal, c.mc, c.cm_buf, c.scan_tmp, c.terms, c.inst, c.inorm, c.node_inst, c.bk, c.bk_i};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c.h_inorm) cudaFreeHost(c.h_inorm);
  if (c.h_bk) cudaFreeHost(c.h_bk);
  if (c.h_err) cudaFreeHost(c.h_err);
  if (c.h_scalar) cudaFreeHost(c.h_scalar);
  if (c.h_terms) cudaFreeHost(c.h_terms);
  if (c.own_stream && c.st) cudaStreamDestroy(c.st);
  c.st = nullptr;
}

}  // namespace
}  // namespace upmpm

using namespace upmpm;

struct mpm_ctx {
  Ctx c;
};

namespace upmpm {
namespace {

// The context of one or several instances: grid is the background grid of the
// context, P / mat / permeability the points of all instances (instance-major,
// each in its own grid's coordinates), insts the instance table and pinst the
// instance of every point (NULL: all instance 0).
// Why the calling thread's last mpm_create / mpm_create_batch failed (its
// context is gone by then); empty after a successful create.
thread_local std::string g_create_error;

int create_fail(int rc, const char *why) {
  g_create_error = why;
  return rc;
}

// a context that failed part-way: keep its message, free it
int create_abort(mpm_ctx *h, int rc, const char *fallback) {
  g_create_error = h->c.last_error.empty() ? fallback : h->c.last_error;
  delete h;
  return rc;
}

int create_impl(const mpm_grid *grid, const mpm_particles *P, const mpm_material *mat,
                const double *permeability, const mpm_options *opt, const std::vector<InstDev> &insts,
                const int32_t *pinst, mpm_ctx **out) {
  constexpr int BAD = MPM_ERR_BAD_ARG;
  g_create_error.clear();
  if (!out) return create_fail(BAD, "out is NULL");
  *out = nullptr;
  if (!grid || !P || !mat || !permeability || !opt)
    return create_fail(BAD, "grid, particles, material, permeability and options must not be NULL");
  if (grid->dim != 2 && grid->dim != 3) return create_fail(BAD, "grid.dim must be 2 or 3");
  if (!(grid->h > 0.0)) return create_fail(BAD, "grid.h must be positive");
  if (P->n <= 0 || !P->x || !P->vol || !P->lp || !mat->E || !mat->nu)
    return create_fail(BAD, "need n > 0 points with x, vol, lp, E and nu");
  for (int k = 0; k < grid->dim; ++k)
    if (grid->ncell[k] < 1) return create_fail(BAD, "grid.ncell must be at least 1 on every axis");
  if (P->n > INT32_MAX / 2) return create_fail(BAD, "more than 2^30 points");
  if (P->n > INT32_MAX / pn_nslot(grid->dim)) return create_fail(BAD, "too many points for the Jacobian staging");
  if (opt->krylov_restart < 1 || opt->krylov_restart > 128)
    return create_fail(BAD, "krylov_restart must be in 1..128");
  if (opt->precond_lag < 0 || opt->precond_lag > MPM_MAX_NEWTON)
    return create_fail(BAD, "precond_lag must be in 0..MPM_MAX_NEWTON");
  if (opt->precond_reuse < 0 || opt->precond_reuse > 1000000)
    return create_fail(BAD, "precond_reuse must be in 0..1000000");
  if (opt->schur_approx < MPM_SCHUR_AUTO || opt->schur_approx > MPM_SCHUR_FIXED_STRESS)
    return create_fail(BAD, "unknown schur_approx");
  if (opt->tau_kind < MPM_TAU_WHITE || opt->tau_kind > MPM_TAU_MONFORTE) return create_fail(BAD, "unknown tau_kind");
  if (opt->permeability != MPM_PERM_CONSTANT && opt->permeability != MPM_PERM_KOZENY_CARMAN)
    return create_fail(BAD, "unknown permeability");
  if (opt->p2g_mass != MPM_P2G_LUMPED && opt->p2g_mass != MPM_P2G_CONSISTENT)
    return create_fail(BAD, "unknown p2g_mass");
  if (opt->model != MPM_MODEL_NEOHOOKE && opt->model != MPM_MODEL_HENCKY) return create_fail(BAD, "unknown model");
  if (opt->permeability == MPM_PERM_KOZENY_CARMAN && !(mat->phi0 > 0.0 && mat->phi0 < 1.0))
    return create_fail(BAD, "MPM_PERM_KOZENY_CARMAN needs 0 < material.phi0 < 1");
  // tau_M uses the Newmark parameters: dynamic steps only (Sec. 4.3)
  if (opt->stabilize && opt->tau_kind == MPM_TAU_MONFORTE && opt->scheme != MPM_NEWMARK)
    return create_fail(BAD, "MPM_TAU_MONFORTE needs the Newmark scheme");
  if (opt->precond != MPM_PRECOND_BLOCK_JACOBI && opt->precond != MPM_PRECOND_SCHUR_MG)
    return create_fail(BAD, "unknown precond");
  if (opt->schur_order != MPM_SCHUR_LOWER && opt->schur_order != MPM_SCHUR_UPPER)
    return create_fail(BAD, "unknown schur_order");
  if (opt->mg_sweeps < 0 || opt->mg_sweeps > 3) return create_fail(BAD, "mg_sweeps must be in 0..3");
  if (!(opt->mg_omega >= 0.0 && opt->mg_omega <= 1.0)) return create_fail(BAD, "mg_omega must be in [0, 1]");
  if (opt->precision != MPM_FP64 && opt->precision != MPM_MIXED) return create_fail(BAD, "unknown precision");
  if (P->n_surf < 0 || (P->n_surf > 0 && (!P->surf_id || !P->surf_normal || !P->surf_area)))
    return create_fail(BAD, "n_surf > 0 needs surf_id, surf_normal and surf_area");
  if (!(mat->mu_f > 0.0)) return create_fail(BAD, "material.mu_f must be positive");
  if (!(opt->min_volume_fraction >= 0.0)) return create_fail(BAD, "min_volume_fraction must be >= 0");
  // the points' own data: finite positions, positive volumes, a positive
  // Young's modulus with -1 < nu < 1/2, a non-negative permeability (the
  // initial pressure and the loads are not checked here: a non-finite value
  // there surfaces as MPM_ERR_NONFINITE at the first residual of a step)
  for (int64_t i = 0; i < P->n; ++i) {
    for (int k = 0; k < grid->dim; ++k)
      if (!isfinite(P->x[i * grid->dim + k])) return create_fail(BAD, "non-finite point position");
    if (!(P->vol[i] > 0.0) || !isfinite(P->vol[i])) return create_fail(BAD, "point volume must be positive and finite");
    if (!(mat->E[i] > 0.0) || !isfinite(mat->E[i])) return create_fail(BAD, "E must be positive and finite");
    if (!(mat->nu[i] > -1.0 && mat->nu[i] < 0.5)) return create_fail(BAD, "nu must lie in (-1, 1/2)");
    if (!(permeability[i] >= 0.0) || !isfinite(permeability[i]))
      return create_fail(BAD, "permeability must be non-negative and finite");
  }
  // every surface id must address an entry of the load arrays
  if (P->surf_id)
    for (int64_t i = 0; i < P->n; ++i)
      if (P->surf_id[i] < -1 || P->surf_id[i] >= P->n_surf)
        return create_fail(BAD, "surf_id outside -1..n_surf-1");

  mpm_ctx *h = new (std::nothrow) mpm_ctx();
  if (!h) return create_fail(MPM_ERR_NO_MEMORY, "out of host memory");
  Ctx &c = h->c;
  c.opt = *opt;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      c.nsm = nsm;
  }
  c.st = (cudaStream_t)opt->stream;
  if (!c.st) {
    // a stream of our own (blocking, so it stays ordered with the legacy
    // default stream); needed for CUDA graph capture
    if (cudaStreamCreate(&c.st) != cudaSuccess) return create_abort(h, MPM_ERR_CUDA, "cudaStreamCreate failed");
    c.own_stream = true;
  }
  c.d = grid->dim;
  c.nb = c.d + 1;
  c.shape = opt->shape;
  c.dyn = opt->scheme == MPM_NEWMARK;
  c.stabilize = opt->stabilize;
  c.tau_scale = opt->tau_scale;
  c.precision = opt->precision;
  c.m_restart = opt->krylov_restart;
  GridP &g = c.g;
  g.d = c.d;
  g.nnodes = 1;
  g.ncells = 1;
  for (int k = 0; k < 3; ++k) {
    const bool used = k < c.d;
    g.nc[k] = used ? grid->ncell[k] : 1;
    g.nn[k] = used ? grid->ncell[k] + 1 : 1;
    g.org[k] = used ? grid->origin[k] : 0.0;
    g.nnodes *= g.nn[k];
    g.ncells *= g.nc[k];
  }
  g.h = grid->h;
  if (g.nnodes > INT32_MAX / 16) return create_abort(h, MPM_ERR_BAD_ARG, "grid has more than 2^27 nodes");
  StepP &s = c.s;
  s.beta = opt->beta;
  s.gamma = opt->gamma;
  s.rho_f = mat->rho_f;
  s.rho_s = mat->rho_s;
  s.phi0 = mat->phi0;
  s.alpha_vis = c.dyn ? mat->alpha_vis : 0.0;
  s.phi_min = opt->min_volume_fraction;
  s.kozeny = opt->permeability == MPM_PERM_KOZENY_CARMAN;
  s.hencky = opt->model == MPM_MODEL_HENCKY;
  // the FP32 Jacobian's direct form has no Hencky tangent: staged only
  if (s.hencky) c.jac_cfg[1].form = Ctx::JAC_STAGED;
  for (int k = 0; k < 3; ++k) s.g[k] = k < c.d ? mat->g[k] : 0.0;
  c.n = P->n;
  c.n_surf = P->n_surf;
  c.ninst = (int)insts.size();
  c.inst_h = insts;

  const int64_t n = c.n, nn = g.nnodes, nc = g.ncells, N = (int64_t)c.nb * nn;
  const int d = c.d, nb = c.nb, m = c.m_restart;
  int rc = MPM_OK;
  auto A = [&](auto **p, int64_t cnt) {
    if (!rc) rc = dalloc(c, p, cnt);
  };
  A(&c.pf, PF_COUNT * n);
  A(&c.pf_alt, PF_COUNT * n);
  A(&c.pid, n);
  A(&c.pid_alt, n);
  A(&c.surf, n);
  A(&c.surf_alt, n);
  A(&c.cell, n);
  A(&c.cell_tmp, n);
  A(&c.cell_start, nc + 1);
  A(&c.cell_cursor, nc + 1);
  A(&c.perm, n);
  A(&c.sh_first, 3 * n);
  A(&c.sh_cnt, n);
  A(&c.sh_box, n);
  A(&c.fb_key, n);
  A(&c.fb_perm, n);
  A(&c.fb_start, nn + 1);
  A(&c.fb_cursor, nn + 1);
  A(&c.fb_cmax, 4);
  A(&c.pn_cnt, n + 1);
  A(&c.pn_base, n + 1);
  A(&c.sh_S, 3 * MAXS * n);
  A(&c.sh_dS, 3 * MAXS * n);
  A(&c.sh_S0, 3 * MAXS * n);
  A(&c.m, n);
  A(&c.rec, RC_COUNT * n);
  // the FP64 Jacobian's staging (allocated on first use in a mixed context,
  // whose Jacobian is FP32 and unstaged)
  A(&c.M, nn);
  A(&c.Pn, nn);
  A(&c.vn, d * nn);
  A(&c.an, d * nn);
  A(&c.pdn, nn);
  A(&c.pddn, nn);
  A(&c.phi, nn);
  A(&c.act, nn);
  A(&c.fsd, nn);
  A(&c.sh_nrm, 5 * n);
  A(&c.fixed, N);
  A(&c.u_fixed, d * nn);
  A(&c.p_fixed, nn);
  A(&c.u_value, d * nn);
  A(&c.p_value, nn);
  A(&c.trac, (int64_t)c.n_surf * d);
  A(&c.trac_raw, (int64_t)c.n_surf * d);
  A(&c.flux, c.n_surf);
  A(&c.err, 1);
  A(&c.row_nnz, nn + 1);
  A(&c.row_ptr, nn + 1);
  A(&c.row_mask, nn * 6);
  A(&c.X, N);
  A(&c.R, N);
  A(&c.dX, N);
  A(&c.stage, std::max<int64_t>(N, 9 * n));
  A(&c.H, (int64_t)(m + 1) * m);
  A(&c.gvec, m + 1);
  A(&c.cs, m);
  A(&c.sn, m);
  A(&c.yv, m);
  A(&c.hcol, 2 * 129);
  A(&c.part, 304 * 129);
  A(&c.scal, 8);
  c.scan_cap = 4096;
  A(&c.scan_tmp, c.scan_cap);
  c.have32 = c.precision == MPM_MIXED;
  if (c.have32) {
    auto F = [&](float **p, int64_t cnt) {
      if (!rc && cudaMalloc((void **)p, sizeof(float) * cnt) != cudaSuccess) rc = MPM_ERR_NO_MEMORY;
    };
    F(&c.sh_Sf, 3 * MAXS * n);
    F(&c.sh_dSf, 3 * MAXS * n);
    F(&c.sh_S0f, 3 * MAXS * n);
    F(&c.sh_nrmf, 5 * n);
    F(&c.recf, RC_F32 * n);
  }
  if (!rc) rc = linsys_alloc<double>(c, c.L64, !c.have32);
  if (!rc && c.have32) rc = linsys_alloc<float>(c, c.L32, true);
  if (!rc && cudaHostAlloc((void **)&c.h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess)
    rc = MPM_ERR_NO_MEMORY;
  if (!rc && cudaHostAlloc((void **)&c.h_scalar, 8 * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
    rc = MPM_ERR_NO_MEMORY;
  if (!rc && (cudaMalloc((void **)&c.terms, 2 * sizeof(unsigned long long)) != cudaSuccess ||
              cudaHostAlloc((void **)&c.h_terms, 2 * sizeof(unsigned long long), cudaHostAllocDefault) !=
                  cudaSuccess))
    rc = MPM_ERR_NO_MEMORY;
  A(&c.inst, c.ninst);
  A(&c.inorm, c.ninst);
  A(&c.node_inst, nn);
  // batched FGMRES state: H ((m+1) m), g, cs, sn, y (m+1 each), h1, h2 (PSTR
  // each), norm, scale, beta, target, residual per instance
  A(&c.bk, (int64_t)c.ninst * ((int64_t)(m + 1) * m + 5 * (m + 1) + 2 * 129 + 5));
  A(&c.bk_i, 2 * (int64_t)c.ninst + 1);
  if (!rc && (cudaHostAlloc((void **)&c.h_inorm, sizeof(double) * c.ninst, cudaHostAllocDefault) != cudaSuccess ||
              cudaHostAlloc((void **)&c.h_bk, sizeof(double) * 4, cudaHostAllocDefault) != cudaSuccess))
    rc = MPM_ERR_NO_MEMORY;
  if (rc) {
    free_all(c);
    return create_abort(h, rc, "device or pinned host memory allocation failed");
  }
  cudaMemcpyAsync(c.inst, c.inst_h.data(), sizeof(InstDev) * c.ninst, cudaMemcpyHostToDevice, c.st);
  {  // instance of every node (node boxes of the instances; -1 between them)
    std::vector<int32_t> ni(nn, -1);
    for (int i = 0; i < c.ninst; ++i) {
      const InstDev &I = c.inst_h[i];
      const int64_t m0 = I.nc[0] + 1, m1 = d > 1 ? I.nc[1] + 1 : 1, m2 = d > 2 ? I.nc[2] + 1 : 1;
      for (int64_t t = 0; t < m0 * m1 * m2; ++t) {
        const int64_t i0 = t % m0, i1 = (t / m0) % m1, i2 = t / (m0 * m1);
        ni[(i0 + I.off[0]) + (int64_t)g.nn[0] * ((i1 + I.off[1]) + (int64_t)g.nn[1] * (i2 + I.off[2]))] = i;
      }
    }
    cudaMemcpyAsync(c.node_inst, ni.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, c.st);
    cudaStreamSynchronize(c.st);  // ni is a host temporary
  }
  cudaMemsetAsync(c.err, 0, sizeof(int), c.st);
  cudaMemsetAsync(c.row_nnz, 0, sizeof(int32_t) * (nn + 1), c.st);  // [nn] stays 0 for the scan
  cudaMemsetAsync(c.u_fixed, 0, d * nn, c.st);
  cudaMemsetAsync(c.p_fixed, 0, nn, c.st);
  cudaMemsetAsync(c.u_value, 0, sizeof(double) * d * nn, c.st);
  cudaMemsetAsync(c.p_value, 0, sizeof(double) * nn, c.st);
  cudaMemsetAsync(c.vn, 0, sizeof(double) * d * nn, c.st);
  cudaMemsetAsync(c.an, 0, sizeof(double) * d * nn, c.st);
  cudaMemsetAsync(c.pdn, 0, sizeof(double) * nn, c.st);
  cudaMemsetAsync(c.pddn, 0, sizeof(double) * nn, c.st);
  if (c.n_surf > 0) {
    cudaMemsetAsync(c.trac, 0, sizeof(double) * c.n_surf * d, c.st);
    cudaMemsetAsync(c.trac_raw, 0, sizeof(double) * c.n_surf * d, c.st);
  }

  // stage the inputs on the device (temporary buffers), then initialise
  double *tmp = nullptr;
  const int64_t tcount = n * (4 * d + 7) + (n + 1) / 2;  // + instance ids (int32)
  rc = dalloc(c, &tmp, tcount);
  if (rc) {
    free_all(c);
    return create_abort(h, rc, "device memory allocation failed (point staging)");
  }
  double *dx = tmp, *dvol = dx + n * d, *dlp = dvol + n, *dp0 = dlp + n * d, *dv0 = dp0 + n,
         *dE = dv0 + n * d, *dnu = dE + n, *dk = dnu + n, *dsn = dk + n, *dsa = dsn + n * d;
  auto H2D = [&](double *dst, const double *src, int64_t cnt) {
    if (src) cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyHostToDevice, c.st);
  };
  H2D(dx, P->x, n * d);
  H2D(dvol, P->vol, n);
  H2D(dlp, P->lp, n * d);
  H2D(dp0, P->p0, n);
  H2D(dv0, P->v0, n * d);
  H2D(dE, mat->E, n);
  H2D(dnu, mat->nu, n);
  H2D(dk, permeability, n);
  H2D(dsn, P->surf_normal, n * d);
  H2D(dsa, P->surf_area, n);
  int32_t *dinst = reinterpret_cast<int32_t *>(dsa + n);
  if (pinst) cudaMemcpyAsync(dinst, pinst, sizeof(int32_t) * n, cudaMemcpyHostToDevice, c.st);
  if (P->surf_id)
    cudaMemcpyAsync(c.surf, P->surf_id, sizeof(int32_t) * n, cudaMemcpyHostToDevice, c.st);
  else
    cudaMemsetAsync(c.surf, 0xff, sizeof(int32_t) * n, c.st);
  if (d == 2)
    k_init<2><<<nblk(n), TPB, 0, c.st>>>(n, c.pf, dx, dvol, dlp, P->p0 ? dp0 : nullptr,
                                          P->v0 ? dv0 : nullptr, dE, dnu, dk,
                                          P->surf_normal ? dsn : nullptr, P->surf_area ? dsa : nullptr,
                                          mat->mu_f, c.tau_scale, c.stabilize, c.pid,
                                          pinst ? dinst : nullptr);
  else
    k_init<3><<<nblk(n), TPB, 0, c.st>>>(n, c.pf, dx, dvol, dlp, P->p0 ? dp0 : nullptr,
                                          P->v0 ? dv0 : nullptr, dE, dnu, dk,
                                          P->surf_normal ? dsn : nullptr, P->surf_area ? dsa : nullptr,
                                          mat->mu_f, c.tau_scale, c.stabilize, c.pid,
                                          pinst ? dinst : nullptr);
  cudaError_t e = cudaStreamSynchronize(c.st);
  cudaFree(tmp);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    rc = check_cuda(c, e, "create");
    free_all(c);
    return create_abort(h, rc, "CUDA error in create");
  }
  *out = h;
  return MPM_OK;
}

}  // namespace
}  // namespace upmpm


extern "C" {

void mpm_default_options(mpm_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->shape = MPM_SHAPE_GIMP;
  o->scheme = MPM_QUASISTATIC;
  o->beta = 0.3025;
  o->gamma = 0.6;
  o->stabilize = 1;
  o->tau_scale = 1.0;
  o->precision = MPM_FP64;
  o->newton_rtol = 1e-8;
  o->newton_max = 25;
  o->newton_stag = 0.0;
  o->krylov_rtol = 1e-8;
  o->krylov_restart = 120;
  o->krylov_max = 3000;
  o->precond = MPM_PRECOND_SCHUR_MG;
  o->min_volume_fraction = 1e-4;
  o->profile = 0;
  o->precond_lag = 2;
  o->precond_reuse = 0;
  o->schur_approx = MPM_SCHUR_AUTO;
  o->tau_kind = MPM_TAU_WHITE;
  o->permeability = MPM_PERM_CONSTANT;
  o->p2g_mass = MPM_P2G_LUMPED;
  o->model = MPM_MODEL_NEOHOOKE;
  o->stream = nullptr;
}

int mpm_create(const mpm_grid *grid, const mpm_particles *P, const mpm_material *mat,
               const double *permeability, const mpm_options *opt, mpm_ctx **out) {
  g_create_error.clear();
  if (!out) return create_fail(MPM_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  if (!grid) return create_fail(MPM_ERR_BAD_ARG, "grid is NULL");
  InstDev one{};
  for (int k = 0; k < 3; ++k) {
    const bool used = k < grid->dim;
    one.org[k] = used ? grid->origin[k] : 0.0;
    one.off[k] = 0;
    one.nc[k] = used ? grid->ncell[k] : 1;
  }
  return create_impl(grid, P, mat, permeability, opt, std::vector<InstDev>{one}, nullptr, out);
}

// ---- batched instances
int mpm_batch_pack(int32_t count, const mpm_grid *grids, int32_t *offsets, int32_t *ncell) {
  if (count < 1 || !grids || !offsets || !ncell) return MPM_ERR_BAD_ARG;
  const int d = grids[0].dim;
  if (d != 2 && d != 3) return MPM_ERR_BAD_ARG;
  double area = 0.0;
  int32_t wmax = 0, zmax = 1;
  for (int i = 0; i < count; ++i) {
    const mpm_grid &g = grids[i];
    if (g.dim != d || !(g.h > 0.0) || g.h != grids[0].h) return MPM_ERR_BAD_ARG;
    for (int k = 0; k < d; ++k)
      if (g.ncell[k] < 1 || g.ncell[k] > (1 << 20)) return MPM_ERR_BAD_ARG;
    area += (double)(g.ncell[0] + MPM_BATCH_GAP) * (double)(g.ncell[1] + MPM_BATCH_GAP);
    wmax = std::max(wmax, g.ncell[0]);
    if (d == 3) zmax = std::max(zmax, g.ncell[2]);
  }
  // shelves of width W ~ sqrt(total area): tallest instances first, left to
  // right, at least MPM_BATCH_GAP empty cells between neighbours
  const int64_t W = std::max<int64_t>((int64_t)ceil(sqrt(area)), wmax);
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (grids[a].ncell[1] != grids[b].ncell[1]) return grids[a].ncell[1] > grids[b].ncell[1];
    return grids[a].ncell[0] > grids[b].ncell[0];
  });
  int64_t x = 0, y = 0, shelf = 0, xmax = 0;
  for (int i : order) {
    const int64_t nx = grids[i].ncell[0], ny = grids[i].ncell[1];
    if (x > 0 && x + nx > W) {
      y += shelf + MPM_BATCH_GAP;
      x = 0;
      shelf = 0;
    }
    offsets[3 * i + 0] = (int32_t)x;
    offsets[3 * i + 1] = (int32_t)y;
    offsets[3 * i + 2] = 0;
    xmax = std::max(xmax, x + nx);
    x += nx + MPM_BATCH_GAP;
    shelf = std::max(shelf, ny);
  }
  const int64_t ny_all = y + shelf;
  if (xmax > INT32_MAX / 4 || ny_all > INT32_MAX / 4) return MPM_ERR_BAD_ARG;
  ncell[0] = (int32_t)xmax;
  ncell[1] = (int32_t)ny_all;
  ncell[2] = d == 3 ? zmax : 1;
  return MPM_OK;
}

int mpm_create_batch(int32_t count, const mpm_grid *grids, const mpm_particles *parts,
                     const mpm_material *mats, const double *const *permeability, const mpm_options *opt,
                     mpm_ctx **out) {
  g_create_error.clear();
  if (!out) return create_fail(MPM_ERR_BAD_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !grids || !parts || !mats || !permeability || !opt)
    return create_fail(MPM_ERR_BAD_ARG, "need count >= 1 and non-NULL grids, particles, materials, "
                                        "permeabilities and options");
  std::vector<int32_t> offs(3 * (size_t)count);
  mpm_grid big{};
  int rc = mpm_batch_pack(count, grids, offs.data(), big.ncell);
  if (rc) return create_fail(rc, "the grids cannot be packed (mixed dim or h, or an axis out of range)");
  const int d = grids[0].dim;
  big.dim = d;
  big.h = grids[0].h;
  // the material constants are shared; E, nu and k are per point
  const mpm_material &m0 = mats[0];
  for (int i = 1; i < count; ++i) {
    const mpm_material &m = mats[i];
    if (m.rho_s != m0.rho_s || m.rho_f != m0.rho_f || m.phi0 != m0.phi0 || m.mu_f != m0.mu_f ||
        m.alpha_vis != m0.alpha_vis || m.g[0] != m0.g[0] || m.g[1] != m0.g[1] || m.g[2] != m0.g[2])
      return create_fail(MPM_ERR_BAD_ARG, "the instances' material constants differ (only E, nu, k may)");
  }
  int64_t n = 0;
  int32_t nsurf = 0;
  bool any_p0 = false, any_v0 = false, any_surf = false;
  for (int i = 0; i < count; ++i) {
    const mpm_particles &P = parts[i];
    if (P.n <= 0 || !P.x || !P.vol || !P.lp || !mats[i].E || !mats[i].nu || !permeability[i])
      return create_fail(MPM_ERR_BAD_ARG, "an instance needs n > 0 points with x, vol, lp, E, nu and k");
    if (P.n_surf < 0 || (P.n_surf > 0 && (!P.surf_id || !P.surf_normal || !P.surf_area)))
      return create_fail(MPM_ERR_BAD_ARG, "n_surf > 0 needs surf_id, surf_normal and surf_area");
    if (P.surf_id)
      for (int64_t j = 0; j < P.n; ++j)
        if (P.surf_id[j] < -1 || P.surf_id[j] >= P.n_surf)
          return create_fail(MPM_ERR_BAD_ARG, "surf_id outside -1..n_surf-1");
    n += P.n;
    nsurf += P.n_surf;
    any_p0 |= P.p0 != nullptr;
    any_v0 |= P.v0 != nullptr;
    any_surf |= P.n_surf > 0;
  }
  if (n > INT32_MAX / 2) return create_fail(MPM_ERR_BAD_ARG, "more than 2^30 points");
  std::vector<double> x(n * d), vol(n), lp(n * d), p0(any_p0 ? n : 0), v0(any_v0 ? n * d : 0), E(n), nu(n), k(n),
      sn(any_surf ? n * d : 0), sa(any_surf ? n : 0);
  std::vector<int32_t> sid(n, -1), pinst(n);
  std::vector<InstDev> insts(count);
  int64_t at = 0;
  int32_t sbase = 0;
  for (int i = 0; i < count; ++i) {
    const mpm_particles &P = parts[i];
    const int64_t ni = P.n;
    std::copy(P.x, P.x + ni * d, x.begin() + at * d);
    std::copy(P.vol, P.vol + ni, vol.begin() + at);
    std::copy(P.lp, P.lp + ni * d, lp.begin() + at * d);
    if (P.p0) std::copy(P.p0, P.p0 + ni, p0.begin() + at);
    if (P.v0) std::copy(P.v0, P.v0 + ni * d, v0.begin() + at * d);
    std::copy(mats[i].E, mats[i].E + ni, E.begin() + at);
    std::copy(mats[i].nu, mats[i].nu + ni, nu.begin() + at);
    std::copy(permeability[i], permeability[i] + ni, k.begin() + at);
    if (P.n_surf > 0) {
      std::copy(P.surf_normal, P.surf_normal + ni * d, sn.begin() + at * d);
      std::copy(P.surf_area, P.surf_area + ni, sa.begin() + at);
      for (int64_t j = 0; j < ni; ++j) sid[at + j] = P.surf_id[j] < 0 ? -1 : P.surf_id[j] + sbase;
    }
    std::fill(pinst.begin() + at, pinst.begin() + at + ni, i);
    InstDev &I = insts[i];
    for (int a = 0; a < 3; ++a) {
      const bool used = a < d;
      I.org[a] = used ? grids[i].origin[a] : 0.0;
      I.off[a] = used ? offs[3 * i + a] : 0;
      I.nc[a] = used ? grids[i].ncell[a] : 1;
    }
    at += ni;
    sbase += P.n_surf;
  }
  mpm_particles all{};
  all.n = n;
  all.x = x.data();
  all.vol = vol.data();
  all.lp = lp.data();
  all.p0 = any_p0 ? p0.data() : nullptr;
  all.v0 = any_v0 ? v0.data() : nullptr;
  all.surf_id = any_surf ? sid.data() : nullptr;
  all.surf_normal = any_surf ? sn.data() : nullptr;
  all.surf_area = any_surf ? sa.data() : nullptr;
  all.n_surf = nsurf;
  mpm_material mat = m0;
  mat.E = E.data();
  mat.nu = nu.data();
  rc = create_impl(&big, &all, &mat, k.data(), opt, insts, pinst.data(), out);
  if (rc) return rc;
  Ctx &c = (*out)->c;
  const int64_t nn = c.g.nnodes;
  for (int i = 0; i < count; ++i) {
    c.inst_n.push_back(parts[i].n);
    c.inst_nsurf.push_back(parts[i].n_surf);
  }
  c.b_trac.assign((size_t)nsurf * d, 0.0);
  c.b_flux.assign(nsurf, 0.0);
  c.b_ufix.assign((size_t)nn * d, 0);
  c.b_uval.assign((size_t)nn * d, 0.0);
  c.b_pfix.assign(nn, 0);
  c.b_pval.assign(nn, 0.0);
  return MPM_OK;
}

int mpm_step_batch(mpm_ctx *h, double dt, const mpm_loads *loads, const mpm_bcs *bcs) {
  if (!h) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  const int d = c.d, ni = c.ninst;
  if ((int)c.inst_n.size() != ni) {
    c.last_error = "mpm_step_batch needs a context made by mpm_create_batch";
    return MPM_ERR_BAD_ARG;
  }
  mpm_loads L{};
  if (loads) {
    int64_t sb = 0;
    for (int i = 0; i < ni; ++i) {
      const int64_t ns = c.inst_nsurf[i];
      const mpm_loads &li = loads[i];
      if (li.traction)
        for (int64_t j = 0; j < ns * d; ++j) c.b_trac[sb * d + j] = li.scale * li.traction[j];
      if (li.flux) {
        for (int64_t j = 0; j < ns; ++j) c.b_flux[sb + j] = li.flux[j];
        c.b_has_flux = true;
      }
      sb += ns;
    }
    L.traction = c.b_trac.data();
    L.flux = c.b_has_flux ? c.b_flux.data() : nullptr;
    L.scale = 1.0;
  }
  mpm_bcs B{};
  if (bcs) {
    const GridP &g = c.g;
    for (int i = 0; i < ni; ++i) {
      const InstDev &I = c.inst_h[i];
      const mpm_bcs &bi = bcs[i];
      const int64_t m0 = I.nc[0] + 1, m1 = d > 1 ? I.nc[1] + 1 : 1, m2 = d > 2 ? I.nc[2] + 1 : 1;
      for (int64_t t = 0; t < m0 * m1 * m2; ++t) {
        const int64_t i0 = t % m0, i1 = (t / m0) % m1, i2 = t / (m0 * m1);
        const int64_t a = (i0 + I.off[0]) + (int64_t)g.nn[0] * ((i1 + I.off[1]) + (int64_t)g.nn[1] * (i2 + I.off[2]));
        for (int k = 0; k < d; ++k) {
          if (bi.u_fixed) c.b_ufix[a * d + k] = bi.u_fixed[t * d + k];
          if (bi.u_value) c.b_uval[a * d + k] = bi.u_value[t * d + k];
        }
        if (bi.p_fixed) c.b_pfix[a] = bi.p_fixed[t];
        if (bi.p_value) c.b_pval[a] = bi.p_value[t];
      }
    }
    B.u_fixed = c.b_ufix.data();
    B.u_value = c.b_uval.data();
    B.p_fixed = c.b_pfix.data();
    B.p_value = c.b_pval.data();
  }
  return do_step(c, dt, loads ? &L : nullptr, bcs ? &B : nullptr);
}

int mpm_step(mpm_ctx *h, double dt, const mpm_loads *loads, const mpm_bcs *bcs) {
  if (!h) return MPM_ERR_BAD_ARG;
  return do_step(h->c, dt, loads, bcs);
}

int mpm_read(const mpm_ctx *hc, mpm_particles_out *o) {
  if (!hc || !o) return MPM_ERR_BAD_ARG;
  Ctx &c = const_cast<mpm_ctx *>(hc)->c;
  const int64_t n = c.n;
  const int d = c.d;
  struct Item {
    double *dst;
    int f0, comps;
  } items[] = {{o->x, PF_X, d}, {o->u, PF_U, d}, {o->p, PF_P, 1}, {o->v, PF_VEL, d},
               {o->a, PF_ACC, d}, {o->F, PF_F, d * d}, {o->V, PF_V, 1}, {o->lp, PF_LP, d},
               {o->pd, PF_PD, 1}, {o->pdd, PF_PDD, 1}};
  for (const Item &it : items) {
    if (!it.dst) continue;
    k_read_field<<<nblk(n), TPB, 0, c.st>>>(n, c.pf, it.f0, it.comps, c.pid, c.stage);
    cudaMemcpyAsync(it.dst, c.stage, sizeof(double) * n * it.comps, cudaMemcpyDeviceToHost, c.st);
    cudaError_t e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return check_cuda(c, e, "read");
  }
  return check_cuda(c, cudaGetLastError(), "read");
}

int mpm_restore(mpm_ctx *h, const mpm_particles_out *st, double t, int64_t steps) {
  if (!h) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  if (!st || !(t >= 0.0) || steps < 0) {
    c.last_error = "mpm_restore needs a state, t >= 0 and steps >= 0";
    return MPM_ERR_BAD_ARG;
  }
  const int64_t n = c.n;
  const int d = c.d;
  struct Item {
    const double *src;
    int f0, comps;
  } items[] = {{st->x, PF_X, d}, {st->u, PF_U, d}, {st->p, PF_P, 1}, {st->v, PF_VEL, d},
               {st->a, PF_ACC, d}, {st->F, PF_F, d * d}, {st->V, PF_V, 1}, {st->lp, PF_LP, d},
               {st->pd, PF_PD, 1}, {st->pdd, PF_PDD, 1}};
  for (const Item &it : items) {
    if (!it.src) continue;
    cudaMemcpyAsync(c.stage, it.src, sizeof(double) * n * it.comps, cudaMemcpyHostToDevice, c.st);
    k_write_field<<<nblk(n), TPB, 0, c.st>>>(n, c.pf, it.f0, it.comps, c.pid, c.stage);
    cudaError_t e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return check_cuda(c, e, "restore");
  }
  c.t = t;
  c.steps = steps;
  c.stats.t = t;
  c.stats.steps = steps;
  c.prepared = false;
  return check_cuda(c, cudaGetLastError(), "restore");
}

int mpm_get_stats(const mpm_ctx *h, mpm_stats *s) {
  if (!h || !s) return MPM_ERR_BAD_ARG;
  *s = h->c.stats;
  return MPM_OK;
}

const char *mpm_last_error(const mpm_ctx *h) {
  if (!h) return g_create_error.empty() ? "null context" : g_create_error.c_str();
  return h->c.last_error.c_str();
}

void mpm_destroy(mpm_ctx *h) {
  if (!h) return;
  cudaStreamSynchronize(h->c.st);
  free_all(h->c);
  delete h;
}

int mpm_debug_bin(mpm_ctx *h, int32_t *cell, int64_t *order) {
  if (!h || !cell || !order) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  int rc = run_binning(c);
  if (rc) return rc;
  int32_t *tmp = reinterpret_cast<int32_t *>(c.stage);
  k_read_cells<<<nblk(c.n), TPB, 0, c.st>>>(c.n, c.cell, c.pid, tmp);
  cudaMemcpyAsync(cell, tmp, sizeof(int32_t) * c.n, cudaMemcpyDeviceToHost, c.st);
  cudaMemcpyAsync(order, c.pid, sizeof(int64_t) * c.n, cudaMemcpyDeviceToHost, c.st);
  return check_cuda(c, cudaStreamSynchronize(c.st), "debug_bin");
}

int mpm_debug_prepare(mpm_ctx *h, double dt, const mpm_loads *loads, const mpm_bcs *bcs) {
  if (!h) return MPM_ERR_BAD_ARG;
  return prepare_step(h->c, dt, loads, bcs);
}

int64_t mpm_debug_pattern(mpm_ctx *h, int64_t *row_ptr, int32_t *col_idx, int64_t cap) {
  if (!h || !row_ptr) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  if (!c.prepared) {
    c.last_error = "no step prepared: call mpm_debug_prepare first";
    return MPM_ERR_BAD_ARG;
  }
  const int64_t nn = c.g.nnodes;
  int32_t *tmp = new (std::nothrow) int32_t[nn + 1];
  if (!tmp) return MPM_ERR_NO_MEMORY;
  cudaMemcpyAsync(tmp, c.row_ptr, sizeof(int32_t) * (nn + 1), cudaMemcpyDeviceToHost, c.st);
  cudaError_t e = cudaStreamSynchronize(c.st);
  for (int64_t i = 0; i <= nn; ++i) row_ptr[i] = tmp[i];
  delete[] tmp;
  if (e != cudaSuccess) return check_cuda(c, e, "debug_pattern");
  if (col_idx) {
    if (cap < c.nnzb) {
      c.last_error = "col_idx holds fewer entries than the pattern's block count";
      return MPM_ERR_BAD_ARG;
    }
    cudaMemcpyAsync(col_idx, c.col, sizeof(int32_t) * c.nnzb, cudaMemcpyDeviceToHost, c.st);
    e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return check_cuda(c, e, "debug_pattern");
  }
  return c.nnzb;
}

int mpm_debug_nodal(mpm_ctx *h, double *M, double *Pn, double *phi) {
  if (!h) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  if (!c.prepared) {
    c.last_error = "no step prepared: call mpm_debug_prepare first";
    return MPM_ERR_BAD_ARG;
  }
  if (M) cudaMemcpyAsync(M, c.M, sizeof(double) * c.g.nnodes, cudaMemcpyDeviceToHost, c.st);
  if (Pn) cudaMemcpyAsync(Pn, c.Pn, sizeof(double) * c.g.nnodes, cudaMemcpyDeviceToHost, c.st);
  if (phi) cudaMemcpyAsync(phi, c.phi, sizeof(double) * c.g.nnodes, cudaMemcpyDeviceToHost, c.st);
  return check_cuda(c, cudaStreamSynchronize(c.st), "debug_nodal");
}

int mpm_debug_eval(mpm_ctx *h, const double *X, double *R, double *Jv, int32_t apply_bc) {
  if (!h || !X || !R) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  if (!c.prepared) {
    c.last_error = "no step prepared: call mpm_debug_prepare first";
    return MPM_ERR_BAD_ARG;
  }
  const int64_t N = c.N();
  cudaMemcpyAsync(c.dX, X, sizeof(double) * N, cudaMemcpyHostToDevice, c.st);
  run_point_eval(c, c.dX);
  int rc = read_dev_err(c);
  if (rc) return rc;
  run_residual(c, c.dX, c.R, apply_bc);
  cudaMemcpyAsync(R, c.R, sizeof(double) * N, cudaMemcpyDeviceToHost, c.st);
  if (Jv) {
    rc = ensure_jacobian_staging(c);
    if (rc) return rc;
    run_jacobian<double>(c, c.L64.val, apply_bc);
    cudaMemcpyAsync(Jv, c.L64.val, sizeof(double) * c.nnzb * c.nb * c.nb, cudaMemcpyDeviceToHost, c.st);
  }
  return check_cuda(c, cudaStreamSynchronize(c.st), "debug_eval");
}

int mpm_debug_jacobian32(mpm_ctx *h, const double *X, int32_t form, int32_t tpb, float *Jv, int32_t apply_bc) {
  if (!h || !X || !Jv) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  if (!c.prepared) {
    c.last_error = "no step prepared: call mpm_debug_prepare first";
    return MPM_ERR_BAD_ARG;
  }
  if (!c.have32) {
    c.last_error = "the FP32 Jacobian exists in mixed-precision contexts only";
    return MPM_ERR_BAD_ARG;
  }
  if (form < 0 || form >= Ctx::JAC_FORMS || (tpb != 64 && tpb != 128 && tpb != 256)) {
    c.last_error = "form must be 0 or 1 and tpb 64, 128 or 256";
    return MPM_ERR_BAD_ARG;
  }
  if (c.s.hencky && form == Ctx::JAC_DIRECT) {
    c.last_error = "the direct FP32 Jacobian has no Hencky tangent: form 1 only";
    return MPM_ERR_BAD_ARG;
  }
  const int64_t N = c.N();
  cudaMemcpyAsync(c.dX, X, sizeof(double) * N, cudaMemcpyHostToDevice, c.st);
  run_point_eval(c, c.dX);
  int rc = read_dev_err(c);
  if (rc) return rc;
  rc = run_jacobian32_form(c, c.L32.val, apply_bc, form, tpb);
  if (rc) return rc;
  cudaMemcpyAsync(Jv, c.L32.val, sizeof(float) * c.nnzb * c.nb * c.nb, cudaMemcpyDeviceToHost, c.st);
  return check_cuda(c, cudaStreamSynchronize(c.st), "debug_jacobian32");
}

int mpm_debug_precond(mpm_ctx *h, const double *X, const double *v, double *z) {
  if (!h || !X || !v || !z) return MPM_ERR_BAD_ARG;
  Ctx &c = h->c;
  if (!c.prepared) {
    c.last_error = "no step prepared: call mpm_debug_prepare first";
    return MPM_ERR_BAD_ARG;
  }
  const int64_t N = c.N();
  cudaMemcpyAsync(c.X, X, sizeof(double) * N, cudaMemcpyHostToDevice, c.st);
  run_point_eval(c, c.X);
  int rc = read_dev_err(c);
  if (rc) return rc;
  run_residual(c, c.X, c.R, 1);
  LinSys<double> &S = c.L64;
  rc = ensure_jacobian_staging(c);
  if (rc) return rc;
  run_jacobian<double>(c, S.val, 1);
  if (c.opt.precond == MPM_PRECOND_SCHUR_MG) {
    rc = schur_setup<double>(c, S);
    if (rc) return rc;
    run_scale_system<double>(c, S, c.R);
  } else {
    run_scale_system<double>(c, S, c.R);
    run_block_jacobi<double>(c, S);
  }
  cudaMemcpyAsync(S.w, v, sizeof(double) * N, cudaMemcpyHostToDevice, c.st);
  run_precond<double>(c, S, S.w, S.x);
  cudaMemcpyAsync(z, S.x, sizeof(double) * N, cudaMemcpyDeviceToHost, c.st);
  return check_cuda(c, cudaStreamSynchronize(c.st), "debug_precond");
}

}  // extern "C"
