// mpm_assemble.cu -- Stage 2 evaluation of the discrete equations:
//   sparsity of the block Jacobian (node b couples with node a iff one point
//   has both in its support),
//   per-point kinematics, Kirchhoff stress, Darcy flux and PPP terms of the
//   current Newton iterate (Sec. 3.3 pull-back to t_n),
//   residual R = [R_mom; R_mass + R_stab] (Eqs. residual-momentum,
//   residual-mass, stab-term-ppp) gathered per node row,
//   Jacobian blocks [A B1; B2 C + C_stab] (Eq. jacobian-system-stabilized-ppp)
//   gathered per block, with the Newmark linearization of Eq.
//   newmark-linearization and delta ln J = div u for the quasi-static form.
//
// Design: gather, not scatter.  Points are cell-sorted, so the points that
// can touch node a live in a small box of cells around it; the pattern, the
// consistent mass and the Jacobian walk instead the first-node bins (the
// points indexed by the first node of their support box, built per step),
// whose box around a node (or a pair of nodes) is one narrower per axis,
// fewer candidates for the kernels that read little per point or stage their
// reads (the residual, which reads many record fields of each point, keeps the
// cells' contiguous runs of points).  The residual is
// computed by one thread per node row and each Jacobian block by one thread,
// each summing its points in a fixed order: no floating-point atomics, results
// are deterministic, and every (point, a, b) block term is computed exactly
// once.  Per-point quantities that do not depend on (a, b) are computed once
// per Newton iterate by k_point_eval and stored as structure-of-arrays
// records.
#include <math.h>

#include "mpm_internal.cuh"

namespace upmpm {

namespace {

constexpr int TPB = 256;
inline int nblk(int64_t n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

constexpr int MASKW = PATTERN_MASK_WORDS;  // 7^3 = 343 offsets in [-3, 3]^3

// Support box of point q along each axis, and whether node coordinate ac lies in
// it (off = slot of that node).
// The same from the point's packed box word (sh_box, written with the
// renormalisation flag at the end of the step's set-up).
template <int D>
__device__ inline bool in_box4(const int4 bx, const int ac[3], int off[3]) {
  const int first[3] = {bx.x, bx.y, bx.z};
  off[0] = off[1] = off[2] = 0;
  for (int k = 0; k < D; ++k) {
    const int o = ac[k] - first[k];
    if (o < 0 || o >= unpack_cnt(bx.w, k)) return false;
    off[k] = o;
  }
  return true;
}

template <int D>
__device__ inline bool in_box(const DevView &v, int64_t q, const int ac[3], int off[3]) {
  const int64_t n = v.n;
  const int packed = v.sh_cnt[q];
  off[0] = off[1] = off[2] = 0;
  for (int k = 0; k < D; ++k) {
    const int o = ac[k] - v.sh_first[k * n + q];
    if (o < 0 || o >= unpack_cnt(packed, k)) return false;
    off[k] = o;
  }
  return true;
}

// ---- Hencky elasticity (Sec. 2.2): tau' = lambda ln J 1 + G ln b.  With
// b = sum_A x_A n_A n_A, eps_A = ln(x_A) / 2, tau_A = lambda sum_B eps_B +
// 2 G eps_A, the spatial tangent (L_v tau' = c : d) is
//   c = sum_AB (lambda + kappa_A delta_AB) m_A (x) m_B
//     + sum_{A != B} theta_AB (m_AB (x) m_AB + m_AB (x) m_BA),
// kappa_A = 2G - 2 tau_A, theta_AB = (tau_A x_B - tau_B x_A) / (x_A - x_B)
// = G log1p(r) / r - tau_B with r = x_A / x_B - 1 (no cancellation, limit
// G - tau_A at equal stretches); m_A = n_A n_A, m_AB = n_A n_B.  In plane
// strain b is the in-plane block (third stretch 1).
// Cyclic Jacobi rotations: A = Q diag(w) Q^T (columns of Q the eigenvectors).
template <int D>
__device__ inline void sym_eig(const double *A, double w[3], double Q[9]) {
  double M[3][3];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      M[i][j] = A[i * D + j];
      Q[i * D + j] = i == j ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 20; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < D; ++i) {
      diag += M[i][i] * M[i][i];
      for (int j = i + 1; j < D; ++j) off += M[i][j] * M[i][j];
    }
    if (off <= 1e-36 * diag) break;
    for (int p = 0; p < D; ++p)
      for (int q = p + 1; q < D; ++q) {
        if (M[p][q] == 0.0) continue;
        const double th = 0.5 * atan2(2.0 * M[p][q], M[q][q] - M[p][p]);
        const double c = cos(th), s = sin(th);
        for (int k = 0; k < D; ++k) {
          const double mkp = M[k][p], mkq = M[k][q];
          M[k][p] = c * mkp - s * mkq;
          M[k][q] = s * mkp + c * mkq;
        }
        for (int k = 0; k < D; ++k) {
          const double mpk = M[p][k], mqk = M[q][k];
          M[p][k] = c * mpk - s * mqk;
          M[q][k] = s * mpk + c * mqk;
        }
        for (int k = 0; k < D; ++k) {
          const double qkp = Q[k * D + p], qkq = Q[k * D + q];
          Q[k * D + p] = c * qkp - s * qkq;
          Q[k * D + q] = s * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < D; ++i) w[i] = M[i][i];
}

__device__ inline double log1p_ratio(double r) {
  return fabs(r) > 1e-6 ? log1p(r) / r : 1.0 - r / 2.0 + r * r / 3.0;
}

// slot of the pair (A, B), A < B, among (0,1), (0,2), (1,2)
__device__ inline int pair_index(int A, int B) { return A + B - 1; }

// ---------------------------------------------------------------- pattern
template <int D, bool GIMP>
__global__ void k_pattern_count(GridP g, DevView v, uint64_t *__restrict__ mask,
                                int32_t *__restrict__ row_nnz) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  int ac[3];
  node_coords(g, a, ac);
  uint64_t mk[MASKW] = {0, 0, 0, 0, 0, 0};
  {  // self coupling
    const int bit = 3 + 7 * (D > 1 ? 3 : 0) + 49 * (D > 2 ? 3 : 0);
    mk[bit >> 6] |= 1ull << (bit & 63);
  }
  int lo[3], hi[3];
  fb_window<D>(v.fb_cmax, ac, ac, lo, hi);
  const int64_t n = v.n;
  for (int f2 = lo[2]; f2 <= hi[2]; ++f2)
    for (int f1 = lo[1]; f1 <= hi[1]; ++f1) {
      int32_t ib, ie;
      fb_run(g, v.fb_start, lo[0], hi[0], f1, f2, ib, ie);
      for (int32_t i = ib; i < ie; ++i) {
        const int32_t q = v.fb_perm[i];
        int off[3];
        if (!in_box<D>(v, q, ac, off)) continue;
        const int packed = v.sh_cnt[q];
        int ob[3] = {0, 0, 0}, oe[3] = {0, 0, 0};
        for (int k = 0; k < D; ++k) {
          ob[k] = v.sh_first[k * n + q] - ac[k];
          oe[k] = ob[k] + unpack_cnt(packed, k) - 1;
        }
        for (int o2 = ob[2]; o2 <= oe[2]; ++o2)
          for (int o1 = ob[1]; o1 <= oe[1]; ++o1)
            for (int o0 = ob[0]; o0 <= oe[0]; ++o0) {
              const int bit = (o0 + 3) + 7 * (D > 1 ? o1 + 3 : 0) + 49 * (D > 2 ? o2 + 3 : 0);
              mk[bit >> 6] |= 1ull << (bit & 63);
            }
      }
    }
  int cnt = 0;
  for (int w = 0; w < MASKW; ++w) {
    mask[a * MASKW + w] = mk[w];
    cnt += __popcll(mk[w]);
  }
  row_nnz[a] = cnt;
}

// Offsets in ascending bit order are ascending node indices (the z offset is
// most significant, then y, then x), so each row's columns come out sorted.
template <int D>
__global__ void k_pattern_fill(GridP g, const uint64_t *__restrict__ mask,
                               const int32_t *__restrict__ row_ptr, int32_t *__restrict__ col,
                               int32_t *__restrict__ row_of) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  int ac[3];
  node_coords(g, a, ac);
  int32_t pos = row_ptr[a];
  for (int w = 0; w < MASKW; ++w) {
    uint64_t mk = mask[a * MASKW + w];
    while (mk) {
      const int bit = w * 64 + __ffsll((long long)mk) - 1;
      mk &= mk - 1;
      const int o0 = bit % 7 - 3, o1 = (bit / 7) % 7 - 3, o2 = bit / 49 - 3;
      const int bc[3] = {ac[0] + o0, ac[1] + (D > 1 ? o1 : 0), ac[2] + (D > 2 ? o2 : 0)};
      col[pos] = (int32_t)node_index(g, bc);
      row_of[pos] = (int32_t)a;
      ++pos;
    }
  }
}

// ---------------------------------------------------------------- Dirichlet
// Fixed DOFs: Dirichlet data, and every DOF of an inactive node, i.e. a node
// whose volume fraction sum_p S_ip V_p / h^d does not exceed phi_min (a
// support reached only by a sliver of a GIMP domain carries no stiffness,
// mass or storage worth an unknown and would leave the system near-singular).
// Initial Newton guess: dU = prescribed increment or 0, P = p^ or P_n.
template <int D>
__global__ void k_initial_guess(GridP g, double phi_min, DevView v, double *__restrict__ X) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  constexpr int NB = D + 1;
  const bool inactive = !(v.M[a] > 0.0) || !(v.phi[a] > phi_min);
  v.act[a] = inactive ? 0 : 1;
  for (int k = 0; k < D; ++k) {
    const bool uf = v.u_fixed[a * D + k] != 0;
    v.fixed[a * NB + k] = (inactive || uf) ? 1 : 0;
    X[a * NB + k] = inactive ? 0.0 : (uf ? v.u_value[a * D + k] : 0.0);
  }
  const bool pfx = v.p_fixed[a] != 0;
  v.fixed[a * NB + D] = (inactive || pfx) ? 1 : 0;
  X[a * NB + D] = inactive ? 0.0 : (pfx ? v.p_value[a] : v.Pn[a]);
}

// Points whose support box holds an inactive node get their basis
// renormalised over the active box nodes (see basis_at).
// Fixed-stress term of the pressure Schur complement, lumped per node:
// fsd_a = sum_p S_ap b2_p vol_p / (cs_p K_p), K = lambda + 2 (G - lambda ln J) / d
// (the drained bulk modulus of the current records).  Node-centric gather in
// (cell, id) order: these gathers read many record fields per point, and the
// cells' contiguous runs of points serve them better than the first-node bins.
template <int D, bool GIMP>
__global__ void k_fs_diag(GridP g, DevView v, double *__restrict__ out) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  const int64_t n = v.n;
  int ac[3];
  node_coords(g, a, ac);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) cand_range<GIMP>(ac[k], g.nc[k], lo[k], hi[k]);
  const double *rec = v.rec;
  double acc = 0.0;
  for (int c2 = lo[2]; c2 <= hi[2]; ++c2)
    for (int c1 = lo[1]; c1 <= hi[1]; ++c1)
      for (int c0 = lo[0]; c0 <= hi[0]; ++c0) {
        const int64_t cid = cell_index(g, c0, c1, c2);
        for (int32_t q = v.cell_start[cid]; q < v.cell_start[cid + 1]; ++q) {
          int off[3];
          if (!in_box<D>(v, q, ac, off)) continue;
          double Sa, S0a, Gn[3];
          basis_at<D>(v, q, off, a, Sa, S0a, Gn);
          const double K = rec[RC_LAM * n + q] + 2.0 * rec[RC_MUP * n + q] / D;
          acc += Sa * rec[RC_B2 * n + q] * rec[RC_VOL * n + q] / (rec[RC_CS * n + q] * K);
        }
      }
  out[a] = acc;
}

// Work count of the Jacobian assembly: n_p active nodes in point p's support
// give n_p^2 (point, a, b) terms and n_p (point, node) terms.
template <int D>
__global__ void k_count_terms(GridP g, DevView v, unsigned long long *__restrict__ terms) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = v.n;
  unsigned long long np = 0;
  if (p < n) {
    const int packed = v.sh_cnt[p] & ~RENORM_BIT;
    int f[3], cn[3];
    for (int k = 0; k < 3; ++k) {
      f[k] = v.sh_first[k * n + p];
      cn[k] = unpack_cnt(packed, k);
    }
    for (int s2 = 0; s2 < cn[2]; ++s2)
      for (int s1 = 0; s1 < cn[1]; ++s1)
        for (int s0 = 0; s0 < cn[0]; ++s0) {
          const int nc3[3] = {f[0] + s0, f[1] + s1, f[2] + s2};
          np += v.act[node_index(g, nc3)] ? 1 : 0;
        }
  }
  unsigned long long sq = np * np;
  for (int o = 16; o > 0; o >>= 1) {
    np += __shfl_xor_sync(0xffffffffu, np, o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&terms[0], sq);
    atomicAdd(&terms[1], np);
  }
}

template <int D>
__global__ void k_renorm(GridP g, DevView v) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = v.n;
  if (p >= n) return;
  int packed = v.sh_cnt[p] & ~RENORM_BIT;
  int f[3], cn[3];
  for (int k = 0; k < 3; ++k) {
    f[k] = v.sh_first[k * n + p];
    cn[k] = unpack_cnt(packed, k);
  }
  bool any = false;
  double sum = 0.0, sum0 = 0.0, gs[3] = {0.0, 0.0, 0.0};
  for (int s2 = 0; s2 < cn[2]; ++s2)
    for (int s1 = 0; s1 < cn[1]; ++s1)
      for (int s0 = 0; s0 < cn[0]; ++s0) {
        const int nc3[3] = {f[0] + s0, f[1] + s1, f[2] + s2};
        const int64_t a = node_index(g, nc3);
        if (!v.act[a]) {
          any = true;
          continue;
        }
        double s[3] = {1.0, 1.0, 1.0}, ds[3] = {0.0, 0.0, 0.0}, z[3] = {1.0, 1.0, 1.0};
        const int sl[3] = {s0, s1, s2};
        for (int k = 0; k < D; ++k) {
          s[k] = v.sh_S[(k * MAXS + sl[k]) * n + p];
          ds[k] = v.sh_dS[(k * MAXS + sl[k]) * n + p];
          z[k] = v.sh_S0[(k * MAXS + sl[k]) * n + p];
        }
        sum += s[0] * s[1] * s[2];
        sum0 += z[0] * z[1] * z[2];
        gs[0] += ds[0] * s[1] * s[2];
        gs[1] += s[0] * ds[1] * s[2];
        gs[2] += s[0] * s[1] * ds[2];
      }
  if (any) {
    v.sh_nrm[0 * n + p] = 1.0 / sum;
    for (int k = 0; k < 3; ++k) v.sh_nrm[(1 + k) * n + p] = gs[k];
    v.sh_nrm[4 * n + p] = 1.0 / sum0;
    if (v.sh_nrmf)
      for (int k = 0; k < 5; ++k) v.sh_nrmf[k * n + p] = (float)v.sh_nrm[k * n + p];
    packed |= RENORM_BIT;
  }
  v.sh_cnt[p] = packed;
  v.sh_box[p] = make_int4(f[0], f[1], f[2], packed);
}

// ---------------------------------------------------------------- points
template <int D, bool DYN>
__global__ void k_point_eval(GridP g, StepP s, DevView v, const double *__restrict__ X) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = v.n;
  if (p >= n) return;
  constexpr int NB = D + 1;
  const int64_t nn = g.nnodes;
  const double dt = s.dt, b = s.beta, gm = s.gamma;
  const int packed = v.sh_cnt[p];
  int f[3], cn[3];
  for (int k = 0; k < 3; ++k) {
    f[k] = v.sh_first[k * n + p];
    cn[k] = unpack_cnt(packed, k);
  }
  double dF[9] = {0}, gPn[3] = {0, 0, 0}, gVn[9] = {0}, ah[3] = {0, 0, 0};
  double ph = 0.0, pdev = 0.0;
  for (int k = 0; k < D; ++k) dF[k * D + k] = 1.0;
  for (int s2 = 0; s2 < cn[2]; ++s2)
    for (int s1 = 0; s1 < cn[1]; ++s1)
      for (int s0 = 0; s0 < cn[0]; ++s0) {
        const int off[3] = {s0, s1, s2};
        const int nc3[3] = {f[0] + s0, f[1] + s1, f[2] + s2};
        const int64_t a = node_index(g, nc3);
        double Sa, S0a, Gn[3];
        basis_at<D>(v, p, off, a, Sa, S0a, Gn);
        const double P = X[a * NB + D];
        for (int i = 0; i < D; ++i) {
          const double dU = X[a * NB + i];
          for (int k = 0; k < D; ++k) dF[i * D + k] += dU * Gn[k];
        }
        ph += Sa * P;
        for (int k = 0; k < D; ++k) gPn[k] += P * Gn[k];
        if (DYN) {
          for (int i = 0; i < D; ++i) {
            const double dU = X[a * NB + i];
            const double vn = v.vn[i * nn + a], an = v.an[i * nn + a];
            const double aa = dU / (b * dt * dt) - vn / (b * dt) + (1.0 - 1.0 / (2.0 * b)) * an;
            const double va = gm / (b * dt) * dU + (1.0 - gm / b) * vn + (1.0 - gm / (2.0 * b)) * dt * an;
            ah[i] += Sa * aa;
            for (int k = 0; k < D; ++k) gVn[i * D + k] += va * Gn[k];
          }
          const double pda = gm / (b * dt) * (P - v.Pn[a]) + (1.0 - gm / b) * v.pdn[a] +
                             (1.0 - gm / (2.0 * b)) * dt * v.pddn[a];
          pdev += (Sa - S0a) * pda;
        } else {
          pdev += (Sa - S0a) * (P - v.Pn[a]) / dt;
        }
      }
  const double dJ = det_d<D>(dF);
  if (!(dJ > 0.0)) {
    atomicOr(v.err, DE_NEG_J);
    return;
  }
  double fi[9], Fn[9], F[9], bl[9];
  inv_d<D>(dF, fi);
  const double *pf = v.pf;
  for (int i = 0; i < D * D; ++i) Fn[i] = pf[(PF_F + i) * n + p];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int k = 0; k < D; ++k) acc += dF[i * D + k] * Fn[k * D + j];
      F[i * D + j] = acc;
    }
  const double Jn = det_d<D>(Fn), J = det_d<D>(F);
  if (!(J > 0.0)) {
    atomicOr(v.err, DE_NEG_J);
    return;
  }
  const double lnJ = log(J);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int k = 0; k < D; ++k) acc += F[i * D + k] * F[j * D + k];
      bl[i * D + j] = acc;
    }
  const double lam = pf[PF_LAM * n + p], G = pf[PF_G * n + p];
  const double Vn = pf[PF_V * n + p], kap = pf[PF_KAP * n + p], tau = pf[PF_TAU * n + p];
  const double mu_p = G - lam * lnJ;
  const double vol = dJ * Vn;
  double *rec = v.rec;
  float *recf = v.recf;  // FP32 copies (mixed mode), written with the FP64 values
  auto put = [&](int f, double val) {
    rec[f * n + p] = val;
    if (recf) recf[f * n + p] = (float)val;
  };
  double hq[9], hk[3], ht[3];  // Hencky: principal directions, kappa_A, theta_AB
  if (s.hencky) {
    double x[3], eps[3], tA[3], tr = 0.0;
    sym_eig<D>(bl, x, hq);
    for (int A = 0; A < D; ++A) {
      eps[A] = 0.5 * log(x[A]);
      tr += eps[A];
    }
    for (int A = 0; A < D; ++A) {
      tA[A] = lam * tr + 2.0 * G * eps[A];
      hk[A] = 2.0 * G - 2.0 * tA[A];
    }
    for (int A = 0; A < D; ++A)
      for (int B = A + 1; B < D; ++B) ht[pair_index(A, B)] = G * log1p_ratio(x[A] / x[B] - 1.0) - tA[B];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double t = 0.0;
        for (int A = 0; A < D; ++A) t += tA[A] * hq[i * D + A] * hq[j * D + A];
        put(RC_TAU + i * D + j, t);
      }
    for (int i = 0; i < D * D; ++i) put(RC_HQ + i, hq[i]);
    for (int A = 0; A < D; ++A) put(RC_HK + A, hk[A]);
    for (int k = 0; k < D * (D - 1) / 2; ++k) put(RC_HT + k, ht[k]);
  }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      put(RC_FINV + i * D + j, fi[i * D + j]);
      if (!s.hencky)
        put(RC_TAU + i * D + j, G * (bl[i * D + j] - (i == j ? 1.0 : 0.0)) + (i == j ? lam * lnJ : 0.0));
    }
  double gp[3] = {0, 0, 0}, gv[9] = {0};
  for (int j = 0; j < D; ++j) {
    double acc = 0.0;
    for (int k = 0; k < D; ++k) acc += gPn[k] * fi[k * D + j];
    gp[j] = acc;
  }
  double divv;
  if (DYN) {
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double acc = 0.0;
        for (int k = 0; k < D; ++k) acc += gVn[i * D + k] * fi[k * D + j];
        gv[i * D + j] = acc;
      }
    divv = 0.0;
    for (int i = 0; i < D; ++i) divv += gv[i * D + i];
    double trD = divv;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        put(RC_GV + i * D + j, gv[i * D + j]);
        const double Dij = 0.5 * (gv[i * D + j] + gv[j * D + i]);
        put(RC_SVIS + i * D + j, s.alpha_vis * ((i == j ? lam * trD : 0.0) + 2.0 * mu_p * Dij));
      }
    if (s.hencky) {  // alpha c : d with the Hencky tangent, in the principal frame
      double Dh[9], Sh[9];
      for (int A = 0; A < D; ++A)
        for (int B = 0; B < D; ++B) {
          double t = 0.0;
          for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) t += hq[i * D + A] * 0.5 * (gv[i * D + j] + gv[j * D + i]) * hq[j * D + B];
          Dh[A * D + B] = t;
        }
      for (int A = 0; A < D; ++A)
        for (int B = 0; B < D; ++B)
          Sh[A * D + B] = A == B ? lam * trD + hk[A] * Dh[A * D + A]
                                 : 2.0 * ht[pair_index(A < B ? A : B, A < B ? B : A)] * Dh[A * D + B];
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          double t = 0.0;
          for (int A = 0; A < D; ++A)
            for (int B = 0; B < D; ++B) t += hq[i * D + A] * Sh[A * D + B] * hq[j * D + B];
          put(RC_SVIS + i * D + j, s.alpha_vis * t);
        }
    }
  } else {
    divv = log(dJ) / dt;
  }
  const double m = v.m[p];
  for (int j = 0; j < D; ++j) {
    put(RC_GP + j, gp[j]);
    put(RC_W + j, gp[j] - s.rho_f * (s.g[j] - ah[j]));
    put(RC_FRC + j, m * (s.g[j] - ah[j]));
  }
  put(RC_CS, Vn / Jn);
  put(RC_VOL, vol);
  put(RC_PH, ph);
  put(RC_MUP, mu_p);
  put(RC_LAM, lam);
  double kv = vol * kap, dkv = 0.0;
  if (s.kozeny) {  // mobility at the current porosity, Eq. kozeny-carman
    double jdk;
    kv = vol * kozeny_carman(kap, s.phi0, J, &jdk);
    dkv = vol * jdk;
  }
  put(RC_KV, kv);
  put(RC_DKV, dkv);
  put(RC_CST, (DYN ? tau * gm / (b * dt) : tau / dt) * Vn);
  put(RC_RST, tau * Vn * pdev);
  put(RC_DIVV, vol * divv);
  put(RC_B2, DYN ? vol * (gm / (b * dt) + divv) : vol * (1.0 + log(dJ)) / dt);
  put(RC_MS, DYN ? m / (b * dt * dt) : 0.0);
  // The residual's per-point factors.  With g = Gn dF^-1 (Gn the gradient of
  // the basis in the configuration of t_n), the momentum term of a node,
  // -cs g.(tau' + s_vis) + vol p^h g, is Gn.RU, and the Darcy term
  // kappa vol g.w is Gn.KW: the residual's node sums then spend d^2 + d FMAs
  // per (point, node) on them instead of forming g first.
  // (the stress and w read back once into registers: the stores below could
  // alias them for the compiler)
  const double cs = Vn / Jn;
  double sg[9], wv[3];
  for (int i = 0; i < D; ++i) {
    for (int j = 0; j < D; ++j) {
      double sij = rec[(RC_TAU + i * D + j) * n + p];
      if (DYN) sij += rec[(RC_SVIS + i * D + j) * n + p];
      sg[i * D + j] = sij;
    }
    wv[i] = rec[(RC_W + i) * n + p];
  }
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) {
      double acc = vol * ph * fi[k * D + i];
      for (int j = 0; j < D; ++j) acc -= cs * sg[i * D + j] * fi[k * D + j];
      rec[(RC_RU + i * D + k) * n + p] = acc;
    }
  for (int k = 0; k < D; ++k) {
    double acc = 0.0;
    for (int j = 0; j < D; ++j) acc += fi[k * D + j] * wv[j];
    rec[(RC_KW + k) * n + p] = kv * acc;
  }
}

// ---------------------------------------------------------------- residual
template <int D, bool GIMP, bool DYN>
__global__ void k_residual(GridP g, DevView v, double *__restrict__ R, int apply_bc) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  constexpr int NB = D + 1;
  const int64_t n = v.n;
  int ac[3];
  node_coords(g, a, ac);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) cand_range<GIMP>(ac[k], g.nc[k], lo[k], hi[k]);
  double r[NB];
  for (int i = 0; i < NB; ++i) r[i] = 0.0;
  const double *rec = v.rec;
  for (int c2 = lo[2]; c2 <= hi[2]; ++c2)
    for (int c1 = lo[1]; c1 <= hi[1]; ++c1)
      for (int c0 = lo[0]; c0 <= hi[0]; ++c0) {
        const int64_t cid = cell_index(g, c0, c1, c2);
        for (int32_t q = v.cell_start[cid]; q < v.cell_start[cid + 1]; ++q) {
          int off[3];
          if (!in_box4<D>(v.sh_box[q], ac, off)) continue;
          double Sa, S0a, Gn[3];
          basis_at<D>(v, q, off, a, Sa, S0a, Gn);
          for (int i = 0; i < D; ++i) {  // Gn.RU + S_a m (g - a)
            double acc = Sa * rec[(RC_FRC + i) * n + q];
            for (int k = 0; k < D; ++k) acc = fma(Gn[k], rec[(RC_RU + i * D + k) * n + q], acc);
            r[i] += acc;
          }
          double rp = fma(Sa, rec[RC_DIVV * n + q], (Sa - S0a) * rec[RC_RST * n + q]);
          for (int k = 0; k < D; ++k) rp = fma(Gn[k], rec[(RC_KW + k) * n + q], rp);  // Gn.KW
          r[D] += rp;
          const int32_t e = v.surf[q];
          if (e >= 0) {  // Neumann data at the surface point x + lp.n (hat basis)
            const InstDev &I = v.inst[(int)v.pf[PF_INST * n + q]];
            double Ny = 1.0;
            for (int k = 0; k < D; ++k) {
              const double y = v.pf[(PF_X + k) * n + q] + v.pf[(PF_LP + k) * n + q] * v.pf[(PF_SN + k) * n + q];
              const double t = 1.0 - fabs((y - I.org[k]) / g.h - (double)(ac[k] - I.off[k]));
              Ny *= t > 0.0 ? t : 0.0;
            }
            const double A = v.pf[PF_SA * n + q];
            for (int i = 0; i < D; ++i) r[i] += Ny * v.trac[(int64_t)e * D + i] * A;
            if (v.flux) r[D] -= Ny * v.flux[e] * A;
          }
        }
      }
  for (int i = 0; i < NB; ++i) {
    const bool fx = apply_bc && v.fixed[a * NB + i];
    R[a * NB + i] = fx ? 0.0 : r[i];
  }
}

// ---------------------------------------------------------------- Jacobian
// Block values are written in precision T and computed in precision R: FP64
// from the FP64 records, or FP32 from their FP32 copies in the mixed mode.
// One thread per block (a, b) (per symmetric pair of blocks, below), mapped
// so that the 32 lanes of a warp hold the same coupling offset (b - a in
// [-3, 3]^d) in 32 consecutive rows and walk the same number of candidate
// bins; a slot absent from the row's pattern exits.
template <int D>
__device__ inline int64_t block_of_slot(const uint64_t *__restrict__ mask, const int32_t *__restrict__ row_ptr,
                                        int64_t a, int s) {
  const uint64_t *mk = mask + a * MASKW;
  const int w = s >> 6;
  const uint64_t word = mk[w];
  if (!((word >> (s & 63)) & 1ull)) return -1;
  int before = __popcll(word & ((1ull << (s & 63)) - 1ull));
  for (int i = 0; i < w; ++i) before += __popcll(mk[i]);
  return (int64_t)row_ptr[a] + before;
}

// Staging of the Jacobian (FP64, and FP32 in the staged mixed form): the
// point's per-node records (k_point_nodes below: PN_LANES lanes per point),
// so that each (point, a, b) term of the block assembly is a short chain of
// FMAs.  With g = F^-T grad S (current configuration), St = S - S0 and the
// point's coefficients
//   p0 = cs,  p1 = cs (1 + cv) G',
//   p2 = vol p - cs (1 + cv) lambda,  p3 = cs (1 + cv) G' + vol p,
//   p4 = m (Newmark),  p5 = vol,  p6 = b2,  p7 = kappa vol,  p8 = C_stab V
// (cs = V_n / J_n, cv = the Newmark viscous factor, G' = G - lambda ln J), a
// node record holds (PnLay: first the fields a pair term reads at both of its
// nodes, then those it reads at the row node only)
//   g, S, St, p2 g, c = p6 S + (p7 + J dk/dJ vol) g.w, e = p7 g.w, p5 S,
//   g.grad v (Newmark); then p3 g, h = p0 (g^T tau') + p1 g, p7 g, p8 St,
//   p4 S (Newmark),
// and the point's own record (after its node records) holds grad p.  (The
// terms are those of the linearization, Eqs. jacobian-system-stabilized-ppp
// and newmark-linearization, grouped per node.)
// Hencky (HK): the material part of the tangent is not of the lambda / G'
// form, so p1 = 0, p2 = p3 = vol p, and the record ends with the d^3 values
// U_ikl = -cs (1 + cv) sum_j g_j c_ijkl (PnLay::U), so that the term adds
// sum_l U_a,ikl g_b,l to A_ik; from the principal data of the point
//   sum_j g_j c_ijkl = lambda g_i delta_kl + sum_A n_Ai (kappa_A gh_A n_Ak n_Al
//                      + sum_{B != A} theta_AB gh_B (n_Ak n_Bl + n_Bk n_Al)),
// gh_A = g . n_A.
template <int D, bool DYN, bool HK, typename R>
__device__ inline void point_node_record(const GridP &g, const StepP &sp, const DevView &v,
                                         const BasisArrays<R> &BA, const R *__restrict__ rec, int64_t q,
                                         const int off[3], R *__restrict__ out) {
  using L = PnLay<D, DYN, HK, (int)sizeof(R)>;
  const int64_t n = v.n;
  const R cs = rec[RC_CS * n + q], vol = rec[RC_VOL * n + q], ph = rec[RC_PH * n + q];
  const R cv = DYN ? (R)(sp.alpha_vis * sp.gamma / (sp.beta * sp.dt)) : R(0);
  const R csv = cs * (R(1) + cv);
  const R p0 = cs, p1 = HK ? R(0) : csv * rec[RC_MUP * n + q];
  const R p2 = HK ? vol * ph : vol * ph - csv * rec[RC_LAM * n + q];
  const R p3 = HK ? vol * ph : csv * rec[RC_MUP * n + q] + vol * ph;
  const R p5 = vol, p6 = rec[RC_B2 * n + q], p7 = rec[RC_KV * n + q], p8 = rec[RC_CST * n + q];
  int nc[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) nc[k] = v.sh_first[k * n + q] + off[k];
  const int64_t a = node_index(g, nc);
  R Sa, S0a, Gn[3], gs[3];
  basis_at_t<D, R>(BA, q, off, a, Sa, S0a, Gn);
  for (int j = 0; j < D; ++j) {
    R sj = 0;
    for (int k = 0; k < D; ++k) sj += Gn[k] * rec[(RC_FINV + k * D + j) * n + q];
    gs[j] = sj;
  }
  R gw = 0;
  for (int l = 0; l < D; ++l) {
    R tl = 0;
    for (int j = 0; j < D; ++j) tl += gs[j] * rec[(RC_TAU + j * D + l) * n + q];
    out[L::G + l] = gs[l];
    out[L::P2G + l] = p2 * gs[l];
    out[L::P3G + l] = p3 * gs[l];
    out[L::H + l] = p0 * tl + p1 * gs[l];
    out[L::P7G + l] = p7 * gs[l];
    gw += gs[l] * rec[(RC_W + l) * n + q];
  }
  const R St = Sa - S0a;
  out[L::S] = Sa;
  out[L::ST] = St;
  out[L::C] = p6 * Sa + (p7 + rec[RC_DKV * n + q]) * gw;
  out[L::E] = p7 * gw;
  out[L::P5S] = p5 * Sa;
  out[L::P8ST] = p8 * St;
  if (DYN) {
    out[L::MS] = rec[RC_MS * n + q] * Sa;
    for (int k = 0; k < D; ++k) {
      R gv = 0;
      for (int j = 0; j < D; ++j) gv += gs[j] * rec[(RC_GV + j * D + k) * n + q];
      out[L::GV + k] = gv;
    }
  }
  if (HK) {
    R nq[9], kap[3], th[3], gh[3];
    for (int i = 0; i < D * D; ++i) nq[i] = rec[(RC_HQ + i) * n + q];
    for (int A = 0; A < D; ++A) kap[A] = rec[(RC_HK + A) * n + q];
    for (int k = 0; k < D * (D - 1) / 2; ++k) th[k] = rec[(RC_HT + k) * n + q];
    for (int A = 0; A < D; ++A) {
      R t = 0;
      for (int j = 0; j < D; ++j) t += gs[j] * nq[j * D + A];
      gh[A] = t;
    }
    const R lam = rec[RC_LAM * n + q];
    for (int i = 0; i < D; ++i)
      for (int k = 0; k < D; ++k)
        for (int l = 0; l < D; ++l) {
          R u = k == l ? lam * gs[i] : R(0);
          for (int A = 0; A < D; ++A) {
            R w = kap[A] * gh[A] * nq[k * D + A] * nq[l * D + A];
            for (int B = 0; B < D; ++B)
              if (B != A) {
                const R tAB = th[pair_index(A < B ? A : B, A < B ? B : A)];
                w += tAB * gh[B] * (nq[k * D + A] * nq[l * D + B] + nq[k * D + B] * nq[l * D + A]);
              }
            u += nq[i * D + A] * w;
          }
          out[L::U + (i * D + k) * D + l] = -csv * u;
        }
  }
}

// Symmetric pairs.  The Jacobian's blocks (a, b) and (b, a) come from the
// same (point, a, b) terms: A_ba = A_ab^T (the material, geometric, pressure,
// Kelvin and inertia parts of A are each symmetric under (a, i) <-> (b, k):
// tau' and the tangent are symmetric) and C_ba = C_ab (Darcy and C_stab are
// symmetric), while B1 and B2 of the two blocks differ.  One thread takes the
// unordered pair: coupling offset o = b - a in the upper half of [-3, 3]^d
// (slot s >= the centre slot; threads mapped by pair_of_thread) and writes
// block (a, b) and, for o != 0, block (b, a) = row b, slot of -o.  Per
// (point, a, b) term of a pair the A and C parts are formed once and the
// B1 / B2 parts twice.
template <int D>
struct PairSlots {
  static constexpr int NSLOT = D == 2 ? 49 : 343;
  static constexpr int CENTRE = NSLOT / 2;  // offset 0
  static constexpr int COUNT = CENTRE + 1;  // slots >= CENTRE
};

// Thread -> (row a, pair slot), tiled: a tile of PAIR_ROWS consecutive rows
// takes all the pair slots before the next tile, and the lanes of a warp hold
// one slot in PAIR_ROWS consecutive rows.  The warps of a block and their
// neighbours then walk the same candidate points for different offsets, so a
// point's records are reused from L1 and L2 instead of being read again from
// DRAM for every offset (slot-major over the whole grid, each offset swept the
// whole point set).  Returns false past the last row.
constexpr int PAIR_ROWS = 32;
template <int D>
__device__ inline bool pair_of_thread(const GridP &g, int64_t t, int64_t &a, int &slot) {
  using PS = PairSlots<D>;
  constexpr int64_t PER_TILE = (int64_t)PAIR_ROWS * PS::COUNT;
  const int64_t tile = t / PER_TILE;
  const int rem = (int)(t - tile * PER_TILE);
  slot = PS::CENTRE + rem / PAIR_ROWS;
  a = tile * PAIR_ROWS + rem % PAIR_ROWS;
  return a < g.nnodes;
}
inline int64_t pair_threads(int d, int64_t nnodes) {
  const int64_t tiles = (nnodes + PAIR_ROWS - 1) / PAIR_ROWS;
  return tiles * PAIR_ROWS * (d == 2 ? PairSlots<2>::COUNT : PairSlots<3>::COUNT);
}

template <int D, typename R, typename T>
__device__ inline void write_block_bc(const DevView &v, int64_t row, int64_t colnode, const R *B, T *out,
                                      int apply_bc) {
  constexpr int NB = D + 1;
  for (int i = 0; i < NB; ++i) {
    const bool fr = apply_bc && v.fixed[row * NB + i] != 0;
    for (int k = 0; k < NB; ++k) {
      const bool fc = apply_bc && v.fixed[colnode * NB + k] != 0;
      R x = B[i * NB + k];
      if (fr || fc) x = (row == colnode && i == k) ? R(1) : R(0);
      out[i * NB + k] = (T)x;
    }
  }
}

// PNL lanes per point, each taking the point's support nodes PNL apart (the
// box's own nodes only, not the 4^d slots of the record array), so that the
// lanes of a warp are busy with the nodes that exist; lane 0 also writes the
// point's own record (grad p, last slot).
constexpr int PN_LANES = 16;
template <int D, bool DYN, bool HK, typename R>
__global__ void k_point_nodes(GridP g, StepP sp, DevView v, BasisArrays<R> BA, const R *__restrict__ rec,
                              R *__restrict__ pn) {
  using L = PnLay<D, DYN, HK, (int)sizeof(R)>;
  constexpr int NPS = L::STRIDE;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = v.n;
  if (t >= n * PN_LANES) return;
  const int64_t q = t / PN_LANES;
  const int j = (int)(t - q * PN_LANES);
  R *P = pn + (int64_t)v.pn_base[q] * NPS;  // the point's records: box nodes x-fastest, then its own
  const int packed = v.sh_cnt[q];
  const int c0 = unpack_cnt(packed, 0), c1 = D > 1 ? unpack_cnt(packed, 1) : 1,
            c2 = D > 2 ? unpack_cnt(packed, 2) : 1;
  const int nq = c0 * c1 * c2;
  if (j == 0)
    for (int k = 0; k < D; ++k) P[nq * NPS + L::GP + k] = rec[(RC_GP + k) * n + q];
  for (int sc = j; sc < nq; sc += PN_LANES) {
    const int off[3] = {sc % c0, (sc / c0) % c1, sc / (c0 * c1)};
    point_node_record<D, DYN, HK, R>(g, sp, v, BA, rec, q, off, P + sc * NPS);
  }
}

// One staged (point, node) record as the pair kernel reads it: in FP32 the
// whole record is brought into registers with 16-byte vector loads (the FP32
// kernel is bound by the load path, and a record read value by value costs a
// memory transaction per value and lane); in FP64 (bound by the FP64 pipe) the
// values are read where they are used.
template <typename R, int NPS>
struct PnRec {
  static constexpr bool VEC = sizeof(R) == 4;
  R v[VEC ? NPS : 1];
  const R *p;
  __device__ __forceinline__ void load(const R *__restrict__ src) {
    if constexpr (VEC) {
      static_assert(NPS % 4 == 0, "FP32 records are padded to 16 bytes");
#pragma unroll
      for (int i = 0; i < NPS / 4; ++i) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(src) + i);
        v[4 * i] = x.x;
        v[4 * i + 1] = x.y;
        v[4 * i + 2] = x.z;
        v[4 * i + 3] = x.w;
      }
    } else {
      p = src;
    }
  }
  __device__ __forceinline__ R operator[](int i) const {
    if constexpr (VEC) return v[i];
    else return p[i];
  }
};

// Every candidate point q of the node pair (ac, bc), in a fixed order: the
// points of the first-node bins that can hold both nodes (FB), or those of the
// cells around both (each x-run of cells is one contiguous run of the
// cell-sorted points).  The bins visit fewer candidates; the cells visit them
// in storage order, whose locality serves the FP64 staged kernel better (its
// records are read in point order), while the FP32 kernels gain from the
// bins.
template <int D, bool GIMP, bool FB, typename F>
__device__ __forceinline__ void for_pair_candidates(const GridP &g, const DevView &v, const int ac[3],
                                                    const int bc[3], F &&f) {
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  if constexpr (FB) {
    fb_window<D>(v.fb_cmax, ac, bc, lo, hi);
    for (int f2 = lo[2]; f2 <= hi[2]; ++f2)
      for (int f1 = lo[1]; f1 <= hi[1]; ++f1) {
        int32_t ib, ie;
        fb_run(g, v.fb_start, lo[0], hi[0], f1, f2, ib, ie);
        for (int32_t i = ib; i < ie; ++i) f(v.fb_perm[i]);
      }
  } else {
    for (int k = 0; k < D; ++k) {
      int l1, h1, l2, h2;
      cand_range<GIMP>(ac[k], g.nc[k], l1, h1);
      cand_range<GIMP>(bc[k], g.nc[k], l2, h2);
      lo[k] = max(l1, l2);
      hi[k] = min(h1, h2);
    }
    if (lo[0] > hi[0]) return;
    for (int c2 = lo[2]; c2 <= hi[2]; ++c2)
      for (int c1 = lo[1]; c1 <= hi[1]; ++c1) {
        const int64_t c0 = cell_index(g, lo[0], c1, c2);
        const int32_t qb = v.cell_start[c0], qe = v.cell_start[c0 + (hi[0] - lo[0]) + 1];
        for (int32_t q = qb; q < qe; ++q) f(q);
      }
  }
}

template <int D, bool GIMP, bool DYN, bool HK, bool FB, typename T, typename R>
__global__ void k_jacobian(GridP g, StepP s, DevView v, const R *__restrict__ pn,
                           const uint64_t *__restrict__ mask, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, T *__restrict__ val, int apply_bc) {
  using PS = PairSlots<D>;
  using L = PnLay<D, DYN, HK, (int)sizeof(R)>;
  constexpr int NPS = L::STRIDE;
  int64_t a;
  int slot;
  if (!pair_of_thread<D>(g, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, a, slot)) return;
  const int64_t e = block_of_slot<D>(mask, row_ptr, a, slot);
  if (e < 0) return;
  constexpr int NB = D + 1;
  const int64_t bn = col[e];
  const bool diag = slot == PS::CENTRE;
  int ac[3], bc[3];
  node_coords(g, a, ac);
  node_coords(g, bn, bc);
  // pair accumulators: A (shared, for (a, b); (b, a) gets its transpose), C
  // (shared), B1 and B2 of each of the two blocks
  // kgp: the grad p part of B2, (p7 g_a.g_b) grad p, the same for both blocks
  // Dg: the sum of the terms' d (A_ii - d per term, subtracted once at the end)
  R A[D * D], b1ab[D], b1ba[D], b2ab[D], b2ba[D], kgp[D], C = 0, Dg = 0;
  for (int i = 0; i < D * D; ++i) A[i] = 0;
  for (int i = 0; i < D; ++i) b1ab[i] = b1ba[i] = b2ab[i] = b2ba[i] = kgp[i] = 0;
  for_pair_candidates<D, GIMP, FB>(g, v, ac, bc, [&](const int32_t q) {
    int oa[3], ob[3];
    const int4 bx = v.sh_box[q];  // one 16-byte load per visited point
    if (!in_box4<D>(bx, ac, oa) || !in_box4<D>(bx, bc, ob)) return;
    // the point's records: its box nodes x-fastest, then its own
    const R *P = pn + (int64_t)v.pn_base[q] * NPS;
    const int c0 = unpack_cnt(bx.w, 0), c1 = D > 1 ? unpack_cnt(bx.w, 1) : 1,
              c2 = D > 2 ? unpack_cnt(bx.w, 2) : 1;
    PnRec<R, NPS> pa;        // the row node's record: all of it
    PnRec<R, L::BPART> pb;   // the column node's: the fields read for both nodes
    pa.load(P + (oa[0] + c0 * (oa[1] + c1 * oa[2])) * NPS);
    pb.load(P + (ob[0] + c0 * (ob[1] + c1 * ob[2])) * NPS);
    const R *pp = P + (c0 * c1 * c2) * NPS;
    R ga[3], gb[3];
    for (int j = 0; j < D; ++j) {
      ga[j] = pa[L::G + j];
      gb[j] = pb[L::G + j];
    }
    // A_ik = g_a,i (p2 g_b)_k - g_b,i (p3 g_a)_k - delta_ik d,
    // d = h_a.g_b (+ p4 S_a S_b): stress, geometric, pressure, Kelvin
    // and inertia terms with the point's coefficients staged per node
    R kgab = 0;
    for (int j = 0; j < D; ++j) {
      Dg = fma(pa[L::H + j], gb[j], Dg);
      kgab = fma(pa[L::P7G + j], gb[j], kgab);  // p7 g_a.g_b
    }
    if (DYN) Dg = fma(pa[L::MS], pb[L::S], Dg);
    for (int i = 0; i < D; ++i)
      for (int k = 0; k < D; ++k) {
        R acc = fma(ga[i], pb[L::P2G + k], A[i * D + k]);
        acc = fma(-gb[i], pa[L::P3G + k], acc);
        if (HK)  // material part of the Hencky tangent, staged per node
          for (int l = 0; l < D; ++l) acc = fma(pa[L::U + (i * D + k) * D + l], gb[l], acc);
        A[i * D + k] = acc;
      }
    // B1 column of (a, b): (p5 S_b) g_a; of (b, a): (p5 S_a) g_b
    const R p5Sb = pb[L::P5S], p5Sa = pa[L::P5S];
    for (int i = 0; i < D; ++i) b1ab[i] = fma(p5Sb, ga[i], b1ab[i]);
    // B2 row of (a, b): (p6 S_a + p7 g_a.w) g_b - (p7 g_b.w) g_a - (p7 g_a.g_b) grad p
    //                   (- p5 S_a g_b.grad v, Newmark); (b, a): a <-> b
    const R ca = pa[L::C], eb = pb[L::E];
    for (int k = 0; k < D; ++k) {
      R tk = fma(ca, gb[k], b2ab[k]);
      if (DYN) tk = fma(-p5Sa, pb[L::GV + k], tk);
      b2ab[k] = fma(-eb, ga[k], tk);
      kgp[k] = fma(kgab, pp[L::GP + k], kgp[k]);
    }
    if (!diag) {
      for (int i = 0; i < D; ++i) b1ba[i] = fma(p5Sa, gb[i], b1ba[i]);
      const R cb = pb[L::C], ea = pa[L::E];
      for (int k = 0; k < D; ++k) {
        R tk = fma(cb, ga[k], b2ba[k]);
        if (DYN) tk = fma(-p5Sb, pa[L::GV + k], tk);
        b2ba[k] = fma(-ea, gb[k], tk);
      }
    }
    // C + C_stab: p7 g_a.g_b + (p8 St_a) St_b (symmetric)
    C = fma(pa[L::P8ST], pb[L::ST], C + kgab);
  });
  for (int i = 0; i < D; ++i) A[i * D + i] -= Dg;
  R B[NB * NB];
  for (int i = 0; i < D; ++i) {
    for (int k = 0; k < D; ++k) B[i * NB + k] = A[i * D + k];
    B[i * NB + D] = b1ab[i];
    B[D * NB + i] = b2ab[i] - kgp[i];
  }
  B[D * NB + D] = C;
  write_block_bc<D>(v, a, bn, B, val + e * (NB * NB), apply_bc);
  if (diag) return;
  const int64_t e2 = block_of_slot<D>(mask, row_ptr, bn, PS::NSLOT - 1 - slot);
  if (e2 < 0) return;  // the coupling is symmetric: not reached
  for (int i = 0; i < D; ++i) {
    for (int k = 0; k < D; ++k) B[i * NB + k] = A[k * D + i];
    B[i * NB + D] = b1ba[i];
    B[D * NB + i] = b2ba[i] - kgp[i];
  }
  B[D * NB + D] = C;
  write_block_bc<D>(v, bn, a, B, val + e2 * (NB * NB), apply_bc);
}

// FP32 variant (mixed mode): the node vectors are recomputed per term from the
// FP32 basis and records; with FP32 arithmetic plentiful this can beat staging.
// Neo-Hookean only: the Hencky tangent (d^3 values per node) is staged.
// Symmetric pairs as in k_jacobian: one thread per unordered pair (a, b).
template <int D, bool GIMP, bool DYN, bool FB, typename T, typename R>
__global__ void k_jacobian_direct(GridP g, StepP s, DevView v, BasisArrays<R> BA, const R *__restrict__ rec,
                           const uint64_t *__restrict__ mask, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, T *__restrict__ val, int apply_bc) {
  using PS = PairSlots<D>;
  int64_t a;
  int slot;
  if (!pair_of_thread<D>(g, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, a, slot)) return;
  const int64_t e = block_of_slot<D>(mask, row_ptr, a, slot);
  if (e < 0) return;
  constexpr int NB = D + 1;
  const int64_t n = v.n;
  const int64_t bn = col[e];
  const bool diag = slot == PS::CENTRE;
  int ac[3], bc[3];
  node_coords(g, a, ac);
  node_coords(g, bn, bc);
  R A[D * D], b1ab[D], b1ba[D], b2ab[D], b2ba[D], kgp[D], C = 0;
  for (int i = 0; i < D * D; ++i) A[i] = 0;
  for (int i = 0; i < D; ++i) b1ab[i] = b1ba[i] = b2ab[i] = b2ba[i] = kgp[i] = 0;
  const R cvis = DYN ? (R)(s.alpha_vis * s.gamma / (s.beta * s.dt)) : R(0);
  for_pair_candidates<D, GIMP, FB>(g, v, ac, bc, [&](const int32_t q) {
    int oa[3], ob[3];
    const int4 bx = v.sh_box[q];  // one 16-byte load per visited point
    if (!in_box4<D>(bx, ac, oa) || !in_box4<D>(bx, bc, ob)) return;
    R Sa, S0a, Gna[3], Sb, S0b, Gnb[3], ga[3], gb[3];
    basis_at_t<D, R>(BA, q, oa, a, Sa, S0a, Gna);
    basis_at_t<D, R>(BA, q, ob, bn, Sb, S0b, Gnb);
    for (int j = 0; j < D; ++j) {
      R sa = 0, sb = 0;
      for (int k = 0; k < D; ++k) {
        const R fkj = rec[(RC_FINV + k * D + j) * n + q];
        sa += Gna[k] * fkj;
        sb += Gnb[k] * fkj;
      }
      ga[j] = sa;
      gb[j] = sb;
    }
    const R cs = rec[RC_CS * n + q], vol = rec[RC_VOL * n + q], ph = rec[RC_PH * n + q];
    const R mu = rec[RC_MUP * n + q], lam = rec[RC_LAM * n + q], kv = rec[RC_KV * n + q];
    R gab = 0, gtg = 0, gaw = 0, gbw = 0;
    for (int j = 0; j < D; ++j) {
      gab += ga[j] * gb[j];
      const R wj = rec[(RC_W + j) * n + q];
      gaw += ga[j] * wj;
      gbw += gb[j] * wj;
      for (int l = 0; l < D; ++l) gtg += ga[j] * rec[(RC_TAU + j * D + l) * n + q] * gb[l];
    }
    const R ms = DYN ? rec[RC_MS * n + q] * Sa * Sb : R(0);
    for (int i = 0; i < D; ++i)
      for (int k = 0; k < D; ++k) {
        const R dik = i == k ? R(1) : R(0);
        const R sym = mu * (dik * gab + ga[k] * gb[i]);
        R Aik = -cs * (dik * gtg + sym + lam * ga[i] * gb[k]);
        Aik += vol * ph * (ga[i] * gb[k] - ga[k] * gb[i]);
        if (DYN) {
          Aik -= cs * cvis * (lam * ga[i] * gb[k] + sym);
          Aik -= dik * ms;
        }
        A[i * D + k] += Aik;
      }
    const R b2 = rec[RC_B2 * n + q], dkv = rec[RC_DKV * n + q];
    for (int i = 0; i < D; ++i) b1ab[i] += vol * ga[i] * Sb;
    for (int k = 0; k < D; ++k) {
      R t = Sa * b2 * gb[k];
      if (DYN) {
        R gbgv = 0;
        for (int j = 0; j < D; ++j) gbgv += gb[j] * rec[(RC_GV + j * D + k) * n + q];
        t -= vol * Sa * gbgv;
      }
      t += kv * (gb[k] * gaw - ga[k] * gbw);
      t += dkv * gb[k] * gaw;  // dk/dJ (Kozeny-Carman)
      b2ab[k] += t;
      kgp[k] += kv * gab * rec[(RC_GP + k) * n + q];  // grad p part, the same for both blocks
    }
    if (!diag) {
      for (int i = 0; i < D; ++i) b1ba[i] += vol * gb[i] * Sa;
      for (int k = 0; k < D; ++k) {
        R t = Sb * b2 * ga[k];
        if (DYN) {
          R gagv = 0;
          for (int j = 0; j < D; ++j) gagv += ga[j] * rec[(RC_GV + j * D + k) * n + q];
          t -= vol * Sb * gagv;
        }
        t += kv * (ga[k] * gbw - gb[k] * gaw);
        t += dkv * ga[k] * gbw;
        b2ba[k] += t;
      }
    }
    C += kv * gab + rec[RC_CST * n + q] * (Sa - S0a) * (Sb - S0b);
  });
  R B[NB * NB];
  for (int i = 0; i < D; ++i) {
    for (int k = 0; k < D; ++k) B[i * NB + k] = A[i * D + k];
    B[i * NB + D] = b1ab[i];
    B[D * NB + i] = b2ab[i] - kgp[i];
  }
  B[D * NB + D] = C;
  write_block_bc<D>(v, a, bn, B, val + e * (NB * NB), apply_bc);
  if (diag) return;
  const int64_t e2 = block_of_slot<D>(mask, row_ptr, bn, PS::NSLOT - 1 - slot);
  if (e2 < 0) return;
  for (int i = 0; i < D; ++i) {
    for (int k = 0; k < D; ++k) B[i * NB + k] = A[k * D + i];
    B[i * NB + D] = b1ba[i];
    B[D * NB + i] = b2ba[i] - kgp[i];
  }
  B[D * NB + D] = C;
  write_block_bc<D>(v, bn, a, B, val + e2 * (NB * NB), apply_bc);
}

// ---------------------------------------------------------------- consistent-mass Stage 1
// Eq. map-from-particles-to-nodes-consistent: sum_j M_ij f_j = sum_mp S_i m f
// with M_ij = sum_mp S_i S_j m, for every mapped field f (P; Newmark also v,
// a, dp/dt, d2p/dt2), solved for the active nodes (mass and volume fraction
// above phi_min, the active set of the Newton system: the consistent mass of a
// node that a GIMP domain barely reaches is singular); the other nodes keep
// the lumped values (Eq. map-from-particles-to-nodes), their couplings moved to
// the right-hand side, whose point sum is M_i f_i of the lumped mapping.
// Jacobi-preconditioned CG over all fields at once, per-field scalars on the
// device.

// M_ij on the node pattern, one thread per block (i = row_of[e], j = col[e]).
template <int D, bool GIMP>
__global__ void k_consistent_mass(GridP g, DevView v, int64_t nnzb, const int32_t *__restrict__ row_of,
                                  const int32_t *__restrict__ col, double *__restrict__ mc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  const int64_t a = row_of[e], b = col[e], n = v.n;
  int ac[3], bc[3];
  node_coords(g, a, ac);
  node_coords(g, b, bc);
  int lo[3], hi[3];
  fb_window<D>(v.fb_cmax, ac, bc, lo, hi);
  double acc = 0.0;
  for (int f2 = lo[2]; f2 <= hi[2]; ++f2)
    for (int f1 = lo[1]; f1 <= hi[1]; ++f1) {
      int32_t ib, ie;
      fb_run(g, v.fb_start, lo[0], hi[0], f1, f2, ib, ie);
      for (int32_t i = ib; i < ie; ++i) {
        const int32_t q = v.fb_perm[i];
        int oa[3], ob[3];
        if (!in_box<D>(v, q, ac, oa) || !in_box<D>(v, q, bc, ob)) continue;
        double Sa = 1.0, Sb = 1.0;
        for (int k = 0; k < D; ++k) {
          Sa *= v.sh_S[(k * MAXS + oa[k]) * n + q];
          Sb *= v.sh_S[(k * MAXS + ob[k]) * n + q];
        }
        acc += Sa * Sb * v.m[q];
      }
    }
  mc[e] = acc;
}

constexpr int CM_MAXF = 9;  // mapped fields: 2d + 3 (Newmark) at most
struct CMFields {
  double *f[CM_MAXF];
  int K;
};

__device__ inline bool cm_active(const DevView &v, int64_t a, double phi_min) {
  return v.M[a] > 0.0 && v.phi[a] > phi_min;
}

// x = lumped values; rhs = M_a f_a - sum over inactive columns; dinv = 1 / M_aa
__global__ void k_cm_setup(int64_t nn, DevView v, double phi_min, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, const double *__restrict__ mc, CMFields F,
                           double *__restrict__ x, double *__restrict__ rhs, double *__restrict__ dinv) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nn * F.K) return;
  const int f = (int)(t / nn);
  const int64_t a = t - (int64_t)f * nn;
  const double fa = F.f[f][a];
  x[t] = fa;
  if (!cm_active(v, a, phi_min)) {
    rhs[t] = 0.0;
    if (f == 0) dinv[a] = 0.0;
    return;
  }
  double r = v.M[a] * fa, diag = 0.0;
  for (int e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
    const int64_t b = col[e];
    if (b == a) diag = mc[e];
    else if (!cm_active(v, b, phi_min)) r -= mc[e] * F.f[f][b];
  }
  rhs[t] = r;
  if (f == 0) dinv[a] = diag > 0.0 ? 1.0 / diag : 0.0;
}

// y = A x over the active rows and columns (zero on inactive rows)
__global__ void k_cm_spmv(int64_t nn, int K, DevView v, double phi_min, const int32_t *__restrict__ row_ptr,
                          const int32_t *__restrict__ col, const double *__restrict__ mc,
                          const double *__restrict__ x, double *__restrict__ y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nn * K) return;
  const int f = (int)(t / nn);
  const int64_t a = t - (int64_t)f * nn;
  double s = 0.0;
  if (cm_active(v, a, phi_min))
    for (int e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
      const int64_t b = col[e];
      if (cm_active(v, b, phi_min)) s += mc[e] * x[(int64_t)f * nn + b];
    }
  y[t] = s;
}

constexpr int CM_NBLK = 64;  // partial sums per field

// Block sums of s and s2 (every thread's), left in thread 0's s and s2: warp
// butterflies, then warp 0's lane 0 adds the warps' sums in warp order.
__device__ inline void cm_block_sum2(double &s, double &s2) {
  __shared__ double sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s;
    sh[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += sh[0][i];
      b += sh[1][i];
    }
    s = a;
    s2 = b;
  }
}

// per field f: part[f][blk] = sum of u.w (and, with w2, of u.w2) over its slice
__global__ void k_cm_dots(int64_t nn, const double *__restrict__ u, const double *__restrict__ w,
                          const double *__restrict__ w2, double *__restrict__ part, double *__restrict__ part2) {
  const int f = blockIdx.y;
  double s = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double ui = u[(int64_t)f * nn + i];
    s += ui * w[(int64_t)f * nn + i];
    if (w2) s2 += ui * w2[(int64_t)f * nn + i];
  }
  cm_block_sum2(s, s2);
  if (threadIdx.x == 0) {
    part[f * CM_NBLK + blockIdx.x] = s;
    if (part2) part2[f * CM_NBLK + blockIdx.x] = s2;
  }
}

// out[f] = sum of part[f][:] (and out2 from part2), one thread per field
__global__ void k_cm_sum(int K, const double *__restrict__ part, const double *__restrict__ part2,
                         double *__restrict__ out, double *__restrict__ out2) {
  const int f = threadIdx.x;
  if (f >= K) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < CM_NBLK; ++i) {
    a += part[f * CM_NBLK + i];
    if (part2) b += part2[f * CM_NBLK + i];
  }
  out[f] = a;
  if (out2) out2[f] = b;
}

// One CG iteration on the Jacobi-scaled consistent mass is three kernels on a
// (CM_NBLK, K) grid (a block per slice of one field, the slices of k_cm_dots,
// so the partial sums are those of separate product and dot kernels).  The
// convergence test runs on the device: k_cm_next sets *flag to 1 when every
// field's r.r is within rtol^2 of its rhs.rhs (2 for a non-finite r.r), and
// k_cm_qdot and k_cm_update do nothing once it is set, so iterations launched
// past convergence leave x as the converged iteration wrote it and the host
// reads the flag only every few iterations.  rz alternates between two
// buffers (k_cm_next writes the next iteration's while its blocks read the
// current one).

// q = A p over the active rows and columns (zero on inactive rows); part[f][blk] = p.q over the slice
__global__ void k_cm_qdot(int64_t nn, DevView v, double phi_min, const int32_t *__restrict__ row_ptr,
                          const int32_t *__restrict__ col, const double *__restrict__ mc,
                          const double *__restrict__ p, double *__restrict__ q, double *__restrict__ part,
                          const double *__restrict__ flag) {
  pdl_enter();
  if (*flag != 0.0) return;
  const int f = blockIdx.y;
  const double *pf = p + (int64_t)f * nn;
  double s = 0.0, s2 = 0.0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nn; a += (int64_t)gridDim.x * blockDim.x) {
    double y = 0.0;
    if (cm_active(v, a, phi_min))
      for (int e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
        const int64_t b = col[e];
        if (cm_active(v, b, phi_min)) y += mc[e] * pf[b];
      }
    q[(int64_t)f * nn + a] = y;
    s += pf[a] * y;
  }
  cm_block_sum2(s, s2);
  if (threadIdx.x == 0) part[f * CM_NBLK + blockIdx.x] = s;
}

// Sum of one field's CM_NBLK partial sums by a whole warp (two per lane, then
// a butterfly): every lane gets the sum, and every block forms it in the same
// order.  (One thread walking them would chain CM_NBLK dependent loads.)
static_assert(CM_NBLK == 64, "two partial sums per lane");
__device__ inline double cm_warp_sum_parts(const double *__restrict__ part) {
  const int lane = threadIdx.x & 31;
  double s = part[lane] + part[lane + 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// alpha = rz / p.q; x += alpha p, r -= alpha q, z = Dinv r; part_rz / part_rr = r.z / r.r over the slice
__global__ void k_cm_update(int64_t nn, const double *__restrict__ rz, const double *__restrict__ part_pq,
                            const double *__restrict__ dinv, const double *__restrict__ p,
                            const double *__restrict__ q, double *__restrict__ x, double *__restrict__ r,
                            double *__restrict__ z, double *__restrict__ part_rz, double *__restrict__ part_rr,
                            const double *__restrict__ flag) {
  pdl_enter();
  if (*flag != 0.0) return;
  const int f = blockIdx.y;
  __shared__ double s_alpha;
  if (threadIdx.x < 32) {
    const double pq = cm_warp_sum_parts(part_pq + f * CM_NBLK);
    if (threadIdx.x == 0) s_alpha = pq != 0.0 ? rz[f] / pq : 0.0;
  }
  __syncthreads();
  const double alpha = s_alpha;
  double s = 0.0, s2 = 0.0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nn; a += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = (int64_t)f * nn + a;
    x[t] += alpha * p[t];
    const double rv = r[t] - alpha * q[t];
    r[t] = rv;
    const double zv = dinv[a] * rv;
    z[t] = zv;
    s += rv * zv;
    s2 += rv * rv;
  }
  cm_block_sum2(s, s2);
  if (threadIdx.x == 0) {
    part_rz[f * CM_NBLK + blockIdx.x] = s;
    part_rr[f * CM_NBLK + blockIdx.x] = s2;
  }
}

// beta = rz_new / rz; p = z + beta p; rz_next = rz_new; the convergence flag
// (block (0, 0), a warp per field's r.r).  Not skipped after convergence: it
// then recomputes the same values from partial sums nothing changes.
__global__ void k_cm_next(int64_t nn, int K, const double *__restrict__ rz, double *__restrict__ rz_next,
                          const double *__restrict__ part_rz, const double *__restrict__ part_rr,
                          const double *__restrict__ bb, double rtol2, const double *__restrict__ z,
                          double *__restrict__ p, double *__restrict__ flag) {
  pdl_enter();
  const int f = blockIdx.y;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __shared__ double s_rzn, s_st[CM_MAXF];
  if (warp == 0) {
    const double v = cm_warp_sum_parts(part_rz + f * CM_NBLK);
    if (threadIdx.x == 0) s_rzn = v;
  }
  const bool lead = blockIdx.x == 0 && blockIdx.y == 0;
  if (lead)
    for (int g = warp; g < K; g += nwarp) {
      const double rr = cm_warp_sum_parts(part_rr + g * CM_NBLK);
      if ((threadIdx.x & 31) == 0) s_st[g] = !isfinite(rr) ? 2.0 : (rr > rtol2 * bb[g] ? 0.0 : 1.0);
    }
  __syncthreads();
  const double rzn = s_rzn;
  const double beta = rz[f] != 0.0 ? rzn / rz[f] : 0.0;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nn; a += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = (int64_t)f * nn + a;
    p[t] = z[t] + beta * p[t];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rz_next[f] = rzn;
  if (lead && threadIdx.x == 0) {
    double st = 1.0;  // 1 converged, 0 not yet, 2 non-finite
    for (int g = 0; g < K; ++g) {
      if (s_st[g] == 2.0) st = 2.0;
      else if (s_st[g] == 0.0 && st == 1.0) st = 0.0;
    }
    *flag = st;
  }
}

__global__ void k_cm_scatter(int64_t nn, CMFields F, const double *__restrict__ x) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nn * F.K) return;
  const int f = (int)(t / nn);
  F.f[f][t - (int64_t)f * nn] = x[t];
}

// r = rhs - A x, z = Dinv r, p = z (A x in q beforehand)
__global__ void k_cm_init(int64_t nn, int K, const double *__restrict__ rhs, const double *__restrict__ q,
                          const double *__restrict__ dinv, double *__restrict__ r, double *__restrict__ z,
                          double *__restrict__ p) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nn * K) return;
  const int64_t a = t % nn;
  const double rv = rhs[t] - q[t];
  r[t] = rv;
  z[t] = dinv[a] * rv;
  p[t] = z[t];
}

}  // namespace

// ============================================================== launchers
// Staging buffer of at least c.pn_total records of `stride` values: kept
// while large enough, else reallocated with a quarter of headroom (the supports
// grow and shrink a little from step to step as the points move).
template <typename R>
static int grow_staging(R **buf, int64_t *cap, int64_t total, int stride) {
  if (*buf && *cap >= total) return MPM_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  const int64_t want = total + total / 4 + 1024;
  if (cudaMalloc(buf, sizeof(R) * want * stride) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return MPM_ERR_NO_MEMORY;
  }
  *cap = want;
  return MPM_OK;
}

int ensure_jacobian_staging(Ctx &c) {
  const int rc = grow_staging(&c.pn, &c.pn_cap, c.pn_total, pn_stride(c.d, c.dyn, c.s.hencky, 8));
  if (rc) c.last_error = "device allocation of the Jacobian staging failed";
  return rc;
}

int run_consistent_p2g(Ctx &c) {
  const int64_t nn = c.g.nnodes;
  const int D = c.d, K = c.dyn ? 2 * D + 3 : 1;
  CMFields F{};
  F.K = K;
  if (c.dyn) {
    for (int k = 0; k < D; ++k) {
      F.f[k] = c.vn + k * nn;
      F.f[D + k] = c.an + k * nn;
    }
    F.f[2 * D] = c.Pn;
    F.f[2 * D + 1] = c.pdn;
    F.f[2 * D + 2] = c.pddn;
  } else {
    F.f[0] = c.Pn;
  }
  const int64_t need = 6 * (int64_t)K * nn + nn + 4 * (int64_t)CM_NBLK * K + 8 * K;
  if (need > c.cm_cap) {
    cudaFree(c.cm_buf);
    c.cm_buf = nullptr;
    c.cm_cap = 0;
    if (cudaMalloc(&c.cm_buf, sizeof(double) * need) != cudaSuccess) {
      c.last_error = "device allocation of the consistent-mass mapping failed";
      return MPM_ERR_NO_MEMORY;
    }
    c.cm_cap = need;
  }
  const int64_t KN = (int64_t)K * nn;
  double *x = c.cm_buf, *r = x + KN, *z = r + KN, *p = z + KN, *q = p + KN, *rhs = q + KN, *dinv = rhs + KN;
  double *part = dinv + nn, *part_rz = part + CM_NBLK * K, *part_rr = part_rz + CM_NBLK * K;
  double *rz = part_rr + 2 * CM_NBLK * K, *rz2 = rz + K, *bb = rz2 + K, *flag = bb + K;
  if (!c.mc || c.mc_cap < c.nnzb_cap) {
    cudaFree(c.mc);
    c.mc = nullptr;
    c.mc_cap = 0;
    if (cudaMalloc(&c.mc, sizeof(double) * c.nnzb_cap) != cudaSuccess) {
      c.last_error = "device allocation of the consistent mass failed";
      return MPM_ERR_NO_MEMORY;
    }
    c.mc_cap = c.nnzb_cap;
  }
  const DevView v = c.view();
  const bool gimp = c.shape == MPM_SHAPE_GIMP;
  const int ge = nblk(c.nnzb), gk = nblk(KN);
  if (D == 2) {
    if (gimp) k_consistent_mass<2, true><<<ge, TPB, 0, c.st>>>(c.g, v, c.nnzb, c.row_of, c.col, c.mc);
    else k_consistent_mass<2, false><<<ge, TPB, 0, c.st>>>(c.g, v, c.nnzb, c.row_of, c.col, c.mc);
  } else {
    if (gimp) k_consistent_mass<3, true><<<ge, TPB, 0, c.st>>>(c.g, v, c.nnzb, c.row_of, c.col, c.mc);
    else k_consistent_mass<3, false><<<ge, TPB, 0, c.st>>>(c.g, v, c.nnzb, c.row_of, c.col, c.mc);
  }
  const double phm = c.s.phi_min;
  k_cm_setup<<<gk, TPB, 0, c.st>>>(nn, v, phm, c.row_ptr, c.col, c.mc, F, x, rhs, dinv);
  k_cm_spmv<<<gk, TPB, 0, c.st>>>(nn, K, v, phm, c.row_ptr, c.col, c.mc, x, q);
  k_cm_init<<<gk, TPB, 0, c.st>>>(nn, K, rhs, q, dinv, r, z, p);
  k_cm_dots<<<dim3(CM_NBLK, K), TPB, 0, c.st>>>(nn, r, z, nullptr, part, nullptr);  // r.z
  k_cm_sum<<<1, 32, 0, c.st>>>(K, part, nullptr, rz, nullptr);
  k_cm_dots<<<dim3(CM_NBLK, K), TPB, 0, c.st>>>(nn, rhs, rhs, nullptr, part, nullptr);
  k_cm_sum<<<1, 32, 0, c.st>>>(K, part, nullptr, bb, nullptr);
  c.launches += 8;
  // each field to a relative residual of CM_RTOL (CG on the Jacobi-scaled
  // mass), tested on the device; the host reads the flag every CM_CHECK
  // iterations
  const double CM_RTOL = 1e-14;
  const int CM_MAXIT = 1000, CM_CHECK = 8;
  cudaMemsetAsync(flag, 0, sizeof(double), c.st);
  double hflag = 0.0;
  const dim3 gcm(CM_NBLK, K);
  for (int it = 0; it < CM_MAXIT && hflag == 0.0;) {
    for (int k = 0; k < CM_CHECK && it < CM_MAXIT; ++k, ++it) {
      double *rzc = (it & 1) ? rz2 : rz, *rzx = (it & 1) ? rz : rz2;
      launch_pdl(c, k_cm_qdot, gcm, TPB, 0, nn, v, phm, (const int32_t *)c.row_ptr, (const int32_t *)c.col,
                 (const double *)c.mc, (const double *)p, q, part, (const double *)flag);
      launch_pdl(c, k_cm_update, gcm, TPB, 0, nn, (const double *)rzc, (const double *)part,
                 (const double *)dinv, (const double *)p, (const double *)q, x, r, z, part_rz, part_rr,
                 (const double *)flag);
      launch_pdl(c, k_cm_next, gcm, TPB, 0, nn, K, (const double *)rzc, rzx, (const double *)part_rz,
                 (const double *)part_rr, (const double *)bb, CM_RTOL * CM_RTOL, (const double *)z, p, flag);
    }
    cudaMemcpyAsync(&hflag, flag, sizeof(double), cudaMemcpyDeviceToHost, c.st);
    if (check_cuda(c, cudaStreamSynchronize(c.st), "consistent mass")) return MPM_ERR_CUDA;
  }
  if (hflag == 2.0) {
    c.last_error = "non-finite value in the consistent-mass mapping";
    return MPM_ERR_NONFINITE;
  }
  if (hflag != 1.0) {
    c.last_error = "consistent-mass mapping: CG did not reach its tolerance (ill-conditioned mass)";
    return MPM_ERR_KRYLOV_STAGNATED;
  }
  k_cm_scatter<<<gk, TPB, 0, c.st>>>(nn, F, x);
  UPMPM_LAUNCH(c);
  return check_cuda(c, cudaGetLastError(), "consistent mass");
}

int run_pattern(Ctx &c) {
  const DevView v = c.view();
  const int nbk = nblk(c.g.nnodes, 128);
  const bool gimp = c.shape == MPM_SHAPE_GIMP;
  if (c.d == 2) {
    if (gimp) k_pattern_count<2, true><<<nbk, 128, 0, c.st>>>(c.g, v, c.row_mask, c.row_nnz);
    else k_pattern_count<2, false><<<nbk, 128, 0, c.st>>>(c.g, v, c.row_mask, c.row_nnz);
  } else {
    if (gimp) k_pattern_count<3, true><<<nbk, 128, 0, c.st>>>(c.g, v, c.row_mask, c.row_nnz);
    else k_pattern_count<3, false><<<nbk, 128, 0, c.st>>>(c.g, v, c.row_mask, c.row_nnz);
  }
  UPMPM_LAUNCH(c);
  const int64_t nnzb = scan_exclusive(c, c.row_nnz, c.row_ptr, c.g.nnodes + 1);
  if (nnzb < 0) return MPM_ERR_CUDA;
  if (nnzb > c.nnzb_cap) {
    const int64_t cap = nnzb + nnzb / 4 + 1024;
    cudaFree(c.col);
    cudaFree(c.row_of);
    c.col = c.row_of = nullptr;
    if (cudaMalloc(&c.col, sizeof(int32_t) * cap) != cudaSuccess ||
        cudaMalloc(&c.row_of, sizeof(int32_t) * cap) != cudaSuccess) {
      c.nnzb_cap = 0;
      c.last_error = "device allocation of the block-CSR matrix failed";
      return MPM_ERR_NO_MEMORY;
    }
    c.nnzb_cap = cap;
  }
  c.nnzb = nnzb;
  if (c.d == 2) k_pattern_fill<2><<<nbk, 128, 0, c.st>>>(c.g, c.row_mask, c.row_ptr, c.col, c.row_of);
  else k_pattern_fill<3><<<nbk, 128, 0, c.st>>>(c.g, c.row_mask, c.row_ptr, c.col, c.row_of);
  UPMPM_LAUNCH(c);
  return check_cuda(c, cudaGetLastError(), "pattern");
}

void run_initial_guess(Ctx &c) {
  const DevView v = c.view();
  if (c.d == 2) k_initial_guess<2><<<nblk(c.g.nnodes), TPB, 0, c.st>>>(c.g, c.s.phi_min, v, c.X);
  else k_initial_guess<3><<<nblk(c.g.nnodes), TPB, 0, c.st>>>(c.g, c.s.phi_min, v, c.X);
  UPMPM_LAUNCH(c);
}

void run_fs_diag(Ctx &c) {
  const DevView v = c.view();
  const int nbk = nblk(c.g.nnodes, 128);
  const bool gimp = c.shape == MPM_SHAPE_GIMP;
  if (c.d == 2) {
    if (gimp) k_fs_diag<2, true><<<nbk, 128, 0, c.st>>>(c.g, v, c.fsd);
    else k_fs_diag<2, false><<<nbk, 128, 0, c.st>>>(c.g, v, c.fsd);
  } else {
    if (gimp) k_fs_diag<3, true><<<nbk, 128, 0, c.st>>>(c.g, v, c.fsd);
    else k_fs_diag<3, false><<<nbk, 128, 0, c.st>>>(c.g, v, c.fsd);
  }
  UPMPM_LAUNCH(c);
}

void run_count_terms(Ctx &c) {
  const DevView v = c.view();
  cudaMemsetAsync(c.terms, 0, 2 * sizeof(unsigned long long), c.st);
  if (c.d == 2) k_count_terms<2><<<nblk(c.n), TPB, 0, c.st>>>(c.g, v, c.terms);
  else k_count_terms<3><<<nblk(c.n), TPB, 0, c.st>>>(c.g, v, c.terms);
  UPMPM_LAUNCH(c);
}

// n_q + 1 records of point q (its support box's nodes and its own), 0 at q = n
__global__ void k_pn_count(int64_t n, const int32_t *__restrict__ cnt, int32_t *__restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p > n) return;
  if (p == n) {
    out[p] = 0;
    return;
  }
  const int packed = cnt[p];
  out[p] = unpack_cnt(packed, 0) * unpack_cnt(packed, 1) * max(unpack_cnt(packed, 2), 1) + 1;
}

int run_pn_layout(Ctx &c) {
  k_pn_count<<<nblk(c.n + 1), TPB, 0, c.st>>>(c.n, c.sh_cnt, c.pn_cnt);
  UPMPM_LAUNCH(c);
  const int64_t total = scan_exclusive(c, c.pn_cnt, c.pn_base, c.n + 1);
  if (total < 0 || total > (int64_t)pn_nslot(c.d) * c.n) {
    if (c.last_error.empty()) c.last_error = "Jacobian staging layout";
    return MPM_ERR_CUDA;
  }
  c.pn_total = total;
  return MPM_OK;
}



void run_renorm(Ctx &c) {
  const DevView v = c.view();
  if (c.d == 2) k_renorm<2><<<nblk(c.n), TPB, 0, c.st>>>(c.g, v);
  else k_renorm<3><<<nblk(c.n), TPB, 0, c.st>>>(c.g, v);
  UPMPM_LAUNCH(c);
}

void run_point_eval(Ctx &c, const double *X) {
  prof_begin(c, MPM_PROF_POINT);
  const DevView v = c.view();
  const int nbk = nblk(c.n);
  if (c.d == 2) {
    if (c.dyn) k_point_eval<2, true><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, X);
    else k_point_eval<2, false><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, X);
  } else {
    if (c.dyn) k_point_eval<3, true><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, X);
    else k_point_eval<3, false><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, X);
  }
  UPMPM_LAUNCH(c);
  prof_end(c, MPM_PROF_POINT);
}

void run_residual(Ctx &c, const double *X, double *R, int apply_bc) {
  (void)X;
  prof_begin(c, MPM_PROF_RESIDUAL);
  const DevView v = c.view();
  const int nbk = nblk(c.g.nnodes, 128);
  const bool gimp = c.shape == MPM_SHAPE_GIMP;
#define RES(D, G, Y) k_residual<D, G, Y><<<nbk, 128, 0, c.st>>>(c.g, v, R, apply_bc)
  if (c.d == 2) {
    if (gimp) { if (c.dyn) RES(2, true, true); else RES(2, true, false); }
    else { if (c.dyn) RES(2, false, true); else RES(2, false, false); }
  } else {
    if (gimp) { if (c.dyn) RES(3, true, true); else RES(3, true, false); }
    else { if (c.dyn) RES(3, false, true); else RES(3, false, false); }
  }
#undef RES
  UPMPM_LAUNCH(c);
  prof_end(c, MPM_PROF_RESIDUAL);
}

// FP32 copy of the staging (allocated for the staged FP32 variant only)
int ensure_jacobian_staging32(Ctx &c) {
  return grow_staging(&c.pn32, &c.pn32_cap, c.pn_total, pn_stride(c.d, c.dyn, c.s.hencky, 4));
}

// One assembly with a given kernel configuration: staged (k_point_nodes then
// k_jacobian on the per-(point, node) vectors) or direct (k_jacobian_direct),
// tpb threads per block.  Values in precision T computed
// in precision T from the FP64 records or their FP32 copies.
template <typename T>
void launch_jacobian(Ctx &c, T *val, int apply_bc, int form, int tpb) {
  const DevView v = c.view();
  const bool staged = form == Ctx::JAC_STAGED;
  // the Jacobian kernels take symmetric pairs: half the offsets plus the centre
  const int64_t nthr = pair_threads(c.d, c.g.nnodes);
  const int nbk_pair = (int)((nthr + tpb - 1) / tpb);
  const bool gimp = c.shape == MPM_SHAPE_GIMP;
  using R = T;
  // candidates from the first-node bins in FP32, from the cells in FP64
  constexpr bool FB = sizeof(T) == sizeof(float);
  BasisArrays<R> BA;
  BA.n = c.n;
  BA.cnt = c.sh_cnt;
  BA.act = c.act;
  const R *rec;
  R *pn;
  if constexpr (sizeof(T) == sizeof(double)) {
    BA.S = (const R *)c.sh_S; BA.dS = (const R *)c.sh_dS; BA.S0 = (const R *)c.sh_S0;
    BA.nrm = (const R *)c.sh_nrm; rec = (const R *)c.rec;
    pn = (R *)c.pn;
  } else {
    BA.S = (const R *)c.sh_Sf; BA.dS = (const R *)c.sh_dSf; BA.S0 = (const R *)c.sh_S0f;
    BA.nrm = (const R *)c.sh_nrmf; rec = (const R *)c.recf;
    pn = (R *)c.pn32;
  }
  if (staged && !pn) return;  // callers allocate the staging first
  if (staged) {
    const int npb = nblk((int64_t)PN_LANES * c.n, TPB);
#define PNODES(D, Y, H) k_point_nodes<D, Y, H, R><<<npb, TPB, 0, c.st>>>(c.g, c.s, v, BA, rec, pn)
    const bool hk = c.s.hencky;
    if (c.d == 2) {
      if (c.dyn) { if (hk) PNODES(2, true, true); else PNODES(2, true, false); }
      else { if (hk) PNODES(2, false, true); else PNODES(2, false, false); }
    } else {
      if (c.dyn) { if (hk) PNODES(3, true, true); else PNODES(3, true, false); }
      else { if (hk) PNODES(3, false, true); else PNODES(3, false, false); }
    }
#undef PNODES
    UPMPM_LAUNCH(c);
  }
#define JAC(D, G, Y)                                                                                         \
  do {                                                                                                       \
    if (staged && c.s.hencky)                                                                                \
      k_jacobian<D, G, Y, true, FB, T, R><<<nbk_pair, tpb, 0, c.st>>>(c.g, c.s, v, pn, c.row_mask,           \
                                                                      c.row_ptr, c.col, val, apply_bc);      \
    else if (staged)                                                                                         \
      k_jacobian<D, G, Y, false, FB, T, R><<<nbk_pair, tpb, 0, c.st>>>(c.g, c.s, v, pn, c.row_mask,          \
                                                                       c.row_ptr, c.col, val, apply_bc);     \
    else                                                                                                     \
      k_jacobian_direct<D, G, Y, FB, T, R><<<nbk_pair, tpb, 0, c.st>>>(c.g, c.s, v, BA, rec, c.row_mask,     \
                                                                       c.row_ptr, c.col, val, apply_bc);     \
  } while (0)
  if (c.d == 2) {
    if (gimp) { if (c.dyn) JAC(2, true, true); else JAC(2, true, false); }
    else { if (c.dyn) JAC(2, false, true); else JAC(2, false, false); }
  } else {
    if (gimp) { if (c.dyn) JAC(3, true, true); else JAC(3, true, false); }
    else { if (c.dyn) JAC(3, false, true); else JAC(3, false, false); }
  }
#undef JAC
  UPMPM_LAUNCH(c);
}

// Autotuner of the assembly: every candidate configuration is run twice on
// the context's own data (the first run warms caches and page tables), the
// second timed with CUDA events; the fastest is kept for the rest of the
// context's life.  Candidates: 64, 128, 256 threads per block of each form;
// FP64 is always staged (recomputing the node vectors per term costs FP64
// issue slots, the bound of that kernel), FP32 tries the direct and the
// staged form.  The chosen configuration only moves work between threads or
// stages exact copies (a different summation order), so the values agree to
// the precision's rounding.
template <typename T>
void autotune_jacobian(Ctx &c, T *val, int apply_bc) {
  constexpr int pi = sizeof(T) == sizeof(double) ? 0 : 1;
  Ctx::JacCfg &cfg = c.jac_cfg[pi];
  const int tpbs[3] = {64, 128, 256};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  float best = 1e30f;
  for (int k = 0; k < 3 * Ctx::JAC_FORMS; ++k) c.stats.jac_tune_ms[pi][k] = 0.0f;
  for (int form = 0; form < Ctx::JAC_FORMS; ++form) {
    if (pi == 0 && form != Ctx::JAC_STAGED) continue;
    if (pi == 1 && form == Ctx::JAC_DIRECT && c.s.hencky) continue;  // no Hencky tangent there
    if (pi == 1 && form != Ctx::JAC_DIRECT && ensure_jacobian_staging32(c) != MPM_OK) continue;
    for (int k = 0; k < 3; ++k) {
      launch_jacobian<T>(c, val, apply_bc, form, tpbs[k]);
      cudaEventRecord(e0, c.st);
      launch_jacobian<T>(c, val, apply_bc, form, tpbs[k]);
      cudaEventRecord(e1, c.st);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
      c.stats.jac_tune_ms[pi][form * 3 + k] = ms;
      if (ms < best) {
        best = ms;
        cfg.form = form;
        cfg.tpb = tpbs[k];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cfg.tuned = 1;
  if (pi == 1 && cfg.form == Ctx::JAC_DIRECT && c.pn32) {  // not chosen: give the memory back
    cudaFree(c.pn32);
    c.pn32 = nullptr;
    c.pn32_cap = 0;
  }
}

template <typename T>
void run_jacobian(Ctx &c, T *val, int apply_bc) {
  constexpr int pi = sizeof(T) == sizeof(double) ? 0 : 1;
  Ctx::JacCfg &cfg = c.jac_cfg[pi];
  if (c.opt.autotune && !cfg.tuned && !c.capturing) autotune_jacobian<T>(c, val, apply_bc);
  // without room for the FP32 staging the direct form serves, except for
  // Hencky (whose Newton loop allocates the staging first and stops on failure)
  if (pi == 1 && cfg.form != Ctx::JAC_DIRECT && !c.s.hencky && ensure_jacobian_staging32(c) != MPM_OK)
    cfg.form = Ctx::JAC_DIRECT;
  c.stats.jac_config[pi] = cfg.tpb + 1000 * cfg.form;
  c.stats.jac_tuned[pi] = cfg.tuned;
  prof_begin(c, MPM_PROF_JACOBIAN);
  launch_jacobian<T>(c, val, apply_bc, cfg.form, cfg.tpb);
  prof_end(c, MPM_PROF_JACOBIAN);
}

// One FP32 assembly by a given form and block size (inspection of every
// candidate of the autotuner).
int run_jacobian32_form(Ctx &c, float *val, int apply_bc, int form, int tpb) {
  if (form != Ctx::JAC_DIRECT) {
    const int rc = ensure_jacobian_staging32(c);
    if (rc) return rc;
  }
  launch_jacobian<float>(c, val, apply_bc, form, tpb);
  return check_cuda(c, cudaGetLastError(), "jacobian32");
}

template void run_jacobian<double>(Ctx &, double *, int);
template void run_jacobian<float>(Ctx &, float *, int);

}  // namespace upmpm
