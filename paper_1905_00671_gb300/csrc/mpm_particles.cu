// mpm_particles.cu -- material-point side of one load step:
//   binning + cell sort (Stage 4 "reset" / Stage 1 preparation),
//   closed-form shape functions (Sec. 3.1, Eqs. gimp-basis / gimp-basis-gradient,
//   constant basis S0 of Sec. 4.4),
//   mixture mass of the step (Sec. 2.1, incompressible constituents),
//   Stage 1 lumped P2G (Eq. map-from-particles-to-nodes) as a node-centric gather,
//   Stages 3-4 G2P / FLIP / convection / GIMP domain update (Sec. 3.5).
// Every kernel is HBM- or latency-bound plain FP64 arithmetic; no atomics on
// floating point (node values are gathered in a fixed order), so results are
// run-to-run deterministic.
#include <math.h>

#include "mpm_internal.cuh"

namespace upmpm {

namespace {

constexpr int TPB = 256;

inline int nblk(int64_t n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

// ---------------------------------------------------------------- binning
// Cell of the point centre: floor((x - origin) / h) per axis with IEEE
// round-to-nearest subtract and divide (no contraction), so the key is
// bit-identical to any IEEE implementation of the same expression.
// The cell is taken on the point's own instance grid (its origin and extent)
// and shifted by the instance's offset on the context's background grid.
template <int D>
__global__ void k_bin_keys(GridP g, int64_t n, const double *__restrict__ pf, const InstDev *__restrict__ inst,
                           int32_t *__restrict__ cell, int32_t *__restrict__ count, int *err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const InstDev &I = inst[(int)pf[PF_INST * n + p]];
  int c[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    const double xi = __ddiv_rn(__dsub_rn(pf[(PF_X + k) * n + p], I.org[k]), g.h);
    const double cf = floor(xi);
    if (!(cf >= 0.0) || !(cf <= (double)(I.nc[k] - 1))) {
      atomicOr(err, DE_OUT_OF_GRID);
      cell[p] = -1;
      return;
    }
    c[k] = (int)cf + I.off[k];
  }
  const int32_t id = (int32_t)cell_index(g, c[0], c[1], c[2]);
  cell[p] = id;
  atomicAdd(&count[id], 1);
}

__global__ void k_bin_scatter(int64_t n, const int32_t *__restrict__ cell,
                              const int32_t *__restrict__ start, int32_t *__restrict__ cursor,
                              int32_t *__restrict__ perm) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t c = cell[p];
  if (c < 0) return;
  const int32_t pos = start[c] + atomicAdd(&cursor[c], 1);
  perm[pos] = (int32_t)p;
}

// Within each cell, order the points by original id (insertion sort of a
// short segment): the final order is (cell, id), independent of the order in
// which the scatter's atomics were served.
__global__ void k_bin_sort_cells(int64_t ncells, const int32_t *__restrict__ start,
                                 int32_t *__restrict__ perm, const int64_t *__restrict__ pid) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int32_t b = start[c], e = start[c + 1];
  for (int32_t i = b + 1; i < e; ++i) {
    const int32_t v = perm[i];
    const int64_t key = pid[v];
    int32_t j = i - 1;
    while (j >= b && pid[perm[j]] > key) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

// First-node bins (a second index of the cell-sorted points, for the
// node-centric gathers): key = node index of the point's box origin, and the
// largest box extent per axis (a warp maximum, then one atomic per warp).
template <int D>
__global__ void k_fb_count(GridP g, int64_t n, const int32_t *__restrict__ first,
                           const int32_t *__restrict__ cnt_packed, int32_t *__restrict__ key,
                           int32_t *__restrict__ count, int *__restrict__ cmax, int *err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int ext[3] = {0, 0, 0};
  if (p < n) {
    const int packed = cnt_packed[p];
    int f[3] = {0, 0, 0};
    bool in = true;
    for (int k = 0; k < D; ++k) {
      f[k] = first[k * n + p];
      ext[k] = unpack_cnt(packed, k);
      if (f[k] < 0 || ext[k] < 1 || f[k] + ext[k] > g.nn[k]) in = false;
    }
    if (in) {
      const int32_t id = (int32_t)node_index(g, f);
      key[p] = id;
      atomicAdd(&count[id], 1);
    } else {  // not reached: k_shape clips the box to the grid
      atomicOr(err, DE_SUPPORT);
      key[p] = -1;
      ext[0] = ext[1] = ext[2] = 0;
    }
  }
  for (int k = 0; k < D; ++k) {
    const int m = __reduce_max_sync(0xffffffffu, ext[k]);
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&cmax[k], m);
  }
}

// Within each bin, ascending point index (insertion sort of a short run), so
// that the gathers sum in an order independent of the scatter's atomics.
__global__ void k_fb_sort(int64_t nbins, const int32_t *__restrict__ start, int32_t *__restrict__ perm) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nbins) return;
  const int32_t b = start[f], e = start[f + 1];
  for (int32_t i = b + 1; i < e; ++i) {
    const int32_t v = perm[i];
    int32_t j = i - 1;
    while (j >= b && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

__global__ void k_permute(int64_t n, int nf, const int32_t *__restrict__ perm,
                          const double *__restrict__ src, double *__restrict__ dst,
                          const int64_t *__restrict__ pid, int64_t *__restrict__ pid_dst,
                          const int32_t *__restrict__ surf, int32_t *__restrict__ surf_dst,
                          const int32_t *__restrict__ cell, int32_t *__restrict__ cell_dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t s = perm[i];
  for (int f = 0; f < nf; ++f) dst[f * n + i] = src[f * n + s];
  pid_dst[i] = pid[s];
  surf_dst[i] = surf[s];
  cell_dst[i] = cell[s];
}

// ---------------------------------------------------------------- shape
// Closed form of the GIMP integrals: on each linear piece [a,b] of the hat the
// integral of N is (b - a) N((a + b) / 2); the gradient integral is +-(b - a);
// the constant basis of Sec. 4.4 integrates 1/2.  The domain is the point's
// domain intersected with the grid box, normalised by its length.
template <int D, bool GIMP>
__global__ void k_shape(GridP g, int64_t n, const double *__restrict__ pf, const InstDev *__restrict__ inst,
                        int32_t *__restrict__ first, int32_t *__restrict__ cnt_packed,
                        double *__restrict__ S, double *__restrict__ dS, double *__restrict__ S0,
                        float *__restrict__ Sf, float *__restrict__ dSf, float *__restrict__ S0f,
                        int *err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const InstDev &I = inst[(int)pf[PF_INST * n + p]];
  int packed = 0;
  for (int k = 0; k < 3; ++k) {
    double s[MAXS] = {0, 0, 0, 0}, ds[MAXS] = {0, 0, 0, 0}, s0[MAXS] = {0, 0, 0, 0};
    int f0 = 0, cn = 1;
    if (k >= D) {
      s[0] = 1.0;
      s0[0] = 1.0;
    } else {
      // on the point's own instance grid: its box clips the GIMP domain
      const double dx = __dsub_rn(pf[(PF_X + k) * n + p], I.org[k]);
      const double h = g.h;
      const double cf = floor(__ddiv_rn(dx, h));
      if (!(cf >= 0.0) || !(cf <= (double)(I.nc[k] - 1))) {
        atomicOr(err, DE_OUT_OF_GRID);
        return;
      }
      if (!GIMP) {
        const double t = __dsub_rn(__ddiv_rn(dx, h), cf);
        f0 = (int)cf;
        cn = 2;
        s[0] = 1.0 - t;
        s[1] = t;
        ds[0] = -1.0 / h;
        ds[1] = 1.0 / h;
        s0[0] = 0.5;
        s0[1] = 0.5;
      } else {
        const double lp = pf[(PF_LP + k) * n + p];
        if (!(lp > 0.0) || !(lp < h)) {
          atomicOr(err, DE_SUPPORT);
          return;
        }
        const double lo = fmax(__ddiv_rn(__dsub_rn(dx, lp), h), 0.0);
        const double hi = fmin(__ddiv_rn(__dadd_rn(dx, lp), h), (double)I.nc[k]);
        const int i0 = (int)floor(lo), i1 = (int)ceil(hi);
        if (i1 - i0 + 1 > MAXS) {
          atomicOr(err, DE_SUPPORT);
          return;
        }
        f0 = i0;
        cn = i1 - i0 + 1;
        const double inv_len = 1.0 / (hi - lo);
        for (int i = i0; i <= i1; ++i) {
          double iN = 0.0, idN = 0.0, iH = 0.0;
          const double a = fmax(lo, (double)(i - 1)), b = fmin(hi, (double)i);
          if (b > a) {  // rising piece, N = 1 + (xi - i)
            iN += (b - a) * (1.0 + (0.5 * (a + b) - (double)i));
            idN += (b - a);
            iH += 0.5 * (b - a);
          }
          const double c = fmax(lo, (double)i), e = fmin(hi, (double)(i + 1));
          if (e > c) {  // falling piece, N = 1 - (xi - i)
            iN += (e - c) * (1.0 - (0.5 * (c + e) - (double)i));
            idN -= (e - c);
            iH += 0.5 * (e - c);
          }
          s[i - i0] = iN * inv_len;
          ds[i - i0] = idN * inv_len / h;
          s0[i - i0] = iH * inv_len;
        }
      }
    }
    first[k * n + p] = f0 + (k < D ? I.off[k] : 0);
    packed |= cn << (4 * k);
    for (int q = 0; q < MAXS; ++q) {
      S[(k * MAXS + q) * n + p] = s[q];
      dS[(k * MAXS + q) * n + p] = ds[q];
      S0[(k * MAXS + q) * n + p] = s0[q];
      if (Sf) {
        Sf[(k * MAXS + q) * n + p] = (float)s[q];
        dSf[(k * MAXS + q) * n + p] = (float)ds[q];
        S0f[(k * MAXS + q) * n + p] = (float)s0[q];
      }
    }
  }
  cnt_packed[p] = packed;
}

// ---------------------------------------------------------------- mass
// Incompressible constituents: porosity phi = 1 - (1 - phi0) / J, mixture
// density rho = (1 - phi) rho_s + phi rho_f, point mass rho V at t_n (frozen
// over the step).
template <int D>
__global__ void k_mass(int64_t n, StepP s, const double *__restrict__ pf, double *__restrict__ m) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  double F[9];
  for (int i = 0; i < D * D; ++i) F[i] = pf[(PF_F + i) * n + p];
  const double J = det_d<D>(F);
  const double phi = 1.0 - (1.0 - s.phi0) / J;
  const double rho = (1.0 - phi) * s.rho_s + phi * s.rho_f;
  m[p] = rho * pf[PF_V * n + p];
}

// ---------------------------------------------------------------- Stage 1
// Node-centric gather: each thread owns one node and sums S m f over the
// points of the first-node bins that can hold it, in (bin, index) order.
template <int D, bool GIMP, bool DYN>
__global__ void k_p2g(GridP g, DevView v) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= g.nnodes) return;
  const int64_t n = v.n;
  int ac[3];
  node_coords(g, a, ac);
  int lo[3], hi[3];
  fb_window<D>(v.fb_cmax, ac, ac, lo, hi);
  double Msum = 0.0, Vsum = 0.0, mp = 0.0, mv[3] = {0, 0, 0}, ma[3] = {0, 0, 0}, mpd = 0.0, mpdd = 0.0;
  for (int f2 = lo[2]; f2 <= hi[2]; ++f2)
    for (int f1 = lo[1]; f1 <= hi[1]; ++f1) {
      int32_t ib, ie;
      fb_run(g, v.fb_start, lo[0], hi[0], f1, f2, ib, ie);
      for (int32_t i = ib; i < ie; ++i) {
        const int32_t q = v.fb_perm[i];
        const int packed = v.sh_cnt[q];
        double S = 1.0;
        bool in = true;
        for (int k = 0; k < D; ++k) {
          const int off = ac[k] - v.sh_first[k * n + q];
          if (off < 0 || off >= unpack_cnt(packed, k)) {
            in = false;
            break;
          }
          S *= v.sh_S[(k * MAXS + off) * n + q];
        }
        if (!in) continue;
        const double w = S * v.m[q];
        Msum += w;
        Vsum += S * v.pf[PF_V * n + q];
        mp += w * v.pf[PF_P * n + q];
        if (DYN) {
          for (int k = 0; k < D; ++k) {
            mv[k] += w * v.pf[(PF_VEL + k) * n + q];
            ma[k] += w * v.pf[(PF_ACC + k) * n + q];
          }
          mpd += w * v.pf[PF_PD * n + q];
          mpdd += w * v.pf[PF_PDD * n + q];
        }
      }
    }
  const int64_t nn = g.nnodes;
  v.M[a] = Msum;
  double hd = g.h;
  for (int k = 1; k < D; ++k) hd *= g.h;
  v.phi[a] = Vsum / hd;
  const double inv = Msum > 0.0 ? 1.0 / Msum : 0.0;
  v.Pn[a] = mp * inv;
  if (DYN) {
    for (int k = 0; k < D; ++k) {
      v.vn[k * nn + a] = mv[k] * inv;
      v.an[k * nn + a] = ma[k] * inv;
    }
    v.pdn[a] = mpd * inv;
    v.pddn[a] = mpdd * inv;
  }
}

// ---------------------------------------------------------------- Stages 3-4
// Diagonal of the right stretch U = (F^T F)^{1/2} from the eigenvalues of
// C = F^T F only (Hoger & Carlson's closed form in the invariants of U):
//   U = (-C^2 + (i^2 - ii) C + i iii 1) / (i ii - iii),
// with i, ii, iii the invariants of U (principal stretches sqrt(eig C)).  In 2D
// U = (C + sqrt(det C) 1) / sqrt(tr C + 2 sqrt(det C)).
template <int D>
__device__ inline void stretch_diag(const double *F, double *Ud) {
  double C[9];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
      for (int k = 0; k < D; ++k) s += F[k * D + i] * F[k * D + j];
      C[i * D + j] = s;
    }
  if (D == 2) {
    const double sd = sqrt(C[0] * C[3] - C[1] * C[2]);
    const double den = sqrt(C[0] + C[3] + 2.0 * sd);
    Ud[0] = (C[0] + sd) / den;
    Ud[1] = (C[3] + sd) / den;
    return;
  }
  // eigenvalues of the symmetric C (trigonometric method)
  const double q = (C[0] + C[4] + C[8]) / 3.0;
  const double p1 = C[1] * C[1] + C[2] * C[2] + C[5] * C[5];
  const double p2 = (C[0] - q) * (C[0] - q) + (C[4] - q) * (C[4] - q) + (C[8] - q) * (C[8] - q) + 2.0 * p1;
  double e1, e2, e3;
  if (p2 <= 1e-30 * q * q) {
    e1 = e2 = e3 = q;
  } else {
    const double pp = sqrt(p2 / 6.0);
    double B[9];
    for (int i = 0; i < 9; ++i) B[i] = C[i] / pp;
    B[0] -= q / pp;
    B[4] -= q / pp;
    B[8] -= q / pp;
    double r = 0.5 * det_d<3>(B);
    r = fmin(1.0, fmax(-1.0, r));
    const double phi = acos(r) / 3.0;
    e1 = q + 2.0 * pp * cos(phi);
    e3 = q + 2.0 * pp * cos(phi + 2.0943951023931957);  // + 2 pi / 3
    e2 = 3.0 * q - e1 - e3;
  }
  const double l1 = sqrt(e1), l2 = sqrt(e2), l3 = sqrt(e3);
  const double i1 = l1 + l2 + l3, i2 = l1 * l2 + l2 * l3 + l3 * l1, i3 = l1 * l2 * l3;
  const double den = i1 * i2 - i3;
  for (int k = 0; k < 3; ++k) {
    double c2 = 0.0;  // (C^2)_kk
    for (int m = 0; m < 3; ++m) c2 += C[k * 3 + m] * C[m * 3 + k];
    Ud[k] = (-c2 + (i1 * i1 - i2) * C[k * 3 + k] + i1 * i3) / den;
  }
}

template <int D, bool DYN>
__global__ void k_g2p(GridP g, StepP s, DevView v, const double *__restrict__ X) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = v.n;
  if (p >= n) return;
  constexpr int NB = D + 1;
  const int64_t nn = g.nnodes;
  const int packed = v.sh_cnt[p];
  int f[3], cn[3];
  for (int k = 0; k < 3; ++k) {
    f[k] = v.sh_first[k * n + p];
    cn[k] = unpack_cnt(packed, k);
  }
  double dF[9] = {0}, du[3] = {0, 0, 0}, ph = 0.0;
  double anew[3] = {0, 0, 0}, vinc[3] = {0, 0, 0}, pdh = 0.0, pddh = 0.0;
  for (int k = 0; k < D; ++k) dF[k * D + k] = 1.0;
  const double b = s.beta, gm = s.gamma, dt = s.dt;
  for (int s2 = 0; s2 < cn[2]; ++s2)
    for (int s1 = 0; s1 < cn[1]; ++s1)
      for (int s0 = 0; s0 < cn[0]; ++s0) {
        const int sl[3] = {s0, s1, s2};
        const int nc3[3] = {f[0] + s0, f[1] + s1, f[2] + s2};
        const int64_t a = node_index(g, nc3);
        double Sa, S0a, Gn[3];
        basis_at<D>(v, p, sl, a, Sa, S0a, Gn);
        for (int i = 0; i < D; ++i) {
          const double dU = X[a * NB + i];
          du[i] += Sa * dU;
          for (int k = 0; k < D; ++k) dF[i * D + k] += dU * Gn[k];
        }
        const double P = X[a * NB + D];
        ph += Sa * P;
        if (DYN) {
          for (int i = 0; i < D; ++i) {
            const double dU = X[a * NB + i];
            const double vn = v.vn[i * nn + a], an = v.an[i * nn + a];
            const double aa = dU / (b * dt * dt) - vn / (b * dt) + (1.0 - 1.0 / (2.0 * b)) * an;
            anew[i] += Sa * aa;
            vinc[i] += Sa * ((1.0 - gm) * an + gm * aa);
          }
          const double dP = P - v.Pn[a];
          const double pdn = v.pdn[a], pddn = v.pddn[a];
          pdh += Sa * (gm / (b * dt) * dP + (1.0 - gm / b) * pdn + (1.0 - gm / (2.0 * b)) * dt * pddn);
          pddh += Sa * (dP / (b * dt * dt) - pdn / (b * dt) + (1.0 - 1.0 / (2.0 * b)) * pddn);
        }
      }
  const double dJ = det_d<D>(dF);
  if (!(dJ > 0.0)) {
    atomicOr(v.err, DE_NEG_J);
    return;
  }
  double* pf = v.pf;
  if (DYN) {
    for (int i = 0; i < D; ++i) {
      pf[(PF_ACC + i) * n + p] = anew[i];
      pf[(PF_VEL + i) * n + p] += dt * vinc[i];
    }
    pf[PF_PD * n + p] = pdh;
    pf[PF_PDD * n + p] = pddh;
  }
  double Fn[9], Fw[9];
  for (int i = 0; i < D * D; ++i) Fn[i] = pf[(PF_F + i) * n + p];
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int k = 0; k < D; ++k) acc += dF[i * D + k] * Fn[k * D + j];
      Fw[i * D + j] = acc;
    }
  for (int i = 0; i < D * D; ++i) pf[(PF_F + i) * n + p] = Fw[i];
  for (int i = 0; i < D; ++i) {
    pf[(PF_X + i) * n + p] += du[i];
    pf[(PF_U + i) * n + p] += du[i];
  }
  pf[PF_V * n + p] = dJ * pf[PF_V * n + p];
  pf[PF_P * n + p] = ph;
  double Ud[3];
  stretch_diag<D>(Fw, Ud);
  for (int k = 0; k < D; ++k) pf[(PF_LP + k) * n + p] = pf[(PF_LP0 + k) * n + p] * Ud[k];
}

}  // namespace

// ============================================================== launchers
int run_binning(Ctx &c) {
  const int64_t n = c.n, nc = c.g.ncells;
  // points per cell (integer atomics: the counts are exact and order-free)
  cudaMemsetAsync(c.cell_cursor, 0, sizeof(int32_t) * (nc + 1), c.st);
  if (c.d == 2)
    k_bin_keys<2><<<nblk(n), TPB, 0, c.st>>>(c.g, n, c.pf, c.inst, c.cell, c.cell_cursor, c.err);
  else
    k_bin_keys<3><<<nblk(n), TPB, 0, c.st>>>(c.g, n, c.pf, c.inst, c.cell, c.cell_cursor, c.err);
  UPMPM_LAUNCH(c);
  int rc = read_dev_err(c);
  if (rc) return rc;
  if (scan_exclusive(c, c.cell_cursor, c.cell_start, nc + 1) != n) {
    c.last_error = "binning lost points";
    return MPM_ERR_CUDA;
  }
  cudaMemsetAsync(c.cell_cursor, 0, sizeof(int32_t) * nc, c.st);
  k_bin_scatter<<<nblk(n), TPB, 0, c.st>>>(n, c.cell, c.cell_start, c.cell_cursor, c.perm);
  k_bin_sort_cells<<<nblk(nc), TPB, 0, c.st>>>(nc, c.cell_start, c.perm, c.pid);
  k_permute<<<nblk(n), TPB, 0, c.st>>>(n, PF_COUNT, c.perm, c.pf, c.pf_alt, c.pid, c.pid_alt,
                                       c.surf, c.surf_alt, c.cell, c.cell_tmp);
  c.launches += 3;
  std::swap(c.pf, c.pf_alt);
  std::swap(c.pid, c.pid_alt);
  std::swap(c.surf, c.surf_alt);
  std::swap(c.cell, c.cell_tmp);
  return check_cuda(c, cudaGetLastError(), "binning");
}

// First-node bins of the step (after run_shape; the box origins and extents
// are fixed over the step): counts and the largest extents, an exclusive scan,
// the scatter, and the per-bin sort.
int run_first_bins(Ctx &c) {
  const int64_t n = c.n, nn = c.g.nnodes;
  cudaMemsetAsync(c.fb_cursor, 0, sizeof(int32_t) * (nn + 1), c.st);
  cudaMemsetAsync(c.fb_cmax, 0, sizeof(int) * 4, c.st);
  if (c.d == 2)
    k_fb_count<2><<<nblk(n), TPB, 0, c.st>>>(c.g, n, c.sh_first, c.sh_cnt, c.fb_key, c.fb_cursor, c.fb_cmax, c.err);
  else
    k_fb_count<3><<<nblk(n), TPB, 0, c.st>>>(c.g, n, c.sh_first, c.sh_cnt, c.fb_key, c.fb_cursor, c.fb_cmax, c.err);
  UPMPM_LAUNCH(c);
  if (scan_exclusive(c, c.fb_cursor, c.fb_start, nn + 1) != n) {
    int rc = read_dev_err(c);
    if (rc) return rc;
    c.last_error = "first-node bins lost points";
    return MPM_ERR_CUDA;
  }
  cudaMemsetAsync(c.fb_cursor, 0, sizeof(int32_t) * nn, c.st);
  k_bin_scatter<<<nblk(n), TPB, 0, c.st>>>(n, c.fb_key, c.fb_start, c.fb_cursor, c.fb_perm);
  k_fb_sort<<<nblk(nn), TPB, 0, c.st>>>(nn, c.fb_start, c.fb_perm);
  c.launches += 2;
  return check_cuda(c, cudaGetLastError(), "first-node bins");
}

void run_shape(Ctx &c) {
  const int64_t n = c.n;
  const int nbk = nblk(n);
  if (c.d == 2) {
    if (c.shape == MPM_SHAPE_GIMP)
      k_shape<2, true><<<nbk, TPB, 0, c.st>>>(c.g, n, c.pf, c.inst, c.sh_first, c.sh_cnt, c.sh_S, c.sh_dS, c.sh_S0, c.sh_Sf, c.sh_dSf, c.sh_S0f, c.err);
    else
      k_shape<2, false><<<nbk, TPB, 0, c.st>>>(c.g, n, c.pf, c.inst, c.sh_first, c.sh_cnt, c.sh_S, c.sh_dS, c.sh_S0, c.sh_Sf, c.sh_dSf, c.sh_S0f, c.err);
  } else {
    if (c.shape == MPM_SHAPE_GIMP)
      k_shape<3, true><<<nbk, TPB, 0, c.st>>>(c.g, n, c.pf, c.inst, c.sh_first, c.sh_cnt, c.sh_S, c.sh_dS, c.sh_S0, c.sh_Sf, c.sh_dSf, c.sh_S0f, c.err);
    else
      k_shape<3, false><<<nbk, TPB, 0, c.st>>>(c.g, n, c.pf, c.inst, c.sh_first, c.sh_cnt, c.sh_S, c.sh_dS, c.sh_S0, c.sh_Sf, c.sh_dSf, c.sh_S0f, c.err);
  }
  UPMPM_LAUNCH(c);
}

void run_mass(Ctx &c) {
  if (c.d == 2) k_mass<2><<<nblk(c.n), TPB, 0, c.st>>>(c.n, c.s, c.pf, c.m);
  else k_mass<3><<<nblk(c.n), TPB, 0, c.st>>>(c.n, c.s, c.pf, c.m);
  UPMPM_LAUNCH(c);
}

void run_p2g(Ctx &c) {
  prof_begin(c, MPM_PROF_P2G);
  const DevView v = c.view();
  const int nbk = nblk(c.g.nnodes, 128);
  const bool gimp = c.shape == MPM_SHAPE_GIMP;
#define P2G(D, G, Y) k_p2g<D, G, Y><<<nbk, 128, 0, c.st>>>(c.g, v)
  if (c.d == 2) {
    if (gimp) { if (c.dyn) P2G(2, true, true); else P2G(2, true, false); }
    else { if (c.dyn) P2G(2, false, true); else P2G(2, false, false); }
  } else {
    if (gimp) { if (c.dyn) P2G(3, true, true); else P2G(3, true, false); }
    else { if (c.dyn) P2G(3, false, true); else P2G(3, false, false); }
  }
#undef P2G
  UPMPM_LAUNCH(c);
  prof_end(c, MPM_PROF_P2G);
}

void run_g2p(Ctx &c) {
  prof_begin(c, MPM_PROF_G2P);
  const DevView v = c.view();
  const int nbk = nblk(c.n);
  if (c.d == 2) {
    if (c.dyn) k_g2p<2, true><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, c.X);
    else k_g2p<2, false><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, c.X);
  } else {
    if (c.dyn) k_g2p<3, true><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, c.X);
    else k_g2p<3, false><<<nbk, TPB, 0, c.st>>>(c.g, c.s, v, c.X);
  }
  UPMPM_LAUNCH(c);
  prof_end(c, MPM_PROF_G2P);
}

}  // namespace upmpm
