/*
 * upmpm_oracle.c -- plain FP64 CPU oracle of the stabilized implicit u-p
 * material point method (Zhao & Choo, arXiv 1905.00671).
 *
 * TEST INFRASTRUCTURE ONLY (see upmpm_oracle.h).  Written for a reader who
 * checks it against the paper line by line: every loop runs over material
 * points in their input order and accumulates exactly the integrands of the
 * paper, with no blocking, fusion or reordering.
 *
 * Pins (tests/test_oracle_*.py): partition of unity and linear reproduction of
 * both bases, GIMP == original MPM when no domain crosses a cell (Sec. 4.4),
 * P2G mass conservation, stabilization block symmetric PSD with cellwise
 * constants in its null space, central finite differences of the residual
 * against the analytic Jacobian, Terzaghi consolidation against its series
 * (Sec. 5.1), zero stress at F = 1 and the small-strain limit of the stress.
 * Parity status per function is listed at each function.
 */
#include "upmpm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXD 3
#define MAXS 4 /* nodes per axis in a support (GIMP half length < h) */

int64_t orc_nnodes(const orc_grid *g) {
  int64_t n = 1;
  for (int k = 0; k < g->dim; ++k) n *= (int64_t)(g->ncell[k] + 1);
  return n;
}

int64_t orc_ncells(const orc_grid *g) {
  int64_t n = 1;
  for (int k = 0; k < g->dim; ++k) n *= (int64_t)g->ncell[k];
  return n;
}

/* ------------------------------------------------------------------------
 * Shape functions (Sec. 3.1, Eqs. gimp-basis / gimp-basis-gradient; the
 * constant basis S0 of Sec. 4.4).  The GIMP values are integrated numerically:
 * the linear hat N_i is split at its node and each linear piece is integrated
 * with 2-point Gauss-Legendre (exact for linear integrands).
 * Pinned: partition of unity, linear reproduction, GIMP == FE when domains
 * touch cell faces only, sum S0 = 1.
 * ---------------------------------------------------------------------- */
static double hat(double t) { return 1.0 - fabs(t); }

static void gl2_piece(double a, double b, double node, double *intN, double *intdN,
                      double *intHalf, double slope) {
  /* 2-point Gauss-Legendre on [a,b] of N(xi) = 1 - |xi - node|, of its slope
   * (constant on the piece) and of the constant 1/2. */
  if (!(b > a)) return;
  const double r = 1.0 / sqrt(3.0);
  const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
  const double q1 = mid - half * r, q2 = mid + half * r;
  *intN += half * (hat(q1 - node) + hat(q2 - node));
  *intdN += half * (slope + slope);
  *intHalf += half * (0.5 + 0.5);
}

/* dx = x - origin along the axis. */
static int shape_axis(int32_t shape, double dx, double lp, double h, int32_t ncell,
                      int32_t *first, int32_t *count, double *S, double *dS, double *S0) {
  for (int s = 0; s < MAXS; ++s) S[s] = dS[s] = S0[s] = 0.0;
  if (shape == 0) {
    const double xi = dx / h;
    const double c = floor(xi);
    if (!(c >= 0.0) || !(c <= (double)(ncell - 1))) return ORC_ERR_OUT_OF_GRID;
    const double t = xi - c;
    *first = (int32_t)c;
    *count = 2;
    S[0] = 1.0 - t;   /* N_c(x)   */
    S[1] = t;         /* N_c+1(x) */
    dS[0] = -1.0 / h;
    dS[1] = 1.0 / h;
    S0[0] = 0.5;      /* R5: a point domain puts 1/2 on each node of its cell */
    S0[1] = 0.5;
    return ORC_OK;
  }
  if (!(lp > 0.0) || !(lp < h)) return ORC_ERR_BAD_ARG;
  /* the centre must lie in a cell of the grid (same rule as the binning) */
  const double c = floor(dx / h);
  if (!(c >= 0.0) || !(c <= (double)(ncell - 1))) return ORC_ERR_OUT_OF_GRID;
  /* Omega_mp intersected with the grid box; the basis is normalised by the
   * length of that intersection so that it still sums to one. */
  const double lo = fmax((dx - lp) / h, 0.0), hi = fmin((dx + lp) / h, (double)ncell);
  const int32_t i0 = (int32_t)floor(lo), i1 = (int32_t)ceil(hi);
  if (i1 - i0 + 1 > MAXS) return ORC_ERR_BAD_ARG;
  *first = i0;
  *count = i1 - i0 + 1;
  const double len = hi - lo;
  for (int32_t i = i0; i <= i1; ++i) {
    double iN = 0.0, idN = 0.0, iH = 0.0;
    /* left piece of the hat: xi in [i-1, i], slope +1 */
    gl2_piece(fmax(lo, (double)i - 1.0), fmin(hi, (double)i), (double)i, &iN, &idN, &iH, 1.0);
    /* right piece: xi in [i, i+1], slope -1 */
    gl2_piece(fmax(lo, (double)i), fmin(hi, (double)i + 1.0), (double)i, &iN, &idN, &iH, -1.0);
    S[i - i0] = iN / len;
    dS[i - i0] = idN / len / h; /* d/dx = (1/h) d/dxi */
    S0[i - i0] = iH / len;
  }
  return ORC_OK;
}

int orc_shape_1d(int32_t shape, double dx, double lp, double h, int32_t ncell,
                 int32_t *first, int32_t *count, double *S, double *dS, double *S0) {
  return shape_axis(shape, dx, lp, h, ncell, first, count, S, dS, S0);
}

int orc_shape(const orc_grid *g, int64_t n, const double *x, const double *lp,
              int32_t *first, int32_t *count, double *S, double *dS, double *S0) {
  const int d = g->dim;
  for (int64_t p = 0; p < n; ++p) {
    for (int k = 0; k < d; ++k) {
      const int64_t o = p * 3 + k;
      int rc = shape_axis(g->shape, x[p * d + k] - g->origin[k], lp ? lp[p * d + k] : 0.0,
                          g->h, g->ncell[k], &first[o], &count[o], &S[o * MAXS],
                          &dS[o * MAXS], &S0[o * MAXS]);
      if (rc) return rc;
    }
    for (int k = d; k < 3; ++k) {
      const int64_t o = p * 3 + k;
      first[o] = 0;
      count[o] = 1;
      for (int s = 0; s < MAXS; ++s) S[o * MAXS + s] = dS[o * MAXS + s] = S0[o * MAXS + s] = 0.0;
      S[o * MAXS] = 1.0;
      S0[o * MAXS] = 1.0;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Binning: cell of the material point centre, then all points ordered by
 * (cell, input index).  Bit-exact reference for the GPU's cell sort.
 * ---------------------------------------------------------------------- */
typedef struct { int64_t key; int64_t idx; } orc_pair;
static int cmp_pair(const void *a, const void *b) {
  const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

int orc_bin(const orc_grid *g, int64_t n, const double *x, int32_t *cell, int64_t *order) {
  const int d = g->dim;
  orc_pair *pr = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(n > 0 ? n : 1));
  for (int64_t p = 0; p < n; ++p) {
    int64_t id = 0, stride = 1;
    for (int k = 0; k < d; ++k) {
      const double c = floor((x[p * d + k] - g->origin[k]) / g->h);
      if (!(c >= 0.0) || !(c <= (double)(g->ncell[k] - 1))) {
        free(pr);
        return ORC_ERR_OUT_OF_GRID;
      }
      id += (int64_t)c * stride;
      stride *= g->ncell[k];
    }
    cell[p] = (int32_t)id;
    pr[p].key = id;
    pr[p].idx = p;
  }
  qsort(pr, (size_t)n, sizeof(orc_pair), cmp_pair);
  for (int64_t p = 0; p < n; ++p) order[p] = pr[p].idx;
  free(pr);
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Support helpers.
 * ---------------------------------------------------------------------- */
typedef struct {
  int ns;                   /* number of support nodes */
  int64_t node[MAXS * MAXS * MAXS];
  double S[MAXS * MAXS * MAXS];
  double S0[MAXS * MAXS * MAXS];
  double Gn[MAXS * MAXS * MAXS][MAXD]; /* gradient in the t_n configuration */
  int ax[MAXS * MAXS * MAXS][MAXD];    /* node index per axis */
} support;

/* Nodes of the point's support box with their S, S0 and t_n gradient.  When
 * `active` is given and some box node is inactive (its volume fraction is at
 * or below the threshold), that node is removed from this point's basis and
 * the rest is renormalised so that constants stay exactly reproduced:
 *   S'_a = S_a / sum S,  grad S'_a = (grad S_a - S'_a grad sum S) / sum S,
 *   S0'_a = S0_a / sum S0   (sums over the active box nodes). */
static void build_support_active(const orc_grid *g, int64_t p, const int32_t *first,
                                 const int32_t *count, const double *S, const double *dS,
                                 const double *S0, const uint8_t *active, support *sp);

static void build_support(const orc_grid *g, int64_t p, const int32_t *first, const int32_t *count,
                          const double *S, const double *dS, const double *S0, support *sp) {
  const int d = g->dim;
  const int64_t nn0 = g->ncell[0] + 1, nn1 = g->ncell[1] + 1;
  int cnt[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) cnt[k] = count[p * 3 + k];
  sp->ns = 0;
  for (int s2 = 0; s2 < cnt[2]; ++s2)
    for (int s1 = 0; s1 < cnt[1]; ++s1)
      for (int s0 = 0; s0 < cnt[0]; ++s0) {
        const int s[3] = {s0, s1, s2};
        int idx[3] = {0, 0, 0};
        double w = 1.0, w0 = 1.0;
        for (int k = 0; k < d; ++k) {
          idx[k] = first[p * 3 + k] + s[k];
          w *= S[(p * 3 + k) * MAXS + s[k]];
          w0 *= S0[(p * 3 + k) * MAXS + s[k]];
        }
        const int q = sp->ns++;
        sp->node[q] = idx[0] + nn0 * (idx[1] + nn1 * idx[2]);
        sp->S[q] = w;
        sp->S0[q] = w0;
        for (int k = 0; k < d; ++k) {
          double gk = dS ? dS[(p * 3 + k) * MAXS + s[k]] : 0.0;
          for (int l = 0; l < d; ++l)
            if (l != k) gk *= S[(p * 3 + l) * MAXS + s[l]];
          sp->Gn[q][k] = gk;
          sp->ax[q][k] = idx[k];
        }
      }
}

static void build_support_active(const orc_grid *g, int64_t p, const int32_t *first,
                                 const int32_t *count, const double *S, const double *dS,
                                 const double *S0, const uint8_t *active, support *sp) {
  build_support(g, p, first, count, S, dS, S0, sp);
  if (!active) return;
  int any = 0;
  for (int q = 0; q < sp->ns; ++q)
    if (!active[sp->node[q]]) any = 1;
  if (!any) return;
  const int d = g->dim;
  double sum = 0.0, sum0 = 0.0, gsum[MAXD] = {0.0, 0.0, 0.0};
  for (int q = 0; q < sp->ns; ++q) {
    if (!active[sp->node[q]]) continue;
    sum += sp->S[q];
    sum0 += sp->S0[q];
    for (int k = 0; k < d; ++k) gsum[k] += sp->Gn[q][k];
  }
  for (int q = 0; q < sp->ns; ++q) {
    if (!active[sp->node[q]]) {
      sp->S[q] = sp->S0[q] = 0.0;
      for (int k = 0; k < d; ++k) sp->Gn[q][k] = 0.0;
      continue;
    }
    const double Sr = sp->S[q] / sum;
    for (int k = 0; k < d; ++k) sp->Gn[q][k] = (sp->Gn[q][k] - Sr * gsum[k]) / sum;
    sp->S[q] = Sr;
    sp->S0[q] = sp->S0[q] / sum0;
  }
}

/* The basis of one point as orc_eval and orc_g2p use it: the nodes of its
 * support box with S, S0 and the t_n gradient, inactive nodes removed and the
 * rest renormalised (reading R7).  Exposed for the pins of that rule; returns
 * the number of box nodes written (at most MAXS^d) or ORC_ERR_BAD_ARG. */
int orc_point_basis(const orc_grid *g, int64_t p, const int32_t *first, const int32_t *count,
                    const double *S, const double *dS, const double *S0, const uint8_t *active,
                    int64_t *node, double *Sv, double *Gv, double *S0v) {
  if (!g || p < 0 || !first || !count || !S || !dS || !S0 || !node || !Sv || !Gv || !S0v)
    return ORC_ERR_BAD_ARG;
  const int d = g->dim;
  support *sp = (support *)malloc(sizeof(support));
  if (!sp) return ORC_ERR_BAD_ARG;
  build_support_active(g, p, first, count, S, dS, S0, active, sp);
  const int ns = sp->ns;
  for (int q = 0; q < ns; ++q) {
    node[q] = sp->node[q];
    Sv[q] = sp->S[q];
    S0v[q] = sp->S0[q];
    for (int k = 0; k < d; ++k) Gv[q * d + k] = sp->Gn[q][k];
  }
  free(sp);
  return ns;
}

/* ------------------------------------------------------------------------
 * Sparsity: node b couples with node a iff some material point has both in
 * its support; every node couples with itself.  Rows over all grid nodes,
 * columns ascending.  Bit-exact reference for the GPU's block-CSR pattern.
 * ---------------------------------------------------------------------- */
static int cmp_i64(const void *a, const void *b) {
  const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

int64_t orc_pattern(const orc_grid *g, int64_t n, const int32_t *first, const int32_t *count,
                    int64_t *row_ptr, int32_t *col_idx, int64_t cap) {
  const int d = g->dim;
  const int64_t nn = orc_nnodes(g);
  const int64_t nn0 = g->ncell[0] + 1, nn1 = g->ncell[1] + 1;
  int64_t npairs = nn;
  for (int64_t p = 0; p < n; ++p) {
    int64_t ns = 1;
    for (int k = 0; k < d; ++k) ns *= count[p * 3 + k];
    npairs += ns * ns;
  }
  int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)npairs);
  int64_t q = 0;
  for (int64_t a = 0; a < nn; ++a) key[q++] = a * nn + a;
  for (int64_t p = 0; p < n; ++p) {
    int cnt[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) cnt[k] = count[p * 3 + k];
    int64_t nodes[MAXS * MAXS * MAXS];
    int ns = 0;
    for (int s2 = 0; s2 < cnt[2]; ++s2)
      for (int s1 = 0; s1 < cnt[1]; ++s1)
        for (int s0 = 0; s0 < cnt[0]; ++s0) {
          const int64_t i0 = first[p * 3 + 0] + s0;
          const int64_t i1 = d > 1 ? first[p * 3 + 1] + s1 : 0;
          const int64_t i2 = d > 2 ? first[p * 3 + 2] + s2 : 0;
          nodes[ns++] = i0 + nn0 * (i1 + nn1 * i2);
        }
    for (int i = 0; i < ns; ++i)
      for (int j = 0; j < ns; ++j) key[q++] = nodes[i] * nn + nodes[j];
  }
  qsort(key, (size_t)q, sizeof(int64_t), cmp_i64);
  int64_t nnz = 0;
  for (int64_t a = 0; a <= nn; ++a) row_ptr[a] = 0;
  for (int64_t i = 0; i < q; ++i) {
    if (i > 0 && key[i] == key[i - 1]) continue;
    const int64_t a = key[i] / nn, b = key[i] % nn;
    if (col_idx) {
      if (nnz >= cap) {
        free(key);
        return ORC_ERR_BAD_ARG;
      }
      col_idx[nnz] = (int32_t)b;
    }
    row_ptr[a + 1] += 1;
    ++nnz;
  }
  for (int64_t a = 0; a < nn; ++a) row_ptr[a + 1] += row_ptr[a];
  free(key);
  return nnz;
}

/* ------------------------------------------------------------------------
 * Stage 1 (Eq. map-from-particles-to-nodes): lumped mass M_i = sum S m and
 * mass-weighted nodal values f_i = sum S m f / M_i.  Pinned: sum M = sum m.
 * ---------------------------------------------------------------------- */
int orc_p2g(const orc_grid *g, int64_t n, const int32_t *first, const int32_t *count,
            const double *S, const double *m, int32_t nf, const double *fld,
            double *M, double *out) {
  const int64_t nn = orc_nnodes(g);
  for (int64_t a = 0; a < nn; ++a) {
    M[a] = 0.0;
    for (int f = 0; f < nf; ++f) out[a * nf + f] = 0.0;
  }
  support *sp = (support *)malloc(sizeof(support));
  for (int64_t p = 0; p < n; ++p) {
    build_support(g, p, first, count, S, NULL, S, sp);
    for (int q = 0; q < sp->ns; ++q) {
      const int64_t a = sp->node[q];
      M[a] += sp->S[q] * m[p];
      for (int f = 0; f < nf; ++f) out[a * nf + f] += sp->S[q] * m[p] * fld[p * nf + f];
    }
  }
  for (int64_t a = 0; a < nn; ++a)
    for (int f = 0; f < nf; ++f) out[a * nf + f] = M[a] > 0.0 ? out[a * nf + f] / M[a] : 0.0;
  free(sp);
  return ORC_OK;
}

static int64_t find_block(const int64_t *row_ptr, const int32_t *col_idx, int64_t a, int64_t b);

int orc_consistent_mass(const orc_grid *g, int64_t n, const int32_t *first, const int32_t *count,
                        const double *S, const double *m, const int64_t *row_ptr, const int32_t *col_idx,
                        double *mc) {
  const int64_t nn = orc_nnodes(g);
  for (int64_t e = 0; e < row_ptr[nn]; ++e) mc[e] = 0.0;
  support *sp = (support *)malloc(sizeof(support));
  int rc = ORC_OK;
  for (int64_t p = 0; p < n && rc == ORC_OK; ++p) {
    build_support(g, p, first, count, S, NULL, S, sp);
    for (int qa = 0; qa < sp->ns; ++qa)
      for (int qb = 0; qb < sp->ns; ++qb) {
        const int64_t e = find_block(row_ptr, col_idx, sp->node[qa], sp->node[qb]);
        if (e < 0) {
          rc = ORC_ERR_BAD_ARG;
          break;
        }
        mc[e] += sp->S[qa] * sp->S[qb] * m[p];
      }
  }
  free(sp);
  return rc;
}

/* ------------------------------------------------------------------------
 * Hencky elasticity (Sec. 2.2): Psi = lambda/2 (ln J)^2 + G tr((1/2 ln b)^2),
 * so tau' = 2 b dPsi/db = lambda ln J 1 + G ln b.  With b = sum_A x_A n_A n_A
 * (x_A = squared principal stretches), eps_A = ln(x_A)/2 and the principal
 * Kirchhoff stresses tau_A = lambda sum_B eps_B + 2 G eps_A, the spatial
 * tangent of tau' (its Lie derivative, L_v tau' = c : d) is, in the principal
 * basis (m_A = n_A n_A, m_AB = n_A n_B),
 *   c = sum_AB (lambda + (2G - 2 tau_A) delta_AB) m_A (x) m_B
 *     + sum_{A != B} theta_AB (m_AB (x) m_AB + m_AB (x) m_BA),
 *   theta_AB = (tau_A x_B - tau_B x_A) / (x_A - x_B)
 *            = G log1p(r) / r - tau_B,  r = x_A / x_B - 1,
 * the second form without cancellation and with its limit G - tau_A at equal
 * stretches.  (The same formulas give the neo-Hookean tangent lambda 1 (x) 1 +
 * 2 (G - lambda ln J) I when tau_A = G (x_A - 1) + lambda ln J.)  In plane
 * strain b is the in-plane 2 x 2 block (the third stretch is 1).
 * ---------------------------------------------------------------------- */
static void jacobi_eig(int d, const double *A, double *w, double *Q) {
  double M[3][3];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      M[i][j] = A[i * d + j];
      Q[i * d + j] = i == j ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < d; ++i) {
      diag += M[i][i] * M[i][i];
      for (int j = i + 1; j < d; ++j) off += M[i][j] * M[i][j];
    }
    if (off <= 1e-36 * diag) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        if (M[p][q] == 0.0) continue;
        const double th = 0.5 * atan2(2.0 * M[p][q], M[q][q] - M[p][p]);
        const double c = cos(th), s = sin(th);
        for (int k = 0; k < d; ++k) {  /* columns p, q of M */
          const double mkp = M[k][p], mkq = M[k][q];
          M[k][p] = c * mkp - s * mkq;
          M[k][q] = s * mkp + c * mkq;
        }
        for (int k = 0; k < d; ++k) {  /* rows p, q */
          const double mpk = M[p][k], mqk = M[q][k];
          M[p][k] = c * mpk - s * mqk;
          M[q][k] = s * mpk + c * mqk;
        }
        for (int k = 0; k < d; ++k) {
          const double qkp = Q[k * d + p], qkq = Q[k * d + q];
          Q[k * d + p] = c * qkp - s * qkq;
          Q[k * d + q] = s * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < d; ++i) w[i] = M[i][i];
}

static double log1p_ratio(double r) { return fabs(r) > 1e-6 ? log1p(r) / r : 1.0 - r / 2.0 + r * r / 3.0; }

/* tau' and the tangent c (d^4, index ((i d + j) d + k) d + l) of Hencky elasticity */
static void hencky(int d, const double *bL, double lam, double G, double *tau, double *c) {
  double x[3], Q[9], eps[3], tA[3], tr = 0.0;
  jacobi_eig(d, bL, x, Q);
  for (int A = 0; A < d; ++A) {
    eps[A] = 0.5 * log(x[A]);
    tr += eps[A];
  }
  for (int A = 0; A < d; ++A) tA[A] = lam * tr + 2.0 * G * eps[A];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int A = 0; A < d; ++A) s += tA[A] * Q[i * d + A] * Q[j * d + A];
      tau[i * d + j] = s;
    }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      for (int k = 0; k < d; ++k)
        for (int l = 0; l < d; ++l) {
          double s = 0.0;
          for (int A = 0; A < d; ++A)
            for (int B = 0; B < d; ++B) {
              const double nAi = Q[i * d + A], nAj = Q[j * d + A];
              const double nBk = Q[k * d + B], nBl = Q[l * d + B];
              s += (lam + (A == B ? 2.0 * G - 2.0 * tA[A] : 0.0)) * nAi * nAj * nBk * nBl;
              if (A != B) {
                const double th = G * log1p_ratio(x[A] / x[B] - 1.0) - tA[B];
                /* m_AB (x) m_AB: n_Ai n_Bj n_Ak n_Bl;  m_AB (x) m_BA: n_Ai n_Bj n_Bk n_Al */
                s += th * (nAi * Q[j * d + B] * Q[k * d + A] * nBl + nAi * Q[j * d + B] * nBk * Q[l * d + A]);
              }
            }
          c[((i * d + j) * d + k) * d + l] = s;
        }
}

/* ------------------------------------------------------------------------
 * Small dense helpers (d x d, row-major).
 * ---------------------------------------------------------------------- */
static double det_d(int d, const double *A) {
  if (d == 2) return A[0] * A[3] - A[1] * A[2];
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static void inv_d(int d, const double *A, double *B) {
  const double det = det_d(d, A);
  if (d == 2) {
    B[0] = A[3] / det;
    B[1] = -A[1] / det;
    B[2] = -A[2] / det;
    B[3] = A[0] / det;
    return;
  }
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

static int64_t find_block(const int64_t *row_ptr, const int32_t *col_idx, int64_t a, int64_t b) {
  int64_t lo = row_ptr[a], hi = row_ptr[a + 1] - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) / 2;
    if (col_idx[mid] == b) return mid;
    if (col_idx[mid] < b) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

/* Newmark nodal kinematics (Eq. newmark, Eq. p-dot-newmark) at one node. */
static void newmark_node(const orc_step *sp, int d, const orc_nodal *nd, int64_t a,
                         const double *X, double *va, double *aa, double *pda, double *pdda) {
  const int nb = d + 1;
  const double b = sp->beta, gm = sp->gamma, dt = sp->dt;
  for (int k = 0; k < d; ++k) {
    const double dU = X[a * nb + k];
    const double vn = nd->v[a * d + k], an = nd->a[a * d + k];
    aa[k] = dU / (b * dt * dt) - vn / (b * dt) + (1.0 - 1.0 / (2.0 * b)) * an;
    va[k] = gm / (b * dt) * dU + (1.0 - gm / b) * vn + (1.0 - gm / (2.0 * b)) * dt * an;
  }
  const double dP = X[a * nb + d] - nd->P[a];
  *pda = gm / (b * dt) * dP + (1.0 - gm / b) * nd->pd[a] + (1.0 - gm / (2.0 * b)) * dt * nd->pdd[a];
  *pdda = dP / (b * dt * dt) - nd->pd[a] / (b * dt) + (1.0 - 1.0 / (2.0 * b)) * nd->pdd[a];
}

/* ------------------------------------------------------------------------
 * Residual (Eqs. residual-momentum, residual-mass, stab-term-ppp) and its
 * analytic Jacobian (Eq. jacobian-system-stabilized-ppp), integrated at the
 * material points with the pull-back of Sec. 3.3:
 *   dF = 1 + sum_b dU_b (x) Gn_b,  dJ = det dF,  F = dF Fn,  J = det F,
 *   grad S_a = Gn_a . dF^{-1},     dv = dJ dV_n.
 * Unknowns X per node: [dU (increment from t_n, grid reset), P (total)].
 * Constitutive law: compressible neo-Hookean in Kirchhoff form
 *   tau' = G (b - 1) + lambda ln J 1.
 * Quasi-static: div v = (ln J - ln J_n)/dt = ln dJ / dt (Eq. implicit-euler).
 * Dynamic: Newmark at the nodes, Kelvin viscous stress, inertia.
 * Not linearized (the paper leaves inertia/damping terms unlinearized): the
 * geometric dependence of the viscous term, the acceleration inside Darcy's
 * law; the mixture mass is frozen over the step.
 * Pinned: central finite differences (quasi-static; dynamic with
 * alpha_vis = 0 and rho_f = 0; dynamic with both, of the residual whose
 * unlinearized terms are frozen, orc_eval_frozen), C_stab symmetric PSD,
 * Terzaghi series.
 *
 * Xf (NULL for the residual itself): the frozen variant.  The terms left
 * unlinearized take their geometry from the iterate Xf instead of X: the
 * Kelvin stress its spatial gradients (in D = grad^s v and in the contraction
 * with grad S_a), its mu' (or the Hencky tangent), and Darcy's law its
 * acceleration; the nodal velocities stay those of X.  The derivative of that
 * residual at X = Xf is what the analytic Jacobian holds.
 * ---------------------------------------------------------------------- */
static int eval_impl(const orc_grid *g, const orc_step *sp, const orc_particles *pp,
                     const int32_t *first, const int32_t *count, const double *S, const double *dS,
                     const double *S0, const uint8_t *active, const orc_nodal *nd, const double *trac,
                     const double *flux, const double *X, const double *Xf, const int64_t *row_ptr,
                     const int32_t *col_idx, double *R, double *Jv) {
  const int d = g->dim, nb = d + 1, nb2 = nb * nb;
  const int64_t nn = orc_nnodes(g);
  const double dt = sp->dt, beta = sp->beta, gam = sp->gamma;
  for (int64_t i = 0; i < nn * nb; ++i) R[i] = 0.0;
  if (Jv) {
    const int64_t nnzb = row_ptr[nn];
    for (int64_t i = 0; i < nnzb * nb2; ++i) Jv[i] = 0.0;
  }
  support *su = (support *)malloc(sizeof(support));
  int rc = ORC_OK;
  for (int64_t p = 0; p < pp->n; ++p) {
    build_support_active(g, p, first, count, S, dS, S0, active, su);
    const int ns = su->ns;
    /* relative deformation gradient dF = 1 + sum dU_b (x) Gn_b */
    double dF[9] = {0}, f[9], Fn[9], F[9] = {0}, bL[9] = {0};
    for (int i = 0; i < d; ++i) dF[i * d + i] = 1.0;
    for (int q = 0; q < ns; ++q)
      for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) dF[i * d + k] += X[su->node[q] * nb + i] * su->Gn[q][k];
    const double dJ = det_d(d, dF);
    if (!(dJ > 0.0)) {
      rc = ORC_ERR_NEGATIVE_J;
      break;
    }
    inv_d(d, dF, f);
    for (int i = 0; i < d * d; ++i) Fn[i] = pp->F[p * d * d + i];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) F[i * d + j] += dF[i * d + k] * Fn[k * d + j];
    const double Jn = det_d(d, Fn);
    const double J = det_d(d, F);
    if (!(J > 0.0)) {
      rc = ORC_ERR_NEGATIVE_J;
      break;
    }
    const double lnJ = log(J);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) bL[i * d + j] += F[i * d + k] * F[j * d + k];
    const double lam = pp->lam[p], Gs = pp->G[p];
    double tau[9], ct[81];
    if (sp->hencky) {
      hencky(d, bL, lam, Gs, tau, ct);
    } else {
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
          tau[i * d + j] = Gs * (bL[i * d + j] - (i == j ? 1.0 : 0.0)) + (i == j ? lam * lnJ : 0.0);
    }
    const double mu_p = Gs - lam * lnJ; /* shear coefficient of the neo-Hookean spatial tangent */
    const double Vn = pp->V[p];
    const double vol = dJ * Vn;         /* current volume */
    const double cs = Vn / Jn;          /* v sigma = (V_n / J_n) tau */
    /* spatial gradients g_a = Gn_a . dF^{-1} */
    double gr[MAXS * MAXS * MAXS][MAXD];
    for (int q = 0; q < ns; ++q)
      for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += su->Gn[q][k] * f[k * d + j];
        gr[q][j] = s;
      }
    /* interpolated pressure and its spatial gradient */
    double ph = 0.0, gp[3] = {0, 0, 0};
    for (int q = 0; q < ns; ++q) {
      const double P = X[su->node[q] * nb + d];
      ph += su->S[q] * P;
      for (int j = 0; j < d; ++j) gp[j] += P * gr[q][j];
    }
    /* time discretization of div v, acceleration, velocity gradient, dp/dt */
    double divv, ah[3] = {0, 0, 0}, gv[9] = {0};
    double pdev = 0.0; /* (pdot^h - Pi pdot^h) at the point, via S - S0 */
    double nva[MAXS * MAXS * MAXS][MAXD], naa[MAXS * MAXS * MAXS][MAXD];
    if (sp->dynamic) {
      for (int q = 0; q < ns; ++q) {
        double pda, pdda;
        newmark_node(sp, d, nd, su->node[q], X, nva[q], naa[q], &pda, &pdda);
        for (int i = 0; i < d; ++i) {
          ah[i] += su->S[q] * naa[q][i];
          for (int j = 0; j < d; ++j) gv[i * d + j] += nva[q][i] * gr[q][j];
        }
        pdev += (su->S[q] - su->S0[q]) * pda;
      }
      divv = 0.0;
      for (int i = 0; i < d; ++i) divv += gv[i * d + i];
    } else {
      for (int q = 0; q < ns; ++q) {
        const int64_t a = su->node[q];
        pdev += (su->S[q] - su->S0[q]) * (X[a * nb + d] - nd->P[a]) / dt;
      }
      divv = log(dJ) / dt;
    }
    /* Darcy: q = -kappa [grad p - rho_f (g - a)]; with Eq. kozeny-carman the
     * mobility follows the porosity phi = 1 - (1 - phi0) / J of the iterate:
     * kappa = kappa_0 (1 - phi0)^2 / phi0^3 * phi^3 / (1 - phi)^2, and
     * dkappa/dJ by the chain rule (dphi/dJ = (1 - phi0) / J^2); closed pores
     * (phi <= 0) conduct nothing */
    double kap = pp->kappa[p], dkap_dJ = 0.0;
    if (sp->kozeny) {
      const double phi0 = sp->phi0, phi = 1.0 - (1.0 - phi0) / J;
      if (phi > 0.0) {
        const double c0 = (1.0 - phi0) * (1.0 - phi0) / (phi0 * phi0 * phi0);
        const double k = kap * c0 * phi * phi * phi / ((1.0 - phi) * (1.0 - phi));
        const double dk_dphi = kap * c0 * (3.0 * phi * phi / ((1.0 - phi) * (1.0 - phi)) +
                                          2.0 * phi * phi * phi / ((1.0 - phi) * (1.0 - phi) * (1.0 - phi)));
        dkap_dJ = dk_dphi * (1.0 - phi0) / (J * J);
        kap = k;
      } else {
        kap = 0.0;
      }
    }
    /* the frozen variant's geometry of the unlinearized terms (see above):
     * gradients grk, mu' muk, Hencky tangent ctk and acceleration ahk at Xf */
    double grf[MAXS * MAXS * MAXS][MAXD], ctf[81], ahf[3] = {0, 0, 0}, muf = 0.0;
    const double(*grk)[MAXD] = gr;
    const double *ctk = ct, *ahk = ah;
    double muk = mu_p;
    if (Xf && sp->dynamic) {
      double dFf[9] = {0}, ff[9], Ff[9] = {0}, bf[9] = {0}, tauf[9];
      for (int i = 0; i < d; ++i) dFf[i * d + i] = 1.0;
      for (int q = 0; q < ns; ++q)
        for (int i = 0; i < d; ++i)
          for (int k = 0; k < d; ++k) dFf[i * d + k] += Xf[su->node[q] * nb + i] * su->Gn[q][k];
      if (!(det_d(d, dFf) > 0.0)) {
        rc = ORC_ERR_NEGATIVE_J;
        break;
      }
      inv_d(d, dFf, ff);
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
          for (int k = 0; k < d; ++k) Ff[i * d + j] += dFf[i * d + k] * Fn[k * d + j];
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
          for (int k = 0; k < d; ++k) bf[i * d + j] += Ff[i * d + k] * Ff[j * d + k];
      if (sp->hencky) hencky(d, bf, lam, Gs, tauf, ctf);
      muf = Gs - lam * log(det_d(d, Ff));
      for (int q = 0; q < ns; ++q) {
        for (int j = 0; j < d; ++j) {
          double s = 0.0;
          for (int k = 0; k < d; ++k) s += su->Gn[q][k] * ff[k * d + j];
          grf[q][j] = s;
        }
        double vf[3], af[3], pdf, pddf;
        newmark_node(sp, d, nd, su->node[q], Xf, vf, af, &pdf, &pddf);
        for (int i = 0; i < d; ++i) ahf[i] += su->S[q] * af[i];
      }
      grk = (const double(*)[MAXD])grf;
      ctk = ctf;
      ahk = ahf;
      muk = muf;
    }
    double w[3];
    for (int j = 0; j < d; ++j) w[j] = gp[j] - sp->rho_f * (sp->g[j] - ahk[j]);
    /* Kelvin viscous stress (v sigma_vis) = (V_n/J_n) alpha (lambda tr D 1 + 2 mu' D) */
    double svis[9] = {0};
    if (sp->dynamic && sp->alpha_vis != 0.0) {
      double gvk[9] = {0}; /* grad v: the velocities of X at the gradients grk */
      if (grk == (const double(*)[MAXD])gr) {
        for (int i = 0; i < d * d; ++i) gvk[i] = gv[i];
      } else {
        for (int q = 0; q < ns; ++q)
          for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) gvk[i * d + j] += nva[q][i] * grk[q][j];
      }
      double trD = 0.0;
      for (int i = 0; i < d; ++i) trD += gvk[i * d + i];
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          const double D = 0.5 * (gvk[i * d + j] + gvk[j * d + i]);
          svis[i * d + j] = sp->alpha_vis * ((i == j ? lam * trD : 0.0) + 2.0 * muk * D);
        }
      if (sp->hencky) /* sigma_vis = alpha c : grad^s v with the Hencky tangent */
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k)
              for (int l = 0; l < d; ++l) s += ctk[((i * d + j) * d + k) * d + l] * 0.5 * (gvk[k * d + l] + gvk[l * d + k]);
            svis[i * d + j] = sp->alpha_vis * s;
          }
    }
    const double mp = pp->m[p];
    const double taus = pp->tau[p];
    const double cstab = sp->dynamic ? taus * gam / (beta * dt) : taus / dt;

    /* ---- residual ---- */
    for (int q = 0; q < ns; ++q) {
      const int64_t a = su->node[q];
      for (int i = 0; i < d; ++i) {
        double r = 0.0;
        for (int j = 0; j < d; ++j) r -= cs * gr[q][j] * tau[i * d + j];   /* -grad^s S : sigma' dv */
        r += vol * gr[q][i] * ph;                                          /* +div S p dv          */
        for (int j = 0; j < d; ++j) r -= cs * grk[q][j] * svis[i * d + j]; /* -grad^s S : sigma_vis */
        r -= su->S[q] * mp * ah[i];                                        /* -S rho a dv          */
        r += su->S[q] * mp * sp->g[i];                                     /* +S rho g dv          */
        R[a * nb + i] += r;
      }
      double rm = vol * su->S[q] * divv;                                  /* S div v dv           */
      double gw = 0.0;
      for (int j = 0; j < d; ++j) gw += gr[q][j] * w[j];
      rm += vol * kap * gw;                                                /* -grad S . q dv       */
      rm += Vn * taus * (su->S[q] - su->S0[q]) * pdev;                    /* R_stab               */
      R[a * nb + d] += rm;
    }
    /* Neumann data carried by surface material points, hat basis at x + lp.n */
    if (pp->surf && pp->surf[p] >= 0) {
      const int32_t e = pp->surf[p];
      double y[3];
      for (int k = 0; k < d; ++k) y[k] = pp->x[p * d + k] + pp->lp[p * d + k] * pp->surf_n[p * d + k];
      for (int q = 0; q < ns; ++q) {
        double Ny = 1.0;
        for (int k = 0; k < d; ++k) {
          const double xi = (y[k] - g->origin[k]) / g->h;
          const double t = 1.0 - fabs(xi - (double)su->ax[q][k]);
          Ny *= t > 0.0 ? t : 0.0;
        }
        const int64_t a = su->node[q];
        for (int i = 0; i < d; ++i) R[a * nb + i] += Ny * trac[(int64_t)e * d + i] * pp->surf_A[p];
        if (flux) R[a * nb + d] -= Ny * flux[e] * pp->surf_A[p];
      }
    }
    if (!Jv) continue;

    /* ---- Jacobian blocks ---- */
    const double kv = vol * kap;
    const double dkv = vol * J * dkap_dJ; /* delta kappa = kappa'(J) J div(delta u) */
    for (int qa = 0; qa < ns; ++qa) {
      const double *ga = gr[qa];
      const double Sa = su->S[qa], Sda = su->S[qa] - su->S0[qa];
      double gaw = 0.0;
      for (int j = 0; j < d; ++j) gaw += ga[j] * w[j];
      for (int qb = 0; qb < ns; ++qb) {
        const double *gb = gr[qb];
        const double Sb = su->S[qb], Sdb = su->S[qb] - su->S0[qb];
        const int64_t e = find_block(row_ptr, col_idx, su->node[qa], su->node[qb]);
        if (e < 0) {
          rc = ORC_ERR_BAD_ARG;
          goto done;
        }
        double *B = &Jv[e * nb2];
        double gab = 0.0, gtg = 0.0, gbw = 0.0;
        for (int j = 0; j < d; ++j) {
          gab += ga[j] * gb[j];
          gbw += gb[j] * w[j];
          for (int l = 0; l < d; ++l) gtg += ga[j] * tau[j * d + l] * gb[l];
        }
        for (int i = 0; i < d; ++i)
          for (int k = 0; k < d; ++k) {
            const double dik = i == k ? 1.0 : 0.0;
            /* material part g_a . c . g_b of the tangent */
            double mat;
            if (sp->hencky) {
              mat = 0.0;
              for (int j = 0; j < d; ++j)
                for (int l = 0; l < d; ++l) mat += ga[j] * ct[((i * d + j) * d + k) * d + l] * gb[l];
            } else {
              mat = mu_p * (dik * gab + ga[k] * gb[i]) + lam * ga[i] * gb[k];
            }
            double A = -cs * (dik * gtg + mat);
            A += vol * ph * (ga[i] * gb[k] - ga[k] * gb[i]);
            if (sp->dynamic) {
              const double cv = sp->alpha_vis * gam / (beta * dt);
              A -= cs * cv * mat;
              A -= dik * mp * Sa * Sb / (beta * dt * dt);
            }
            B[i * nb + k] += A;
          }
        for (int i = 0; i < d; ++i) B[i * nb + d] += vol * ga[i] * Sb; /* B1 */
        for (int k = 0; k < d; ++k) {                                 /* B2 */
          double b2;
          if (sp->dynamic) {
            double gbgv = 0.0;
            for (int j = 0; j < d; ++j) gbgv += gb[j] * gv[j * d + k];
            b2 = vol * Sa * (gam / (beta * dt) * gb[k] + divv * gb[k] - gbgv);
          } else {
            b2 = vol * Sa * (1.0 + log(dJ)) * gb[k] / dt;
          }
          b2 += kv * (gb[k] * gaw - ga[k] * gbw - gp[k] * gab);
          b2 += dkv * gaw * gb[k];
          B[d * nb + k] += b2;
        }
        B[d * nb + d] += kv * gab + cstab * Vn * Sda * Sdb; /* C + C_stab */
      }
    }
  }
done:
  free(su);
  return rc;
}

int orc_eval(const orc_grid *g, const orc_step *sp, const orc_particles *pp,
             const int32_t *first, const int32_t *count, const double *S, const double *dS,
             const double *S0, const uint8_t *active, const orc_nodal *nd, const double *trac,
             const double *flux, const double *X, const int64_t *row_ptr, const int32_t *col_idx,
             double *R, double *Jv) {
  return eval_impl(g, sp, pp, first, count, S, dS, S0, active, nd, trac, flux, X, NULL, row_ptr, col_idx,
                   R, Jv);
}

int orc_eval_frozen(const orc_grid *g, const orc_step *sp, const orc_particles *pp,
                    const int32_t *first, const int32_t *count, const double *S, const double *dS,
                    const double *S0, const uint8_t *active, const orc_nodal *nd, const double *trac,
                    const double *flux, const double *X, const double *Xf, double *R) {
  if (!Xf) return ORC_ERR_BAD_ARG;
  return eval_impl(g, sp, pp, first, count, S, dS, S0, active, nd, trac, flux, X, Xf, NULL, NULL, R, NULL);
}

/* ------------------------------------------------------------------------
 * Right stretch diagonal U_kk of U = (F^T F)^{1/2} by cyclic Jacobi rotations.
 * Used for the GIMP domain update (Charlton et al.), Sec. 3.5.
 * ---------------------------------------------------------------------- */
void orc_stretch_diag(int32_t d, const double *F, double *Udiag) {
  double C[3][3] = {{0}}, Q[3][3] = {{0}};
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += F[k * d + i] * F[k * d + j];
      C[i][j] = s;
    }
  for (int i = 0; i < d; ++i) Q[i][i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < d; ++i)
      for (int j = i + 1; j < d; ++j) off += C[i][j] * C[i][j];
    if (off < 1e-300) break;
    for (int pq = 0; pq < d; ++pq)
      for (int qq = pq + 1; qq < d; ++qq) {
        if (C[pq][qq] == 0.0) continue;
        const double th = 0.5 * atan2(2.0 * C[pq][qq], C[qq][qq] - C[pq][pq]);
        const double c = cos(th), s = sin(th);
        for (int k = 0; k < d; ++k) { /* C <- C R */
          const double ckp = C[k][pq], ckq = C[k][qq];
          C[k][pq] = c * ckp - s * ckq;
          C[k][qq] = s * ckp + c * ckq;
        }
        for (int k = 0; k < d; ++k) { /* C <- R^T C */
          const double cpk = C[pq][k], cqk = C[qq][k];
          C[pq][k] = c * cpk - s * cqk;
          C[qq][k] = s * cpk + c * cqk;
        }
        for (int k = 0; k < d; ++k) { /* Q <- Q R */
          const double qkp = Q[k][pq], qkq = Q[k][qq];
          Q[k][pq] = c * qkp - s * qkq;
          Q[k][qq] = s * qkp + c * qkq;
        }
      }
  }
  for (int k = 0; k < d; ++k) {
    double u = 0.0;
    for (int m = 0; m < d; ++m) u += Q[k][m] * Q[k][m] * sqrt(C[m][m]);
    Udiag[k] = u;
  }
}

/* ------------------------------------------------------------------------
 * Stages 3-4 (Sec. 3.5): PIC for u, p, a, dp/dt, d2p/dt2 (Eq.
 * map-from-nodes-to-particles), FLIP for v, position convection, F = dF Fn,
 * V = dJ Vn, GIMP half lengths from the right stretch.
 * ---------------------------------------------------------------------- */
int orc_g2p(const orc_grid *g, const orc_step *sp, int64_t n, const int32_t *first,
            const int32_t *count, const double *S, const double *dS, const double *S0,
            const uint8_t *active, const orc_nodal *nd, const double *X, double *x, double *u,
            double *F, double *V, double *lp, const double *lp0, double *p, double *v, double *a,
            double *pd, double *pdd) {
  const int d = g->dim, nb = d + 1;
  support *su = (support *)malloc(sizeof(support));
  int rc = ORC_OK;
  for (int64_t q0 = 0; q0 < n; ++q0) {
    build_support_active(g, q0, first, count, S, dS, S0, active, su);
    double dF[9] = {0}, du[3] = {0, 0, 0}, ph = 0.0;
    for (int i = 0; i < d; ++i) dF[i * d + i] = 1.0;
    for (int q = 0; q < su->ns; ++q) {
      const int64_t nd_ = su->node[q];
      for (int i = 0; i < d; ++i) {
        du[i] += su->S[q] * X[nd_ * nb + i];
        for (int k = 0; k < d; ++k) dF[i * d + k] += X[nd_ * nb + i] * su->Gn[q][k];
      }
      ph += su->S[q] * X[nd_ * nb + d];
    }
    const double dJ = det_d(d, dF);
    if (!(dJ > 0.0)) {
      rc = ORC_ERR_NEGATIVE_J;
      break;
    }
    if (sp->dynamic) {
      double anew[3] = {0, 0, 0}, vinc[3] = {0, 0, 0}, pdh = 0.0, pddh = 0.0;
      for (int q = 0; q < su->ns; ++q) {
        double va[3], aa[3], pda, pdda;
        const int64_t nd_ = su->node[q];
        newmark_node(sp, d, nd, nd_, X, va, aa, &pda, &pdda);
        for (int i = 0; i < d; ++i) {
          anew[i] += su->S[q] * aa[i];
          vinc[i] += su->S[q] * ((1.0 - sp->gamma) * nd->a[nd_ * d + i] + sp->gamma * aa[i]);
        }
        pdh += su->S[q] * pda;
        pddh += su->S[q] * pdda;
      }
      for (int i = 0; i < d; ++i) {
        a[q0 * d + i] = anew[i];
        v[q0 * d + i] += sp->dt * vinc[i];
      }
      pd[q0] = pdh;
      pdd[q0] = pddh;
    }
    double Fn[9], Fnew[9] = {0};
    for (int i = 0; i < d * d; ++i) Fn[i] = F[q0 * d * d + i];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) Fnew[i * d + j] += dF[i * d + k] * Fn[k * d + j];
    for (int i = 0; i < d * d; ++i) F[q0 * d * d + i] = Fnew[i];
    for (int i = 0; i < d; ++i) {
      x[q0 * d + i] += du[i];
      u[q0 * d + i] += du[i];
    }
    V[q0] = dJ * V[q0];
    p[q0] = ph;
    double Ud[3];
    orc_stretch_diag(d, Fnew, Ud);
    for (int k = 0; k < d; ++k) lp[q0 * d + k] = lp0[q0 * d + k] * Ud[k];
  }
  free(su);
  return rc;
}
