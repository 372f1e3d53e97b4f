// mpm_solver.cu -- linear algebra of the Newton step (Eq. jacobian-system-
// stabilized-ppp):  J dX = -R  on the block-CSR Jacobian.
//
// The system is first scaled symmetrically, D J D y = -D R with
// D_ii = |J_ii|^{-1/2}, which brings the momentum rows (stiffness ~ 1e7) and
// the mass rows (~ 1e-7) to unit diagonal, so that the Krylov residual norm
// weighs both balance laws; then right-preconditioned restarted FGMRES with
// classical Gram-Schmidt applied twice (CGS2) and node-block Jacobi
// preconditioning solves it.  The Givens rotations and the Hessenberg system
// live in device memory; the host reads one scalar per iteration.
// All reductions use a fixed grid and a fixed tree, so results are
// deterministic.  Plain FP64 HBM-bound kernels, no tensor cores (sparse work).
#include <math.h>

#include "mpm_internal.cuh"

namespace upmpm {

namespace {

constexpr int TPB = 256;
constexpr int NPART = 304;  // partial sums per reduction (2 x 152 SMs)
constexpr int PSTR = 129;   // stride of the per-block partial sums (restart <= 128)
inline int nblk(int64_t n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

__device__ inline double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;  // valid in thread 0
}

// ---------------------------------------------------------------- scan
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_CHUNK = SCAN_T * SCAN_I;

__device__ inline int block_excl_scan(int v, int *total) {
  __shared__ int sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = sh[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const int before = wid > 0 ? sh[wid - 1] : 0;
  *total = sh[31];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_blocks(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                              int32_t *__restrict__ blk) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_I;
  int v[SCAN_I], s = 0;
  for (int i = 0; i < SCAN_I; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int total;
  int run = block_excl_scan(s, &total);
  for (int i = 0; i < SCAN_I; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) blk[blockIdx.x] = total;
}

__global__ void k_scan_top(int32_t *__restrict__ blk, int nb) {
  // one block; nb <= SCAN_CHUNK
  const int base = threadIdx.x * SCAN_I;
  int v[SCAN_I], s = 0;
  for (int i = 0; i < SCAN_I; ++i) {
    v[i] = (base + i < nb) ? blk[base + i] : 0;
    s += v[i];
  }
  int total;
  int run = block_excl_scan(s, &total);
  for (int i = 0; i < SCAN_I; ++i) {
    if (base + i < nb) blk[base + i] = run;
    run += v[i];
  }
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ blk,
                           const int32_t *__restrict__ in, double *__restrict__ total_out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_I;
  const int32_t add = blk[blockIdx.x];
  for (int i = 0; i < SCAN_I; ++i)
    if (base + i < n) {
      out[base + i] += add;
      if (base + i == n - 1) total_out[0] = (double)out[base + i] + (double)in[base + i];
    }
}

// ---------------------------------------------------------------- vectors
__global__ void k_dot_partial(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                              double *__restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_reduce(const double *__restrict__ part, int np, double *__restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[0] = acc;
}

__global__ void k_axpy(double *__restrict__ y, double a, const double *__restrict__ x, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void k_scale_copy(double *__restrict__ y, const double *__restrict__ x, const double *s,
                             int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] * s[0];
}

// y = b - y
__global__ void k_residual_vec(double *__restrict__ y, const double *__restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = b[i] - y[i];
}

// ---------------------------------------------------------------- scaling
template <int NB>
__global__ void k_diag_scale(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const double *__restrict__ val,
                             double *__restrict__ dsc) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  int lo = row_ptr[a], hi = row_ptr[a + 1] - 1, e = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int cm = col[mid];
    if (cm == a) { e = mid; break; }
    if (cm < a) lo = mid + 1; else hi = mid - 1;
  }
  for (int r = 0; r < NB; ++r) {
    const double d = e >= 0 ? fabs(val[(int64_t)e * NB * NB + r * NB + r]) : 0.0;
    dsc[a * NB + r] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
  }
}

template <int NB>
__global__ void k_scale_matrix(int64_t nnzb, const int32_t *__restrict__ row_of,
                               const int32_t *__restrict__ col, double *__restrict__ val,
                               const double *__restrict__ dsc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * NB * NB) return;
  const int64_t e = t / (NB * NB);
  const int rc = (int)(t % (NB * NB));
  const int r = rc / NB, cc = rc % NB;
  val[t] *= dsc[(int64_t)row_of[e] * NB + r] * dsc[(int64_t)col[e] * NB + cc];
}

__global__ void k_scale_rhs(int64_t n, const double *__restrict__ R, const double *__restrict__ dsc,
                            double *__restrict__ rhs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = -dsc[i] * R[i];
}

__global__ void k_unscale_add(int64_t n, double *__restrict__ X, const double *__restrict__ dsc,
                              const double *__restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) X[i] += dsc[i] * y[i];
}

// ---------------------------------------------------------------- block Jacobi
template <int NB>
__global__ void k_block_jacobi(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, const double *__restrict__ val,
                               double *__restrict__ dinv, int *err) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  int lo = row_ptr[a], hi = row_ptr[a + 1] - 1, e = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int cm = col[mid];
    if (cm == a) { e = mid; break; }
    if (cm < a) lo = mid + 1; else hi = mid - 1;
  }
  double A[NB][NB], B[NB][NB];
  for (int i = 0; i < NB; ++i)
    for (int j = 0; j < NB; ++j) {
      A[i][j] = e >= 0 ? val[(int64_t)e * NB * NB + i * NB + j] : (i == j ? 1.0 : 0.0);
      B[i][j] = i == j ? 1.0 : 0.0;
    }
  // Gauss-Jordan with partial pivoting
  bool ok = true;
  for (int k = 0; k < NB; ++k) {
    int piv = k;
    double best = fabs(A[k][k]);
    for (int i = k + 1; i < NB; ++i)
      if (fabs(A[i][k]) > best) { best = fabs(A[i][k]); piv = i; }
    if (!(best > 1e-300)) { ok = false; break; }
    if (piv != k)
      for (int j = 0; j < NB; ++j) {
        double t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t;
        t = B[k][j]; B[k][j] = B[piv][j]; B[piv][j] = t;
      }
    const double inv = 1.0 / A[k][k];
    for (int j = 0; j < NB; ++j) { A[k][j] *= inv; B[k][j] *= inv; }
    for (int i = 0; i < NB; ++i) {
      if (i == k) continue;
      const double f = A[i][k];
      if (f == 0.0) continue;
      for (int j = 0; j < NB; ++j) { A[i][j] -= f * A[k][j]; B[i][j] -= f * B[k][j]; }
    }
  }
  if (!ok) {
    atomicOr(err, DE_SINGULAR);
    for (int i = 0; i < NB; ++i)
      for (int j = 0; j < NB; ++j) B[i][j] = i == j ? 1.0 : 0.0;
  }
  for (int i = 0; i < NB; ++i)
    for (int j = 0; j < NB; ++j) dinv[a * NB * NB + i * NB + j] = B[i][j];
}

template <int NB>
__global__ void k_bj_apply(int64_t nnodes, const double *__restrict__ dinv, const double *__restrict__ x,
                           double *__restrict__ y) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  double xv[NB];
  for (int j = 0; j < NB; ++j) xv[j] = x[a * NB + j];
  for (int i = 0; i < NB; ++i) {
    double s = 0.0;
    for (int j = 0; j < NB; ++j) s += dinv[a * NB * NB + i * NB + j] * xv[j];
    y[a * NB + i] = s;
  }
}

// ---------------------------------------------------------------- SpMV
// LN lanes per block row; each lane takes whole NB x NB blocks (72 / 128
// contiguous bytes, so the lanes of a row read one contiguous span), does one
// FMA per matrix value, and the row's NB sums are reduced across the lanes.
// (The FP64 pipe of GB300 is narrow, so the kernel spends exactly one FP64
// instruction per stored value.)
template <int NB, int LN>
__global__ void k_bsr_spmv(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, const double *__restrict__ val,
                           const double *__restrict__ x, double *__restrict__ y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = t / LN;
  const int lane = (int)(t % LN);
  const bool valid = row < nnodes;
  double acc[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) acc[r] = 0.0;
  if (valid) {
    const int e1 = row_ptr[row + 1];
    for (int e = row_ptr[row] + lane; e < e1; e += LN) {
      const double *blk = val + (int64_t)e * NB * NB;
      const double *xb = x + (int64_t)__ldg(&col[e]) * NB;
      double xv[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) xv[c] = __ldg(&xb[c]);
#pragma unroll
      for (int r = 0; r < NB; ++r)
#pragma unroll
        for (int c = 0; c < NB; ++c) acc[r] = fma(__ldg(&blk[r * NB + c]), xv[c], acc[r]);
    }
  }
#pragma unroll
  for (int o = LN / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < NB; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  if (valid && lane == 0)
#pragma unroll
    for (int r = 0; r < NB; ++r) y[row * NB + r] = acc[r];
}

// ---------------------------------------------------------------- FGMRES
// partial dots of w against V_0..V_{cnt-1}
__global__ void k_multidot_partial(const double *__restrict__ V, int cnt, const double *__restrict__ w,
                                   int64_t n, double *__restrict__ part) {
  for (int i = 0; i < cnt; ++i) {
    const double *vi = V + (int64_t)i * n;
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
      acc += vi[k] * w[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR + i] = acc;
  }
}

__global__ void k_multidot_reduce(const double *__restrict__ part, int np, int cnt,
                                  double *__restrict__ h) {
  // one block per coefficient
  const int i = blockIdx.x;
  if (i >= cnt) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) acc += part[(int64_t)b * PSTR + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) h[i] = acc;
}

// w -= sum_i h_i V_i over the thread's elements, then partial dots of the
// updated w against V_i (second Gram-Schmidt pass) or with itself (norm).
__global__ void k_orth_update(double *__restrict__ w, const double *__restrict__ V, const double *h,
                              int cnt, int64_t n, double *__restrict__ part, int want_norm) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double s = w[k];
    for (int i = 0; i < cnt; ++i) s -= h[i] * V[(int64_t)i * n + k];
    w[k] = s;
  }
  if (want_norm) {
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
      acc += w[k] * w[k];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR] = acc;
  } else {
    for (int i = 0; i < cnt; ++i) {
      double acc = 0.0;
      for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
           k += (int64_t)gridDim.x * blockDim.x)
        acc += V[(int64_t)i * n + k] * w[k];
      acc = block_sum(acc);
      if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR + i] = acc;
    }
  }
}

// Finish Arnoldi column j: ||w|| from the partials, H(:,j) = h1 + h2, apply
// the previous Givens rotations, form the new one, update g.
// scal[0] = |g_{j+1}| (residual estimate), scal[1] = 1 / ||w||.
__global__ void k_arnoldi_finish(const double *__restrict__ part, int np, int j, int m,
                                 const double *__restrict__ h1, const double *__restrict__ h2,
                                 double *__restrict__ H, double *__restrict__ g, double *__restrict__ cs,
                                 double *__restrict__ sn, double *__restrict__ scal) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) acc += part[(int64_t)b * PSTR];
  acc = block_sum(acc);
  if (threadIdx.x != 0) return;
  const double hn = sqrt(acc);
  double col[PSTR];
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double r = hypot(col[j], hn);
  double c = 1.0, s = 0.0;
  if (r > 0.0) {
    c = col[j] / r;
    s = hn / r;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = r;
  for (int i = 0; i <= j; ++i) H[i * m + j] = col[i];
  const double gj = g[j];
  g[j + 1] = -s * gj;
  g[j] = c * gj;
  scal[0] = fabs(g[j + 1]);
  scal[1] = hn > 0.0 ? 1.0 / hn : 0.0;
}

__global__ void k_gmres_init(double *__restrict__ g, int m, const double *beta_sq, double *scal) {
  if (threadIdx.x != 0) return;
  const double beta = sqrt(beta_sq[0]);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  scal[0] = beta;
  scal[1] = beta > 0.0 ? 1.0 / beta : 0.0;
}

__global__ void k_backsolve(const double *__restrict__ H, const double *__restrict__ g, int jc, int m,
                            double *__restrict__ y) {
  if (threadIdx.x != 0) return;
  for (int i = jc - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < jc; ++l) s -= H[i * m + l] * y[l];
    y[i] = s / H[i * m + i];
  }
}

__global__ void k_update_x(double *__restrict__ x, const double *__restrict__ Z, const double *y, int jc,
                           int64_t n) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = x[k];
  for (int i = 0; i < jc; ++i) s += y[i] * Z[(int64_t)i * n + k];
  x[k] = s;
}

template <int NB>
void spmv(Ctx &c, const double *x, double *y) {
  constexpr int LN = NB == 3 ? 8 : 16;
  const int64_t threads = c.g.nnodes * LN;
  prof_begin(c, MPM_PROF_SPMV);
  k_bsr_spmv<NB, LN><<<nblk(threads), TPB, 0, c.st>>>(c.g.nnodes, c.row_ptr, c.col, c.val, x, y);
  prof_end(c, MPM_PROF_SPMV);
  UPMPM_LAUNCH(c);
}

template <int NB>
void precond(Ctx &c, const double *x, double *y) {
  prof_begin(c, MPM_PROF_PRECOND);
  if (c.opt.precond == MPM_PRECOND_SCHUR_MG) {
    schur_apply(c, x, y);
  } else {
    k_bj_apply<NB><<<nblk(c.g.nnodes), TPB, 0, c.st>>>(c.g.nnodes, c.dinv, x, y);
    UPMPM_LAUNCH(c);
  }
  prof_end(c, MPM_PROF_PRECOND);
}

double read_scalar(Ctx &c, const double *dptr) {
  cudaMemcpyAsync(c.h_scalar, dptr, sizeof(double), cudaMemcpyDeviceToHost, c.st);
  cudaStreamSynchronize(c.st);
  return c.h_scalar[0];
}

template <int NB>
int fgmres_impl(Ctx &c, const double *b, double *x, double rtol, int maxit, int *iters) {
  const int64_t N = c.N();
  const int m = c.m_restart;
  const int gN = nblk(N);
  double *w = c.w;
  double *h1 = c.hcol, *h2 = c.hcol + PSTR;
  cudaMemsetAsync(x, 0, sizeof(double) * N, c.st);
  // beta = ||b||, V_0 = b / beta
  k_dot_partial<<<NPART, TPB, 0, c.st>>>(b, b, N, c.part);
  k_reduce<<<1, TPB, 0, c.st>>>(c.part, NPART, c.scal + 2);
  k_gmres_init<<<1, 32, 0, c.st>>>(c.gvec, m, c.scal + 2, c.scal);
  k_scale_copy<<<gN, TPB, 0, c.st>>>(c.V, b, c.scal + 1, N);
  c.launches += 4;
  const double beta0 = read_scalar(c, c.scal);
  *iters = 0;
  if (!(beta0 > 0.0)) return MPM_OK;
  if (!isfinite(beta0)) return MPM_ERR_NONFINITE;
  const double target = rtol * beta0;
  int total = 0;
  bool converged = false;
  while (true) {
    int jc = 0;
    for (int j = 0; j < m; ++j) {
      double *Vj = c.V + (int64_t)j * N, *Zj = c.Z + (int64_t)j * N, *Vn = c.V + (int64_t)(j + 1) * N;
      precond<NB>(c, Vj, Zj);
      spmv<NB>(c, Zj, w);
      prof_begin(c, MPM_PROF_ORTH);
      k_multidot_partial<<<NPART, TPB, 0, c.st>>>(c.V, j + 1, w, N, c.part);
      k_multidot_reduce<<<j + 1, TPB, 0, c.st>>>(c.part, NPART, j + 1, h1);
      k_orth_update<<<NPART, TPB, 0, c.st>>>(w, c.V, h1, j + 1, N, c.part, 0);
      k_multidot_reduce<<<j + 1, TPB, 0, c.st>>>(c.part, NPART, j + 1, h2);
      k_orth_update<<<NPART, TPB, 0, c.st>>>(w, c.V, h2, j + 1, N, c.part, 1);
      prof_end(c, MPM_PROF_ORTH);
      k_arnoldi_finish<<<1, TPB, 0, c.st>>>(c.part, NPART, j, m, h1, h2, c.H, c.gvec, c.cs, c.sn, c.scal);
      k_scale_copy<<<gN, TPB, 0, c.st>>>(Vn, w, c.scal + 1, N);
      c.launches += 7;
      ++total;
      jc = j + 1;
      const double res = read_scalar(c, c.scal);
      if (!isfinite(res)) return MPM_ERR_NONFINITE;
      if (res <= target) {
        converged = true;
        break;
      }
      if (total >= maxit) break;
    }
    k_backsolve<<<1, 32, 0, c.st>>>(c.H, c.gvec, jc, m, c.yv);
    k_update_x<<<gN, TPB, 0, c.st>>>(x, c.Z, c.yv, jc, N);
    c.launches += 2;
    if (converged || total >= maxit) break;
    // restart from the true residual r = b - A M^{-1}... in right
    // preconditioning x is already in the unpreconditioned space: r = b - A x
    spmv<NB>(c, x, w);
    k_residual_vec<<<gN, TPB, 0, c.st>>>(w, b, N);
    k_dot_partial<<<NPART, TPB, 0, c.st>>>(w, w, N, c.part);
    k_reduce<<<1, TPB, 0, c.st>>>(c.part, NPART, c.scal + 2);
    k_gmres_init<<<1, 32, 0, c.st>>>(c.gvec, m, c.scal + 2, c.scal);
    k_scale_copy<<<gN, TPB, 0, c.st>>>(c.V, w, c.scal + 1, N);
    c.launches += 5;
    const double br = read_scalar(c, c.scal);
    if (br <= target) {
      converged = true;
      break;
    }
  }
  *iters = total;
  if (check_cuda(c, cudaGetLastError(), "fgmres")) return MPM_ERR_CUDA;
  return converged ? MPM_OK : MPM_ERR_KRYLOV_STAGNATED;
}

}  // namespace

// ============================================================== launchers
int64_t scan_exclusive(Ctx &c, const int32_t *in, int32_t *out, int64_t n) {
  const int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
  if (nb > SCAN_CHUNK || nb > c.scan_cap) {
    c.last_error = "scan too long";
    return -1;
  }
  k_scan_blocks<<<nb, SCAN_T, 0, c.st>>>(in, out, n, c.scan_tmp);
  k_scan_top<<<1, SCAN_T, 0, c.st>>>(c.scan_tmp, nb);
  k_scan_add<<<nb, SCAN_T, 0, c.st>>>(out, n, c.scan_tmp, in, c.scal + 4);
  c.launches += 3;
  return (int64_t)llround(read_scalar(c, c.scal + 4));
}

double run_norm(Ctx &c, const double *x) {
  k_dot_partial<<<NPART, TPB, 0, c.st>>>(x, x, c.N(), c.part);
  k_reduce<<<1, TPB, 0, c.st>>>(c.part, NPART, c.scal + 3);
  c.launches += 2;
  return sqrt(read_scalar(c, c.scal + 3));
}

void run_axpy(Ctx &c, double *y, double a, const double *x, int64_t n) {
  k_axpy<<<nblk(n), TPB, 0, c.st>>>(y, a, x, n);
  UPMPM_LAUNCH(c);
}

void run_scale_system(Ctx &c, double *rhs_out, const double *R) {
  const int64_t nn = c.g.nnodes;
  if (c.nb == 3) {
    k_diag_scale<3><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, c.val, c.dscale);
    k_scale_matrix<3><<<nblk(c.nnzb * 9), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, c.val, c.dscale);
  } else {
    k_diag_scale<4><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, c.val, c.dscale);
    k_scale_matrix<4><<<nblk(c.nnzb * 16), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, c.val, c.dscale);
  }
  k_scale_rhs<<<nblk(c.N()), TPB, 0, c.st>>>(c.N(), R, c.dscale, rhs_out);
  c.launches += 3;
}

void run_unscale_add(Ctx &c, double *X, const double *xhat) {
  k_unscale_add<<<nblk(c.N()), TPB, 0, c.st>>>(c.N(), X, c.dscale, xhat);
  UPMPM_LAUNCH(c);
}

void run_block_jacobi(Ctx &c) {
  const int64_t nn = c.g.nnodes;
  if (c.nb == 3)
    k_block_jacobi<3><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, c.val, c.dinv, c.err);
  else
    k_block_jacobi<4><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, c.val, c.dinv, c.err);
  UPMPM_LAUNCH(c);
}

void run_precond(Ctx &c, const double *v, double *z) {
  if (c.nb == 3) precond<3>(c, v, z);
  else precond<4>(c, v, z);
}

int run_fgmres(Ctx &c, const double *b, double *x, double rtol, int maxit, int *iters) {
  if (c.nb == 3) return fgmres_impl<3>(c, b, x, rtol, maxit, iters);
  return fgmres_impl<4>(c, b, x, rtol, maxit, iters);
}

}  // namespace upmpm
