// mpm_solver.cu -- linear algebra of the Newton step (Eq. jacobian-system-
// stabilized-ppp):  J dX = -R  on the block-CSR Jacobian.
//
// The system is scaled symmetrically, D J D y = -D R with D_ii = |J_ii|^{-1/2},
// which brings the momentum rows (stiffness ~ 1e7) and the mass rows (~ 1e-7)
// to unit diagonal so that the Krylov residual weighs both balance laws; then
// right-preconditioned restarted FGMRES with classical Gram-Schmidt applied
// twice (CGS2) solves it.  The Hessenberg matrix and the Givens rotations live
// in device memory (FP64); the host reads one scalar per iteration.  Vectors
// and matrix values are in the precision T of the solve: FP64, or FP32 in the
// mixed mode (the Newton residual around it stays FP64).  Reductions use a
// fixed grid and tree (deterministic) and sum each thread's part in T before
// the FP64 block sum.  No tensor cores: the work is sparse.
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
  const int base = threadIdx.x * SCAN_I;  // one block; nb <= SCAN_CHUNK
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
template <typename T>
__global__ void k_dot_partial(const T *__restrict__ x, const T *__restrict__ y, int64_t n,
                              double *__restrict__ part) {
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_reduce(const double *__restrict__ part, int np, double *__restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[0] = acc;
}

template <typename T>
__global__ void k_scale_copy(T *__restrict__ y, const T *__restrict__ x, const double *s, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] * (T)s[0];
}

template <typename T>
__global__ void k_residual_vec(T *__restrict__ y, const T *__restrict__ b, int64_t n) {  // y = b - y
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = b[i] - y[i];
}

// ---------------------------------------------------------------- scaling
__device__ inline int find_diag(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                int64_t a) {
  int lo = row_ptr[a], hi = row_ptr[a + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int cm = col[mid];
    if (cm == a) return mid;
    if (cm < a) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

template <int NB, typename T>
__global__ void k_diag_scale(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const T *__restrict__ val,
                             T *__restrict__ dsc) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  const int e = find_diag(row_ptr, col, a);
  for (int r = 0; r < NB; ++r) {
    const double d = e >= 0 ? fabs((double)val[(int64_t)e * NB * NB + r * NB + r]) : 0.0;
    dsc[a * NB + r] = (T)(d > 0.0 ? 1.0 / sqrt(d) : 1.0);
  }
}

template <int NB, typename T>
__global__ void k_scale_matrix(int64_t nnzb, const int32_t *__restrict__ row_of,
                               const int32_t *__restrict__ col, T *__restrict__ val,
                               const T *__restrict__ dsc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * NB * NB) return;
  const int64_t e = t / (NB * NB);
  const int rc = (int)(t % (NB * NB));
  const int r = rc / NB, cc = rc % NB;
  val[t] *= dsc[(int64_t)row_of[e] * NB + r] * dsc[(int64_t)col[e] * NB + cc];
}

template <typename T>
__global__ void k_scale_rhs(int64_t n, const double *__restrict__ R, const T *__restrict__ dsc,
                            T *__restrict__ rhs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = (T)(-(double)dsc[i] * R[i]);
}

template <typename T>
__global__ void k_unscale_add(int64_t n, double *__restrict__ X, const T *__restrict__ dsc,
                              const T *__restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) X[i] += (double)dsc[i] * (double)y[i];
}

// ---------------------------------------------------------------- block Jacobi
template <int NB, typename T>
__global__ void k_block_jacobi(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ col, const T *__restrict__ val,
                               T *__restrict__ dinv, int *err) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  const int e = find_diag(row_ptr, col, a);
  double A[NB][NB], B[NB][NB];
  for (int i = 0; i < NB; ++i)
    for (int j = 0; j < NB; ++j) {
      A[i][j] = e >= 0 ? (double)val[(int64_t)e * NB * NB + i * NB + j] : (i == j ? 1.0 : 0.0);
      B[i][j] = i == j ? 1.0 : 0.0;
    }
  bool ok = true;  // Gauss-Jordan with partial pivoting
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
    for (int j = 0; j < NB; ++j) dinv[a * NB * NB + i * NB + j] = (T)B[i][j];
}

template <int NB, typename T>
__global__ void k_bj_apply(int64_t nnodes, const T *__restrict__ dinv, const T *__restrict__ x,
                           T *__restrict__ y) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  T xv[NB];
  for (int j = 0; j < NB; ++j) xv[j] = x[a * NB + j];
  for (int i = 0; i < NB; ++i) {
    T s = 0;
    for (int j = 0; j < NB; ++j) s += dinv[a * NB * NB + i * NB + j] * xv[j];
    y[a * NB + i] = s;
  }
}

// ---------------------------------------------------------------- SpMV
// SPL * NB threads per block row: the SPL lanes of output r of a row split the
// row's blocks (lane l takes blocks l, l + SPL, ...) and spend one FMA per
// stored value of block row r; one shuffle sum per output joins them.
// (GB300's FP64 pipe is narrow: an FP64 SpMV should issue one FP64
// instruction per value with all lanes busy; the SPL-fold split gives the SM
// enough warps to cover the load latency.)
template <int NB, int SPL, typename T>
__global__ void k_bsr_spmv(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, const T *__restrict__ val,
                           const T *__restrict__ x, T *__restrict__ y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t o = t / SPL;
  const int part = (int)(t - o * SPL);
  const int64_t row = o / NB;
  const int r = (int)(o - row * NB);
  T acc = 0;
  if (row < nnodes) {
    const int e1 = row_ptr[row + 1];
#pragma unroll 4
    for (int e = row_ptr[row] + part; e < e1; e += SPL) {
      const T *blk = val + (int64_t)e * NB * NB + r * NB;
      const T *xb = x + (int64_t)__ldg(&col[e]) * NB;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc = fma(__ldg(&blk[c]), __ldg(&xb[c]), acc);
    }
  }
#pragma unroll
  for (int s = SPL / 2; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (row < nnodes && part == 0) y[row * NB + r] = acc;
}

// ---------------------------------------------------------------- FGMRES
// partial dots of w against V_0..V_{cnt-1}
template <typename T>
__global__ void k_multidot_partial(const T *__restrict__ V, int cnt, const T *__restrict__ w,
                                   int64_t n, double *__restrict__ part) {
  for (int i = 0; i < cnt; ++i) {
    const T *vi = V + (int64_t)i * n;
    T acc = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
      acc += vi[k] * w[k];
    const double s = block_sum((double)acc);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR + i] = s;
  }
}

__global__ void k_multidot_reduce(const double *__restrict__ part, int np, int cnt,
                                  double *__restrict__ h) {
  const int i = blockIdx.x;  // one block per coefficient
  if (i >= cnt) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) acc += part[(int64_t)b * PSTR + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) h[i] = acc;
}

// w -= sum_i h_i V_i over the thread's elements, then partial dots of the
// updated w against V_i (second Gram-Schmidt pass) or with itself (norm).
template <typename T>
__global__ void k_orth_update(T *__restrict__ w, const T *__restrict__ V, const double *h, int cnt,
                              int64_t n, double *__restrict__ part, int want_norm) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    T s = w[k];
    for (int i = 0; i < cnt; ++i) s -= (T)h[i] * V[(int64_t)i * n + k];
    w[k] = s;
  }
  if (want_norm) {
    T acc = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
      acc += w[k] * w[k];
    const double s = block_sum((double)acc);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR] = s;
  } else {
    for (int i = 0; i < cnt; ++i) {
      T acc = 0;
      for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
           k += (int64_t)gridDim.x * blockDim.x)
        acc += V[(int64_t)i * n + k] * w[k];
      const double s = block_sum((double)acc);
      if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR + i] = s;
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

template <typename T>
__global__ void k_update_x(T *__restrict__ x, const T *__restrict__ Z, const double *y, int jc, int64_t n) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  T s = x[k];
  for (int i = 0; i < jc; ++i) s += (T)y[i] * Z[(int64_t)i * n + k];
  x[k] = s;
}

template <int NB, typename T>
void spmv(Ctx &c, const LinSys<T> &S, const T *x, T *y) {
  constexpr int SPL = NB == 3 ? 2 : 4;  // 25 (2D) / 125 (3D) blocks per GIMP row
  const int64_t threads = c.g.nnodes * NB * SPL;
  prof_begin(c, MPM_PROF_SPMV);
  k_bsr_spmv<NB, SPL, T><<<nblk(threads), TPB, 0, c.st>>>(c.g.nnodes, c.row_ptr, c.col, S.val, x, y);
  prof_end(c, MPM_PROF_SPMV);
  UPMPM_LAUNCH(c);
}

template <int NB, typename T>
void precond(Ctx &c, LinSys<T> &S, const T *x, T *y) {
  prof_begin(c, MPM_PROF_PRECOND);
  if (c.opt.precond == MPM_PRECOND_SCHUR_MG) {
    schur_apply<T>(c, S, x, y);
  } else {
    k_bj_apply<NB, T><<<nblk(c.g.nnodes), TPB, 0, c.st>>>(c.g.nnodes, S.dinv, x, y);
    UPMPM_LAUNCH(c);
  }
  prof_end(c, MPM_PROF_PRECOND);
}

double read_scalar(Ctx &c, const double *dptr) {
  cudaMemcpyAsync(c.h_scalar, dptr, sizeof(double), cudaMemcpyDeviceToHost, c.st);
  cudaStreamSynchronize(c.st);
  return c.h_scalar[0];
}

template <int NB, typename T>
int fgmres_impl(Ctx &c, LinSys<T> &S, double rtol, int maxit, int *iters) {
  const int64_t N = c.N();
  const int m = c.m_restart;
  const int gN = nblk(N);
  const T *b = S.rhs;
  T *x = S.x, *w = S.w;
  double *h1 = c.hcol, *h2 = c.hcol + PSTR;
  cudaMemsetAsync(x, 0, sizeof(T) * N, c.st);
  // beta = ||b||, V_0 = b / beta
  k_dot_partial<T><<<NPART, TPB, 0, c.st>>>(b, b, N, c.part);
  k_reduce<<<1, TPB, 0, c.st>>>(c.part, NPART, c.scal + 2);
  k_gmres_init<<<1, 32, 0, c.st>>>(c.gvec, m, c.scal + 2, c.scal);
  k_scale_copy<T><<<gN, TPB, 0, c.st>>>(S.V, b, c.scal + 1, N);
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
      T *Vj = S.V + (int64_t)j * N, *Zj = S.Z + (int64_t)j * N, *Vn = S.V + (int64_t)(j + 1) * N;
      precond<NB, T>(c, S, Vj, Zj);
      spmv<NB, T>(c, S, Zj, w);
      prof_begin(c, MPM_PROF_ORTH);
      k_multidot_partial<T><<<NPART, TPB, 0, c.st>>>(S.V, j + 1, w, N, c.part);
      k_multidot_reduce<<<j + 1, TPB, 0, c.st>>>(c.part, NPART, j + 1, h1);
      k_orth_update<T><<<NPART, TPB, 0, c.st>>>(w, S.V, h1, j + 1, N, c.part, 0);
      k_multidot_reduce<<<j + 1, TPB, 0, c.st>>>(c.part, NPART, j + 1, h2);
      k_orth_update<T><<<NPART, TPB, 0, c.st>>>(w, S.V, h2, j + 1, N, c.part, 1);
      prof_end(c, MPM_PROF_ORTH);
      k_arnoldi_finish<<<1, TPB, 0, c.st>>>(c.part, NPART, j, m, h1, h2, c.H, c.gvec, c.cs, c.sn, c.scal);
      k_scale_copy<T><<<gN, TPB, 0, c.st>>>(Vn, w, c.scal + 1, N);
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
    k_update_x<T><<<gN, TPB, 0, c.st>>>(x, S.Z, c.yv, jc, N);
    c.launches += 2;
    if (converged || total >= maxit) break;
    // restart from the true residual r = b - A x (right preconditioning: x is
    // already in the unpreconditioned space)
    spmv<NB, T>(c, S, x, w);
    k_residual_vec<T><<<gN, TPB, 0, c.st>>>(w, b, N);
    k_dot_partial<T><<<NPART, TPB, 0, c.st>>>(w, w, N, c.part);
    k_reduce<<<1, TPB, 0, c.st>>>(c.part, NPART, c.scal + 2);
    k_gmres_init<<<1, 32, 0, c.st>>>(c.gvec, m, c.scal + 2, c.scal);
    k_scale_copy<T><<<gN, TPB, 0, c.st>>>(S.V, w, c.scal + 1, N);
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

template <typename T>
int dmalloc(T **p, int64_t n) {
  return cudaMalloc((void **)p, sizeof(T) * (size_t)(n > 0 ? n : 1)) == cudaSuccess ? MPM_OK
                                                                                     : MPM_ERR_NO_MEMORY;
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
  k_dot_partial<double><<<NPART, TPB, 0, c.st>>>(x, x, c.N(), c.part);
  k_reduce<<<1, TPB, 0, c.st>>>(c.part, NPART, c.scal + 3);
  c.launches += 2;
  return sqrt(read_scalar(c, c.scal + 3));
}

template <typename T>
int linsys_alloc(Ctx &c, LinSys<T> &S, bool krylov) {
  const int64_t nn = c.g.nnodes, N = c.N();
  const int nb = c.nb, m = c.m_restart;
  int rc = MPM_OK;
  auto A = [&](T **p, int64_t n) {
    if (!rc) rc = dmalloc(p, n);
  };
  A(&S.dscale, N);
  A(&S.dinv, nn * nb * nb);
  A(&S.rhs, N);
  A(&S.x, N);
  A(&S.w, N);
  if (krylov) {
    A(&S.V, (int64_t)(m + 1) * N);
    A(&S.Z, (int64_t)m * N);
  }
  if (!rc && c.opt.precond == MPM_PRECOND_SCHUR_MG) rc = schur_alloc<T>(c, S);
  return rc;
}

template <typename T>
void linsys_free(LinSys<T> &S) {
  schur_free<T>(S);
  T *ptrs[] = {S.val, S.dscale, S.dinv, S.rhs, S.x, S.w, S.V, S.Z};
  for (T *p : ptrs)
    if (p) cudaFree(p);
  S.val = S.dscale = S.dinv = S.rhs = S.x = S.w = S.V = S.Z = nullptr;
  S.cap = 0;
}

template <typename T>
int linsys_reserve(Ctx &c, LinSys<T> &S) {
  if (S.cap >= c.nnzb_cap && S.val) return MPM_OK;
  if (S.val) cudaFree(S.val);
  S.val = nullptr;
  S.cap = 0;
  if (dmalloc(&S.val, c.nnzb_cap * c.nb * c.nb)) {
    c.last_error = "device allocation of the block-CSR values failed";
    return MPM_ERR_NO_MEMORY;
  }
  S.cap = c.nnzb_cap;
  return MPM_OK;
}

template <typename T>
void run_scale_system(Ctx &c, LinSys<T> &S, const double *R) {
  const int64_t nn = c.g.nnodes;
  if (c.nb == 3) {
    k_diag_scale<3, T><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.dscale);
    k_scale_matrix<3, T><<<nblk(c.nnzb * 9), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, S.val, S.dscale);
  } else {
    k_diag_scale<4, T><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.dscale);
    k_scale_matrix<4, T><<<nblk(c.nnzb * 16), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, S.val, S.dscale);
  }
  k_scale_rhs<T><<<nblk(c.N()), TPB, 0, c.st>>>(c.N(), R, S.dscale, S.rhs);
  c.launches += 3;
}

template <typename T>
__global__ void k_inst_weight(int64_t N, int nb, const int32_t *__restrict__ node_inst,
                              const double *__restrict__ w, T *__restrict__ v, int divide) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int inst = node_inst[i / nb];
  if (inst < 0) return;
  v[i] = divide ? (T)(v[i] / w[inst]) : (T)(v[i] * w[inst]);
}

template <typename T>
void run_inst_weight(Ctx &c, T *v, int divide) {
  k_inst_weight<T><<<nblk(c.N()), TPB, 0, c.st>>>(c.N(), c.nb, c.node_inst, c.iw, v, divide);
  UPMPM_LAUNCH(c);
}
template void run_inst_weight<double>(Ctx &, double *, int);
template void run_inst_weight<float>(Ctx &, float *, int);

template <typename T>
void run_unscale_add(Ctx &c, const LinSys<T> &S, double *X) {
  k_unscale_add<T><<<nblk(c.N()), TPB, 0, c.st>>>(c.N(), X, S.dscale, S.x);
  UPMPM_LAUNCH(c);
}

template <typename T>
void run_block_jacobi(Ctx &c, LinSys<T> &S) {
  const int64_t nn = c.g.nnodes;
  if (c.nb == 3)
    k_block_jacobi<3, T><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.dinv, c.err);
  else
    k_block_jacobi<4, T><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.dinv, c.err);
  UPMPM_LAUNCH(c);
}

template <typename T>
void run_precond(Ctx &c, LinSys<T> &S, const T *v, T *z) {
  if (c.nb == 3) precond<3, T>(c, S, v, z);
  else precond<4, T>(c, S, v, z);
}

template <typename T>
int run_fgmres(Ctx &c, LinSys<T> &S, double rtol, int maxit, int *iters) {
  if (c.nb == 3) return fgmres_impl<3, T>(c, S, rtol, maxit, iters);
  return fgmres_impl<4, T>(c, S, rtol, maxit, iters);
}

#define UPMPM_INST(T)                                                               \
  template int linsys_alloc<T>(Ctx &, LinSys<T> &, bool);                           \
  template void linsys_free<T>(LinSys<T> &);                                        \
  template int linsys_reserve<T>(Ctx &, LinSys<T> &);                               \
  template void run_scale_system<T>(Ctx &, LinSys<T> &, const double *);            \
  template void run_unscale_add<T>(Ctx &, const LinSys<T> &, double *);             \
  template void run_block_jacobi<T>(Ctx &, LinSys<T> &);                            \
  template void run_precond<T>(Ctx &, LinSys<T> &, const T *, T *);                 \
  template int run_fgmres<T>(Ctx &, LinSys<T> &, double, int, int *);
UPMPM_INST(double)
UPMPM_INST(float)
#undef UPMPM_INST

}  // namespace upmpm
