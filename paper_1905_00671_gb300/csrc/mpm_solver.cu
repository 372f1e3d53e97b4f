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
constexpr int ORTH_TPB = 1024;     // threads per block of the Gram-Schmidt update ...
constexpr int64_t ORTH_BIG = 1 << 20;  // ... on systems of at least this many unknowns
// FP64 Gram-Schmidt: the second pass of classical Gram-Schmidt runs when the
// first left less than this fraction of the new vector's norm (it then lost
// more digits than a second pass needs to restore; otherwise one pass keeps
// the basis orthogonal to round-off: on the oracle's Jacobian of a slope piece
// the first pass left 0.2-0.5 of the norm and the basis orthogonal to 4e-15
// with one pass).  FP32 keeps both passes always.
constexpr double REORTH_THETA = 0.01;
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
  pdl_enter();
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_reduce(const double *__restrict__ part, int np, double *__restrict__ out) {
  pdl_enter();
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[0] = acc;
}

template <typename T>
__global__ void k_scale_copy(T *__restrict__ y, const T *__restrict__ x, const double *s, int64_t n) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] * (T)s[0];
}

template <typename T>
__global__ void k_residual_vec(T *__restrict__ y, const T *__restrict__ b, int64_t n) {  // y = b - y
  pdl_enter();
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
                             T *__restrict__ dsc, T *__restrict__ dsci) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  const int e = find_diag(row_ptr, col, a);
  for (int r = 0; r < NB; ++r) {
    const double d = e >= 0 ? fabs((double)val[(int64_t)e * NB * NB + r * NB + r]) : 0.0;
    dsc[a * NB + r] = (T)(d > 0.0 ? 1.0 / sqrt(d) : 1.0);
    dsci[a * NB + r] = (T)(d > 0.0 ? sqrt(d) : 1.0);
  }
}

// D J D in place, FP64: one thread per value (the two multiplications of
// each value are the kernel's FP64 work; one thread per block was slower).
template <int NB, typename T>
__global__ void k_scale_matrix_v(int64_t nnzb, const int32_t *__restrict__ row_of,
                                 const int32_t *__restrict__ col, T *__restrict__ val,
                                 const T *__restrict__ dsc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb * NB * NB) return;
  const int64_t e = t / (NB * NB);
  const int rc = (int)(t % (NB * NB));
  const int r = rc / NB, cc = rc % NB;
  val[t] *= dsc[(int64_t)row_of[e] * NB + r] * dsc[(int64_t)col[e] * NB + cc];
}

// D J D in place, FP32 (bound by memory): one thread per block, the block's
// NB row and NB column scales read once, its NB^2 values in 16-byte words.
template <int NB, typename T>
__global__ void k_scale_matrix(int64_t nnzb, const int32_t *__restrict__ row_of,
                               const int32_t *__restrict__ col, T *__restrict__ val,
                               const T *__restrict__ dsc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  const int64_t ra = (int64_t)row_of[e] * NB, cb = (int64_t)col[e] * NB;
  T rs[NB], cs[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    rs[i] = dsc[ra + i];
    cs[i] = dsc[cb + i];
  }
  T *blk = val + e * NB * NB;
  if constexpr (NB == 4 && sizeof(T) == sizeof(float)) {  // a block row is one 16-byte word
    float4 *b4 = reinterpret_cast<float4 *>(blk);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4 v = b4[i];
      v.x *= rs[i] * cs[0];
      v.y *= rs[i] * cs[1];
      v.z *= rs[i] * cs[2];
      v.w *= rs[i] * cs[3];
      b4[i] = v;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j) blk[i * NB + j] *= rs[i] * cs[j];
  }
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
  pdl_enter();
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
  pdl_enter();
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
// Partial dots of w against V_0..V_{cnt-1}, block (b, i) summing its slice of
// V_i . w: the cnt products run side by side instead of one after another.
// A row i = cnt of blocks (grid y = cnt + 1) sums w . w.  With skip set, the
// kernel does nothing unless *skip is nonzero (a second Gram-Schmidt pass
// that the first pass's norms made unnecessary).
template <typename T>
__global__ void k_multidot2(const T *__restrict__ V, const T *__restrict__ w, int64_t n, int cnt,
                            double *__restrict__ part, const double *__restrict__ skip) {
  pdl_enter();
  if (skip && *skip == 0.0) return;
  const int i = blockIdx.y;
  const T *vi = i < cnt ? V + (int64_t)i * n : w;
  T acc = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    acc += vi[k] * w[k];
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR + i] = s;
}

// w -= sum_i h_i V_i; with want_norm also the partial sums of |w|^2; with
// skip set, nothing unless *skip is nonzero (as k_multidot2)
template <typename T>
__global__ void k_orth_sub(T *__restrict__ w, const T *__restrict__ V, const double *__restrict__ h, int cnt,
                           int64_t n, double *__restrict__ part, int want_norm, const double *__restrict__ skip) {
  pdl_enter();
  if (skip && *skip == 0.0) return;
  T nacc = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    T sv = w[k];
    for (int i = 0; i < cnt; ++i) sv -= (T)h[i] * V[(int64_t)i * n + k];
    w[k] = sv;
    nacc += sv * sv;
  }
  if (want_norm) {
    const double sn = block_sum((double)nacc);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * PSTR] = sn;
  }
}

__global__ void k_multidot_reduce(const double *__restrict__ part, int np, int cnt,
                                  double *__restrict__ h, const double *__restrict__ skip) {
  pdl_enter();
  const int i = blockIdx.x;  // one block per coefficient
  if (i >= cnt) return;
  if (skip && *skip == 0.0) {  // the pass is skipped: its coefficients are zero
    if (threadIdx.x == 0) h[i] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) acc += part[(int64_t)b * PSTR + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) h[i] = acc;
}

// Whether classical Gram-Schmidt needs its second pass: after the first, w
// has lost most of its norm to the basis (|w1|^2 < theta^2 |w0|^2, |w0|^2 in
// h1[cnt] from the first pass's products, |w1|^2 from the first update's
// partials).  Writes 1 (second pass) or 0 into *flag.
__global__ void k_reorth_test(const double *__restrict__ part, int np, const double *__restrict__ h1, int cnt,
                              double theta, double *__restrict__ flag) {
  pdl_enter();
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) acc += part[(int64_t)b * PSTR];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *flag = acc < theta * theta * h1[cnt] ? 1.0 : 0.0;
}

// Finish Arnoldi column j: ||w|| from the partials, H(:,j) = h1 + h2, apply
// the previous Givens rotations, form the new one, update g.
// scal[0] = |g_{j+1}| (residual estimate), scal[1] = 1 / ||w||.
__global__ void k_arnoldi_finish(const double *__restrict__ part, int np, int j, int m,
                                 const double *__restrict__ h1, const double *__restrict__ h2,
                                 double *__restrict__ H, double *__restrict__ g, double *__restrict__ cs,
                                 double *__restrict__ sn, double *__restrict__ scal) {
  pdl_enter();
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
  pdl_enter();
  if (threadIdx.x != 0) return;
  const double beta = sqrt(beta_sq[0]);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  scal[0] = beta;
  scal[1] = beta > 0.0 ? 1.0 / beta : 0.0;
}

__global__ void k_backsolve(const double *__restrict__ H, const double *__restrict__ g, int jc, int m,
                            double *__restrict__ y) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  for (int i = jc - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < jc; ++l) s -= H[i * m + l] * y[l];
    y[i] = s / H[i * m + i];
  }
}

template <typename T>
__global__ void k_update_x(T *__restrict__ x, const T *__restrict__ Z, const double *y, int jc, int64_t n) {
  pdl_enter();
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
  const int32_t *rp = c.row_ptr, *cl = c.col;
  const T *val = S.val;
  launch_pdl(c, k_bsr_spmv<NB, SPL, T>, nblk(threads), TPB, 0, c.g.nnodes, rp, cl, val, x, y);
  prof_end(c, MPM_PROF_SPMV);
}

template <int NB, typename T>
void precond(Ctx &c, LinSys<T> &S, const T *x, T *y) {
  prof_begin(c, MPM_PROF_PRECOND);
  if (c.opt.precond == MPM_PRECOND_SCHUR_MG) {
    schur_apply<T>(c, S, x, y);
  } else {
    launch_pdl(c, k_bj_apply<NB, T>, nblk(c.g.nnodes), TPB, 0, c.g.nnodes, (const T *)S.dinv, x, y);
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
      {  // classical Gram-Schmidt, twice; the j + 1 products of a pass run side by side
        // slices per vector: enough blocks to stream the vectors at HBM speed
        // on large systems (about 8 elements per thread, up to NPART slices),
        // at least NPART / cnt on small ones; the update uses 1024-thread
        // blocks on large systems for the same reason (measured: slope
        // Gram-Schmidt 70 -> 46 ms per step; on the 62k-unknown footing the
        // larger blocks cost more than they gave, 1.4 -> 1.7 ms)
        const int cnt = j + 1;
        const int64_t by_size = N >= ORTH_BIG ? N / (TPB * 8) : 0;
        const int nbx = (int)std::min<int64_t>(NPART, std::max<int64_t>(std::max(16, NPART / cnt), by_size));
        const T *V = S.V, *wc = w;
        const double *ph = c.part;
        const int otpb = N >= ORTH_BIG ? ORTH_TPB : TPB;
        // FP64: the second pass only where the first lost the new direction's
        // digits (REORTH_THETA); FP32 always takes both passes
        const bool sel = sizeof(T) == sizeof(double);
        const double *skip = sel ? (const double *)(c.scal + 6) : nullptr;
        const int c1 = sel ? cnt + 1 : cnt;  // FP64: |w|^2 beside the products
        launch_pdl(c, k_multidot2<T>, dim3(nbx, c1), TPB, 0, V, wc, N, cnt, c.part, (const double *)nullptr);
        launch_pdl(c, k_multidot_reduce, c1, TPB, 0, ph, nbx, c1, h1, (const double *)nullptr);
        launch_pdl(c, k_orth_sub<T>, NPART, otpb, 0, w, V, (const double *)h1, cnt, N, c.part, sel ? 1 : 0,
                   (const double *)nullptr);
        if (sel)
          launch_pdl(c, k_reorth_test, 1, TPB, 0, ph, (int)NPART, (const double *)h1, cnt, REORTH_THETA,
                     c.scal + 6);
        launch_pdl(c, k_multidot2<T>, dim3(nbx, cnt), TPB, 0, V, wc, N, cnt, c.part, skip);
        launch_pdl(c, k_multidot_reduce, cnt, TPB, 0, ph, nbx, cnt, h2, skip);
        launch_pdl(c, k_orth_sub<T>, NPART, otpb, 0, w, V, (const double *)h2, cnt, N, c.part, 1, skip);
      }
      prof_end(c, MPM_PROF_ORTH);
      launch_pdl(c, k_arnoldi_finish, 1, TPB, 0, (const double *)c.part, (int)NPART, j, m, (const double *)h1,
                 (const double *)h2, c.H, c.gvec, c.cs, c.sn, c.scal);
      launch_pdl(c, k_scale_copy<T>, gN, TPB, 0, Vn, (const T *)w, (const double *)(c.scal + 1), N);
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

// ------------------------------------------------ batched FGMRES (instances)
// A batched context solves one block-diagonal system (the instances never
// couple; the preconditioner keeps that structure), so FGMRES runs per
// instance: every inner product, Hessenberg column, Givens rotation and
// convergence test is the instance's own, while each kernel serves all
// instances at once.  An instance that meets its tolerance is frozen (its next
// Krylov vectors are zero) until the others finish.

// out[i * ostride + k] = sum over the DOFs of instance i of V_k . w, k < cnt;
// block (i, k) walks instance i's node box in a fixed order
template <typename T>
__global__ void k_inst_dots(GridP g, int nb, const InstDev *__restrict__ inst, const T *__restrict__ V,
                            int64_t vstride, const T *__restrict__ w, double *__restrict__ out, int ostride) {
  pdl_enter();
  const InstDev I = inst[blockIdx.x];
  const int k = blockIdx.y;
  const T *Vk = V + (int64_t)k * vstride;
  const int64_t m0 = I.nc[0] + 1, m1 = g.d > 1 ? I.nc[1] + 1 : 1, m2 = g.d > 2 ? I.nc[2] + 1 : 1;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < m0 * m1 * m2; t += blockDim.x) {
    const int64_t i0 = t % m0, i1 = (t / m0) % m1, i2 = t / (m0 * m1);
    const int64_t a = (i0 + I.off[0]) + (int64_t)g.nn[0] * ((i1 + I.off[1]) + (int64_t)g.nn[1] * (i2 + I.off[2]));
    for (int d = 0; d < nb; ++d) acc += (double)Vk[a * nb + d] * (double)w[a * nb + d];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[(int64_t)blockIdx.x * ostride + k] = acc;
}

// w -= sum_k h[inst, k] V_k
template <typename T>
__global__ void k_inst_orth(int64_t N, int nb, const int32_t *__restrict__ node_inst, T *__restrict__ w,
                            const T *__restrict__ V, int64_t vstride, const double *__restrict__ h, int cnt) {
  pdl_enter();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  const int i = node_inst[e / nb];
  if (i < 0) return;
  T s = w[e];
  for (int k = 0; k < cnt; ++k) s -= (T)h[(int64_t)i * PSTR + k] * V[(int64_t)k * vstride + e];
  w[e] = s;
}

// out = scale[inst] w (0 between instances)
template <typename T>
__global__ void k_inst_scale(int64_t N, int nb, const int32_t *__restrict__ node_inst, const T *__restrict__ w,
                             const double *__restrict__ scl, T *__restrict__ out) {
  pdl_enter();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  const int i = node_inst[e / nb];
  out[e] = i < 0 ? T(0) : (T)(scl[i] * (double)w[e]);
}

// start of a cycle: beta_i = ||r_i||, g_i = beta_i e_1, scale 1 / beta_i; the
// tolerance rtol beta_i is fixed at the first start; an instance already
// within it is frozen
__global__ void k_inst_init(int ni, int m, const double *__restrict__ nrm, double *__restrict__ g,
                            double *__restrict__ scl, double *__restrict__ tgt, int32_t *__restrict__ frozen,
                            int32_t *__restrict__ jc, int32_t *__restrict__ active, double rtol, int set_target) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni) return;
  const double beta = sqrt(nrm[i]);
  if (set_target) tgt[i] = rtol * beta;
  for (int k = 0; k <= m; ++k) g[(int64_t)i * (m + 1) + k] = 0.0;
  g[(int64_t)i * (m + 1)] = beta;
  jc[i] = 0;
  const bool done = !(beta > tgt[i]);
  frozen[i] = done ? 1 : 0;
  scl[i] = (!done && beta > 0.0) ? 1.0 / beta : 0.0;
  if (!done) atomicAdd(active, 1);
}

// Arnoldi column j of every active instance: H(:, j) = h1 + h2, previous
// rotations, new rotation, g update, residual estimate |g_{j+1}|; an instance
// whose estimate reaches its tolerance (or whose new vector vanishes) freezes
// with j + 1 columns
__global__ void k_inst_arnoldi(int ni, int j, int m, const double *__restrict__ h1, const double *__restrict__ h2,
                               const double *__restrict__ nrm, double *__restrict__ H, double *__restrict__ g,
                               double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ scl,
                               const double *__restrict__ tgt, double *__restrict__ res,
                               int32_t *__restrict__ frozen, int32_t *__restrict__ jc, int32_t *__restrict__ active) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni) return;
  if (frozen[i]) {
    scl[i] = 0.0;
    return;
  }
  double *Hi = H + (int64_t)i * (m + 1) * m, *gi = g + (int64_t)i * (m + 1);
  double *csi = cs + (int64_t)i * (m + 1), *sni = sn + (int64_t)i * (m + 1);
  const double hn = sqrt(nrm[i]);
  double col[PSTR];
  for (int k = 0; k <= j; ++k) col[k] = h1[(int64_t)i * PSTR + k] + h2[(int64_t)i * PSTR + k];
  for (int k = 0; k < j; ++k) {
    const double t = csi[k] * col[k] + sni[k] * col[k + 1];
    col[k + 1] = -sni[k] * col[k] + csi[k] * col[k + 1];
    col[k] = t;
  }
  const double r = hypot(col[j], hn);
  double c = 1.0, sv = 0.0;
  if (r > 0.0) {
    c = col[j] / r;
    sv = hn / r;
  }
  csi[j] = c;
  sni[j] = sv;
  col[j] = r;
  for (int k = 0; k <= j; ++k) Hi[k * m + j] = col[k];
  const double gj = gi[j];
  gi[j + 1] = -sv * gj;
  gi[j] = c * gj;
  res[i] = fabs(gi[j + 1]);
  jc[i] = j + 1;
  if (res[i] <= tgt[i] || !(hn > 0.0)) {
    frozen[i] = 1;
    scl[i] = 0.0;
  } else {
    scl[i] = 1.0 / hn;
    atomicAdd(active, 1);
  }
}

__global__ void k_inst_backsolve(int ni, int m, const double *__restrict__ H, const double *__restrict__ g,
                                 const int32_t *__restrict__ jc, double *__restrict__ y) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni) return;
  const double *Hi = H + (int64_t)i * (m + 1) * m, *gi = g + (int64_t)i * (m + 1);
  double *yi = y + (int64_t)i * (m + 1);
  for (int k = jc[i] - 1; k >= 0; --k) {
    double sv = gi[k];
    for (int l = k + 1; l < jc[i]; ++l) sv -= Hi[k * m + l] * yi[l];
    yi[k] = Hi[k * m + k] != 0.0 ? sv / Hi[k * m + k] : 0.0;
  }
}

template <typename T>
__global__ void k_inst_update_x(int64_t N, int nb, const int32_t *__restrict__ node_inst, T *__restrict__ x,
                                const T *__restrict__ Z, int64_t zstride, const double *__restrict__ y, int m,
                                const int32_t *__restrict__ jc) {
  pdl_enter();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N) return;
  const int i = node_inst[e / nb];
  if (i < 0) return;
  T sv = x[e];
  for (int k = 0; k < jc[i]; ++k) sv += (T)y[(int64_t)i * (m + 1) + k] * Z[(int64_t)k * zstride + e];
  x[e] = sv;
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
  A(&S.dscinv, N);
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
  T *ptrs[] = {S.val, S.dscale, S.dscinv, S.dinv, S.rhs, S.x, S.w, S.V, S.Z};
  for (T *p : ptrs)
    if (p) cudaFree(p);
  S.val = S.dscale = S.dscinv = S.dinv = S.rhs = S.x = S.w = S.V = S.Z = nullptr;
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
    k_diag_scale<3, T><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.dscale, S.dscinv);
    if (sizeof(T) == sizeof(float))
      k_scale_matrix<3, T><<<nblk(c.nnzb), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, S.val, S.dscale);
    else
      k_scale_matrix_v<3, T><<<nblk(c.nnzb * 9), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, S.val, S.dscale);
  } else {
    k_diag_scale<4, T><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.dscale, S.dscinv);
    if (sizeof(T) == sizeof(float))
      k_scale_matrix<4, T><<<nblk(c.nnzb), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, S.val, S.dscale);
    else
      k_scale_matrix_v<4, T><<<nblk(c.nnzb * 16), TPB, 0, c.st>>>(c.nnzb, c.row_of, c.col, S.val, S.dscale);
  }
  k_scale_rhs<T><<<nblk(c.N()), TPB, 0, c.st>>>(c.N(), R, S.dscale, S.rhs);
  c.launches += 3;
}

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

int read_active(Ctx &c, const int32_t *dptr) {
  int32_t *h = reinterpret_cast<int32_t *>(c.h_bk);
  cudaMemcpyAsync(h, dptr, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st);
  cudaStreamSynchronize(c.st);
  return h[0];
}

template <int NB, typename T>
int fgmres_batched_impl(Ctx &c, LinSys<T> &S, double rtol, int maxit, int *iters) {
  const int64_t N = c.N();
  const int m = c.m_restart, ni = c.ninst;
  const int gN = nblk(N);
  const T *b = S.rhs;
  T *x = S.x, *w = S.w;
  double *H = c.bk, *g = H + (int64_t)ni * (m + 1) * m, *cs = g + (int64_t)ni * (m + 1);
  double *sn = cs + (int64_t)ni * (m + 1), *y = sn + (int64_t)ni * (m + 1);
  double *h1 = y + (int64_t)ni * (m + 1), *h2 = h1 + (int64_t)ni * PSTR, *nrm = h2 + (int64_t)ni * PSTR;
  double *scl = nrm + ni, *tgt = scl + ni, *res = tgt + ni;
  int32_t *frozen = c.bk_i, *jc = frozen + ni, *active = jc + ni;
  const int ib = nblk(ni, 128);
  cudaMemsetAsync(x, 0, sizeof(T) * N, c.st);
  auto start = [&](const T *r, int set_target) {
    k_inst_dots<T><<<dim3(ni, 1), TPB, 0, c.st>>>(c.g, NB, c.inst, r, N, r, nrm, 1);
    cudaMemsetAsync(active, 0, sizeof(int32_t), c.st);
    k_inst_init<<<ib, 128, 0, c.st>>>(ni, m, nrm, g, scl, tgt, frozen, jc, active, rtol, set_target);
    k_inst_scale<T><<<gN, TPB, 0, c.st>>>(N, NB, c.node_inst, r, scl, S.V);
    c.launches += 3;
    return read_active(c, active);
  };
  *iters = 0;
  int nact = start(b, 1);
  if (nact == 0) return MPM_OK;
  int total = 0;
  bool converged = false;
  while (true) {
    for (int j = 0; j < m; ++j) {
      T *Vj = S.V + (int64_t)j * N, *Zj = S.Z + (int64_t)j * N, *Vn = S.V + (int64_t)(j + 1) * N;
      precond<NB, T>(c, S, Vj, Zj);
      spmv<NB, T>(c, S, Zj, w);
      prof_begin(c, MPM_PROF_ORTH);
      k_inst_dots<T><<<dim3(ni, j + 1), TPB, 0, c.st>>>(c.g, NB, c.inst, S.V, N, w, h1, PSTR);
      k_inst_orth<T><<<gN, TPB, 0, c.st>>>(N, NB, c.node_inst, w, S.V, N, h1, j + 1);
      k_inst_dots<T><<<dim3(ni, j + 1), TPB, 0, c.st>>>(c.g, NB, c.inst, S.V, N, w, h2, PSTR);
      k_inst_orth<T><<<gN, TPB, 0, c.st>>>(N, NB, c.node_inst, w, S.V, N, h2, j + 1);
      k_inst_dots<T><<<dim3(ni, 1), TPB, 0, c.st>>>(c.g, NB, c.inst, w, N, w, nrm, 1);
      prof_end(c, MPM_PROF_ORTH);
      cudaMemsetAsync(active, 0, sizeof(int32_t), c.st);
      k_inst_arnoldi<<<ib, 128, 0, c.st>>>(ni, j, m, h1, h2, nrm, H, g, cs, sn, scl, tgt, res, frozen, jc,
                                           active);
      k_inst_scale<T><<<gN, TPB, 0, c.st>>>(N, NB, c.node_inst, w, scl, Vn);
      c.launches += 7;
      ++total;
      nact = read_active(c, active);
      if (nact == 0) {
        converged = true;
        break;
      }
      if (total >= maxit) break;
    }
    k_inst_backsolve<<<ib, 128, 0, c.st>>>(ni, m, H, g, jc, y);
    k_inst_update_x<T><<<gN, TPB, 0, c.st>>>(N, NB, c.node_inst, x, S.Z, N, y, m, jc);
    c.launches += 2;
    if (converged || total >= maxit) break;
    // restart every instance from its true residual r = b - A x
    spmv<NB, T>(c, S, x, w);
    k_residual_vec<T><<<gN, TPB, 0, c.st>>>(w, b, N);
    UPMPM_LAUNCH(c);
    if (start(w, 0) == 0) {
      converged = true;
      break;
    }
  }
  *iters = total;
  if (check_cuda(c, cudaGetLastError(), "fgmres")) return MPM_ERR_CUDA;
  return converged ? MPM_OK : MPM_ERR_KRYLOV_STAGNATED;
}

template <typename T>
int run_fgmres(Ctx &c, LinSys<T> &S, double rtol, int maxit, int *iters) {
  if (c.ninst > 1)
    return c.nb == 3 ? fgmres_batched_impl<3, T>(c, S, rtol, maxit, iters)
                     : fgmres_batched_impl<4, T>(c, S, rtol, maxit, iters);
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
