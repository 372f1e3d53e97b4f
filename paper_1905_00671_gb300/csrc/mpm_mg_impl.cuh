// mpm_mg_impl.cuh -- precision-generic body of mpm_mg.cu (included twice, with
// MG_REAL = double / float and MG_NS naming the namespace of that precision).

namespace MG_NS {
using real = MG_REAL;


constexpr int TPB = 256;
inline int nblk(int64_t n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

// Block size for a launch of `threads` threads: the largest of 256, 128, 64, 32
// that still gives two blocks per SM, so that small multigrid levels spread
// over the whole GPU (one SM's FP64 pipe is narrow; a level's rows packed into
// a few 256-thread blocks would run on a few SMs).
struct Geom {
  int blocks, tpb;
};
inline Geom geom(const Ctx &c, int64_t threads) {
  int t = 256;
  while (t > 32 && threads < (int64_t)t * 2 * c.nsm) t >>= 1;
  return {nblk(threads > 0 ? threads : 1, t), t};
}

template <int D>
struct NS_ {
  static constexpr int v = D == 2 ? 25 : 125;
};

// Small dense inverse with partial pivoting (B <= 4); identity on failure.
template <int B>
__device__ inline bool invert_small(real A[B][B], real Inv[B][B]) {
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) Inv[i][j] = i == j ? 1.0 : 0.0;
  for (int k = 0; k < B; ++k) {
    int piv = k;
    real best = fabs(A[k][k]);
    for (int i = k + 1; i < B; ++i)
      if (fabs(A[i][k]) > best) { best = fabs(A[i][k]); piv = i; }
    if (!(best > 1e-300)) {
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) Inv[i][j] = i == j ? 1.0 : 0.0;
      return false;
    }
    if (piv != k)
      for (int j = 0; j < B; ++j) {
        real t = A[k][j]; A[k][j] = A[piv][j]; A[piv][j] = t;
        t = Inv[k][j]; Inv[k][j] = Inv[piv][j]; Inv[piv][j] = t;
      }
    const real inv = 1.0 / A[k][k];
    for (int j = 0; j < B; ++j) { A[k][j] *= inv; Inv[k][j] *= inv; }
    for (int i = 0; i < B; ++i) {
      if (i == k) continue;
      const real f = A[i][k];
      if (f == 0.0) continue;
      for (int j = 0; j < B; ++j) { A[i][j] -= f * A[k][j]; Inv[i][j] -= f * Inv[k][j]; }
    }
  }
  return true;
}

__device__ inline int find_col(const int32_t *__restrict__ col, int lo, int hi, int key) {
  hi -= 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = col[mid];
    if (c == key) return mid;
    if (c < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// ------------------------------------------------------------ block split
template <int D>
__global__ void k_extract_A(int64_t nnzb, const real *__restrict__ J, real *__restrict__ A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  constexpr int NB = D + 1;
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) A[e * D * D + i * D + k] = J[e * NB * NB + i * NB + k];
}

// Block of row a coupling with node a + o, from the per-node coupling mask of
// the block sparsity (columns of a row are in mask-bit order); -1 if absent.
template <int D>
__device__ inline int mask_block(const uint64_t *__restrict__ mask, const int32_t *__restrict__ row_ptr,
                                 int a, int o0, int o1, int o2) {
  if (o0 < -3 || o0 > 3 || o1 < -3 || o1 > 3 || (D == 3 && (o2 < -3 || o2 > 3))) return -1;
  const int sl = (o0 + 3) + 7 * (o1 + 3) + (D == 3 ? 49 * (o2 + 3) : 0);
  const uint64_t *mk = mask + (int64_t)a * PATTERN_MASK_WORDS;
  const int w = sl >> 6;
  const uint64_t word = mk[w];
  if (!((word >> (sl & 63)) & 1ull)) return -1;
  int before = __popcll(word & ((1ull << (sl & 63)) - 1ull));
  for (int i = 0; i < w; ++i) before += __popcll(mk[i]);
  return row_ptr[a] + before;
}

__device__ inline void grid_xyz(const int nn0, const int nn1, int a, int c[3]) {
  const int r = a / nn0;
  c[0] = a - r * nn0;
  c[1] = r % nn1;
  c[2] = r / nn1;
}

// diag(A)_a^{-1} and the row sum of the B1 blocks of row a
template <int D>
__global__ void k_diag_inv_A(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const real *__restrict__ A,
                             const real *__restrict__ J, real *__restrict__ DAinv,
                             real *__restrict__ B1rs) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  constexpr int NB = D + 1;
  const int e = find_col(col, row_ptr[a], row_ptr[a + 1], (int)a);
  real M[D][D], Inv[D][D];
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) M[i][k] = e >= 0 ? A[(int64_t)e * D * D + i * D + k] : (i == k);
  invert_small<D>(M, Inv);
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) DAinv[a * D * D + i * D + k] = Inv[i][k];
  real rs[D];
  for (int k = 0; k < D; ++k) rs[k] = 0.0;
  for (int eb = row_ptr[a]; eb < row_ptr[a + 1]; ++eb)
    for (int k = 0; k < D; ++k) rs[k] += J[(int64_t)eb * NB * NB + k * NB + D];
  for (int k = 0; k < D; ++k) B1rs[a * D + k] = rs[k];
}

// W_ac = B2_ac diag(A)_c^{-1} (a 1 x D row per block)
template <int D>
__global__ void k_schur_w(int64_t nnzb, const int32_t *__restrict__ col, const real *__restrict__ J,
                          const real *__restrict__ DAinv, real *__restrict__ W) {
  const int64_t ec = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ec >= nnzb) return;
  constexpr int NB = D + 1;
  const int64_t c = col[ec];
  for (int k = 0; k < D; ++k) {
    real w = 0.0;
    for (int i = 0; i < D; ++i) w += J[ec * NB * NB + D * NB + i] * DAinv[c * D * D + i * D + k];
    W[ec * D + k] = w;
  }
}

// S_ab = C_ab - sum_c W_ac B1_cb on J's sparsity, one thread per block (a, b),
// offset-major (thread t: offset slot t / nnodes of row t % nnodes) so that a
// warp's lanes share the offset; (c, b) is found from c's coupling mask.
template <int D>
__global__ void k_schur_rows(int nn0, int nn1, int64_t nnodes, const uint64_t *__restrict__ mask,
                             const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                             const real *__restrict__ J, const real *__restrict__ W,
                             real *__restrict__ S) {
  constexpr int NB = D + 1, NSL = D == 2 ? 49 : 343;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= NSL * nnodes) return;
  const int a = (int)(t % nnodes);
  const int sl = (int)(t / nnodes);
  const int o0 = sl % 7 - 3, o1 = (sl / 7) % 7 - 3, o2 = D == 3 ? sl / 49 - 3 : 0;
  const int eb = mask_block<D>(mask, row_ptr, a, o0, o1, o2);
  if (eb < 0) return;
  int ac[3];
  grid_xyz(nn0, nn1, a, ac);
  const int b0 = ac[0] + o0, b1 = ac[1] + o1, b2 = ac[2] + o2;
  real prod = 0.0;
  const int r1 = row_ptr[a + 1];
  for (int ec = row_ptr[a]; ec < r1; ++ec) {
    const int cn = col[ec];
    int cc[3];
    grid_xyz(nn0, nn1, cn, cc);
    const int e_cb = mask_block<D>(mask, row_ptr, cn, b0 - cc[0], b1 - cc[1], b2 - cc[2]);
    if (e_cb < 0) continue;
    for (int k = 0; k < D; ++k) prod += W[(int64_t)ec * D + k] * J[(int64_t)e_cb * NB * NB + k * NB + D];
  }
  S[eb] = J[(int64_t)eb * NB * NB + D * NB + D] - prod;
}

// Fixed-stress approximation: S_ab = C_ab, plus the lumped fixed-stress term
// on the diagonal of free pressure rows.
template <int D>
__global__ void k_schur_fs(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, const real *__restrict__ J,
                           const double *__restrict__ fsd, const uint8_t *__restrict__ fixed,
                           real *__restrict__ S) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  constexpr int NB = D + 1;
  const bool free_p = !fixed[a * NB + D];
  for (int e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
    real v = J[(int64_t)e * NB * NB + D * NB + D];
    if (col[e] == a && free_p) v += (real)fsd[a];
    S[e] = v;
  }
}

// The part of row a's full product sum_c W_ac (sum_b B1_cb) that fell outside
// the sparsity is added to S_aa.
template <int D>
__global__ void k_schur_lump(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const real *__restrict__ J,
                             const real *__restrict__ W, const real *__restrict__ B1rs,
                             real *__restrict__ S) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  constexpr int NB = D + 1;
  real total = 0.0, kept = 0.0;
  int diag = -1;
  for (int e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
    const int cn = col[e];
    if (cn == a) diag = e;
    for (int k = 0; k < D; ++k) total += W[(int64_t)e * D + k] * B1rs[(int64_t)cn * D + k];
    kept += J[(int64_t)e * NB * NB + D * NB + D] - S[e];
  }
  if (diag >= 0) S[diag] -= (total - kept);
}

// ------------------------------------------------------------ Schur apply
// The Krylov solver works on D J D (D = dsc); the blocks below are the
// unscaled physical ones, so the preconditioner of D J D is D^-1 M^-1 D^-1,
// applied with the stored D^-1 (dsi = |diag J|^{1/2}: products instead of
// FP64 divisions, which run long on the narrow FP64 pipe).
// v_u, v_p of the unscaled system; v_p is the S-cycle's level-0 rhs, whose
// first smoothing sweep from zero (x = omega Dinv b, pointwise) is done here.
template <int D>
__global__ void k_split(int64_t nnodes, const real *__restrict__ v, const real *__restrict__ dsi,
                        real *__restrict__ vu, real *__restrict__ bs0, real *__restrict__ xs0,
                        const real *__restrict__ dinvs0, real omega) {
  pdl_enter();
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  for (int k = 0; k < D; ++k) vu[a * D + k] = v[a * (D + 1) + k] * dsi[a * (D + 1) + k];
  const real vp = v[a * (D + 1) + D] * dsi[a * (D + 1) + D];
  bs0[a] = vp;
  xs0[a] = omega * (dinvs0[a] * vp);
}

// Lower-triangular order: v_u is the A-cycle's level-0 rhs, with its first
// smoothing sweep from zero (x = omega Dinv_A v_u, a D x D block per node);
// v_p is kept for the S-cycle's rhs v_p - B2 z_u.
template <int D>
__global__ void k_split_lower(int64_t nnodes, const real *__restrict__ v, const real *__restrict__ dsi,
                              real *__restrict__ ba0, real *__restrict__ xa0, const real *__restrict__ dinva0,
                              real *__restrict__ vp, real omega) {
  pdl_enter();
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  real vu[D];
  for (int k = 0; k < D; ++k) {
    vu[k] = v[a * (D + 1) + k] * dsi[a * (D + 1) + k];
    ba0[a * D + k] = vu[k];
  }
  for (int i = 0; i < D; ++i) {
    real sv = 0.0;
    for (int j = 0; j < D; ++j) sv = fma(dinva0[a * D * D + i * D + j], vu[j], sv);
    xa0[a * D + i] = omega * sv;
  }
  vp[a] = v[a * (D + 1) + D] * dsi[a * (D + 1) + D];
}

// Compact unscaled B2 (row D, u columns, of the unscaled J): D values per block.
template <int D>
__global__ void k_extract_B2(int64_t nnzb, const real *__restrict__ J, real *__restrict__ B2) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  constexpr int NB = D + 1;
  for (int k = 0; k < D; ++k) B2[e * D + k] = J[e * NB * NB + D * NB + k];
}

// w_p = v_p - B2 z_u with the compact unscaled B2: the S-cycle's level-0 rhs,
// with its first smoothing sweep from zero (x = omega Dinv_S w_p).  B1C_LANES
// lanes per row.
template <int D>
__global__ void k_b2c_update(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const real *__restrict__ B2,
                             const real *__restrict__ zu, const real *__restrict__ vp,
                             real *__restrict__ bs0, real *__restrict__ xs0,
                             const real *__restrict__ dinvs0, real omega);

// Compact unscaled B1 (column D of the u rows of the unscaled J): D values
// per block instead of the whole (D+1)^2 block.
template <int D>
__global__ void k_extract_B1(int64_t nnzb, const real *__restrict__ J, real *__restrict__ B1) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  constexpr int NB = D + 1;
  for (int k = 0; k < D; ++k) B1[e * D + k] = J[e * NB * NB + k * NB + D];
}

// w_u = v_u - B1 z_p with the compact unscaled B1: the A-cycle's level-0 rhs,
// with its first smoothing sweep from zero (x = omega Dinv w_u).  B1C_LANES
// lanes per row.
constexpr int B1C_LANES = 8;
template <int D>
__global__ void k_b1c_update(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const real *__restrict__ B1,
                             const real *__restrict__ zp, const real *__restrict__ vu,
                             real *__restrict__ ba0, real *__restrict__ xa0,
                             const real *__restrict__ dinva0, real omega) {
  pdl_enter();
  constexpr int LN = B1C_LANES;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t a = t / LN;
  const int lane = (int)(t % LN);
  const bool valid = a < nnodes;
  real acc[D];
  for (int k = 0; k < D; ++k) acc[k] = 0;
  if (valid) {
    const int e1 = row_ptr[a + 1];
    for (int e = row_ptr[a] + lane; e < e1; e += LN) {
      const real z = zp[col[e]];
      for (int k = 0; k < D; ++k) acc[k] = fma(B1[(int64_t)e * D + k], z, acc[k]);
    }
  }
  for (int o = LN / 2; o > 0; o >>= 1)
    for (int k = 0; k < D; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if (!valid || lane >= D) return;
  // lane i < D finishes component i
  real s = 0.0, wi = 0.0;
  for (int j = 0; j < D; ++j) {
    const real wj = vu[a * D + j] - acc[j];
    wi = lane == j ? wj : wi;
    s = fma(dinva0[a * D * D + lane * D + j], wj, s);
  }
  ba0[a * D + lane] = wi;
  xa0[a * D + lane] = omega * s;
}

template <int D>
__global__ void k_b2c_update(int64_t nnodes, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const real *__restrict__ B2,
                             const real *__restrict__ zu, const real *__restrict__ vp,
                             real *__restrict__ bs0, real *__restrict__ xs0,
                             const real *__restrict__ dinvs0, real omega) {
  pdl_enter();
  constexpr int LN = B1C_LANES;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t a = t / LN;
  const int lane = (int)(t % LN);
  const bool valid = a < nnodes;
  real acc = 0;
  if (valid) {
    const int e1 = row_ptr[a + 1];
    for (int e = row_ptr[a] + lane; e < e1; e += LN) {
      const int64_t b = col[e];
      for (int k = 0; k < D; ++k) acc = fma(B2[(int64_t)e * D + k], zu[b * D + k], acc);
    }
  }
  for (int o = LN / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (!valid || lane != 0) return;
  const real w = vp[a] - acc;
  bs0[a] = w;
  xs0[a] = omega * (dinvs0[a] * w);
}

template <int D>
__global__ void k_merge(int64_t nnodes, const real *__restrict__ zu, const real *__restrict__ zp,
                        const real *__restrict__ dsi, real *__restrict__ z) {
  pdl_enter();
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= nnodes) return;
  for (int k = 0; k < D; ++k) z[a * (D + 1) + k] = zu[a * D + k] * dsi[a * (D + 1) + k];
  z[a * (D + 1) + D] = zp[a] * dsi[a * (D + 1) + D];
}

// ------------------------------------------------------------ multigrid
struct LevelDev {
  int nn[3];
  int64_t nnodes;
  const int32_t *row_ptr, *col;  // level 0 only
  const real *val;              // level 0: block-CSR values
  real *sval;                   // coarse levels: dense 5^d stencil values
  uint8_t *nslot;               // coarse levels: nonzero blocks of each row (0: a node without coupling)
  real *dinv;
  // level 0 only: Dirichlet / inactive DOFs are left out of the transfers
  const uint8_t *fixed;           // fixed[a * mstride + moff + i] != 0: DOF fixed
  int mstride, moff;
  const uint64_t *mask;           // level 0 only: coupling mask of the block sparsity
  // instance of every node (-1 between instances): the transfers connect a
  // fine and a coarse node only within one instance, so the hierarchy of a
  // batched context never mixes instances (null for a single instance)
  const int32_t *inst;
};

__device__ inline real free_w(const LevelDev &L, int64_t a, int i) {
  return (L.fixed && L.fixed[a * L.mstride + L.moff + i]) ? 0.0 : 1.0;
}

// Lanes per row of the row kernels (a row is one node: up to 49 blocks of the
// fine block-CSR in 2D, 125 in 3D, 5^d slots of a coarse stencil).  Eight
// lanes keep the shuffle reduction (log2 LN steps per block row) small next to
// the row's FMAs on GB300's narrow FP64 pipe; FP32 3D rows take 16 (latency).
template <int D>
struct LN_ {
  static constexpr int v = (sizeof(real) == sizeof(double) || D == 2) ? 8 : 16;
};

// Component `lane` (< B) of a B-vector held in registers, without indexing
// the register array by a run-time value.
template <int B>
__device__ inline real pick(const real v[B], int lane) {
  real o = v[0];
#pragma unroll
  for (int i = 1; i < B; ++i) o = lane == i ? v[i] : o;
  return o;
}

// Partial sum over the blocks of row a handled by `lane` (of LN lanes):
// acc += A_ab x_b, one FMA per matrix value.
template <int B, int D, bool ST, int LN>
__device__ inline void row_partial(const LevelDev &L, int64_t a, int lane, const real *__restrict__ x,
                                   real acc[B]) {
  if (!ST) {
    const int e1 = L.row_ptr[a + 1];
    for (int e = L.row_ptr[a] + lane; e < e1; e += LN) {
      const int64_t b = L.col[e];
      const real *blk = L.val + (int64_t)e * B * B;
      real xb[B];
      for (int j = 0; j < B; ++j) xb[j] = x[b * B + j];
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) acc[i] = fma(blk[i * B + j], xb[j], acc[i]);
    }
  } else {
    int ac[3];
    grid_xyz(L.nn[0], L.nn[1], (int)a, ac);
    constexpr int NS = NS_<D>::v;
    const real *base = L.sval + a * NS * B * B;
    // rows without coupling (grid nodes outside the material: half of the
    // slope's coarse grids) are skipped whole
    if (L.nslot[a] == 0) return;
#pragma unroll
    for (int k = 0; k < (NS + LN - 1) / LN; ++k) {
      const int s = lane + k * LN;
      const int o0 = s % 5 - 2, o1 = (s / 5) % 5 - 2, o2 = D == 3 ? s / 25 - 2 : 0;
      const int b0 = ac[0] + o0, b1 = ac[1] + o1, b2 = ac[2] + o2;
      if (s >= NS || b0 < 0 || b0 >= L.nn[0] || b1 < 0 || b1 >= L.nn[1] || b2 < 0 || b2 >= L.nn[2]) continue;
      const int64_t b = b0 + L.nn[0] * (b1 + L.nn[1] * b2);
      const real *blk = base + s * B * B;
      real xb[B];
      for (int j = 0; j < B; ++j) xb[j] = x[b * B + j];
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) acc[i] = fma(blk[i * B + j], xb[j], acc[i]);
    }
  }
}

template <int B, int LN>
__device__ inline void lane_reduce(real acc[B]) {
  for (int o = LN / 2; o > 0; o >>= 1)
    for (int i = 0; i < B; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
}

template <int B, int D, bool ST>
__global__ void k_mg_dinv(LevelDev L, int *err) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= L.nnodes) return;
  real M[B][B], Inv[B][B];
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) M[i][j] = (i == j) ? 1.0 : 0.0;
  if (!ST) {
    const int e = find_col(L.col, L.row_ptr[a], L.row_ptr[a + 1], (int)a);
    if (e >= 0)
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) M[i][j] = L.val[(int64_t)e * B * B + i * B + j];
  } else {
    constexpr int NS = NS_<D>::v;
    const int s = D == 2 ? 12 : 62;  // centre slot of the 5^d stencil
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j) M[i][j] = L.sval[(a * NS + s) * B * B + i * B + j];
  }
  if (!invert_small<B>(M, Inv)) {
    // an all-zero diagonal block (e.g. a node without coupling) acts as identity
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j) Inv[i][j] = i == j ? 1.0 : 0.0;
  }
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) L.dinv[a * B * B + i * B + j] = Inv[i][j];
}

// One damped block-Jacobi sweep: xo = xi + w Dinv (b - A xi); zero_init: xi = 0.
// LN lanes per row.
template <int B, int D, bool ST>
__global__ void k_mg_smooth(LevelDev L, const real *__restrict__ xi, real *__restrict__ xo,
                            const real *__restrict__ b, real omega, int zero_init) {
  pdl_enter();
  constexpr int LN = LN_<D>::v;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t a = t / LN;
  const int lane = (int)(t % LN);
  const bool valid = a < L.nnodes;
  real ax[B];
  for (int i = 0; i < B; ++i) ax[i] = 0.0;
  if (valid && !zero_init) row_partial<B, D, ST, LN>(L, a, lane, xi, ax);
  lane_reduce<B, LN>(ax);  // every lane of the row now holds (A xi)_a
  if (!valid || lane >= B) return;
  // lane i < B finishes component i: B FMAs of row i of Dinv
  real s = 0.0;
  for (int j = 0; j < B; ++j) s = fma(L.dinv[a * B * B + lane * B + j], b[a * B + j] - ax[j], s);
  xo[a * B + lane] = (zero_init ? 0.0 : xi[a * B + lane]) + omega * s;
}

// Fine (block-CSR) level with B <= 2, a group of GS = B * SPL lanes per row:
// lane (r, part) sums block row r over the row's blocks part, part + SPL, ...
// (one FMA per stored value, all lanes busy), one shuffle sum over the SPL
// parts gives (A x)_r, and for a sweep the row's B residuals are exchanged
// inside the group: out = b - A x (residual) or x + omega Dinv (b - A x).
template <int B, int SPL, bool SMOOTH>
__global__ void k_mg_csr_row(LevelDev L, const real *__restrict__ x, real *__restrict__ out,
                             const real *__restrict__ b, real omega) {
  pdl_enter();
  constexpr int GS = B * SPL;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t a = t / GS;
  const int lg = (int)(t - a * GS);
  const int r = lg / SPL, part = lg - r * SPL;
  const bool valid = a < L.nnodes;
  real acc = 0;
  if (valid) {
    const int e1 = L.row_ptr[a + 1];
#pragma unroll 4
    for (int e = L.row_ptr[a] + part; e < e1; e += SPL) {
      const real *blk = L.val + (int64_t)e * B * B + r * B;
      const real *xb = x + (int64_t)L.col[e] * B;
#pragma unroll
      for (int c = 0; c < B; ++c) acc = fma(blk[c], xb[c], acc);
    }
  }
#pragma unroll
  for (int o = SPL / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const real res = valid ? b[a * B + r] - acc : real(0);
  if (!SMOOTH) {
    if (valid && part == 0) out[a * B + r] = res;
    return;
  }
  const int base = (int)(threadIdx.x & 31) - lg;
  real rv[B];
#pragma unroll
  for (int c = 0; c < B; ++c) rv[c] = __shfl_sync(0xffffffffu, res, base + c * SPL);
  if (!valid || part != 0) return;
  real sum = 0;
#pragma unroll
  for (int c = 0; c < B; ++c) sum = fma(L.dinv[a * B * B + r * B + c], rv[c], sum);
  out[a * B + r] = x[a * B + r] + omega * sum;
}

template <int B, int D, bool ST>
__global__ void k_mg_resid(LevelDev L, const real *__restrict__ x, const real *__restrict__ b,
                           real *__restrict__ r) {
  pdl_enter();
  constexpr int LN = LN_<D>::v;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t a = t / LN;
  const int lane = (int)(t % LN);
  const bool valid = a < L.nnodes;
  real ax[B];
  for (int i = 0; i < B; ++i) ax[i] = 0.0;
  if (valid) row_partial<B, D, ST, LN>(L, a, lane, x, ax);
  lane_reduce<B, LN>(ax);
  if (!valid || lane >= B) return;
  r[a * B + lane] = b[a * B + lane] - pick<B>(ax, lane);
}

// ---- coarsest level: exact solve with a dense inverse built at set-up
// Dense copy of the coarsest operator (n = nnodes * B unknowns).
template <int B, int D, bool ST>
__global__ void k_dense_fill(LevelDev L, real *__restrict__ Ad) {
  const int64_t n = L.nnodes * B;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int64_t ri = t / n, ci = t % n;
  const int64_t a = ri / B, b = ci / B;
  const int i = (int)(ri % B), j = (int)(ci % B);
  real v = 0.0;
  if (!ST) {
    const int e = find_col(L.col, L.row_ptr[a], L.row_ptr[a + 1], (int)b);
    if (e >= 0) v = L.val[(int64_t)e * B * B + i * B + j];
  } else {
    int ac[3], bc[3];
    ac[0] = (int)(a % L.nn[0]); ac[1] = (int)((a / L.nn[0]) % L.nn[1]); ac[2] = (int)(a / ((int64_t)L.nn[0] * L.nn[1]));
    bc[0] = (int)(b % L.nn[0]); bc[1] = (int)((b / L.nn[0]) % L.nn[1]); bc[2] = (int)(b / ((int64_t)L.nn[0] * L.nn[1]));
    const int o0 = bc[0] - ac[0], o1 = bc[1] - ac[1], o2 = bc[2] - ac[2];
    if (o0 >= -2 && o0 <= 2 && o1 >= -2 && o1 <= 2 && o2 >= -2 && o2 <= 2) {
      constexpr int NS = NS_<D>::v;
      const int sl = (o0 + 2) + 5 * (o1 + 2) + (D == 3 ? 25 * (o2 + 2) : 0);
      v = L.sval[(a * NS + sl) * B * B + i * B + j];
    }
  }
  Ad[t] = v;
}

// Inverse of the dense coarsest operator Ad (n x n, row-major) into Ai, for
// the two hierarchies side by side (job 0, job 1), in two kernels:
//   k_dense_lu: LU factorisation with partial pivoting, one block per job,
//     in place in Ad (in dynamic shared memory when n <= DENSE_SMEM_MAX_N),
//     row interchanges in piv[k] (LAPACK order), n^3 / 3 FMAs;
//   k_dense_inv_cols: column c of the inverse from P A = L U (forward and
//     back substitution on e_c), one block per column, so the n^3 FMAs of the
//     inverse spread over many SMs (GB300's FP64 pipe does 2 FMAs per clock
//     per SM: one block inverting a 126 x 126 matrix took over a millisecond).
// Columns with no usable pivot (below 1e-14 of the largest entry: nodes
// without material on the coarsest grid) are singular directions: their
// unknowns get zero in every column of the inverse, so the coarse correction
// leaves them alone.
struct DenseJob {
  int n;
  real *Ad, *Ai;
  int *piv;  // n: row interchanged with row k; -1 marks a singular column
};

constexpr int DENSE_LU_THREADS = 512;

__global__ void __launch_bounds__(DENSE_LU_THREADS) k_dense_lu(DenseJob j0, DenseJob j1, int smem) {
  const DenseJob job = blockIdx.x == 0 ? j0 : j1;
  const int n = job.n;
  __shared__ int piv;
  __shared__ real red_v[32];
  __shared__ int red_i[32];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  real *M = smem ? reinterpret_cast<real *>(dyn_smem) : job.Ad;
  if (smem)
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) M[t] = job.Ad[t];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // largest magnitude, for the singular-pivot threshold
  real amax = 0;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) amax = fmax(amax, fabs(M[t]));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (lane == 0) red_v[wid] = amax;
  __syncthreads();
  amax = 0;
  for (int i = 0; i < nw; ++i) amax = fmax(amax, red_v[i]);
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: largest |M[i][k]|, i >= k (warp argmax, then across warps)
    real best = -1;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const real v = fabs(M[i * n + k]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const real ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      real b = -1;
      int p = k;
      for (int i = 0; i < nw; ++i)
        if (red_v[i] > b || (red_v[i] == b && red_i[i] < p)) { b = red_v[i]; p = red_i[i]; }
      piv = b > real(1e-14) * amax ? p : -1;
      job.piv[k] = piv;
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) {  // singular column: no elimination, zero multipliers
      for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) M[i * n + k] = 0;
      __syncthreads();
      continue;
    }
    if (p != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const real t1 = M[k * n + j];
        M[k * n + j] = M[p * n + j];
        M[p * n + j] = t1;
      }
    __syncthreads();
    const real inv = real(1) / M[k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) M[i * n + k] *= inv;
    __syncthreads();
    const int w = n - k - 1;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      const int i = k + 1 + t / w, j = k + 1 + t % w;
      M[i * n + j] = fma(-M[i * n + k], M[k * n + j], M[i * n + j]);
    }
    __syncthreads();
  }
  if (smem)
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) job.Ad[t] = M[t];
}

// block (c, job): column c of the job's inverse; dynamic shared memory n values
__global__ void k_dense_inv_cols(DenseJob j0, DenseJob j1) {
  const DenseJob job = blockIdx.y == 0 ? j0 : j1;
  const int n = job.n, c = blockIdx.x;
  if (c >= n) return;  // block-uniform
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  real *y = reinterpret_cast<real *>(dyn_smem);
  const real *LU = job.Ad;
  const int *pv = job.piv;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = i == c ? real(1) : real(0);
  __syncthreads();
  if (threadIdx.x == 0)  // y = P e_c (the interchanges in order)
    for (int k = 0; k < n; ++k) {
      const int p = pv[k];
      if (p > k) { const real t = y[k]; y[k] = y[p]; y[p] = t; }
    }
  __syncthreads();
  for (int i = 0; i < n; ++i) {  // L y = P e_c (unit lower triangle)
    const real yi = y[i];
    if (yi != real(0))
      for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) y[k] = fma(-LU[k * n + i], yi, y[k]);
    __syncthreads();
  }
  for (int i = n - 1; i >= 0; --i) {  // U x = y
    const real xi = pv[i] < 0 ? real(0) : y[i] / LU[i * n + i];
    __syncthreads();
    if (threadIdx.x == 0) y[i] = xi;
    if (xi != real(0))
      for (int k = threadIdx.x; k < i; k += blockDim.x) y[k] = fma(-LU[k * n + i], xi, y[k]);
    __syncthreads();
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) job.Ai[(int64_t)k * n + c] = y[k];
}

// largest coarsest system factorised in shared memory (n^2 values)
constexpr int DENSE_SMEM_MAX_N = 160;

// x = Ai b
// one warp per row i; lanes split the row and reduce
__global__ void k_dense_apply(int n, const real *__restrict__ Ai, const real *__restrict__ b,
                              real *__restrict__ x) {
  pdl_enter();
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  real s = 0.0;
  if (i < n)
    for (int j = lane; j < n; j += 32) s = fma(Ai[(int64_t)i * n + j], b[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (i < n && lane == 0) x[i] = s;
}

// weight of coarse node I for fine node a along one axis
__device__ inline real pw(int a, int I) {
  const int dlt = a - 2 * I;
  return dlt == 0 ? 1.0 : ((dlt == 1 || dlt == -1) ? 0.5 : 0.0);
}

// b_c(I) = sum_a P_aI r_a over the fine nodes within one fine cell of 2I; if
// xc is given, also the coarse level's first smoothing sweep from zero,
// x_c = omega Dinv_c b_c.
template <int B, int D>
__global__ void k_mg_restrict(LevelDev F, LevelDev Cl, const real *__restrict__ rf,
                              real *__restrict__ bc, real *__restrict__ xc, real omega) {
  pdl_enter();
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= Cl.nnodes) return;
  int Ic[3];
  grid_xyz(Cl.nn[0], Cl.nn[1], (int)I, Ic);
  real acc[B];
  for (int i = 0; i < B; ++i) acc[i] = 0.0;
  const int lo2 = D == 3 ? -1 : 0, hi2 = D == 3 ? 1 : 0;
  for (int d2 = lo2; d2 <= hi2; ++d2)
    for (int d1 = -1; d1 <= 1; ++d1)
      for (int d0 = -1; d0 <= 1; ++d0) {
        const int a0 = 2 * Ic[0] + d0, a1 = 2 * Ic[1] + d1, a2 = D == 3 ? 2 * Ic[2] + d2 : 0;
        if (a0 < 0 || a0 >= F.nn[0] || a1 < 0 || a1 >= F.nn[1] || a2 < 0 || a2 >= F.nn[2]) continue;
        const real wgt = pw(a0, Ic[0]) * pw(a1, Ic[1]) * (D == 3 ? pw(a2, Ic[2]) : 1.0);
        const int64_t a = a0 + (int64_t)F.nn[0] * (a1 + (int64_t)F.nn[1] * a2);
        if (F.inst && F.inst[a] != Cl.inst[I]) continue;
        for (int i = 0; i < B; ++i) acc[i] += wgt * free_w(F, a, i) * rf[a * B + i];
      }
  for (int i = 0; i < B; ++i) bc[I * B + i] = acc[i];
  if (xc)
    for (int i = 0; i < B; ++i) {
      real s = 0.0;
      for (int j = 0; j < B; ++j) s = fma(Cl.dinv[I * B * B + i * B + j], acc[j], s);
      xc[I * B + i] = omega * s;
    }
}

// (P x_c)(a) at fine node a from its 2^d candidate coarse parents: per axis
// I = a/2 (weight 1 if a is even, 1/2 if odd) and I + 1 (weight 1/2 if a is
// odd and I + 1 exists, else 0, with its index clamped), so all loads are
// issued without branches.
template <int B, int D>
__device__ inline void prolong_at(const LevelDev &Cl, const real *__restrict__ xc, const int ac[3],
                                  int inst_a, real out[B]) {
  int i0[3], i1[3];
  real w0[3], w1[3];
  for (int k = 0; k < 3; ++k) {
    const int odd = ac[k] & 1;
    i0[k] = ac[k] >> 1;
    const bool up = odd && i0[k] + 1 < Cl.nn[k];
    i1[k] = up ? i0[k] + 1 : i0[k];
    w0[k] = odd ? 0.5 : 1.0;
    w1[k] = up ? 0.5 : 0.0;
  }
  for (int i = 0; i < B; ++i) out[i] = 0.0;
#pragma unroll
  for (int cmb = 0; cmb < (1 << D); ++cmb) {
    const int s0 = cmb & 1, s1 = (cmb >> 1) & 1, s2 = (cmb >> 2) & 1;
    const real wgt = (s0 ? w1[0] : w0[0]) * (s1 ? w1[1] : w0[1]) * (D == 3 ? (s2 ? w1[2] : w0[2]) : 1.0);
    const int64_t I = (s0 ? i1[0] : i0[0]) +
                      (int64_t)Cl.nn[0] * ((s1 ? i1[1] : i0[1]) + (int64_t)Cl.nn[1] * (D == 3 ? (s2 ? i1[2] : i0[2]) : 0));
    const real w = (!Cl.inst || Cl.inst[I] == inst_a) ? wgt : real(0);
    for (int i = 0; i < B; ++i) out[i] = fma(w, xc[I * B + i], out[i]);
  }
}

// x_f(a) += sum_I P_aI x_c(I)
template <int B, int D>
__global__ void k_mg_prolong(LevelDev F, LevelDev Cl, real *__restrict__ xf,
                             const real *__restrict__ xc) {
  pdl_enter();
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= F.nnodes) return;
  int ac[3];
  grid_xyz(F.nn[0], F.nn[1], (int)a, ac);
  real acc[B];
  prolong_at<B, D>(Cl, xc, ac, F.inst ? F.inst[a] : 0, acc);
  for (int i = 0; i < B; ++i) xf[a * B + i] += free_w(F, a, i) * acc[i];
}

// ---- coarse tail of a V-cycle in one thread block (FP32 hierarchies)
// On the small coarse levels each kernel of a V-cycle is a few microseconds
// of launch and drain for very little work; one block of 1024 threads runs the
// whole tail (every level below a size limit down to the dense coarsest
// solve) with a block barrier between the phases.  Same operations and order
// of levels as the kernel-per-phase V(k, k) cycle.
constexpr int TAIL_MAX_LEVELS = 8;
constexpr int TAIL_MAX_NODES = 128;  // one pass of the block per phase: larger levels are latency-bound here
constexpr int TAIL_THREADS = 1024;

struct TailLevel {
  LevelDev L;
  real *x, *x2, *b, *r;
};
struct TailArgs {
  int nl;  // levels of the tail, the last one the dense coarsest level
  TailLevel lv[TAIL_MAX_LEVELS];
  const real *Ai;
  int ncoarse;
  real omega;
  int nsw;  // sweeps before and after the coarse correction
};

template <int B, int D, bool SMOOTH>
__device__ inline void tail_rows(const LevelDev &L, const real *x, real *out, const real *b, real omega) {
  constexpr int LN = LN_<D>::v;
  const int64_t total = L.nnodes * LN;
  for (int64_t base = 0; base < total; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    const int64_t a = t / LN;
    const int lane = (int)(t % LN);
    const bool valid = a < L.nnodes;
    real ax[B];
    for (int i = 0; i < B; ++i) ax[i] = 0.0;
    if (valid) row_partial<B, D, true, LN>(L, a, lane, x, ax);
    lane_reduce<B, LN>(ax);
    if (!valid || lane != 0) continue;
    real r[B];
    for (int i = 0; i < B; ++i) r[i] = b[a * B + i] - ax[i];
    if (!SMOOTH) {
      for (int i = 0; i < B; ++i) out[a * B + i] = r[i];
      continue;
    }
    for (int i = 0; i < B; ++i) {
      real sv = 0.0;
      for (int j = 0; j < B; ++j) sv = fma(L.dinv[a * B * B + i * B + j], r[j], sv);
      out[a * B + i] = x[a * B + i] + omega * sv;
    }
  }
}

template <int B, int D>
__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(TailArgs A) {
  pdl_enter();
  real *xs[TAIL_MAX_LEVELS], *x2s[TAIL_MAX_LEVELS];
  for (int l = 0; l < A.nl; ++l) {
    xs[l] = A.lv[l].x;
    x2s[l] = A.lv[l].x2;
  }
  for (int l = 0; l + 1 < A.nl; ++l) {
    const LevelDev &L = A.lv[l].L, &Ln = A.lv[l + 1].L;
    for (int k = 1; k < A.nsw; ++k) {  // pre-smoothing sweeps after the first (from zero)
      tail_rows<B, D, true>(L, xs[l], x2s[l], A.lv[l].b, A.omega);
      __syncthreads();
      real *t = xs[l]; xs[l] = x2s[l]; x2s[l] = t;
    }
    tail_rows<B, D, false>(L, xs[l], A.lv[l].r, A.lv[l].b, A.omega);
    __syncthreads();
    real *xc = l + 2 < A.nl ? xs[l + 1] : nullptr;  // first sweep from zero of the next level
    for (int64_t I = threadIdx.x; I < Ln.nnodes; I += blockDim.x) {
      int Ic[3];
      grid_xyz(Ln.nn[0], Ln.nn[1], (int)I, Ic);
      real acc[B];
      for (int i = 0; i < B; ++i) acc[i] = 0.0;
      const int lo2 = D == 3 ? -1 : 0, hi2 = D == 3 ? 1 : 0;
      for (int d2 = lo2; d2 <= hi2; ++d2)
        for (int d1 = -1; d1 <= 1; ++d1)
          for (int d0 = -1; d0 <= 1; ++d0) {
            const int a0 = 2 * Ic[0] + d0, a1 = 2 * Ic[1] + d1, a2 = D == 3 ? 2 * Ic[2] + d2 : 0;
            if (a0 < 0 || a0 >= L.nn[0] || a1 < 0 || a1 >= L.nn[1] || a2 < 0 || a2 >= L.nn[2]) continue;
            const real wgt = pw(a0, Ic[0]) * pw(a1, Ic[1]) * (D == 3 ? pw(a2, Ic[2]) : 1.0);
            const int64_t a = a0 + (int64_t)L.nn[0] * (a1 + (int64_t)L.nn[1] * a2);
            if (L.inst && L.inst[a] != Ln.inst[I]) continue;
            for (int i = 0; i < B; ++i) acc[i] += wgt * A.lv[l].r[a * B + i];
          }
      for (int i = 0; i < B; ++i) A.lv[l + 1].b[I * B + i] = acc[i];
      if (xc)
        for (int i = 0; i < B; ++i) {
          real sv = 0.0;
          for (int j = 0; j < B; ++j) sv = fma(Ln.dinv[I * B * B + i * B + j], acc[j], sv);
          xc[I * B + i] = A.omega * sv;
        }
    }
    __syncthreads();
  }
  {  // dense coarsest solve, one warp per row
    const int lc = A.nl - 1;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < A.ncoarse; i += blockDim.x >> 5) {
      real sv = 0.0;
      for (int j = lane; j < A.ncoarse; j += 32) sv = fma(A.Ai[(int64_t)i * A.ncoarse + j], A.lv[lc].b[j], sv);
      for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
      if (lane == 0) xs[lc][i] = sv;
    }
    __syncthreads();
  }
  for (int l = A.nl - 2; l >= 0; --l) {
    const LevelDev &L = A.lv[l].L, &Ln = A.lv[l + 1].L;
    for (int64_t a = threadIdx.x; a < L.nnodes; a += blockDim.x) {
      int ac[3];
      grid_xyz(L.nn[0], L.nn[1], (int)a, ac);
      real acc[B];
      prolong_at<B, D>(Ln, xs[l + 1], ac, L.inst ? L.inst[a] : 0, acc);
      for (int i = 0; i < B; ++i) xs[l][a * B + i] += acc[i];
    }
    __syncthreads();
    for (int k = 0; k < A.nsw; ++k) {  // post-smoothing sweeps
      tail_rows<B, D, true>(L, xs[l], x2s[l], A.lv[l].b, A.omega);
      __syncthreads();
      real *t = xs[l]; xs[l] = x2s[l]; x2s[l] = t;
    }
  }
}

// Galerkin product P^T A P in two passes, from the block-CSR finest level
// (couplings up to 3 apart per axis) or a stencil level (up to 2 apart):
//   k_mg_ap:   T_a(J) = sum_b w_bJ A_ab over the children b of J, for every
//              fine row a and coarse node J of the 5^d window centred on
//              floor(a / 2) (the coarse nodes a row can reach); thread per
//              (window slot, a), T stored slot-major;
//   k_mg_rap2: A_c(I, J) = sum_a w_aI T_a(J) over the 3^d children a of I;
//              thread per (stencil slot, I).
// Dirichlet DOFs are masked out of the finest level's transfers only, and
// instances are kept apart on every level; grouped as (P^T (A P)), a coarse
// entry costs a few lookups and 3^d FMA blocks instead of one per (a, b) pair
// (measured on the slope's stencil levels: the one-pass product took 20 ms
// per set-up).
// A fine row that contributes nothing to the Galerkin product: a stencil row
// without coupling, or a finest-level row whose DOFs are all fixed (its
// transfers are masked).  k_mg_ap leaves such a row's T unwritten and
// k_mg_rap2 skips it (on the slope, the grid nodes outside the material).
template <int B, bool FST>
__device__ inline bool row_void(const LevelDev &F, int64_t a) {
  if (FST) return F.nslot[a] == 0;
  if (!F.fixed) return false;
  for (int i = 0; i < B; ++i)
    if (!F.fixed[a * F.mstride + F.moff + i]) return false;
  return true;
}

template <int B, int D, bool FST>
__global__ void k_mg_ap(LevelDev F, LevelDev Cl, real *__restrict__ T) {
  constexpr int NS = NS_<D>::v;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= F.nnodes * NS) return;
  // slot-major: the lanes of a warp take one window slot of consecutive fine
  // rows (the same loop bounds up to the parity of a), and T is stored
  // slot-major ([s][a]) so that their results are written side by side
  const int64_t a = t % F.nnodes;
  const int s = (int)(t / F.nnodes);
  if (row_void<B, FST>(F, a)) return;
  int fa[3], Jc[3];
  grid_xyz(F.nn[0], F.nn[1], (int)a, fa);
  Jc[0] = (fa[0] >> 1) + s % 5 - 2;
  Jc[1] = (fa[1] >> 1) + (s / 5) % 5 - 2;
  Jc[2] = D == 3 ? (fa[2] >> 1) + s / 25 - 2 : 0;
  real acc[B * B];
  for (int i = 0; i < B * B; ++i) acc[i] = 0.0;
  if (Jc[0] >= 0 && Jc[0] < Cl.nn[0] && Jc[1] >= 0 && Jc[1] < Cl.nn[1] && Jc[2] >= 0 && Jc[2] < Cl.nn[2]) {
    const int64_t Jn = Jc[0] + (int64_t)Cl.nn[0] * (Jc[1] + (int64_t)Cl.nn[1] * Jc[2]);
    int blo[3], bhi[3];  // children of J within reach of a (and inside the grid)
    for (int k = 0; k < 3; ++k) {
      const int lo = 2 * Jc[k] - 1 > fa[k] - 3 ? 2 * Jc[k] - 1 : fa[k] - 3;
      const int hi = 2 * Jc[k] + 1 < fa[k] + 3 ? 2 * Jc[k] + 1 : fa[k] + 3;
      blo[k] = lo > 0 ? lo : 0;
      bhi[k] = hi < F.nn[k] - 1 ? hi : F.nn[k] - 1;
    }
    if (D == 2) blo[2] = bhi[2] = 0;
    for (int b2 = blo[2]; b2 <= bhi[2]; ++b2)
      for (int b1 = blo[1]; b1 <= bhi[1]; ++b1)
        for (int b0 = blo[0]; b0 <= bhi[0]; ++b0) {
          const int64_t b = b0 + (int64_t)F.nn[0] * (b1 + (int64_t)F.nn[1] * b2);
          if (F.inst && F.inst[b] != Cl.inst[Jn]) continue;
          const real *blk;
          if (!FST) {  // finest level: block-CSR, found by the coupling mask
            const int e = mask_block<D>(F.mask, F.row_ptr, (int)a, b0 - fa[0], b1 - fa[1], b2 - fa[2]);
            if (e < 0) continue;
            blk = F.val + (int64_t)e * B * B;
          } else {     // stencil level: the 5^d slot of b - a
            const int d0 = b0 - fa[0], d1 = b1 - fa[1], d2 = b2 - fa[2];
            if (d0 < -2 || d0 > 2 || d1 < -2 || d1 > 2 || d2 < -2 || d2 > 2) continue;
            blk = F.sval + (a * NS + (d0 + 2) + 5 * (d1 + 2) + (D == 3 ? 25 * (d2 + 2) : 0)) * B * B;
          }
          const real w = pw(b0, Jc[0]) * pw(b1, Jc[1]) * (D == 3 ? pw(b2, Jc[2]) : 1.0);
          for (int j = 0; j < B; ++j) {
            const real wj = FST ? w : w * free_w(F, b, j);  // Dirichlet masks: finest transfers only
            for (int i = 0; i < B; ++i) acc[i * B + j] = fma(wj, blk[i * B + j], acc[i * B + j]);
          }
        }
  }
  for (int i = 0; i < B * B; ++i) T[t * B * B + i] = acc[i];  // t = s * nnodes + a
}

template <int B, int D, bool FST>
__global__ void k_mg_rap2(LevelDev F, LevelDev Cl, const real *__restrict__ T) {
  constexpr int NS = NS_<D>::v;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Cl.nnodes * NS) return;
  // slot-major as k_mg_ap: the lanes take consecutive coarse nodes I of one
  // stencil slot, so a child a = 2 I + d of every lane reads the same window
  // slot of T at every other fine row
  const int64_t I = t % Cl.nnodes;
  const int s = (int)(t / Cl.nnodes);
  int Ic[3], Jc[3];
  grid_xyz(Cl.nn[0], Cl.nn[1], (int)I, Ic);
  Jc[0] = Ic[0] + s % 5 - 2;
  Jc[1] = Ic[1] + (s / 5) % 5 - 2;
  Jc[2] = D == 3 ? Ic[2] + s / 25 - 2 : 0;
  real acc[B * B];
  for (int i = 0; i < B * B; ++i) acc[i] = 0.0;
  if (Jc[0] >= 0 && Jc[0] < Cl.nn[0] && Jc[1] >= 0 && Jc[1] < Cl.nn[1] && Jc[2] >= 0 && Jc[2] < Cl.nn[2]) {
    const int lo2 = D == 3 ? -1 : 0, hi2 = D == 3 ? 1 : 0;
    for (int a2 = lo2; a2 <= hi2; ++a2)
      for (int a1 = -1; a1 <= 1; ++a1)
        for (int a0 = -1; a0 <= 1; ++a0) {
          const int fa[3] = {2 * Ic[0] + a0, 2 * Ic[1] + a1, D == 3 ? 2 * Ic[2] + a2 : 0};
          if (fa[0] < 0 || fa[0] >= F.nn[0] || fa[1] < 0 || fa[1] >= F.nn[1] || fa[2] < 0 || fa[2] >= F.nn[2])
            continue;
          // slot of J in a's window; outside it, T_a(J) is zero (J out of reach)
          const int d0 = Jc[0] - (fa[0] >> 1), d1 = Jc[1] - (fa[1] >> 1), d2 = D == 3 ? Jc[2] - (fa[2] >> 1) : 0;
          if (d0 < -2 || d0 > 2 || d1 < -2 || d1 > 2 || d2 < -2 || d2 > 2) continue;
          const int64_t a = fa[0] + (int64_t)F.nn[0] * (fa[1] + (int64_t)F.nn[1] * fa[2]);
          if (F.inst && F.inst[a] != Cl.inst[I]) continue;
          const real wa = pw(fa[0], Ic[0]) * pw(fa[1], Ic[1]) * (D == 3 ? pw(fa[2], Ic[2]) : 1.0);
          real wi[B];
          bool any = false;
          for (int i = 0; i < B; ++i) {
            wi[i] = FST ? wa : wa * free_w(F, a, i);
            any |= wi[i] != real(0);
          }
          // a row without contribution (row_void): T_a was not written
          if (FST ? F.nslot[a] == 0 : !any) continue;
          const int sl = (d0 + 2) + 5 * (d1 + 2) + (D == 3 ? 25 * (d2 + 2) : 0);
          const real *ta = T + ((int64_t)sl * F.nnodes + a) * B * B;
          for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) acc[i * B + j] = fma(wi[i], ta[i * B + j], acc[i * B + j]);
        }
  }
  for (int i = 0; i < B * B; ++i) Cl.sval[(I * NS + s) * B * B + i] = acc[i];
}

// Nonzero blocks of each coarse row (a block is zero when the product never
// reached it: the coupling is absent), so that the row kernels skip the rows
// of nodes without coupling.  Thread per row.
template <int B, int D>
__global__ void k_mg_rowcount(LevelDev Cl) {
  constexpr int NS = NS_<D>::v;
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= Cl.nnodes) return;
  const real *row = Cl.sval + I * NS * B * B;
  int cnt = 0;
  for (int s = 0; s < NS; ++s) {
    bool nz = false;
    for (int e = 0; e < B * B; ++e) nz |= row[s * B * B + e] != real(0);
    cnt += nz ? 1 : 0;
  }
  Cl.nslot[I] = (uint8_t)cnt;
}

}  // namespace MG_NS

// ============================================================== hierarchy
template <>
struct MGHier<MG_REAL> {
  int B = 1, nlev = 0;
  MG_NS::LevelDev L[16];
  MG_REAL *x[16], *x2[16], *b[16], *r[16];
  MG_REAL *Ad = nullptr, *Ai = nullptr;  // dense coarsest operator (LU factors after set-up) and its inverse
  int *piv = nullptr;                    // row interchanges of the LU factorisation
  MG_REAL *apT = nullptr;                // finest level x 5^d window: A P, first pass of a level's product
  int ncoarse = 0;                       // unknowns of the coarsest level
};

namespace MG_NS {

template <int B, int D>
void mg_setup_t(Ctx &c, MGHier<real> &H) {
  for (int l = 0; l < H.nlev; ++l) {
    LevelDev &L = H.L[l];
    const int nbk = nblk(L.nnodes);
    if (l > 0) {
      constexpr int NS = NS_<D>::v;
      const int g2 = nblk(L.nnodes * NS);
      // two passes, P^T (A P), on every level (the intermediate of the finest
      // level is the largest): on the stencil levels a few lookups and 3^d
      // FMA blocks per coarse entry instead of 3^d x 3^d in one pass
      if (l == 1) {
        k_mg_ap<B, D, false><<<nblk(H.L[0].nnodes * NS), TPB, 0, c.st>>>(H.L[0], L, H.apT);
        k_mg_rap2<B, D, false><<<g2, TPB, 0, c.st>>>(H.L[0], L, H.apT);
      } else {
        k_mg_ap<B, D, true><<<nblk(H.L[l - 1].nnodes * NS), TPB, 0, c.st>>>(H.L[l - 1], L, H.apT);
        k_mg_rap2<B, D, true><<<g2, TPB, 0, c.st>>>(H.L[l - 1], L, H.apT);
      }
      k_mg_rowcount<B, D><<<nbk, TPB, 0, c.st>>>(L);
      UPMPM_LAUNCH(c);
      UPMPM_LAUNCH(c);
      UPMPM_LAUNCH(c);
      k_mg_dinv<B, D, true><<<nbk, TPB, 0, c.st>>>(L, c.err);
    } else {
      k_mg_dinv<B, D, false><<<nbk, TPB, 0, c.st>>>(L, c.err);
    }
    UPMPM_LAUNCH(c);
  }
  // coarsest level: dense inverse
  LevelDev &Lc = H.L[H.nlev - 1];
  const int64_t n = H.ncoarse;
  if (H.nlev == 1) k_dense_fill<B, D, false><<<nblk(n * n), TPB, 0, c.st>>>(Lc, H.Ad);
  else k_dense_fill<B, D, true><<<nblk(n * n), TPB, 0, c.st>>>(Lc, H.Ad);
  UPMPM_LAUNCH(c);
}

// Inverses of the coarsest operators of two hierarchies, in one launch.
void dense_invert_pair(Ctx &c, MGHier<real> &H0, MGHier<real> &H1) {
  const int nmax = H0.ncoarse > H1.ncoarse ? H0.ncoarse : H1.ncoarse;
  const int smem = nmax <= DENSE_SMEM_MAX_N;
  const size_t bytes = smem ? sizeof(real) * nmax * nmax : 0;
  if (smem && bytes > 48 * 1024)
    cudaFuncSetAttribute(k_dense_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  const DenseJob a{H0.ncoarse, H0.Ad, H0.Ai, H0.piv}, b{H1.ncoarse, H1.Ad, H1.Ai, H1.piv};
  k_dense_lu<<<2, DENSE_LU_THREADS, bytes, c.st>>>(a, b, smem);
  k_dense_inv_cols<<<dim3(nmax, 2), 128, sizeof(real) * nmax, c.st>>>(a, b);
  c.launches += 2;
}

// Damping of the block-Jacobi smoother.  A damped Jacobi sweep is stable only
// while omega * lambda_max(Dinv A) < 2 on every level.  Measured lambda_max:
// at most 2.5 for the plane-strain blocks of the strip footing (2D), 3.25 on
// the 3D consolidation block and 3.5 next to the inclined free surface of the
// 3D slope, where 0.6 made the V(2,2)-cycle diverge (FGMRES at its cap; 14
// iterations instead of 232 with 0.5 on a 32 x 32 x 16 slope).  The default
// cycle is V(1,1) (0.7 in 2D, 0.5 in 3D): on the full-size slope it took
// fewer FGMRES iterations than V(2,2) at 0.56 of its cost per application,
// and V(3,3) stalled there.
// (the defaults of Ctx::mg_omega; mpm_options.mg_omega overrides them)
inline real mg_omega(const Ctx &c) { return (real)c.mg_omega(); }

// one damped block-Jacobi sweep on level l: x <- x + omega Dinv (b - A x)
template <int B, int D>
void sweep(Ctx &c, MGHier<real> &H, int l) {
  LevelDev &L = H.L[l];
  if (l == 0 && B <= 2) {
    constexpr int SPL = B <= 2 ? 4 / B : 1;
    const Geom g = geom(c, L.nnodes * B * SPL);
    launch_pdl(c, k_mg_csr_row<B, SPL, true>, g.blocks, g.tpb, 0, L, (const real *)H.x[l], H.x2[l],
               (const real *)H.b[l], mg_omega(c));
  } else {
    const Geom g = geom(c, L.nnodes * LN_<D>::v);
    if (l == 0)
      launch_pdl(c, k_mg_smooth<B, D, false>, g.blocks, g.tpb, 0, L, (const real *)H.x[l], H.x2[l],
                 (const real *)H.b[l], mg_omega(c), 0);
    else
      launch_pdl(c, k_mg_smooth<B, D, true>, g.blocks, g.tpb, 0, L, (const real *)H.x[l], H.x2[l],
                 (const real *)H.b[l], mg_omega(c), 0);
  }
  std::swap(H.x[l], H.x2[l]);
}

// V(k,k)-cycle on level l (k = c.mg_sweeps(), default 2).  On entry b[l]
// holds the rhs and x[l] the first pre-smoothing sweep from zero (omega Dinv
// b, pointwise), done by the kernel that produced b[l]; on return x[l] holds
// the result.
template <int B, int D>
void vcycle_t(Ctx &c, MGHier<real> &H, int l) {
  if (sizeof(real) == sizeof(float) && l >= 1 && l < H.nlev - 1 && H.L[l].nnodes <= TAIL_MAX_NODES &&
      H.nlev - l <= TAIL_MAX_LEVELS) {  // the rest of the cycle in one block
    TailArgs A{};
    A.nl = H.nlev - l;
    for (int k = 0; k < A.nl; ++k) A.lv[k] = TailLevel{H.L[l + k], H.x[l + k], H.x2[l + k], H.b[l + k], H.r[l + k]};
    A.Ai = H.Ai;
    A.ncoarse = H.ncoarse;
    A.omega = mg_omega(c);
    A.nsw = c.mg_sweeps();
    launch_pdl(c, k_mg_tail<B, D>, 1, TAIL_THREADS, 0, A);
    // 2 nsw - 1 sweeps per level (odd) swapped x and x2 (as sweep() does on the host)
    for (int k = l; k < H.nlev - 1; ++k) std::swap(H.x[k], H.x2[k]);
    return;
  }
  if (l == H.nlev - 1) {  // exact solve on the coarsest grid
    const Geom g = geom(c, (int64_t)H.ncoarse * 32);
    launch_pdl(c, k_dense_apply, g.blocks, g.tpb, 0, H.ncoarse, (const real *)H.Ai, (const real *)H.b[l], H.x[l]);
    return;
  }
  LevelDev &L = H.L[l], &Ln = H.L[l + 1];
  real *xn_first = l + 1 == H.nlev - 1 ? nullptr : H.x[l + 1];
  for (int k = 1; k < c.mg_sweeps(); ++k) sweep<B, D>(c, H, l);  // pre-smoothing after the first
  const Geom gr = geom(c, L.nnodes * LN_<D>::v), gc = geom(c, Ln.nnodes), gf = geom(c, L.nnodes);
  if (l == 0 && B <= 2) {
    constexpr int SPL = B <= 2 ? 4 / B : 1;
    const Geom g0 = geom(c, L.nnodes * B * SPL);
    launch_pdl(c, k_mg_csr_row<B, SPL, false>, g0.blocks, g0.tpb, 0, L, (const real *)H.x[l], H.r[l],
               (const real *)H.b[l], mg_omega(c));
  } else if (l == 0) {
    launch_pdl(c, k_mg_resid<B, D, false>, gr.blocks, gr.tpb, 0, L, (const real *)H.x[l], (const real *)H.b[l],
               H.r[l]);
  } else {
    launch_pdl(c, k_mg_resid<B, D, true>, gr.blocks, gr.tpb, 0, L, (const real *)H.x[l], (const real *)H.b[l],
               H.r[l]);
  }
  launch_pdl(c, k_mg_restrict<B, D>, gc.blocks, gc.tpb, 0, L, Ln, (const real *)H.r[l], H.b[l + 1], xn_first,
             mg_omega(c));
  vcycle_t<B, D>(c, H, l + 1);
  launch_pdl(c, k_mg_prolong<B, D>, gf.blocks, gf.tpb, 0, L, Ln, H.x[l], (const real *)H.x[l + 1]);
  for (int k = 0; k < c.mg_sweeps(); ++k) sweep<B, D>(c, H, l);  // post-smoothing sweeps
}

// Allocate a hierarchy for block size B over the grid's node lattice; level 0
// refers to a block-CSR operator given at setup.
int mg_alloc(Ctx &c, MGHier<real> &H, int B) {
  H.B = B;
  const int D = c.d;
  const int NS = D == 2 ? 25 : 125;
  int nn[3] = {c.g.nn[0], c.g.nn[1], c.g.nn[2]};
  // instance of every node of the current level (host); level l + 1 takes
  // the instance of the fine node at the same place (2I)
  std::vector<int32_t> imap((size_t)nn[0] * nn[1] * nn[2], -1), inext;
  for (size_t i = 0; i < c.inst_h.size(); ++i) {
    const InstDev &I = c.inst_h[i];
    const int64_t m0 = I.nc[0] + 1, m1 = D > 1 ? I.nc[1] + 1 : 1, m2 = D > 2 ? I.nc[2] + 1 : 1;
    for (int64_t t = 0; t < m0 * m1 * m2; ++t) {
      const int64_t i0 = t % m0, i1 = (t / m0) % m1, i2 = t / (m0 * m1);
      imap[(i0 + I.off[0]) + (int64_t)nn[0] * ((i1 + I.off[1]) + (int64_t)nn[1] * (i2 + I.off[2]))] = (int32_t)i;
    }
  }
  int l = 0;
  while (true) {
    LevelDev &L = H.L[l];
    for (int k = 0; k < 3; ++k) L.nn[k] = nn[k];
    L.nnodes = (int64_t)nn[0] * nn[1] * nn[2];
    L.row_ptr = nullptr;
    L.col = nullptr;
    L.val = nullptr;
    L.sval = nullptr;
    L.nslot = nullptr;
    L.fixed = nullptr;
    L.mask = nullptr;
    L.mstride = 1;
    L.moff = 0;
    const int64_t vb = L.nnodes * B;
    if (cudaMalloc(&L.dinv, sizeof(real) * L.nnodes * B * B) ||
        cudaMalloc(&H.x[l], sizeof(real) * vb) || cudaMalloc(&H.x2[l], sizeof(real) * vb) ||
        cudaMalloc(&H.b[l], sizeof(real) * vb) || cudaMalloc(&H.r[l], sizeof(real) * vb))
      return MPM_ERR_NO_MEMORY;
    if (l > 0 && (cudaMalloc(&L.sval, sizeof(real) * L.nnodes * NS * B * B) || cudaMalloc(&L.nslot, L.nnodes)))
      return MPM_ERR_NO_MEMORY;
    int32_t *dinst = nullptr;
    if (c.ninst > 1) {
      if (cudaMalloc(&dinst, sizeof(int32_t) * L.nnodes) != cudaSuccess) return MPM_ERR_NO_MEMORY;
      cudaMemcpy(dinst, imap.data(), sizeof(int32_t) * L.nnodes, cudaMemcpyHostToDevice);
    }
    L.inst = dinst;
    ++l;
    int mn = 1 << 30;
    for (int k = 0; k < D; ++k) mn = nn[k] < mn ? nn[k] : mn;
    // the coarsest level is solved exactly: stop at <= 64 nodes or a 2-node axis
    if (mn <= 2 || L.nnodes <= 64 || l >= 15) break;
    int nc[3] = {nn[0], nn[1], nn[2]};
    for (int k = 0; k < D; ++k) nc[k] = (nn[k] + 1) / 2;
    inext.assign((size_t)nc[0] * nc[1] * nc[2], -1);
    for (int64_t I2 = 0; I2 < nc[2]; ++I2)
      for (int64_t I1 = 0; I1 < nc[1]; ++I1)
        for (int64_t I0 = 0; I0 < nc[0]; ++I0) {
          const int64_t f0 = 2 * I0, f1 = D > 1 ? 2 * I1 : I1, f2 = D > 2 ? 2 * I2 : I2;
          inext[I0 + nc[0] * (I1 + nc[1] * I2)] = imap[f0 + nn[0] * (f1 + nn[1] * f2)];
        }
    imap.swap(inext);
    for (int k = 0; k < 3; ++k) nn[k] = nc[k];
  }
  H.nlev = l;
  H.ncoarse = (int)(H.L[l - 1].nnodes * B);
  if (H.ncoarse > 1024) {  // an axis of 2 nodes stops the coarsening early (a thin grid)
    c.last_error = "multigrid: the coarsest level has more than 1024 unknowns (one grid axis of very few "
                   "cells against a long one)";
    return MPM_ERR_BAD_ARG;
  }
  if (cudaMalloc(&H.Ad, sizeof(real) * H.ncoarse * H.ncoarse) ||
      cudaMalloc(&H.Ai, sizeof(real) * H.ncoarse * H.ncoarse) || cudaMalloc(&H.piv, sizeof(int) * H.ncoarse))
    return MPM_ERR_NO_MEMORY;
  if (H.nlev > 1 && cudaMalloc(&H.apT, sizeof(real) * H.L[0].nnodes * NS * B * B)) return MPM_ERR_NO_MEMORY;
  return MPM_OK;
}

void mg_free(MGHier<real> &H) {
  cudaFree(H.Ad);
  cudaFree(H.Ai);
  cudaFree(H.piv);
  cudaFree(H.apT);
  H.Ad = H.Ai = H.apT = nullptr;
  H.piv = nullptr;
  for (int l = 0; l < H.nlev; ++l) {
    cudaFree(const_cast<int32_t *>(H.L[l].inst));
    H.L[l].inst = nullptr;
    cudaFree(H.L[l].dinv);
    cudaFree(H.L[l].sval);
    cudaFree(H.L[l].nslot);
    cudaFree(H.x[l]);
    cudaFree(H.x2[l]);
    cudaFree(H.b[l]);
    cudaFree(H.r[l]);
  }
  H.nlev = 0;
}

// The finest level's block-Jacobi inverses only: the coarse levels keep the
// Galerkin product of an earlier set-up (mpm_options.precond_reuse).
template <int B, int D>
void mg_refresh_t(Ctx &c, MGHier<real> &H) {
  k_mg_dinv<B, D, false><<<nblk(H.L[0].nnodes), TPB, 0, c.st>>>(H.L[0], c.err);
  UPMPM_LAUNCH(c);
}

void mg_setup(Ctx &c, MGHier<real> &H, const int32_t *row_ptr, const int32_t *col, const real *val,
              int moff, bool coarse) {
  H.L[0].row_ptr = row_ptr;
  H.L[0].col = col;
  H.L[0].val = val;
  H.L[0].fixed = c.fixed;
  H.L[0].mstride = c.nb;
  H.L[0].moff = moff;
  H.L[0].mask = c.row_mask;
  if (c.d == 2) {
    if (H.B == 1) coarse ? mg_setup_t<1, 2>(c, H) : mg_refresh_t<1, 2>(c, H);
    else coarse ? mg_setup_t<2, 2>(c, H) : mg_refresh_t<2, 2>(c, H);
  } else {
    if (H.B == 1) coarse ? mg_setup_t<1, 3>(c, H) : mg_refresh_t<1, 3>(c, H);
    else coarse ? mg_setup_t<3, 3>(c, H) : mg_refresh_t<3, 3>(c, H);
  }
}

// V-cycle on H's level-0 vectors (b[0] and the first sweep in x[0] set by the
// caller); the result is left in x[0].
void mg_vcycle(Ctx &c, MGHier<real> &H) {
  if (c.d == 2) {
    if (H.B == 1) vcycle_t<1, 2>(c, H, 0);
    else vcycle_t<2, 2>(c, H, 0);
  } else {
    if (H.B == 1) vcycle_t<1, 3>(c, H, 0);
    else vcycle_t<3, 3>(c, H, 0);
  }
}

}  // namespace MG_NS

// ============================================================== Schur
template <>
int schur_alloc<MG_REAL>(Ctx &c, LinSys<MG_REAL> &S) {
  using namespace MG_NS;
  const int64_t nn = c.g.nnodes;
  const int d = c.d;
  if (!S.mgA) S.mgA = new MGHier<MG_REAL>();
  if (!S.mgS) S.mgS = new MGHier<MG_REAL>();
  int rc = mg_alloc(c, *S.mgA, d);
  if (!rc) rc = mg_alloc(c, *S.mgS, 1);
  if (rc) return rc;
  if (cudaMalloc(&S.DAinv, sizeof(real) * nn * d * d) || cudaMalloc(&S.vu, sizeof(real) * nn * d) ||
      cudaMalloc(&S.B1rs, sizeof(real) * nn * d) || (c.schur_lower() && cudaMalloc(&S.vp, sizeof(real) * nn)))
    return MPM_ERR_NO_MEMORY;
  return MPM_OK;
}

template <>
void schur_free<MG_REAL>(LinSys<MG_REAL> &S) {
  using namespace MG_NS;
  if (S.mgA) { mg_free(*S.mgA); delete S.mgA; S.mgA = nullptr; }
  if (S.mgS) { mg_free(*S.mgS); delete S.mgS; S.mgS = nullptr; }
  MG_REAL *ptrs[] = {S.Aval, S.Sval, S.B1c, S.W, S.B1rs, S.DAinv, S.vu, S.B2c, S.vp};
  for (MG_REAL *p : ptrs) cudaFree(p);
  S.Aval = S.Sval = S.B1c = S.W = S.B1rs = S.DAinv = S.vu = S.B2c = S.vp = nullptr;
  if (S.gexec) cudaGraphExecDestroy(S.gexec);
  S.gexec = nullptr;
  S.gkey_col = S.gkey_val = nullptr;
  S.g_x0 = S.g_zp = S.g_zu = nullptr;
  S.sub_cap = 0;
}

// Split the unscaled Jacobian (after Dirichlet elimination) into A and S and
// build both hierarchies.
template <>
int schur_setup<MG_REAL>(Ctx &c, LinSys<MG_REAL> &S, bool coarse) {
  using namespace MG_NS;
  const int64_t nn = c.g.nnodes, nnzb = c.nnzb;
  const int d = c.d;
  if (nnzb > S.sub_cap) {
    // the captured graph reads these buffers (B1c, and Aval / Sval through
    // the finest multigrid level): drop it, it is re-captured on next use
    if (S.gexec) cudaGraphExecDestroy(S.gexec);
    S.gexec = nullptr;
    MG_REAL *ptrs[] = {S.Aval, S.Sval, S.B1c, S.W, S.B2c};
    for (MG_REAL *p : ptrs) cudaFree(p);
    S.Aval = S.Sval = S.B1c = S.W = S.B2c = nullptr;
    const int64_t cap = c.nnzb_cap;
    if (cudaMalloc(&S.Aval, sizeof(real) * cap * d * d) || cudaMalloc(&S.Sval, sizeof(real) * cap) ||
        cudaMalloc(&S.B1c, sizeof(real) * cap * d) || cudaMalloc(&S.W, sizeof(real) * cap * d) ||
        (c.schur_lower() && cudaMalloc(&S.B2c, sizeof(real) * cap * d))) {
      S.sub_cap = 0;
      c.last_error = "device allocation of the block preconditioner failed";
      return MPM_ERR_NO_MEMORY;
    }
    S.sub_cap = cap;
  }
  const int nsl = d == 2 ? 49 : 343;
  if (c.fixed_stress()) {
    run_fs_diag(c);
    if (d == 2) {
      k_extract_A<2><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.Aval);
      k_extract_B1<2><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.B1c);
      k_schur_fs<2><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, c.fsd, c.fixed, S.Sval);
    } else {
      k_extract_A<3><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.Aval);
      k_extract_B1<3><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.B1c);
      k_schur_fs<3><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, c.fsd, c.fixed, S.Sval);
    }
    c.launches += 3;
  } else if (d == 2) {
    k_extract_A<2><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.Aval);
    k_extract_B1<2><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.B1c);
    k_diag_inv_A<2><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.Aval, S.val, S.DAinv, S.B1rs);
    k_schur_w<2><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, c.col, S.val, S.DAinv, S.W);
    k_schur_rows<2><<<nblk(nsl * nn), TPB, 0, c.st>>>(c.g.nn[0], c.g.nn[1], nn, c.row_mask, c.row_ptr, c.col,
                                                      S.val, S.W, S.Sval);
    k_schur_lump<2><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.W, S.B1rs, S.Sval);
  } else {
    k_extract_A<3><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.Aval);
    k_extract_B1<3><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.B1c);
    k_diag_inv_A<3><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.Aval, S.val, S.DAinv, S.B1rs);
    k_schur_w<3><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, c.col, S.val, S.DAinv, S.W);
    k_schur_rows<3><<<nblk(nsl * nn), TPB, 0, c.st>>>(c.g.nn[0], c.g.nn[1], nn, c.row_mask, c.row_ptr, c.col,
                                                      S.val, S.W, S.Sval);
    k_schur_lump<3><<<nblk(nn), TPB, 0, c.st>>>(nn, c.row_ptr, c.col, S.val, S.W, S.B1rs, S.Sval);
  }
  if (!c.fixed_stress()) c.launches += 6;
  if (c.schur_lower()) {
    if (d == 2) k_extract_B2<2><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.B2c);
    else k_extract_B2<3><<<nblk(nnzb), TPB, 0, c.st>>>(nnzb, S.val, S.B2c);
    c.launches += 1;
  }
  // the coarse levels and the coarsest inverses: a new Galerkin product, or
  // (coarse = false, after one exists) the product of an earlier set-up kept,
  // the finest levels' values and block-Jacobi inverses refreshed
  const bool full = coarse || !S.coarse_built;
  mg_setup(c, *S.mgA, c.row_ptr, c.col, S.Aval, 0, full);
  mg_setup(c, *S.mgS, c.row_ptr, c.col, S.Sval, d, full);
  if (full) {
    dense_invert_pair(c, *S.mgA, *S.mgS);
    S.coarse_built = true;
    S.coarse_step = c.steps;
  }
  return check_cuda(c, cudaGetLastError(), "schur setup");
}

// z = M^{-1} v (block triangular, multigrid sub-solves) in three parts:
// split (v -> the first sub-solve's rhs and first sweep, and the other
// block's part of v), the multigrid core (first V-cycle, coupling update,
// second V-cycle), merge (-> z).  Upper order: S-cycle, B1 update, A-cycle;
// lower order: A-cycle, B2 update, S-cycle.
namespace MG_NS {
// x0: where the first sub-solve's first sweep goes (its hierarchy's x[0])
void schur_split(Ctx &c, LinSys<MG_REAL> &S, const MG_REAL *v, MG_REAL *x0) {
  const int64_t nn = c.g.nnodes;
  MGHier<real> &HS = *S.mgS, &HA = *S.mgA;
  const Geom g = geom(c, nn);
  const real *dsc = S.dscinv;  // D^-1: the unscaled v is D^-1 times the scaled one
  const real om = mg_omega(c);
  if (c.schur_lower()) {
    const real *dinv = HA.L[0].dinv;
    if (c.d == 2) launch_pdl(c, k_split_lower<2>, g.blocks, g.tpb, 0, nn, v, dsc, HA.b[0], x0, dinv, S.vp, om);
    else launch_pdl(c, k_split_lower<3>, g.blocks, g.tpb, 0, nn, v, dsc, HA.b[0], x0, dinv, S.vp, om);
    return;
  }
  const real *dinv = HS.L[0].dinv;
  if (c.d == 2) launch_pdl(c, k_split<2>, g.blocks, g.tpb, 0, nn, v, dsc, S.vu, HS.b[0], x0, dinv, om);
  else launch_pdl(c, k_split<3>, g.blocks, g.tpb, 0, nn, v, dsc, S.vu, HS.b[0], x0, dinv, om);
}

// x0 of the hierarchy whose V-cycle comes first
MG_REAL *schur_first_x0(Ctx &c, LinSys<MG_REAL> &S) { return c.schur_lower() ? S.mgA->x[0] : S.mgS->x[0]; }

void schur_core(Ctx &c, LinSys<MG_REAL> &S) {
  const int64_t nn = c.g.nnodes;
  MGHier<real> &HS = *S.mgS, &HA = *S.mgA;
  const Geom g = geom(c, nn * B1C_LANES);
  const int32_t *rp = c.row_ptr, *cl = c.col;
  const real om = mg_omega(c);
  if (c.schur_lower()) {
    mg_vcycle(c, HA);
    const real *b2 = S.B2c, *zu = HA.x[0], *vp = S.vp, *dinv = HS.L[0].dinv;
    if (c.d == 2)
      launch_pdl(c, k_b2c_update<2>, g.blocks, g.tpb, 0, nn, rp, cl, b2, zu, vp, HS.b[0], HS.x[0], dinv, om);
    else
      launch_pdl(c, k_b2c_update<3>, g.blocks, g.tpb, 0, nn, rp, cl, b2, zu, vp, HS.b[0], HS.x[0], dinv, om);
    mg_vcycle(c, HS);
    return;
  }
  mg_vcycle(c, HS);
  const real *b1 = S.B1c, *zp = HS.x[0], *vu = S.vu, *dinv = HA.L[0].dinv;
  if (c.d == 2)
    launch_pdl(c, k_b1c_update<2>, g.blocks, g.tpb, 0, nn, rp, cl, b1, zp, vu, HA.b[0], HA.x[0], dinv, om);
  else
    launch_pdl(c, k_b1c_update<3>, g.blocks, g.tpb, 0, nn, rp, cl, b1, zp, vu, HA.b[0], HA.x[0], dinv, om);
  mg_vcycle(c, HA);
}

void schur_merge(Ctx &c, LinSys<MG_REAL> &S, const MG_REAL *zu, const MG_REAL *zp, MG_REAL *z) {
  const int64_t nn = c.g.nnodes;
  const Geom g = geom(c, nn);
  const real *dsc = S.dscinv;  // D^-1: the unscaled v is D^-1 times the scaled one
  if (c.d == 2) launch_pdl(c, k_merge<2>, g.blocks, g.tpb, 0, nn, zu, zp, dsc, z);
  else launch_pdl(c, k_merge<3>, g.blocks, g.tpb, 0, nn, zu, zp, dsc, z);
}
}  // namespace MG_NS

// The multigrid core is a fixed sequence of small kernels on fixed buffers: it
// is captured once into a CUDA graph and replayed between the split and merge
// kernels, which take the caller's v and z.  It is re-captured when a buffer
// it reads moves: the block columns (key below) or the Schur / multigrid
// matrices (schur_setup drops the graph when it reallocates them; a freed and
// reallocated buffer may come back at another address while col does not).
template <>
void schur_apply<MG_REAL>(Ctx &c, LinSys<MG_REAL> &S, const MG_REAL *v, MG_REAL *z) {
  using namespace MG_NS;
  if (!c.capturing && (!S.gexec || S.gkey_col != c.col || S.gkey_val != S.val ||
                       S.g_lower != (int)c.schur_lower())) {
    if (S.gexec) cudaGraphExecDestroy(S.gexec);
    S.gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const int64_t before = c.launches;
    MG_REAL *x0 = schur_first_x0(c, S);
    bool ok = cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      c.capturing = true;
      schur_core(c, S);
      c.capturing = false;
      ok = cudaStreamEndCapture(c.st, &graph) == cudaSuccess && graph;
    }
    if (ok) ok = cudaGraphInstantiate(&S.gexec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    S.gkernels = c.launches - before;
    c.launches = before;
    if (ok) {
      S.g_x0 = x0;
      S.g_lower = (int)c.schur_lower();
      S.g_zp = S.mgS->x[0];
      S.g_zu = S.mgA->x[0];
      S.gkey_col = c.col;
      S.gkey_val = S.val;
    } else {  // capture unavailable: launch directly from now on
      cudaGetLastError();
      S.gexec = nullptr;
    }
  }
  if (S.gexec && !c.capturing) {
    schur_split(c, S, v, S.g_x0);
    cudaGraphLaunch(S.gexec, c.st);
    c.launches += S.gkernels;
    schur_merge(c, S, S.g_zu, S.g_zp, z);
    return;
  }
  schur_split(c, S, v, schur_first_x0(c, S));
  schur_core(c, S);
  schur_merge(c, S, S.mgA->x[0], S.mgS->x[0], z);
}
