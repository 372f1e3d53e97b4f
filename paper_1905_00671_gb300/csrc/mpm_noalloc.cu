// mpm_noalloc.cu -- mpm_bin_noalloc: the cell binning and (cell, index)
// ordering of material points, for callers that cannot allocate device memory.
//
// Who needs it: code that may not call cudaMalloc at the point where it bins
// points -- for example a solver embedded in a host application that owns all
// device memory through its own pool and gives libraries no allocator, or a
// latency-critical loop where the implicit device synchronisation of
// cudaMalloc / cudaFree is not acceptable.  The caller passes the positions and
// the two output arrays; the per-cell counters live in the fixed array below.
//
// The scratch array is a file-scope __device__ variable: every GPU that loads
// this library holds it (about 3 MiB) until the process exits, and every call
// on that GPU shares it.  Host code cannot use the array's name as a device
// address; the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and keeps it.  Because that
// first call does this set-up (and synchronises), it should be made before any
// stream capture.  Every call, not only the first, copies an error word to the
// host and waits for its stream before it returns.  The counters a call needs
// at zero are cleared by the call; two calls that overlap on the GPU
// (different streams, or host threads that do not order them) race on the
// shared array and give wrong results.
#include <math.h>
#include <string.h>

#include <atomic>

#include "mpm_internal.cuh"

namespace upmpm {
namespace {

constexpr int64_t NOALLOC_MAX_CELLS = 1 << 18;   // 262,144 cells
constexpr int NOALLOC_MAX_DEVICES = 64;
// layout: [0, C] counts, [C+1, 2C+1] cell starts, [2C+2, 3C+2] cursors, then
// the error word
constexpr int64_t NOALLOC_INTS = 3 * (NOALLOC_MAX_CELLS + 1) + 64;

static __device__ __align__(256) int32_t g_noalloc_scratch[NOALLOC_INTS];

std::atomic<int32_t *> g_scratch_ptr[NOALLOC_MAX_DEVICES];

int scratch_for_current_device(int32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MPM_ERR_CUDA;
  int32_t *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void *addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return MPM_ERR_CUDA;
    p = static_cast<int32_t *>(addr);
    g_scratch_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return MPM_OK;
}

template <int D>
__global__ void k_na_keys(GridP g, int64_t n, const double *__restrict__ x, int32_t *__restrict__ cell,
                          int32_t *__restrict__ count, int32_t *__restrict__ err) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  int c[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    const double cf = floor(__ddiv_rn(__dsub_rn(x[p * D + k], g.org[k]), g.h));
    if (!(cf >= 0.0) || !(cf <= (double)(g.nc[k] - 1))) {
      atomicOr(err, 1);
      cell[p] = -1;
      return;
    }
    c[k] = (int)cf;
  }
  const int32_t id = (int32_t)cell_index(g, c[0], c[1], c[2]);
  cell[p] = id;
  atomicAdd(&count[id], 1);
}

// exclusive scan of count[0..m) into start[0..m] by one block of 1024 threads
__global__ void k_na_scan(const int32_t *__restrict__ count, int64_t m, int32_t *__restrict__ start) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (m + 1023) / 1024;
  const int64_t b = t * chunk, e = b + chunk < m ? b + chunk : m;
  int32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += count[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int32_t v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = t > 0 ? part[t - 1] : 0;
  for (int64_t i = b; i < e; ++i) {
    start[i] = run;
    run += count[i];
  }
  if (t == 1023) start[m] = part[1023];
}

__global__ void k_na_scatter(int64_t n, const int32_t *__restrict__ cell, const int32_t *__restrict__ start,
                             int32_t *__restrict__ cursor, int64_t *__restrict__ order) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t c = cell[p];
  if (c < 0) return;
  order[start[c] + atomicAdd(&cursor[c], 1)] = p;
}

__global__ void k_na_sort(int64_t ncells, const int32_t *__restrict__ start, int64_t *__restrict__ order) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int32_t b = start[c], e = start[c + 1];
  for (int32_t i = b + 1; i < e; ++i) {
    const int64_t v = order[i];
    int32_t j = i - 1;
    while (j >= b && order[j] > v) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = v;
  }
}

}  // namespace
}  // namespace upmpm

using namespace upmpm;

extern "C" int mpm_bin_noalloc(const mpm_grid *grid, int64_t n, const double *x_dev,
                               int32_t *cell_dev, int64_t *order_dev, void *stream) {
  if (!grid || n < 0 || (n > 0 && (!x_dev || !cell_dev || !order_dev))) return MPM_ERR_BAD_ARG;
  if (grid->dim != 2 && grid->dim != 3) return MPM_ERR_BAD_ARG;
  if (!(grid->h > 0.0) || n > INT32_MAX) return MPM_ERR_BAD_ARG;
  // Each axis is bounded before the product is formed, so the product of at
  // most three factors <= 2^18 cannot overflow int64 and a grid whose cell
  // count would wrap is rejected rather than indexed.  Only the cell fields
  // of GridP are used here.
  GridP g{};
  g.d = grid->dim;
  g.ncells = 1;
  for (int k = 0; k < 3; ++k) {
    const bool used = k < g.d;
    if (used && grid->ncell[k] < 1) return MPM_ERR_BAD_ARG;
    if (used && grid->ncell[k] > NOALLOC_MAX_CELLS) return MPM_ERR_TOO_LARGE;
    g.nc[k] = used ? grid->ncell[k] : 1;
    g.org[k] = used ? grid->origin[k] : 0.0;
    g.ncells *= g.nc[k];
  }
  g.h = grid->h;
  if (g.ncells > NOALLOC_MAX_CELLS) return MPM_ERR_TOO_LARGE;
  int32_t *scr = nullptr;
  int rc = scratch_for_current_device(&scr);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t C = g.ncells;
  int32_t *count = scr, *start = scr + (C + 1), *cursor = scr + 2 * (C + 1);
  int32_t *err = scr + 3 * (NOALLOC_MAX_CELLS + 1);
  // everything this call reads before writing starts at zero
  if (cudaMemsetAsync(count, 0, sizeof(int32_t) * (C + 1), st) != cudaSuccess ||
      cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (C + 1), st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int32_t), st) != cudaSuccess)
    return MPM_ERR_CUDA;
  if (n > 0) {
    const int nbk = (int)((n + 255) / 256);
    if (g.d == 2) k_na_keys<2><<<nbk, 256, 0, st>>>(g, n, x_dev, cell_dev, count, err);
    else k_na_keys<3><<<nbk, 256, 0, st>>>(g, n, x_dev, cell_dev, count, err);
  }
  int32_t herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MPM_ERR_CUDA;
  if (herr) return MPM_ERR_OUT_OF_GRID;
  if (n == 0) return MPM_OK;
  k_na_scan<<<1, 1024, 0, st>>>(count, C, start);
  k_na_scatter<<<(int)((n + 255) / 256), 256, 0, st>>>(n, cell_dev, start, cursor, order_dev);
  k_na_sort<<<(int)((C + 255) / 256), 256, 0, st>>>(C, start, order_dev);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return MPM_ERR_CUDA;
  return MPM_OK;
}
