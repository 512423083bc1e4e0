// Allocation-free CFL time step (mrfv_cfl_dt_noalloc): the reduction of
// k_dt (with its last-CTA finalisation) over a caller-owned dense array of cells, with its scratch
// in a file-scope device array instead of the context arena.
//
// Some callers cannot allocate device memory: code that issues its work while a
// CUDA stream is being captured into a graph (cudaMalloc is not allowed there),
// host frameworks that own every byte of device memory through their own pool,
// and latency-critical loops that cannot afford cudaMalloc's implicit device
// synchronisation.  This entry point allocates nothing: the caller passes the
// state and the output, and the per-tile partial minima live in g_dt_partial,
// which every GPU that loads this library keeps until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "mrfv.h"

namespace {

constexpr int kTileCells = MRFV_NOALLOC_DT_TILE_CELLS;
constexpr int kMaxTiles = MRFV_NOALLOC_DT_MAX_TILES;
constexpr int kThreads = 256;

// one partial minimum per tile of kTileCells cells; -1 marks a tile with a
// non-physical cell.  Every tile the second pass reads is written by the first
// pass of the same call, so nothing has to start at zero.
static __device__ __align__(256) double g_dt_partial[kMaxTiles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_partial_ptr[kMaxDevices] = {nullptr};

template <typename T, int D>
__global__ void k_dt_tiles(const T *__restrict__ U, long long ncell, double dx0, double dx1, double dx2,
                           double gamma, double *partial) {
  __shared__ T wmin[kThreads / 32];
  __shared__ int wbad[kThreads / 32];
  const T gam = T(gamma), gm1 = T(gamma - 1.0);
  const T dx[3] = {T(dx0), T(dx1), T(dx2)};
  const long long t0 = (long long)blockIdx.x * kTileCells;
  T best = T(INFINITY);
  int bad = 0;
  for (int k = threadIdx.x; k < kTileCells; k += kThreads) {
    long long c = t0 + k;
    if (c >= ncell) break;
    T rho = U[c];
    T v[3] = {T(0), T(0), T(0)};
    for (int d = 0; d < D; d++) v[d] = U[(long long)(1 + d) * ncell + c] / rho;
    T vv = (v[0] * v[0]) + (v[1] * v[1]);
    if (D == 3) vv = vv + (v[2] * v[2]);
    T p = gm1 * (U[(long long)(D + 1) * ncell + c] - ((T(0.5) * rho) * vv));
    if (!(rho > T(0)) || !(p > T(0))) {
      bad = 1;
      continue;
    }
    T cs = sqrt((gam * p) / rho);
    for (int d = 0; d < D; d++) {
      T r = dx[d] / (fabs(v[d]) + cs);
      if (r < best) best = r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(0xffffffffu, best, o);
    if (x < best) best = x;
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    wmin[threadIdx.x >> 5] = best;
    wbad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T m = wmin[0];
    int b = wbad[0];
    for (int w = 1; w < kThreads / 32; w++) {
      if (wmin[w] < m) m = wmin[w];
      b |= wbad[w];
    }
    partial[blockIdx.x] = b ? -1.0 : (double)m;
  }
}

__global__ void k_dt_tiles_final(const double *partial, int ntiles, double cfl, double *dt_out) {
  __shared__ double wmin[kThreads / 32];
  __shared__ int wbad[kThreads / 32];
  double best = INFINITY;
  int bad = 0;
  for (int i = threadIdx.x; i < ntiles; i += kThreads) {
    double x = partial[i];
    if (x < 0.0) bad = 1;
    else if (x < best) best = x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    double x = __shfl_xor_sync(0xffffffffu, best, o);
    if (x < best) best = x;
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    wmin[threadIdx.x >> 5] = best;
    wbad[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = wmin[0];
    int b = wbad[0];
    for (int w = 1; w < kThreads / 32; w++) {
      if (wmin[w] < m) m = wmin[w];
      b |= wbad[w];
    }
    *dt_out = b ? -1.0 : cfl * m;
  }
}

// Device address of g_dt_partial for the current device, looked up once per
// device (the array's name is only a host-side stand-in in host code).  The
// cached address belongs to the device's primary context: it does not survive
// cudaDeviceReset (or any other teardown of that context) in this process.
int partial_for_current_device(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MRFV_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dt_partial) != cudaSuccess || !p) {
      cudaGetLastError();
      return MRFV_ERR_CUDA;
    }
    g_partial_ptr[dev] = (double *)p;
  }
  *out = g_partial_ptr[dev];
  return MRFV_OK;
}

}  // namespace

extern "C" int mrfv_cfl_dt_noalloc(int dim, int precision, const void *state, int64_t n0, int64_t n1, int64_t n2,
                                   const double *dx, double gamma, double cfl, double *dt_out, void *stream) {
  if ((dim != 2 && dim != 3) || (precision != MRFV_FP32 && precision != MRFV_FP64) || !state || !dx || !dt_out)
    return MRFV_ERR_ARG;
  if (n0 < 1 || n1 < 1 || n2 < 1 || (dim == 2 && n2 != 1) || !(gamma > 1.0) || !(cfl > 0.0)) return MRFV_ERR_ARG;
  // the cell count, checked against the maximum before each multiply (no overflow)
  const int64_t maxc = MRFV_NOALLOC_DT_MAX_CELLS;
  if (n0 > maxc || n1 > maxc || n2 > maxc) return MRFV_ERR_ARG;
  if (n1 > maxc / n0) return MRFV_ERR_ARG;
  long long ncell = (long long)n0 * n1;
  if (n2 > maxc / ncell) return MRFV_ERR_ARG;
  ncell *= n2;
  long long ntiles = (ncell + kTileCells - 1) / kTileCells;
  if (ntiles > kMaxTiles) return MRFV_ERR_ARG;  // more than MRFV_NOALLOC_DT_MAX_CELLS cells
  double *partial = nullptr;
  int rc = partial_for_current_device(&partial);
  if (rc != MRFV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int nt = (int)ntiles;
  if (precision == MRFV_FP64) {
    if (dim == 2) k_dt_tiles<double, 2><<<nt, kThreads, 0, st>>>((const double *)state, ncell, dx[0], dx[1], dx[2], gamma, partial);
    else k_dt_tiles<double, 3><<<nt, kThreads, 0, st>>>((const double *)state, ncell, dx[0], dx[1], dx[2], gamma, partial);
  } else {
    if (dim == 2) k_dt_tiles<float, 2><<<nt, kThreads, 0, st>>>((const float *)state, ncell, dx[0], dx[1], dx[2], gamma, partial);
    else k_dt_tiles<float, 3><<<nt, kThreads, 0, st>>>((const float *)state, ncell, dx[0], dx[1], dx[2], gamma, partial);
  }
  k_dt_tiles_final<<<1, kThreads, 0, st>>>(partial, nt, cfl, dt_out);
  if (cudaGetLastError() != cudaSuccess) return MRFV_ERR_CUDA;
  return MRFV_OK;
}
