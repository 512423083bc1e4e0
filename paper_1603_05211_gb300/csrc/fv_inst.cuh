// Launchers of the finite-volume stage and CFL kernels for one precision
// (included by fv_f32.cu and fv_f64.cu).
#pragma once
#include "fv.cuh"
#include "fvh.cuh"
#include "launch.h"

namespace mrfv {

template <typename T>
void launch_fv(const Geo &g, const FVArgs<T> &a, int grid, cudaStream_t st) {
  if (g.dim == 2) {
    constexpr size_t sm = fv_smem_bytes<T, 2>();
    k_fv<T, 2><<<grid, FVShape<T, 2>::NT, sm, st>>>(g, a);
  } else {
    constexpr size_t sm = fv_smem_bytes<T, 3>();
    k_fv<T, 3><<<grid, FVShape<T, 3>::NT, sm, st>>>(g, a);
  }
}

// Opt in to the dynamic shared memory the stage kernel needs and report how
// many CTAs fit on one SM (sizes the persistent grid).
template <typename T>
int fv_ctas_per_sm(int dim) {
  int n = 0;
  if (dim == 2) {
    constexpr size_t sm = fv_smem_bytes<T, 2>();
    cudaFuncSetAttribute(k_fv<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fv<T, 2>, FVShape<T, 2>::NT, sm);
  } else {
    constexpr size_t sm = fv_smem_bytes<T, 3>();
    cudaFuncSetAttribute(k_fv<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fv<T, 3>, FVShape<T, 3>::NT, sm);
  }
  return n > 0 ? n : 1;
}

template <typename T>
void launch_fvh(const Geo &g, const FVArgs<T> &a, int grid, cudaStream_t st) {
  if (g.dim == 2) k_fvh<T, 2><<<grid, FVH<T, 2>::NT, fvh_smem_bytes<T, 2>(), st>>>(g, a);
  else k_fvh<T, 3><<<grid, FVH<T, 3>::NT, fvh_smem_bytes<T, 3>(), st>>>(g, a);
}

// the same for the MUSCL-Hancock stage kernel
template <typename T>
int fvh_ctas_per_sm(int dim) {
  int n = 0;
  if (dim == 2) {
    constexpr size_t sm = fvh_smem_bytes<T, 2>();
    cudaFuncSetAttribute(k_fvh<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fvh<T, 2>, FVH<T, 2>::NT, sm);
  } else {
    constexpr size_t sm = fvh_smem_bytes<T, 3>();
    cudaFuncSetAttribute(k_fvh<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fvh<T, 3>, FVH<T, 3>::NT, sm);
  }
  return n > 0 ? n : 1;
}

template <typename T>
void launch_dt(const Geo &g, const T *A, int lts, unsigned long long *red, unsigned *done, double cfl, double t_end,
               double *dsc, double *lev, float *levf, int grid, cudaStream_t st) {
  cudaMemsetAsync(red, 0x7f, sizeof(unsigned long long), st);  // a huge positive double
  cudaMemsetAsync(done, 0, sizeof(unsigned), st);
  if (g.dim == 2) k_dt<T, 2><<<grid, 256, 0, st>>>(g, A, lts, red, done, cfl, t_end, dsc, lev, levf);
  else k_dt<T, 3><<<grid, 256, 0, st>>>(g, A, lts, red, done, cfl, t_end, dsc, lev, levf);
}

#define MRFV_INSTANTIATE_FV(T)                                                                  \
  template void launch_fv<T>(const Geo &, const FVArgs<T> &, int, cudaStream_t);                \
  template int fv_ctas_per_sm<T>(int);                                                          \
  template void launch_fvh<T>(const Geo &, const FVArgs<T> &, int, cudaStream_t);               \
  template int fvh_ctas_per_sm<T>(int);                                                         \
  template void launch_dt<T>(const Geo &, const T *, int, unsigned long long *, unsigned *, double, double, double *, \
                             double *, float *, int, cudaStream_t);

}  // namespace mrfv
