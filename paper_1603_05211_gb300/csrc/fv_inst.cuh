// Launchers of the finite-volume stage and CFL kernels for one precision
// (included by fv_f32.cu and fv_f64.cu).
#pragma once
#include "fv.cuh"
#include "fvh.cuh"
#include "launch.h"

namespace mrfv {

template <typename T, int D, int SPLIT>
void launch_fv_shape(const Geo &g, const FVArgs<T> &a, int grid, cudaStream_t st) {
  constexpr size_t sm = fv_smem_bytes<T, D, SPLIT>();
  k_fv<T, D, SPLIT><<<grid, FVShape<T, D, SPLIT>::NT, sm, st>>>(g, a);
}
template <typename T>
void launch_fv(const Geo &g, const FVArgs<T> &a, bool split, int grid, cudaStream_t st) {
  if (g.dim == 2) {
    if (split) launch_fv_shape<T, 2, 2>(g, a, grid, st);
    else launch_fv_shape<T, 2, 1>(g, a, grid, st);
  } else {
    if (split) launch_fv_shape<T, 3, 2>(g, a, grid, st);
    else launch_fv_shape<T, 3, 1>(g, a, grid, st);
  }
}

// Opt in to the dynamic shared memory the pencil kernel needs and report how many
// CTAs fit on one SM (sizes the persistent grid).
template <typename T, int D, int SPLIT>
int fv_occupancy_of() {
  int n = 0;
  constexpr size_t sm = fv_smem_bytes<T, D, SPLIT>();
  cudaFuncSetAttribute(k_fv<T, D, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fv<T, D, SPLIT>, FVShape<T, D, SPLIT>::NT, sm);
  return n > 0 ? n : 1;
}
template <typename T>
int fv_ctas_per_sm(int dim, bool split) {
  if (dim == 2) return split ? fv_occupancy_of<T, 2, 2>() : fv_occupancy_of<T, 2, 1>();
  return split ? fv_occupancy_of<T, 3, 2>() : fv_occupancy_of<T, 3, 1>();
}

// pencil kernel reading primitives staged in shared memory
template <typename T>
void launch_fvp(const Geo &g, const FVArgs<T> &a, int grid, cudaStream_t st) {
  if (g.dim == 2) k_fvp<T, 2><<<grid, FVPShape<T, 2>::NT, fvp_smem_bytes<T, 2>(), st>>>(g, a);
  else k_fvp<T, 3><<<grid, FVPShape<T, 3>::NT, fvp_smem_bytes<T, 3>(), st>>>(g, a);
}
template <typename T, int D>
int fvp_occupancy_of() {
  int n = 0;
  constexpr size_t sm = fvp_smem_bytes<T, D>();
  cudaFuncSetAttribute(k_fvp<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fvp<T, D>, FVPShape<T, D>::NT, sm);
  return n > 0 ? n : 1;
}
template <typename T>
int fvp_ctas_per_sm(int dim) { return dim == 2 ? fvp_occupancy_of<T, 2>() : fvp_occupancy_of<T, 3>(); }
template <typename T>
int fvp_blocks_per_cta(int dim) { return dim == 2 ? FVPShape<T, 2>::BPC : FVPShape<T, 3>::BPC; }

// staged stage kernel (fvh.cuh): the MUSCL-Hancock stage, or the MR-scheme
// stage in the thread-per-face form
template <typename T>
void launch_fvs(const Geo &g, const FVArgs<T> &a, bool hancock, int grid, cudaStream_t st) {
  if (g.dim == 2) {
    if (hancock) k_fvs<T, 2, true><<<grid, FVS<T, 2, true>::NT, fvs_smem_bytes<T, 2, true>(), st>>>(g, a);
    else k_fvs<T, 2, false><<<grid, FVS<T, 2, false>::NT, fvs_smem_bytes<T, 2, false>(), st>>>(g, a);
  } else {
    if (hancock) k_fvs<T, 3, true><<<grid, FVS<T, 3, true>::NT, fvs_smem_bytes<T, 3, true>(), st>>>(g, a);
    else k_fvs<T, 3, false><<<grid, FVS<T, 3, false>::NT, fvs_smem_bytes<T, 3, false>(), st>>>(g, a);
  }
}

template <typename T, int D, bool H>
int fvs_occupancy() {
  int n = 0;
  constexpr size_t sm = fvs_smem_bytes<T, D, H>();
  cudaFuncSetAttribute(k_fvs<T, D, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fvs<T, D, H>, FVS<T, D, H>::NT, sm);
  return n > 0 ? n : 1;
}
// the same for the staged kernel
template <typename T>
int fvs_ctas_per_sm(int dim, bool hancock) {
  if (dim == 2) return hancock ? fvs_occupancy<T, 2, true>() : fvs_occupancy<T, 2, false>();
  return hancock ? fvs_occupancy<T, 3, true>() : fvs_occupancy<T, 3, false>();
}

// blocks one CTA takes per iteration: pencil kernel, or the staged kernel
template <typename T>
int fv_blocks_per_cta(int dim, bool staged) {
  if (staged) return dim == 2 ? FVS<T, 2, true>::BPC : FVS<T, 3, true>::BPC;
  return dim == 2 ? FVShape<T, 2>::BPC : FVShape<T, 3>::BPC;
}

template <typename T>
void launch_dt(const Geo &g, const T *A, int lts, unsigned long long *red, unsigned *done, double cfl, double t_end,
               double *dsc, double *lev, float *levf, int grid, cudaStream_t st) {
  // red (a huge positive double) and done are set at context creation and reset
  // by the reduction's last CTA
  if (g.dim == 2) k_dt<T, 2><<<grid, 256, 0, st>>>(g, A, lts, red, done, cfl, t_end, dsc, lev, levf);
  else k_dt<T, 3><<<grid, 256, 0, st>>>(g, A, lts, red, done, cfl, t_end, dsc, lev, levf);
}

#define MRFV_INSTANTIATE_FV(T)                                                                  \
  template void launch_fv<T>(const Geo &, const FVArgs<T> &, bool, int, cudaStream_t);          \
  template int fv_ctas_per_sm<T>(int, bool);                                                    \
  template void launch_fvs<T>(const Geo &, const FVArgs<T> &, bool, int, cudaStream_t);         \
  template void launch_fvp<T>(const Geo &, const FVArgs<T> &, int, cudaStream_t);               \
  template int fvp_ctas_per_sm<T>(int);                                                         \
  template int fvp_blocks_per_cta<T>(int);                                                      \
  template int fvs_ctas_per_sm<T>(int, bool);                                                   \
  template int fv_blocks_per_cta<T>(int, bool);                                                 \
  template void launch_dt<T>(const Geo &, const T *, int, unsigned long long *, unsigned *, double, double, double *, \
                             double *, float *, int, cudaStream_t);

}  // namespace mrfv
