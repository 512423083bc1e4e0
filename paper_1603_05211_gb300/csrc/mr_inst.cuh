// Launchers of the multiresolution kernels for one precision (included by
// mr_f32.cu and mr_f64.cu, which are compiled without FMA contraction so the
// prediction, details and projection round exactly as written).
#pragma once
#include "launch.h"
#include "mr.cuh"
#include "rich.cuh"

namespace mrfv {

template <typename T>
void launch_restrict(const Geo &g, int l, T *A, int grid, cudaStream_t st) {
  if (g.dim == 2) k_restrict<T, 2><<<grid, 256, 0, st>>>(g, l, A);
  else k_restrict<T, 3><<<grid, 512, 0, st>>>(g, l, A);
}
template <typename T>
void launch_restrict_pos(const Geo &g, int l, T *A, int grid, cudaStream_t st) {
  if (g.dim == 2) k_restrict_pos<T, 2><<<grid, 256, 0, st>>>(g, l, A);
  else k_restrict_pos<T, 3><<<grid, 512, 0, st>>>(g, l, A);
}
template <typename T>
void launch_reflux_restrict(const Geo &g, T *A, const T *FR, int nr, int np, cudaStream_t st) {
  if (g.dim == 2) k_reflux_restrict<T, 2><<<nr + np, 256, 0, st>>>(g, nr, A, FR);
  else k_reflux_restrict<T, 3><<<nr + np, 512, 0, st>>>(g, nr, A, FR);
}
template <typename T>
void launch_restrict_tail(const Geo &g, int lhi, T *A, cudaStream_t st) {
  if (g.dim == 2) k_restrict_tail<T, 2><<<1, kTailThreads, 0, st>>>(g, lhi, A);
  else k_restrict_tail<T, 3><<<1, kTailThreads, 0, st>>>(g, lhi, A);
}
template <typename T>
void launch_prolong_tail(const Geo &g, int lhi, const int32_t *newlist, const int *nnew, T *A, cudaStream_t st) {
  if (g.dim == 2) k_prolong_tail<T, 2><<<1, 64, 0, st>>>(g, lhi, newlist, nnew, A);
  else k_prolong_tail<T, 3><<<1, 512, 0, st>>>(g, lhi, newlist, nnew, A);
}
template <typename T>
void launch_ghost_edge(const Geo &g, T *A, T *G, int ng, int ne, cudaStream_t st) {
  if (g.dim == 2) k_ghost_edge<T, 2><<<ng + ne, 64, 4 * 64 * sizeof(T), st>>>(g, ng, A, G);
  else k_ghost_edge<T, 3><<<ng + ne, 256, 5 * 512 * sizeof(T), st>>>(g, ng, A, G);
}
template <typename T>
void launch_gather_var(const Geo &g, int l, int v, int f, const T *A, double *out, cudaStream_t st) {
  if (g.dim == 2) k_gather_var<T, 2><<<1024, 256, 0, st>>>(g, l, v, f, A, out);
  else k_gather_var<T, 3><<<1024, 256, 0, st>>>(g, l, v, f, A, out);
}
template <typename T>
void launch_scales(const Geo &g, const T *A, unsigned long long *red, unsigned *done, T *scale, int grid,
                   cudaStream_t st) {
  if (g.dim == 2) {
    k_scale_max<T, 2><<<grid, 256, 0, st>>>(g, A, red, done, scale);
  } else {
    k_scale_max<T, 3><<<grid, 256, 0, st>>>(g, A, red, done, scale);
  }
}
template <typename T>
void launch_details(const Geo &g, const T *A, const T *scale, double eps, uint8_t *sig, double *maxdet, int l0,
                    const T *A0, double theta, int grid, cudaStream_t st, T *own_scale, uint8_t *need) {
  if (g.dim == 2)
    k_details<T, 2><<<grid, 64, 0, st>>>(g, A, scale, T(eps), sig, maxdet, l0, A0, T(theta), own_scale, need);
  else
    k_details<T, 3><<<grid, 512, 0, st>>>(g, A, scale, T(eps), sig, maxdet, l0, A0, T(theta), own_scale, need);
}
template <typename T>
void launch_prolong(const Geo &g, int l, const int32_t *newlist, const int *nnew, T *A, int grid, cudaStream_t st) {
  if (g.dim == 2) k_prolong<T, 2><<<grid, 64, 0, st>>>(g, l, newlist, nnew, A);
  else k_prolong<T, 3><<<grid, 512, 0, st>>>(g, l, newlist, nnew, A);
}
template <typename T>
void launch_ghost(const Geo &g, int l0, int l1, const T *A, const T *A0, double theta, T *G, int grid,
                  cudaStream_t st) {
  if (g.dim == 2) k_ghost<T, 2><<<grid, 64, 4 * 64 * sizeof(T), st>>>(g, l0, l1, A, A0, T(theta), G);
  else k_ghost<T, 3><<<grid, 256, 5 * 512 * sizeof(T), st>>>(g, l0, l1, A, A0, T(theta), G);
}
template <typename T>
void launch_init(const Geo &g, const ICParams &ic, const double *hi, T *A, int grid, cudaStream_t st) {
  if (g.dim == 2) k_init<T, 2><<<grid, 256, 0, st>>>(g, ic, hi[0], hi[1], hi[2], A);
  else k_init<T, 3><<<grid, 256, 0, st>>>(g, ic, hi[0], hi[1], hi[2], A);
}
template <typename T>
void launch_gather(const Geo &g, int l, const T *A, double *out, cudaStream_t st) {
  if (g.dim == 2) k_gather_level<T, 2><<<1024, 256, 0, st>>>(g, l, A, out);
  else k_gather_level<T, 3><<<1024, 256, 0, st>>>(g, l, A, out);
}
template <typename T>
void launch_scatter(const Geo &g, int l, const double *in, T *A, cudaStream_t st) {
  if (g.dim == 2) k_scatter_level<T, 2><<<1024, 256, 0, st>>>(g, l, in, A);
  else k_scatter_level<T, 3><<<1024, 256, 0, st>>>(g, l, in, A);
}
template <typename T>
void launch_totals(const Geo &g, const T *A, double *out, int grid, cudaStream_t st) {
  cudaMemsetAsync(out, 0, 5 * sizeof(double), st);
  if (g.dim == 2) k_totals<T, 2><<<grid, 256, 0, st>>>(g, A, out);
  else k_totals<T, 3><<<grid, 256, 0, st>>>(g, A, out);
}
template <typename T>
void launch_reflux(const Geo &g, int l0, int l1, T *A, const T *FR, int grid, cudaStream_t st) {
  if (g.dim == 2) k_reflux<T, 2><<<grid, 256, 0, st>>>(g, l0, l1, A, FR);
  else k_reflux<T, 3><<<grid, 256, 0, st>>>(g, l0, l1, A, FR);
}
template <typename T>
void launch_copy_level(const Geo &g, int kind, int l0, int l1, const T *src, T *dst, int grid, cudaStream_t st) {
  if (g.dim == 2) k_copy_level<T, 2><<<grid, 256, 0, st>>>(g, kind, l0, l1, src, dst);
  else k_copy_level<T, 3><<<grid, 256, 0, st>>>(g, kind, l0, l1, src, dst);
}
template <typename T>
void launch_gradflags(const Geo &g, const T *A, double epsw, double epsp, uint8_t *gflag, int l0, const T *A0,
                      double theta, int grid, cudaStream_t st) {
  if (g.dim == 2) k_gradflags<T, 2><<<grid, 128, 0, st>>>(g, A, T(epsw), T(epsp), gflag, l0, A0, T(theta));
  else k_gradflags<T, 3><<<grid, 256, 0, st>>>(g, A, T(epsw), T(epsp), gflag, l0, A0, T(theta));
}

template <typename T>
void launch_rich(const Geo &g, int hancock, const T *A, const T *A0, double theta, int l0, const double *lev,
                 double eps_r, unsigned long long *rmask, double *maxdet, uint8_t *gflag, T *scratch, int ctas,
                 int grid, unsigned long long *nblk, cudaStream_t st) {
  const T th = T(theta);
  if (g.dim == 2) {
    constexpr size_t sh = RichShape<2, true>::PER * sizeof(T), sm = RichShape<2, false>::PER * sizeof(T);
    if (hancock)
      k_rich<T, 2, true><<<ctas, RichShape<2, true>::NT, sh, st>>>(g, A, A0, th, l0, lev, eps_r, rmask, maxdet, scratch, nblk);
    else
      k_rich<T, 2, false><<<ctas, RichShape<2, false>::NT, sm, st>>>(g, A, A0, th, l0, lev, eps_r, rmask, maxdet, scratch, nblk);
    k_rich_flags<2><<<grid, 256, 0, st>>>(g, l0, rmask, gflag);
  } else {
    if (hancock)
      k_rich<T, 3, true><<<ctas, RichShape<3, true>::NT, 0, st>>>(g, A, A0, th, l0, lev, eps_r, rmask, maxdet, scratch, nblk);
    else
      k_rich<T, 3, false><<<ctas, RichShape<3, false>::NT, 0, st>>>(g, A, A0, th, l0, lev, eps_r, rmask, maxdet, scratch, nblk);
    k_rich_flags<3><<<grid, 256, 0, st>>>(g, l0, rmask, gflag);
  }
}
// global scratch per CTA (2D patches live in shared memory: none)
template <typename T>
long long rich_scratch_bytes(int dim, int hancock) {
  if (dim == 2) return 0;
  return (hancock ? RichShape<3, true>::PER : RichShape<3, false>::PER) * (long long)sizeof(T);
}
// the 2D estimate's dynamic shared memory above the default limit (once, before
// any graph capture); *per_sm = CTAs of the scheme's 2D kernel one SM holds with
// that shared memory (0 in 3D, whose patches live in global scratch)
template <typename T>
cudaError_t prepare_rich(int dim, int hancock, int *per_sm) {
  *per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(k_rich<T, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(RichShape<2, true>::PER * sizeof(T)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_rich<T, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(RichShape<2, false>::PER * sizeof(T)));
  if (e != cudaSuccess || dim != 2) return e;
  if (hancock)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_rich<T, 2, true>, RichShape<2, true>::NT,
                                                      RichShape<2, true>::PER * sizeof(T));
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_rich<T, 2, false>, RichShape<2, false>::NT,
                                                      RichShape<2, false>::PER * sizeof(T));
  return e;
}

template <typename T>
void launch_project_level(const Geo &g, int l, const T *A, const double *coarse, double *out, cudaStream_t st) {
  if (g.dim == 2) k_project_level<T, 2><<<1024, 256, 0, st>>>(g, l, A, coarse, out);
  else k_project_level<T, 3><<<1024, 256, 0, st>>>(g, l, A, coarse, out);
}

#define MRFV_INSTANTIATE_MR(T)                                                                              \
  template void launch_restrict<T>(const Geo &, int, T *, int, cudaStream_t);                               \
  template void launch_ghost_edge<T>(const Geo &, T *, T *, int, int, cudaStream_t);                       \
  template void launch_restrict_pos<T>(const Geo &, int, T *, int, cudaStream_t);                           \
  template void launch_restrict_tail<T>(const Geo &, int, T *, cudaStream_t);                               \
  template void launch_reflux_restrict<T>(const Geo &, T *, const T *, int, int, cudaStream_t);            \
  template void launch_prolong_tail<T>(const Geo &, int, const int32_t *, const int *, T *, cudaStream_t);  \
  template void launch_scales<T>(const Geo &, const T *, unsigned long long *, unsigned *, T *, int, cudaStream_t); \
  template void launch_details<T>(const Geo &, const T *, const T *, double, uint8_t *, double *, int,      \
                                  const T *, double, int, cudaStream_t, T *, uint8_t *);                    \
  template void launch_prolong<T>(const Geo &, int, const int32_t *, const int *, T *, int, cudaStream_t);  \
  template void launch_ghost<T>(const Geo &, int, int, const T *, const T *, double, T *, int, cudaStream_t); \
  template void launch_init<T>(const Geo &, const ICParams &, const double *, T *, int, cudaStream_t);      \
  template void launch_gather<T>(const Geo &, int, const T *, double *, cudaStream_t);                      \
  template void launch_scatter<T>(const Geo &, int, const double *, T *, cudaStream_t);                     \
  template void launch_totals<T>(const Geo &, const T *, double *, int, cudaStream_t);                      \
  template void launch_reflux<T>(const Geo &, int, int, T *, const T *, int, cudaStream_t);                 \
  template void launch_gather_var<T>(const Geo &, int, int, int, const T *, double *, cudaStream_t);        \
  template void launch_copy_level<T>(const Geo &, int, int, int, const T *, T *, int, cudaStream_t);                  \
  template void launch_gradflags<T>(const Geo &, const T *, double, double, uint8_t *, int, const T *, double, int, \
                                    cudaStream_t);         \
  template void launch_project_level<T>(const Geo &, int, const T *, const double *, double *, cudaStream_t); \
  template void launch_rich<T>(const Geo &, int, const T *, const T *, double, int, const double *, double,     \
                               unsigned long long *, double *, uint8_t *, T *, int, int, unsigned long long *, \
                               cudaStream_t);                                                                   \
  template long long rich_scratch_bytes<T>(int, int);                                                      \
  template cudaError_t prepare_rich<T>(int, int, int *);

}  // namespace mrfv
