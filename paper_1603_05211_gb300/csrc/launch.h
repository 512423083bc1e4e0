// Host-side launchers of the kernels (one definition per precision, see the
// *_f32.cu / *_f64.cu translation units).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "common.h"

namespace mrfv {

// multiresolution / bookkeeping kernels (mr_f32.cu, mr_f64.cu)
template <typename T> void launch_restrict(const Geo &, int l, T *A, int grid, cudaStream_t);
// the same as a sweep of the dense maps of level l (levels with few positions)
template <typename T> void launch_restrict_pos(const Geo &, int l, T *A, int grid, cudaStream_t);
// threads of the single-CTA kernels that take several coarse levels in one launch
constexpr int kTailThreads = 1024;
// flux correction of levels 0..L-1 on nr CTAs and projection of level L-1 (list
// form) on np CTAs, in one launch
template <typename T> void launch_reflux_restrict(const Geo &, T *A, const T *FR, int nr, int np, cudaStream_t);
// levels lhi..0 in one single-CTA launch (levels whose positions one CTA covers)
template <typename T> void launch_restrict_tail(const Geo &, int lhi, T *A, cudaStream_t);
// new blocks of levels 1..lhi in one single-CTA launch
template <typename T> void launch_prolong_tail(const Geo &, int lhi, const int32_t *newlist, const int *nnew, T *A,
                                               cudaStream_t);
// between the stages of the MR step: the ghost strips of every level (ng CTAs, the
// coarse cells over refined blocks projected on the fly) and the projection of
// restrict_edge_dev (ne CTAs: the parent quadrants of the leaves next to an absent
// block, all levels) in one launch
template <typename T> void launch_ghost_edge(const Geo &, T *A, T *G, int ng, int ne, cudaStream_t);
template <typename T> void launch_scales(const Geo &, const T *A, unsigned long long *red, unsigned *done, T *scale,
                                         int grid, cudaStream_t);
// own_scale (optional): every CTA computes the level-0 normalisation itself and CTA
// 0 stores it there (no k_scale_max before); need (optional): the MR criterion's
// needed-block marks made here (no k_need_mark after)
template <typename T> void launch_details(const Geo &, const T *A, const T *scale, double eps, uint8_t *sig, double *maxdet,
                                         int l0, const T *A0, double theta, int grid, cudaStream_t,
                                         T *own_scale = nullptr, uint8_t *need = nullptr);
template <typename T> void launch_prolong(const Geo &, int l, const int32_t *newlist, const int *nnew, T *A, int grid, cudaStream_t);
template <typename T> void launch_ghost(const Geo &, int l0, int l1, const T *A, const T *A0, double theta, T *G, int grid, cudaStream_t);
template <typename T> void launch_init(const Geo &, const ICParams &, const double *hi, T *A, int grid, cudaStream_t);
template <typename T> void launch_gather(const Geo &, int l, const T *A, double *out, cudaStream_t);
template <typename T> void launch_gather_var(const Geo &, int l, int v, int f, const T *A, double *out, cudaStream_t);
template <typename T> void launch_scatter(const Geo &, int l, const double *in, T *A, cudaStream_t);
template <typename T> void launch_totals(const Geo &, const T *A, double *out, int grid, cudaStream_t);
template <typename T> void launch_reflux(const Geo &, int l0, int l1, T *A, const T *FR, int grid, cudaStream_t);
template <typename T> void launch_copy_level(const Geo &, int kind, int l0, int l1, const T *src, T *dst, int grid,
                                             cudaStream_t);
template <typename T> void launch_gradflags(const Geo &, const T *A, double epsw, double epsp, uint8_t *gflag, int l0,
                                           const T *A0, double theta, int grid, cudaStream_t);
// Richardson estimate of levels l0..L-1 (ctas CTAs, each with rich_scratch_bytes
// of scratch), then gflag |= its block flags; nblk (optional) += blocks estimated
template <typename T> void launch_rich(const Geo &, int hancock, const T *A, const T *A0, double theta, int l0,
                                       const double *lev, double eps_r, unsigned long long *rmask, double *maxdet,
                                       uint8_t *gflag, T *scratch, int ctas, int grid, unsigned long long *nblk,
                                       cudaStream_t);
template <typename T> long long rich_scratch_bytes(int dim, int hancock);
template <typename T> cudaError_t prepare_rich(int dim, int hancock, int *per_sm);
template <typename T> void launch_project_level(const Geo &, int l, const T *A, const double *coarse, double *out, cudaStream_t);
// finite-volume stage and CFL reduction (fv_f32.cu, fv_f64.cu)
template <typename T> void launch_fv(const Geo &, const FVArgs<T> &, bool split, int grid, cudaStream_t);
template <typename T> void launch_fvs(const Geo &, const FVArgs<T> &, bool hancock, int grid, cudaStream_t);
template <typename T> int fvs_ctas_per_sm(int dim, bool hancock);
template <typename T> int fv_blocks_per_cta(int dim, bool staged);
template <typename T> void launch_fvp(const Geo &, const FVArgs<T> &, int grid, cudaStream_t);
template <typename T> int fvp_ctas_per_sm(int dim);
template <typename T> int fvp_blocks_per_cta(int dim);
template <typename T> void launch_dt(const Geo &, const T *A, int lts, unsigned long long *red, unsigned *done, double cfl,
                                     double t_end, double *dsc, double *lev, float *levf, int grid, cudaStream_t);
template <typename T> int fv_ctas_per_sm(int dim, bool split);

// TMA-staged stage kernel of the MR scheme, 2D single precision (fvt.cu): tensor
// maps of the state buffers (own block, x-halo and y-halo boxes) and the ghost
// strips, built once per context
struct FvtMaps {
  CUtensorMap in_own, in_xh, in_yh, u0_own, ghost;
};
struct FvtSet {
  CUtensorMap own[3], xh[3], yh[3], ghost;
  const void *buf[3];   // the state buffers the maps describe (U, Us, U0; null: none)
  int ctas_per_sm;
  bool ok;
};
bool fvt_prepare(FvtSet &, const Geo &, const void *U, const void *Us, const void *U0, const void *G);
int fvt_blocks_per_cta();
// false (nothing launched) when a buffer of the launch has no tensor map
bool launch_fvt(const Geo &, const FVArgs<float> &, const FvtSet &, int grid, cudaStream_t);

// integer tree work (tree.cu)
void launch_need_mark(const Geo &, const uint8_t *sig, uint8_t *need, int crit, int grid, cudaStream_t, int lkeep = 0);
void prepare_br();
void launch_need_close(const Geo &, int l, uint8_t *need, int grid, cudaStream_t, bool parents = true);
// the closure of levels lhi..1 (with parents) in one single-CTA launch, in shared
// memory: the need map of levels 0..lhi must fit in kTailNeedBytes
constexpr int kTailNeedBytes = 4096;
void launch_need_close_tail(const Geo &, int lhi, uint8_t *need, cudaStream_t);
void launch_remesh_begin(const Geo &, long long total, uint8_t *sig, uint8_t *gflag, uint8_t *need, int *nnew, int l0,
                         int grid, cudaStream_t);
void launch_need_prune(const Geo &, int l, uint8_t *need, int grid, cudaStream_t);
void launch_list_level(const Geo &, int l, int32_t *newlist, int *nnew, int grid, cudaStream_t);
void launch_adapt_begin(const Geo &, long long total, uint8_t *sig, double *maxdet, uint8_t *gflag, uint8_t *need,
                        int *nnew, double *t, const double *dt, double factor, long long *counter, int lts,
                        int32_t *pub, int grid, cudaStream_t);
void launch_free(const Geo &, const uint8_t *need, int32_t *fs, int *ft, int grid, cudaStream_t);
void launch_alloc(const Geo &, const uint8_t *need, int32_t *fs, int *ft, int32_t *nl, int *nn, int grid, cudaStream_t);
void launch_init_freestack(int32_t *fs, int *ft, long long cap, int grid, cudaStream_t);
void launch_rebuild_lists(const Geo &, uint8_t *kbits, int32_t *tcount, int32_t *toff, int ntiles, int grid, cudaStream_t);
int scan_tile_entries();
int rebuild_launches(int ntiles);  // kernels launch_rebuild_lists issues
void launch_cluster(const Geo &, const uint8_t *gflag, uint8_t *sig, double eta, int grid, cudaStream_t);
size_t br_scratch_bytes(const Geo &, long long maptotal, int maxside);
void launch_br(const Geo &, const uint8_t *gflag, uint8_t *sig, double eta, void *scratch, long long maptotal,
               int maxside, cudaStream_t);
void launch_set_double(double *p, double v, cudaStream_t);
void launch_level_params(const Geo &, const double *dt, int lts, double *lev, float *levf, cudaStream_t);
void launch_advance(const Geo &, double *t, const double *dt, double factor, long long *counter, int lts,
                    int32_t *pub, cudaStream_t);

// learned refinement proposer (proposer.cu)
template <typename T> void launch_prop_features(const Geo &, const T *U, const double *maxdet, const T *scale, double eps,
                                                float *feat, int grid, cudaStream_t);
void prop_setup();
void launch_wait_selftest(int *err, unsigned limit, int arrive, cudaStream_t);
// the 128-position tiles each layer of the proposer needs (flags: 3 x ntp bytes); count
// (optional): tiles flagged per layer are added to count[3]
void launch_prop_tiles(const Geo &, uint8_t *flags, long long ntp, unsigned long long *count, int grid, cudaStream_t);
// tneed: flags of launch_prop_tiles (only those tiles are computed), or null (every tile)
void launch_prop_infer(const Geo &, const float *feat, __nv_bfloat16 *a0, __nv_bfloat16 *a1, __nv_bfloat16 *a2,
                       const __nv_bfloat16 *w1, const float *b1, const __nv_bfloat16 *w2, const float *b2,
                       const __nv_bfloat16 *w3, const float *b3, float *logits, int nsm, cudaEvent_t conv_begin,
                       cudaEvent_t conv_end, const uint8_t *tneed, cudaStream_t);
void launch_prop_mark(const Geo &, const float *logits, uint8_t *need, int grid, cudaStream_t);
void launch_pack_weights(const float *blob, __nv_bfloat16 *w1, float *b1, __nv_bfloat16 *w2, float *b2,
                         __nv_bfloat16 *w3, float *b3, cudaStream_t);
// adam = 0: gradient and loss only (weights and moments untouched); a0..a2, w1..b3:
// the inference buffers and operands (overwritten); w3t, w2t: the mirrored-tap
// operands of the backward-data convolutions
void launch_prop_train_step(const Geo &, const float *feat, const uint8_t *target, int ns, float *blob, float *grad,
                            float *m1, float *m2, int t, float lr, float *work, double *loss, int adam,
                            __nv_bfloat16 *a0, __nv_bfloat16 *a1, __nv_bfloat16 *a2, __nv_bfloat16 *w1, float *b1,
                            __nv_bfloat16 *w2, float *b2, __nv_bfloat16 *w3, float *b3, __nv_bfloat16 *w3t,
                            __nv_bfloat16 *w2t, int nsm, cudaStream_t);

}  // namespace mrfv
