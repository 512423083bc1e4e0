// Multiresolution and bookkeeping kernels (arXiv:1603.05211, Section 2.1 and
// Section 2.2): projection (restriction), details + eps-thresholding, prediction
// of new blocks, ghost strips of coarse-fine faces, initial data, dense
// download/upload, CFL reduction and conserved totals.
//
// Every kernel is a persistent grid-stride loop over a device work list whose
// length lives in device memory, so the launch shape never depends on the
// tree and the launches can be captured in a CUDA graph.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"

namespace mrfv {

// ---------------------------------------------------------------- projection
// Parent cell = mean of its 2^d children, summed in lexicographic child order
// (x offset fastest), on every refined block of level l.
template <typename T, int D>
__device__ __forceinline__ void restrict_level_dev(const Geo &g, int l, T *__restrict__ A, int cta, int ncta) {
  constexpr int B = (D == 2) ? 64 : 512;
  constexpr int BPC = (D == 2) ? 4 : 1;
  int b, e;
  list_range(g, LK_INTERNAL, l, l, b, e);
  const int sub = threadIdx.x / B, c = threadIdx.x % B;
  const int x = c & 7, y = (c >> 3) & 7, z = (D == 3) ? (c >> 6) : 0;
  const long long cap = g.cap;
  for (int i = b + cta * BPC + sub; i < e; i += ncta * BPC) {
    int s = g.lists[LK_INTERNAL * cap + i];
    int cs = g.kids[8 * s + (x >> 2) + 2 * (y >> 2) + ((D == 3) ? 4 * (z >> 2) : 0)];
    if (cs < 0) {
      set_err(g, EB_TREE);
      continue;
    }
    int f = 2 * (x & 3) + 16 * (y & 3) + ((D == 3) ? 128 * (z & 3) : 0);
    for (int v = 0; v < D + 2; v++) {
      const T *C = A + ((long long)v * cap + cs) * B + f;
      T sum = C[0];
      sum = sum + C[1];
      sum = sum + C[8];
      sum = sum + C[9];
      if (D == 3) {
        sum = sum + C[64];
        sum = sum + C[65];
        sum = sum + C[72];
        sum = sum + C[73];
      }
      A[((long long)v * cap + s) * B + c] = sum * T(D == 2 ? 0.25 : 0.125);
    }
  }
}

template <typename T, int D>
__global__ void k_restrict(Geo g, int l, T *__restrict__ A) {
  restrict_level_dev<T, D>(g, l, A, blockIdx.x, gridDim.x);
}

// The same projection as a sweep over the block positions of level l: the slots
// of the block and of its child come from the dense maps, two independent reads,
// where the list form reads the list offsets, the list and the child table one
// after the other.  A position whose child is absent holds no refined block.
template <typename T, int D>
__device__ __forceinline__ void restrict_pos_dev(const Geo &g, int l, T *__restrict__ A) {
  constexpr int B = (D == 2) ? 64 : 512;
  const int BPC = blockDim.x / B;  // blocks per CTA and pass
  const int sub = threadIdx.x / B, c = threadIdx.x % B;
  const int x = c & 7, y = (c >> 3) & 7, z = (D == 3) ? (c >> 6) : 0;
  const int nx = g.nb[l][0], ny = g.nb[l][1];
  const int n = (int)(g.mapoff[l + 1] - g.mapoff[l]);
  const long long cap = g.cap;
  const int f = 2 * (x & 3) + 16 * (y & 3) + ((D == 3) ? 128 * (z & 3) : 0);
  for (int u = blockIdx.x * BPC + sub; u < n; u += gridDim.x * BPC) {
    const int r = u / nx, bx = u - r * nx, by = r % ny, bz = r / ny;
    const int cs = g.idx[map_index(g, l + 1, 2 * bx + (x >> 2), 2 * by + (y >> 2), (D == 3) ? 2 * bz + (z >> 2) : 0)];
    const int s = g.idx[g.mapoff[l] + u];
    if (cs < 0) continue;
    if (s < 0) {
      set_err(g, EB_TREE);
      continue;
    }
    for (int v = 0; v < D + 2; v++) {
      const T *C = A + ((long long)v * cap + cs) * B + f;
      T sum = C[0];
      sum = sum + C[1];
      sum = sum + C[8];
      sum = sum + C[9];
      if (D == 3) {
        sum = sum + C[64];
        sum = sum + C[65];
        sum = sum + C[72];
        sum = sum + C[73];
      }
      A[((long long)v * cap + s) * B + c] = sum * T(D == 2 ? 0.25 : 0.125);
    }
  }
}
template <typename T, int D>
__global__ void k_restrict_pos(Geo g, int l, T *__restrict__ A) {
  restrict_pos_dev<T, D>(g, l, A);
}
// Levels lhi..0 projected by one CTA (the coarse levels, whose few positions one
// CTA covers in a pass: 16 blocks of level lhi at most in 2D, 2 in 3D).  Two passes
// of global reads: the slots of every position of levels 0..lhi and of their
// children, then the values of every block there (leaves final, refined blocks of
// level lhi projected from their children of level lhi+1); the coarser levels
// are then projected from shared memory, finest first, a CTA barrier per level.
// Every projected block is also stored.  Same sums in the same order as
// restrict_level_dev.
template <int D>
struct TailShape {
  static constexpr int B = (D == 2) ? 64 : 512;
  static constexpr int MAXB = (D == 2) ? kRestrictTailBlocks2D : kRestrictTailBlocks3D;  // positions of levels 0..lhi
};
// the projection of one cell from its children's cells at C (C[0]: the first child
// cell in x, y, z order), the sums of restrict_level_dev in their order
template <typename T, int D>
__device__ __forceinline__ T project_cell(const T *C) {
  T sum = C[0];
  sum = sum + C[1];
  sum = sum + C[8];
  sum = sum + C[9];
  if (D == 3) {
    sum = sum + C[64];
    sum = sum + C[65];
    sum = sum + C[72];
    sum = sum + C[73];
  }
  return sum * T(D == 2 ? 0.25 : 0.125);
}
template <typename T, int D>
__global__ void k_restrict_tail(Geo g, int lhi, T *__restrict__ A) {
  constexpr int B = TailShape<D>::B, MAXB = TailShape<D>::MAXB, NV = D + 2, NK = (D == 2) ? 4 : 8;
  __shared__ T sv[MAXB * NV * B];
  __shared__ int sslot[MAXB], skid[MAXB][NK];
  const long long cap = g.cap;
  const int np = (int)g.mapoff[lhi + 1];
  // first pass of reads: slots of the positions and of their children
  for (int k = threadIdx.x; k < np * (NK + 1); k += blockDim.x) {
    const int pos = k / (NK + 1), q = k % (NK + 1) - 1;
    int l = 0;
    while (l < lhi && pos >= g.mapoff[l + 1]) l++;
    const int u = pos - (int)g.mapoff[l], nx = g.nb[l][0], ny = g.nb[l][1];
    const int r = u / nx, bx = u - r * nx, by = r % ny, bz = r / ny;
    if (q < 0) sslot[pos] = g.idx[pos];
    else
      skid[pos][q] = g.idx[map_index(g, l + 1, 2 * bx + (q & 1), 2 * by + ((q >> 1) & 1), (D == 3) ? 2 * bz + (q >> 2) : 0)];
  }
  __syncthreads();
  // second pass of reads: every block's values; refined blocks of level lhi from their children
  const int p0 = (int)g.mapoff[lhi];
  for (int k = threadIdx.x; k < np * B; k += blockDim.x) {
    const int pos = k / B, c = k % B, s = sslot[pos];
    if (s < 0) continue;
    if (pos >= p0 && skid[pos][0] >= 0) {
      const int x = c & 7, y = (c >> 3) & 7, z = (D == 3) ? (c >> 6) : 0;
      const int cs = skid[pos][(x >> 2) + 2 * (y >> 2) + ((D == 3) ? 4 * (z >> 2) : 0)];
      const int f = 2 * (x & 3) + 16 * (y & 3) + ((D == 3) ? 128 * (z & 3) : 0);
      if (cs < 0) {
        set_err(g, EB_TREE);
        continue;
      }
      for (int v = 0; v < NV; v++) {
        const T val = project_cell<T, D>(A + ((long long)v * cap + cs) * B + f);
        sv[(pos * NV + v) * B + c] = val;
        A[((long long)v * cap + s) * B + c] = val;
      }
    } else {
      for (int v = 0; v < NV; v++) sv[(pos * NV + v) * B + c] = A[((long long)v * cap + s) * B + c];
    }
  }
  __syncthreads();
  for (int l = lhi - 1; l >= 0; l--) {
    const int b = (int)g.mapoff[l], e = (int)g.mapoff[l + 1];
    const int nxf = g.nb[l + 1][0], nyf = g.nb[l + 1][1], nx = g.nb[l][0], ny = g.nb[l][1];
    for (int k = threadIdx.x; k < (e - b) * B; k += blockDim.x) {
      const int pos = b + k / B, c = k % B, s = sslot[pos];
      if (s < 0 || skid[pos][0] < 0) continue;
      const int u = pos - b, r = u / nx, bx = u - r * nx, by = r % ny, bz = r / ny;
      const int x = c & 7, y = (c >> 3) & 7, z = (D == 3) ? (c >> 6) : 0;
      // the child holding this cell's children, as a position of level l+1
      const int cpos = (int)g.mapoff[l + 1] + (2 * bx + (x >> 2)) + nxf * ((2 * by + (y >> 2)) + nyf * ((D == 3) ? 2 * bz + (z >> 2) : 0));
      const int f = 2 * (x & 3) + 16 * (y & 3) + ((D == 3) ? 128 * (z & 3) : 0);
      for (int v = 0; v < NV; v++) {
        const T val = project_cell<T, D>(sv + (cpos * NV + v) * B + f);
        sv[(pos * NV + v) * B + c] = val;
        A[((long long)v * cap + s) * B + c] = val;
      }
    }
    __syncthreads();
  }
}

// Projection between the two stages of the MR step.  Before the step's closing
// projection, the second stage reads only two kinds of coarse cells of refined
// blocks: the parent-level cells that the ghost-strip prediction of a block with
// an absent same-level neighbour reads (three cells across the face, six along
// it, around the block's quadrant), and the two cells next to a coarse-fine face
// that the coarse side's reconstruction reads.  In a graded tree a block next to
// an absent position (across a face, an edge or a corner) is a leaf, and every
// such cell lies over a leaf of that kind; so projecting, on all levels at once,
// the parent quadrant of every leaf that has an absent position among its 3^d-1
// neighbours gives those cells the values of the full projection (one level, the
// same sums in the same order).  Cells of refined blocks over other children keep
// older values that nothing reads before the closing projection.
template <typename T, int D>
__device__ __forceinline__ void restrict_edge_dev(const Geo &g, T *__restrict__ A, int cta, int ncta) {
  constexpr int B = (D == 2) ? 64 : 512;
  constexpr int Q = (D == 2) ? 16 : 64;  // cells of a parent quadrant
  const int PER = blockDim.x / Q;        // leaves per CTA and pass
  const int sub = threadIdx.x / Q, c = threadIdx.x % Q;
  const int qx = c & 3, qy = (c >> 2) & 3, qz = (D == 3) ? (c >> 4) : 0;
  const long long cap = g.cap;
  int b, e;
  list_range(g, LK_LEAF, 1, g.L, b, e);
  for (int i = b + cta * PER + sub; i < e; i += ncta * PER) {
    const int s = g.lists[LK_LEAF * cap + i];
    const int l = g.slot_level[s];
    const int bx = g.slot_coord[3 * s], by = g.slot_coord[3 * s + 1], bz = g.slot_coord[3 * s + 2];
    bool edge = false;
    for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const int x = bc_block(g, l, 0, bx + dx), y = bc_block(g, l, 1, by + dy), z = bc_block(g, l, 2, bz + dz);
          if (x < 0 || y < 0 || z < 0) continue;  // outside a transmissive domain: not an absent block
          if (g.idx[map_index(g, l, x, y, z)] < 0) edge = true;
        }
    const int p = g.idx[map_index(g, l - 1, bx >> 1, by >> 1, bz >> 1)];
    if (!edge) continue;
    if (p < 0) {
      set_err(g, EB_TREE);
      continue;
    }
    const int pc = ((bx & 1) * 4 + qx) + 8 * ((by & 1) * 4 + qy) + ((D == 3) ? 64 * ((bz & 1) * 4 + qz) : 0);
    const int f = 2 * qx + 16 * qy + ((D == 3) ? 128 * qz : 0);
    for (int v = 0; v < D + 2; v++) {
      const T *C = A + ((long long)v * cap + s) * B + f;
      T sum = C[0];
      sum = sum + C[1];
      sum = sum + C[8];
      sum = sum + C[9];
      if (D == 3) {
        sum = sum + C[64];
        sum = sum + C[65];
        sum = sum + C[72];
        sum = sum + C[73];
      }
      A[((long long)v * cap + p) * B + pc] = sum * T(D == 2 ? 0.25 : 0.125);
    }
  }
}

// ---------------------------------------------------------------- MR analysis
// Normalisation maxima over level 0: |rho|, |rho e|, max_n |v_n| (as the bit
// patterns of non-negative doubles, so atomicMax on the integer orders them).
// This thread's maxima over the level-0 cells start, start + stride, ..., then
// the warp's (every lane holds them).
template <typename T, int D>
__device__ __forceinline__ void level0_maxima(const Geo &g, const T *__restrict__ A, long long start, long long stride,
                                              T &mr, T &mE, T &mv) {
  constexpr int B = (D == 2) ? 64 : 512;
  int b, e;
  list_range(g, LK_EXIST, 0, 0, b, e);
  const long long cap = g.cap;
  mr = 0;
  mE = 0;
  mv = 0;
  for (long long t = (long long)b * B + start; t < (long long)e * B; t += stride) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[LK_EXIST * cap + i];
    T rho = A[((long long)0 * cap + s) * B + c];
    T E = A[((long long)(D + 1) * cap + s) * B + c];
    if (fabs(rho) > mr) mr = fabs(rho);
    if (fabs(E) > mE) mE = fabs(E);
    for (int d = 0; d < D; d++) {
      T v = fabs(A[((long long)(1 + d) * cap + s) * B + c] / rho);
      if (v > mv) mv = v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mE = fmax(mE, __shfl_xor_sync(0xffffffffu, mE, o));
    mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
  }
}
template <typename T, int D>
__device__ __forceinline__ void scale_max_dev(const Geo &g, const T *__restrict__ A, unsigned long long *red) {
  T mr, mE, mv;
  level0_maxima<T, D>(g, A, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x, mr,
                      mE, mv);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(red + 0, (unsigned long long)__double_as_longlong((double)mr));
    atomicMax(red + 1, (unsigned long long)__double_as_longlong((double)mE));
    atomicMax(red + 2, (unsigned long long)__double_as_longlong((double)mv));
  }
}

template <typename T, int D>
__device__ __forceinline__ void scale_final_dev(const unsigned long long *red, T *scale);

// maxima of level 0, then (last CTA) the scales; the last CTA also clears the
// maxima and its counter for the next launch
template <typename T, int D>
__global__ void k_scale_max(Geo g, const T *__restrict__ A, unsigned long long *red, unsigned *done, T *scale) {
  scale_max_dev<T, D>(g, A, red);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      __threadfence();
      unsigned long long r[3];
      for (int k = 0; k < 3; k++) r[k] = atomicAdd(red + k, 0ull);
      scale_final_dev<T, D>(r, scale);
      for (int k = 0; k < 3; k++) red[k] = 0ull;
      *done = 0u;
      __threadfence();
    }
  }
}

// s_rho = max|rho|, s_E = max|rho e|, s_m = max|rho| * max|v_n|, each at least
// 1e-14 * max|rho| (reading of the paper's unstated normalisation), in T.
template <typename T, int D>
__device__ __forceinline__ void scale_final_dev(const unsigned long long *red, T *scale) {
  T mr = (T)__longlong_as_double((long long)red[0]);
  T mE = (T)__longlong_as_double((long long)red[1]);
  T mv = (T)__longlong_as_double((long long)red[2]);
  T fl = T(1e-14) * mr;
  T sm = mr * mv;
  scale[0] = mr > fl ? mr : fl;
  for (int d = 0; d < D; d++) scale[1 + d] = sm > fl ? sm : fl;
  scale[D + 1] = mE > fl ? mE : fl;
}

template <typename T, int D>
__global__ void k_scale_final(const unsigned long long *red, T *scale) {
  scale_final_dev<T, D>(red, scale);
}

// Details of every existing block of levels 1..L against the prediction from
// its parent level; block flag = max over cells and variables of |d_v|/s_v > eps.
template <typename T, int D>
__device__ __forceinline__ void details_dev(const Geo &g, const T *__restrict__ A, const T *__restrict__ scale,
                                            T eps, uint8_t *sig, double *maxdet, T *patch, T *wmax, int l0,
                                            const T *__restrict__ A0, T theta, T *own_scale, uint8_t *need) {
  constexpr int B = (D == 2) ? 64 : 512;
  constexpr int EXT = 6;
  constexpr int NP = (D == 2) ? EXT * EXT : EXT * EXT * EXT;
  int b, e;
  if (l0 < 1) l0 = 1;
  if (l0 > g.L) return;
  list_range(g, LK_EXIST, l0, g.L, b, e);
  const long long cap = g.cap;
  const int c = threadIdx.x;
  const int x = c & 7, y = (c >> 3) & 7, z = (D == 3) ? (c >> 6) : 0;
  T sc[D + 2];
  if (own_scale) {
    // the normalisation of k_scale_max computed by this CTA alone (a level 0 of a
    // few blocks): the same maxima, so the same scales; CTA 0 stores them
    T mr, mE, mv;
    level0_maxima<T, D>(g, A, c, B, mr, mE, mv);
    if ((c & 31) == 0) {
      patch[3 * (c >> 5)] = mr;
      patch[3 * (c >> 5) + 1] = mE;
      patch[3 * (c >> 5) + 2] = mv;
    }
    __syncthreads();
    if (c == 0) {
      for (int w = 1; w < B / 32; w++) {
        mr = fmax(mr, patch[3 * w]);
        mE = fmax(mE, patch[3 * w + 1]);
        mv = fmax(mv, patch[3 * w + 2]);
      }
      unsigned long long r[3] = {(unsigned long long)__double_as_longlong((double)mr),
                                 (unsigned long long)__double_as_longlong((double)mE),
                                 (unsigned long long)__double_as_longlong((double)mv)};
      scale_final_dev<T, D>(r, wmax);
      if (blockIdx.x == 0)
        for (int v = 0; v < D + 2; v++) own_scale[v] = wmax[v];
    }
    __syncthreads();
    for (int v = 0; v < D + 2; v++) sc[v] = wmax[v];
  } else {
    for (int v = 0; v < D + 2; v++) sc[v] = scale[v];
  }
  for (int i = b + blockIdx.x; i < e; i += gridDim.x) {
    int s = g.lists[LK_EXIST * cap + i];
    int l = g.slot_level[s];
    int bx = g.slot_coord[3 * s], by = g.slot_coord[3 * s + 1], bz = g.slot_coord[3 * s + 2];
    __syncthreads();
    // (level l0 of a remesh: the parent level interpolated in time)
    gather_patch<T, D, EXT>(g, l - 1, A, l == l0 ? A0 : (const T *)nullptr, theta, 4 * bx - 1, 4 * by - 1, 4 * bz - 1,
                            patch, c, B);
    __syncthreads();
    // this cell's parent inside the patch and its child signs
    int px = (x >> 1) + 1, py = (y >> 1) + 1, pz = (D == 3) ? (z >> 1) + 1 : 0;
    T si = (x & 1) ? T(-1) : T(1), sj = (y & 1) ? T(-1) : T(1), sk = (z & 1) ? T(-1) : T(1);
    T md = 0;
    for (int v = 0; v < D + 2; v++) {
      T q = A[((long long)v * cap + s) * B + c];
      T qh = predict<T, D, EXT>(patch + v * NP, px, py, pz, si, sj, sk);
      T r = fabs(q - qh) / sc[v];
      if (r > md) md = r;
    }
    for (int o = 16; o > 0; o >>= 1) {
      T t = __shfl_xor_sync(0xffffffffu, md, o);
      if (t > md) md = t;
    }
    if ((c & 31) == 0) wmax[c >> 5] = md;
    __syncthreads();
    if (c == 0) {
      T m = wmax[0];
      for (int w = 1; w < B / 32; w++)
        if (wmax[w] > m) m = wmax[w];
      long long mi = map_index(g, l, bx, by, bz);
      sig[mi] = (m > eps) ? 1 : 0;
      maxdet[mi] = (double)m;
      wmax[31] = (need && m > eps) ? T(1) : T(0);
    }
    if (need) {
      // the MR marks of k_need_mark for a significant block (level >= 1): the block
      // and its 3^d-1 neighbours (one per thread), below the finest level its children
      __syncthreads();
      if (wmax[31] != T(0)) {
        constexpr int NN = (D == 2) ? 9 : 27;
        if (c < NN) {
          const int a = c % 3 - 1, bb = (c / 3) % 3 - 1, cc = (D == 3) ? c / 9 - 1 : 0;
          const int nx = bc_block(g, l, 0, bx + a), ny = bc_block(g, l, 1, by + bb), nz = bc_block(g, l, 2, bz + cc);
          if (nx >= 0 && ny >= 0 && nz >= 0) need[map_index(g, l, nx, ny, nz)] = 1;
        } else if (c < NN + (D == 2 ? 4 : 8) && l < g.L) {
          const int q = c - NN;
          need[map_index(g, l + 1, 2 * bx + (q & 1), 2 * by + ((q >> 1) & 1), (D == 3) ? 2 * bz + (q >> 2) : 0)] = 1;
        }
      }
    }
  }
}

// own_scale: compute the level-0 normalisation in every CTA (and store it there)
// instead of reading it; need: mark the needed blocks of the MR criterion here
// instead of in k_need_mark (the adaptation of a step)
template <typename T, int D>
__global__ void k_details(Geo g, const T *__restrict__ A, const T *__restrict__ scale, T eps, uint8_t *sig,
                          double *maxdet, int l0, const T *__restrict__ A0, T theta, T *own_scale, uint8_t *need) {
  __shared__ T patch[(D + 2) * ((D == 2) ? 36 : 216)];
  __shared__ T wmax[32];
  details_dev<T, D>(g, A, scale, eps, sig, maxdet, patch, wmax, l0, A0, theta, own_scale, need);
}

// ---------------------------------------------------------------- prediction of new blocks
template <typename T, int D>
__device__ __forceinline__ void prolong_level_dev(const Geo &g, int l, const int32_t *__restrict__ newlist,
                                                  const int *__restrict__ nnew, T *__restrict__ A, T *patch) {
  constexpr int B = (D == 2) ? 64 : 512;
  constexpr int EXT = 6;
  constexpr int NP = (D == 2) ? EXT * EXT : EXT * EXT * EXT;
  const long long cap = g.cap;
  const int n = nnew[l];
  const int c = threadIdx.x;
  const int x = c & 7, y = (c >> 3) & 7, z = (D == 3) ? (c >> 6) : 0;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    int s = newlist[g.mapoff[l] + i];
    int bx = g.slot_coord[3 * s], by = g.slot_coord[3 * s + 1], bz = g.slot_coord[3 * s + 2];
    __syncthreads();
    gather_patch<T, D, EXT>(g, l - 1, A, (const T *)nullptr, T(0), 4 * bx - 1, 4 * by - 1, 4 * bz - 1, patch, c, B);
    __syncthreads();
    int px = (x >> 1) + 1, py = (y >> 1) + 1, pz = (D == 3) ? (z >> 1) + 1 : 0;
    T si = (x & 1) ? T(-1) : T(1), sj = (y & 1) ? T(-1) : T(1), sk = (z & 1) ? T(-1) : T(1);
    for (int v = 0; v < D + 2; v++)
      A[((long long)v * cap + s) * B + c] = predict<T, D, EXT>(patch + v * NP, px, py, pz, si, sj, sk);
  }
}

template <typename T, int D>
__global__ void k_prolong(Geo g, int l, const int32_t *__restrict__ newlist, const int *__restrict__ nnew,
                          T *__restrict__ A) {
  __shared__ T patch[(D + 2) * ((D == 2) ? 36 : 216)];
  prolong_level_dev<T, D>(g, l, newlist, nnew, A, patch);
}
// New blocks of levels 1..lhi predicted by one CTA, coarsest first (a new block
// may read new blocks of the level above), a CTA barrier between the levels.
template <typename T, int D>
__global__ void k_prolong_tail(Geo g, int lhi, const int32_t *__restrict__ newlist, const int *__restrict__ nnew,
                               T *__restrict__ A) {
  __shared__ T patch[(D + 2) * ((D == 2) ? 36 : 216)];
  for (int l = 1; l <= lhi; l++) {
    prolong_level_dev<T, D>(g, l, newlist, nnew, A, patch);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- ghost strips
// For every block of level l in the ghost list, each face whose same-level
// neighbour is absent gets its two outer cell layers predicted from level l-1
// (A, or A0 + theta (A - A0) for level-dependent steps).  Strip layout:
// G[v][slot][face][depth][tangential], depth 0 touches the block.
template <typename T, int D, bool PROJ>
__device__ __forceinline__ void ghost_dev(const Geo &g, int l0, int l1, const T *__restrict__ A,
                                          const T *__restrict__ A0, T theta, T *__restrict__ G, T *patch, int cta,
                                          int ncta) {
  constexpr int TF = (D == 2) ? 8 : 64;
  constexpr int GS = 2 * D * 2 * TF;
  constexpr int EXT = 8;
  constexpr int NP = (D == 2) ? EXT * EXT : EXT * EXT * EXT;
  int b, e;
  list_range(g, LK_GHOST, l0, l1, b, e);
  const long long cap = g.cap;
  for (int i = b + cta; i < e; i += ncta) {
    int s = g.lists[LK_GHOST * cap + i];
    int l = g.slot_level[s];
    int bx = g.slot_coord[3 * s], by = g.slot_coord[3 * s + 1], bz = g.slot_coord[3 * s + 2];
    __syncthreads();
    if (PROJ)
      gather_patch_proj<T, D, EXT>(g, l - 1, A, 4 * bx - 2, 4 * by - 2, 4 * bz - 2, patch, threadIdx.x, blockDim.x);
    else
      gather_patch<T, D, EXT>(g, l - 1, A, A0, theta, 4 * bx - 2, 4 * by - 2, 4 * bz - 2, patch, threadIdx.x,
                              blockDim.x);
    __syncthreads();
    for (int q = threadIdx.x; q < GS; q += blockDim.x) {
      int f = q / (2 * TF), dd = (q / TF) & 1, t = q % TF;
      if (g.nbr[6 * s + f] != NBR_MISSING) continue;
      int n = f >> 1, side = f & 1;
      int rel[3];
      int ta = t & 7, tb = t >> 3;  // tangential coordinates, lower dimension first
      int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
      rel[n] = side ? 8 + dd : -1 - dd;
      rel[t1] = ta;
      rel[t2] = (D == 3) ? tb : 0;
      // fine coordinate relative to the block origin -> patch coordinates of its parent
      int px = ((rel[0] + 8) >> 1) - 2, py = ((rel[1] + 8) >> 1) - 2, pz = (D == 3) ? ((rel[2] + 8) >> 1) - 2 : 0;
      T si = (rel[0] & 1) ? T(-1) : T(1), sj = (rel[1] & 1) ? T(-1) : T(1), sk = (rel[2] & 1) ? T(-1) : T(1);
      for (int v = 0; v < D + 2; v++)
        G[((long long)v * cap + s) * GS + q] = predict<T, D, EXT>(patch + v * NP, px, py, pz, si, sj, sk);
    }
  }
}
template <typename T, int D>
__global__ void k_ghost(Geo g, int l0, int l1, const T *__restrict__ A, const T *__restrict__ A0, T theta,
                        T *__restrict__ G) {
  extern __shared__ unsigned char smem_raw[];
  ghost_dev<T, D, false>(g, l0, l1, A, A0, theta, G, reinterpret_cast<T *>(smem_raw), blockIdx.x, gridDim.x);
}
// Between the stages of the MR step, in one launch: the ghost strips of every
// level (the first ng CTAs), their coarse cells over refined blocks projected on
// the fly from the children, and the projection of restrict_edge_dev (the
// others), which the stage's coarse-side fluxes read.  The two parts read the
// stage state and write disjoint buffers.
template <typename T, int D>
__global__ void k_ghost_edge(Geo g, int ng, T *__restrict__ A, T *__restrict__ G) {
  extern __shared__ unsigned char smem_raw[];
  if ((int)blockIdx.x < ng)
    ghost_dev<T, D, true>(g, 1, g.L, A, (const T *)nullptr, T(0), G, reinterpret_cast<T *>(smem_raw), blockIdx.x, ng);
  else
    restrict_edge_dev<T, D>(g, A, blockIdx.x - ng, gridDim.x - ng);
}

// ---------------------------------------------------------------- initial data

__device__ inline void ic_point(const ICParams &ic, int dim, double gamma, const double *lo, const double *hi,
                                const double *x, double *w) {
  w[0] = 1.0;
  w[1] = w[2] = w[3] = 0.0;
  w[4] = 1.0;
  const double *P = ic.p;
  if (ic.kind == 0) {  // quadrants I..IV (Table 1 order)
    double xc = 0.5 * (lo[0] + hi[0]), yc = 0.5 * (lo[1] + hi[1]);
    int quad;
    if (x[1] >= yc) quad = (x[0] >= xc) ? 0 : 1;
    else quad = (x[0] >= xc) ? 3 : 2;
    w[0] = P[4 * quad];
    w[1] = P[4 * quad + 1];
    w[2] = P[4 * quad + 2];
    w[4] = P[4 * quad + 3];
  } else if (ic.kind == 1) {  // axis-aligned ellipsoid
    double r2 = 0.0;
    for (int d = 0; d < 3; d++) {
      double t = (x[d] - P[d]) / P[3 + d];
      r2 = r2 + t * t;
    }
    if (r2 < 1.0) { w[0] = P[6]; w[4] = P[7]; }
    else { w[0] = P[8]; w[4] = P[9]; }
  } else if (ic.kind == 2) {  // shock tube
    int ax = (int)P[0];
    bool left = x[ax] < P[1];
    w[0] = left ? P[2] : P[5];
    w[1 + ax] = left ? P[3] : P[6];
    w[4] = left ? P[4] : P[7];
  } else if (ic.kind == 3) {  // uniform
    w[0] = P[0]; w[1] = P[1]; w[2] = P[2]; w[3] = P[3]; w[4] = P[4];
  } else if (ic.kind == 4) {  // smooth wave
    double s = x[0] + x[1];
    if (dim == 3) s = s + x[2];
    w[0] = 1.0 + P[0] * sin(2.0 * 3.14159265358979323846 * s);
    w[1] = P[1]; w[2] = P[2]; w[3] = P[3]; w[4] = P[4];
  } else if (ic.kind == 5) {  // rotated ellipsoid (Section 4.2)
    double a = P[0], b = P[1], c = P[2], rc = P[3], th = P[4], ph = P[5];
    double x1 = x[0] * cos(th) - x[1] * sin(th);
    double t = x[0] * sin(th) + x[1] * cos(th);
    double x2 = t * cos(ph) - x[2] * sin(ph);
    double x3 = t * sin(ph) + x[2] * cos(ph);
    double r = sqrt((x1 / a) * (x1 / a) + (x2 / b) * (x2 / b) + (x3 / c) * (x3 / c));
    bool in = r < rc;
    w[0] = in ? P[6] : P[8];
    w[4] = (gamma - 1.0) * (in ? P[7] : P[9]);
  }
  if (dim == 2) w[3] = 0.0;
}

// Sample the finest level at cell centres (conservative variables from the
// primitive state in double, then rounded to T).
template <typename T, int D>
__global__ void k_init(Geo g, ICParams ic, double hi0, double hi1, double hi2, T *__restrict__ A) {
  constexpr int B = (D == 2) ? 64 : 512;
  int b, e;
  const int L = g.L;
  list_range(g, LK_EXIST, L, L, b, e);
  const long long cap = g.cap;
  double lo[3] = {g.lo[0], g.lo[1], g.lo[2]}, hi[3] = {hi0, hi1, hi2};
  for (long long t = (long long)b * B + blockIdx.x * blockDim.x + threadIdx.x; t < (long long)e * B;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[LK_EXIST * cap + i];
    int id[3] = {g.slot_coord[3 * s] * 8 + (c & 7), g.slot_coord[3 * s + 1] * 8 + ((c >> 3) & 7),
                 (D == 3) ? g.slot_coord[3 * s + 2] * 8 + (c >> 6) : 0};
    double x[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; d++) x[d] = g.lo[d] + ((double)id[d] + 0.5) * g.dx[L][d];
    double w[5];
    ic_point(ic, D, g.gamma, lo, hi, x, w);
    double vv = ((w[1] * w[1]) + (w[2] * w[2])) + (w[3] * w[3]);
    double Q[5];
    Q[0] = w[0];
    for (int d = 0; d < D; d++) Q[1 + d] = w[0] * w[1 + d];
    Q[D + 1] = (w[4] / (g.gamma - 1.0)) + ((0.5 * w[0]) * vv);
    for (int v = 0; v < D + 2; v++) A[((long long)v * cap + s) * B + c] = (T)Q[v];
  }
}

// ---------------------------------------------------------------- dense copies
template <typename T, int D>
__global__ void k_gather_level(Geo g, int l, const T *__restrict__ A, double *__restrict__ out) {
  constexpr int B = (D == 2) ? 64 : 512;
  long long n0 = (long long)g.nb[l][0] * 8, n1 = (long long)g.nb[l][1] * 8, n2 = (D == 3) ? (long long)g.nb[l][2] * 8 : 1;
  long long nc = n0 * n1 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / (n0 * n1));
    int32_t s = g.idx[map_index(g, l, i >> 3, j >> 3, k >> 3)];
    int c = (i & 7) + 8 * (j & 7) + ((D == 3) ? 64 * (k & 7) : 0);
    for (int v = 0; v < D + 2; v++)
      out[(long long)v * nc + t] = (s >= 0) ? (double)A[((long long)v * g.cap + s) * B + c] : (double)nan_val<T>();
  }
}

// one variable of level l, averaged over cubes of f^d cells (x fastest within
// the cube, then y, then z); NaN where the block is absent
template <typename T, int D>
__global__ void k_gather_var(Geo g, int l, int v, int f, const T *__restrict__ A, double *__restrict__ out) {
  constexpr int B = (D == 2) ? 64 : 512;
  long long n0 = (long long)g.nb[l][0] * 8 / f, n1 = (long long)g.nb[l][1] * 8 / f;
  long long n2 = (D == 3) ? (long long)g.nb[l][2] * 8 / f : 1;
  long long nc = n0 * n1 * n2;
  const double w = 1.0 / (double)(D == 3 ? f * f * f : f * f);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
    int i0 = (int)(t % n0) * f, j0 = (int)((t / n0) % n1) * f, k0 = (D == 3) ? (int)(t / (n0 * n1)) * f : 0;
    double sum = 0.0;
    bool absent = false;
    for (int c3 = 0; c3 < (D == 3 ? f : 1); c3++)
      for (int b = 0; b < f; b++)
        for (int a = 0; a < f; a++) {
          int i = i0 + a, j = j0 + b, k = k0 + c3;
          int32_t s = g.idx[map_index(g, l, i >> 3, j >> 3, k >> 3)];
          if (s < 0) {
            absent = true;
            continue;
          }
          int c = (i & 7) + 8 * (j & 7) + ((D == 3) ? 64 * (k & 7) : 0);
          sum = sum + (double)A[((long long)v * g.cap + s) * B + c];
        }
    out[t] = absent ? (double)nan_val<T>() : sum * w;
  }
}

template <typename T, int D>
__global__ void k_scatter_level(Geo g, int l, const double *__restrict__ in, T *__restrict__ A) {
  constexpr int B = (D == 2) ? 64 : 512;
  long long n0 = (long long)g.nb[l][0] * 8, n1 = (long long)g.nb[l][1] * 8, n2 = (D == 3) ? (long long)g.nb[l][2] * 8 : 1;
  long long nc = n0 * n1 * n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / (n0 * n1));
    int32_t s = g.idx[map_index(g, l, i >> 3, j >> 3, k >> 3)];
    if (s < 0) continue;
    int c = (i & 7) + 8 * (j & 7) + ((D == 3) ? 64 * (k & 7) : 0);
    for (int v = 0; v < D + 2; v++) A[((long long)v * g.cap + s) * B + c] = (T)in[(long long)v * nc + t];
  }
}

// ---------------------------------------------------------------- projection to the finest level
// Dense level-l array of the leaf representation (Section 3, error assessment
// for MR): existing cells from the pool, every other cell predicted (third
// order, in double) from the dense level l-1 array built the same way.
template <typename T, int D>
__global__ void k_project_level(Geo g, int l, const T *__restrict__ A, const double *__restrict__ coarse,
                                double *__restrict__ out) {
  constexpr int B = (D == 2) ? 64 : 512;
  const long long n0 = (long long)g.nb[l][0] * 8, n1 = (long long)g.nb[l][1] * 8;
  const long long n2 = (D == 3) ? (long long)g.nb[l][2] * 8 : 1;
  const long long nc = n0 * n1 * n2;
  const long long c0 = n0 / 2, c1 = n1 / 2, c2 = (D == 3) ? n2 / 2 : 1, ncc = c0 * c1 * c2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n0), j = (int)((t / n0) % n1), k = (int)(t / (n0 * n1));
    int32_t s = g.idx[map_index(g, l, i >> 3, j >> 3, k >> 3)];
    if (s >= 0) {
      int c = (i & 7) + 8 * (j & 7) + ((D == 3) ? 64 * (k & 7) : 0);
      for (int v = 0; v < D + 2; v++) out[(long long)v * nc + t] = (double)A[((long long)v * g.cap + s) * B + c];
      continue;
    }
    // 3^d coarse stencil around the parent cell (boundary rule at level l-1)
    double Pch[27];
    for (int v = 0; v < D + 2; v++) {
      for (int cz = 0; cz < ((D == 3) ? 3 : 1); cz++)
        for (int cy = 0; cy < 3; cy++)
          for (int cx = 0; cx < 3; cx++) {
            int x = bc_cell(g, l - 1, 0, (i >> 1) + cx - 1), y = bc_cell(g, l - 1, 1, (j >> 1) + cy - 1);
            int z = (D == 3) ? bc_cell(g, l - 1, 2, (k >> 1) + cz - 1) : 0;
            Pch[cx + 3 * (cy + 3 * cz)] = coarse[(long long)v * ncc + x + c0 * (y + c1 * z)];
          }
      double si = (i & 1) ? -1.0 : 1.0, sj = (j & 1) ? -1.0 : 1.0, sk = (k & 1) ? -1.0 : 1.0;
      out[(long long)v * nc + t] = predict<double, D, 3>(Pch, 1, 1, (D == 3) ? 1 : 0, si, sj, sk);
    }
  }
}

// ---------------------------------------------------------------- totals
template <typename T, int D>
__global__ void k_totals(Geo g, const T *__restrict__ A, double *out) {
  constexpr int B = (D == 2) ? 64 : 512;
  int b, e;
  list_range(g, LK_LEAF, 0, g.L, b, e);
  const long long cap = g.cap;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long t = (long long)b * B + blockIdx.x * blockDim.x + threadIdx.x; t < (long long)e * B;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[LK_LEAF * cap + i];
    int l = g.slot_level[s];
    double vol = g.dx[l][0] * g.dx[l][1];
    if (D == 3) vol = vol * g.dx[l][2];
    for (int v = 0; v < D + 2; v++) acc[v] += (double)A[((long long)v * cap + s) * B + c] * vol;
  }
  for (int v = 0; v < D + 2; v++) {
    double a = acc[v];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out + v, a);
  }
}

// ---------------------------------------------------------------- flux correction
// Coarse leaf cells bordering a refined same-level neighbour (Section 2.2, Fig. 2;
// virtual leaves of Section 2.1): the time-integrated coarse flux R_c = dt_l F_c is
// replaced by the mean of the 2^(d-1) time-integrated fine fluxes on that face,
// q += s (R_c - mean R_f) / dx (s = +1 high face, -1 low face).  One thread per
// cell applies its faces in direction order, low side first; the fine faces are
// averaged in the order (first tangential offset fastest).
template <typename T, int D>
__device__ __forceinline__ void reflux_dev(const Geo &g, int l0, int l1, T *__restrict__ A, const T *__restrict__ FR,
                                           int cta, int ncta) {
  constexpr int B = (D == 2) ? 64 : 512;
  constexpr int TF = (D == 2) ? 8 : 64;
  constexpr int FS = 2 * D * TF;
  int b, e;
  list_range(g, LK_REFLUX, l0, l1, b, e);
  const long long cap = g.cap;
  for (long long t = (long long)b * B + cta * (long long)blockDim.x + threadIdx.x; t < (long long)e * B;
       t += (long long)ncta * blockDim.x) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[LK_REFLUX * cap + i];
    int l = g.slot_level[s];
    int cm = g.cmask[s];
    int cc[3] = {c & 7, (c >> 3) & 7, (D == 3) ? (c >> 6) : 0};
    for (int f = 0; f < 2 * D; f++) {
      if (!((cm >> f) & 1)) continue;
      int n = f >> 1, side = f & 1;
      if (cc[n] != (side ? 7 : 0)) continue;
      int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
      int u = cc[t1], w = (D == 3) ? cc[t2] : 0;
      int P = g.nbr[6 * s + f];
      // the child of the refined neighbour P that touches this face
      int ch[3] = {0, 0, 0};
      ch[n] = side ? 0 : 1;
      ch[t1] = u >> 2;
      if (D == 3) ch[t2] = w >> 2;
      int fs = g.kids[8 * P + ch[0] + 2 * ch[1] + 4 * ch[2]];
      if (fs < 0) {
        set_err(g, EB_TREE);
        continue;
      }
      int ff = 2 * n + (1 - side);
      const T dx = T(g.dx[l][n]);
      for (int v = 0; v < D + 2; v++) {
        const T *Rf = FR + ((long long)v * cap + fs) * FS + ff * TF;
        T m;
        if (D == 2) {
          m = Rf[2 * (u & 3)];
          m = m + Rf[2 * (u & 3) + 1];
          m = m * T(0.5);
        } else {
          int fu = 2 * (u & 3), fw = 2 * (w & 3);
          m = Rf[fu + 8 * fw];
          m = m + Rf[fu + 1 + 8 * fw];
          m = m + Rf[fu + 8 * (fw + 1)];
          m = m + Rf[fu + 1 + 8 * (fw + 1)];
          m = m * T(0.25);
        }
        T rc = FR[((long long)v * cap + s) * FS + f * TF + u + ((D == 3) ? 8 * w : 0)];
        T corr = (rc - m) / dx;
        long long o = ((long long)v * cap + s) * B + c;
        A[o] = side ? A[o] + corr : A[o] - corr;
      }
    }
  }
}
template <typename T, int D>
__global__ void k_reflux(Geo g, int l0, int l1, T *__restrict__ A, const T *__restrict__ FR) {
  reflux_dev<T, D>(g, l0, l1, A, FR, blockIdx.x, gridDim.x);
}
// Flux correction of levels 0..L-1 (the first nr CTAs) beside the projection of
// level L-1 (the others): the projection reads only leaves of level L, which the
// correction never changes (no block of the finest level has a refined
// neighbour), and writes only refined blocks, which the correction never reads.
template <typename T, int D>
__global__ void k_reflux_restrict(Geo g, int nr, T *__restrict__ A, const T *__restrict__ FR) {
  if ((int)blockIdx.x < nr) reflux_dev<T, D>(g, 0, g.L - 1, A, FR, blockIdx.x, nr);
  else restrict_level_dev<T, D>(g, g.L - 1, A, blockIdx.x - nr, gridDim.x - nr);
}

// copy the blocks of list `kind` on levels l0..l1 from src to dst
template <typename T, int D>
__global__ void k_copy_level(Geo g, int kind, int l0, int l1, const T *__restrict__ src, T *__restrict__ dst) {
  constexpr int B = (D == 2) ? 64 : 512;
  int b, e;
  list_range(g, kind, l0, l1, b, e);
  const long long cap = g.cap;
  for (long long t = (long long)b * B + blockIdx.x * blockDim.x + threadIdx.x; t < (long long)e * B;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[kind * cap + i];
    for (int v = 0; v < D + 2; v++) {
      long long o = ((long long)v * cap + s) * B + c;
      dst[o] = src[o];
    }
  }
}

// ---------------------------------------------------------------- scaled-gradient flags
// density of level l at global cell (i, j, k) (already inside the domain):
// the block's value, or the prediction from level l-1 when the block is absent
template <typename T, int D>
__device__ T var_ext(const Geo &g, int l, const T *__restrict__ Abase, int v, int i, int j, int k,
                     const T *__restrict__ C0base = nullptr, T theta = T(0)) {
  constexpr int B = (D == 2) ? 64 : 512;
  const T *__restrict__ A = Abase + (long long)v * g.cap * B;
  int32_t s = g.idx[map_index(g, l, i >> 3, j >> 3, k >> 3)];
  if (s >= 0) return A[(long long)s * B + (i & 7) + 8 * (j & 7) + ((D == 3) ? 64 * (k & 7) : 0)];
  if (l == 0) {
    set_err(g, EB_TREE);
    return nan_val<T>();
  }
  T P[27];
  int ci = i >> 1, cj = j >> 1, ck = k >> 1;
  for (int c = 0; c < ((D == 3) ? 3 : 1); c++)
    for (int bb = 0; bb < 3; bb++)
      for (int a = 0; a < 3; a++) {
        int x = bc_cell(g, l - 1, 0, ci + a - 1), y = bc_cell(g, l - 1, 1, cj + bb - 1);
        int z = (D == 3) ? bc_cell(g, l - 1, 2, ck + c - 1) : 0;
        int32_t cs = g.idx[map_index(g, l - 1, x >> 3, y >> 3, z >> 3)];
        T val;
        if (cs < 0) {
          set_err(g, EB_TREE);
          val = nan_val<T>();
        } else {
          const long long off = (long long)cs * B + (x & 7) + 8 * (y & 7) + ((D == 3) ? 64 * (z & 7) : 0);
          val = A[off];
          if (C0base) {  // level l-1 interpolated in time, as for ghost cells
            const T a0 = C0base[(long long)v * g.cap * B + off];
            val = a0 + theta * (val - a0);
          }
        }
        P[a + 3 * (bb + 3 * c)] = val;
      }
  T si = (i & 1) ? T(-1) : T(1), sj = (j & 1) ? T(-1) : T(1), sk = (k & 1) ? T(-1) : T(1);
  return predict<T, D, 3>(P, 1, 1, (D == 3) ? 1 : 0, si, sj, sk);
}
// pressure of the same (possibly predicted) conserved state
template <typename T, int D>
__device__ T pres_ext(const Geo &g, int l, const T *__restrict__ A, int i, int j, int k,
                      const T *__restrict__ C0 = nullptr, T theta = T(0)) {
  T Q[D + 2];
  for (int v = 0; v < D + 2; v++) Q[v] = var_ext<T, D>(g, l, A, v, i, j, k, C0, theta);
  const T rho = Q[0];
  T vel[3] = {T(0), T(0), T(0)};
  for (int d = 0; d < D; d++) vel[d] = Q[1 + d] / rho;
  const T vv = ((vel[0] * vel[0]) + (vel[1] * vel[1])) + (vel[2] * vel[2]);
  return T(g.gamma - 1.0) * (Q[D + 1] - ((T(0.5) * rho) * vv));
}

// Block flag (before clustering) of every existing block of level l < L: a cell
// within one cell of the block (and inside the domain) has
// |rho(Q_{i+alpha}) - rho(Q_i)| > eps_w, or with eps_p > 0
// |p(Q_{i+alpha}) - p(Q_i)| > eps_p, for some alpha in {0,1}^d \ {0}.
template <typename T, int D>
// Levels l0..L-1 only; with A0 set, the absent cells of level l0 are predicted
// from level l0-1 interpolated in time, A0 + theta (A - A0) (a remesh inside the
// level recursion, where level l0-1 is at another time).
__global__ void k_gradflags(Geo g, const T *__restrict__ A, T epsw, T epsp, uint8_t *gflag, int l0,
                            const T *__restrict__ A0, T theta) {
  constexpr int EXT = 11;  // relative cells -1 .. 9
  constexpr int NP = (D == 2) ? EXT * EXT : EXT * EXT * EXT;
  __shared__ T rp[NP], pp[NP];
  const bool use_p = epsp > T(0);
  int b, e;
  if (g.L < 1 || l0 > g.L - 1) return;
  list_range(g, LK_EXIST, l0, g.L - 1, b, e);
  const long long cap = g.cap;
  for (int it = b + blockIdx.x; it < e; it += gridDim.x) {
    int s = g.lists[LK_EXIST * cap + it];
    int l = g.slot_level[s];
    int bc3[3] = {g.slot_coord[3 * s], g.slot_coord[3 * s + 1], g.slot_coord[3 * s + 2]};
    __syncthreads();
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
      int r[3] = {p % EXT - 1, (p / EXT) % EXT - 1, (D == 3) ? p / (EXT * EXT) - 1 : 0};
      int gc[3];
      for (int d = 0; d < 3; d++) gc[d] = (d < D) ? bc_cell(g, l, d, 8 * bc3[d] + r[d]) : 0;
      const T *C0 = (l == l0) ? A0 : nullptr;
      rp[p] = var_ext<T, D>(g, l, A, 0, gc[0], gc[1], gc[2], C0, theta);
      if (use_p) pp[p] = pres_ext<T, D>(g, l, A, gc[0], gc[1], gc[2], C0, theta);
    }
    __syncthreads();
    int hit = 0;
    constexpr int NC = (D == 2) ? 100 : 1000;  // cells -1 .. 8
    for (int q = threadIdx.x; q < NC && !hit; q += blockDim.x) {
      int r[3] = {q % 10 - 1, (q / 10) % 10 - 1, (D == 3) ? q / 100 - 1 : 0};
      bool inside = true;
      for (int d = 0; d < D; d++) {
        int gcd = 8 * bc3[d] + r[d];
        if (g.bc != 1 && (gcd < 0 || gcd >= g.nb[l][d] * 8)) inside = false;
      }
      if (!inside) continue;
      int p0 = (r[0] + 1) + EXT * ((r[1] + 1) + ((D == 3) ? EXT * (r[2] + 1) : 0));
      T r0 = rp[p0];
      for (int al = 1; al < (1 << D); al++) {
        int pa = p0 + (al & 1) + EXT * (((al >> 1) & 1) + ((D == 3) ? EXT * ((al >> 2) & 1) : 0));
        if (fabs(rp[pa] - r0) > epsw) hit = 1;
        if (use_p && fabs(pp[pa] - pp[p0]) > epsp) hit = 1;
      }
    }
    hit = __syncthreads_or(hit);
    if (threadIdx.x == 0) gflag[map_index(g, l, bc3[0], bc3[1], bc3[2])] = (uint8_t)(hit ? 1 : 0);
  }
}

}  // namespace mrfv
