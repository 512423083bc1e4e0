// Device helpers: indexing, boundary rule, list ranges, coarse patches and the
// third-order multiresolution prediction (Section 2.1 of arXiv:1603.05211).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"

namespace mrfv {

__device__ __forceinline__ long long map_index(const Geo &g, int l, int bx, int by, int bz) {
  return g.mapoff[l] + (long long)bx + (long long)g.nb[l][0] * ((long long)by + (long long)g.nb[l][1] * bz);
}

// Boundary rule on a cell coordinate of level l: transmissive = nearest interior
// cell (zero-gradient copy into every ghost layer), periodic = wrap.
__device__ __forceinline__ int bc_cell(const Geo &g, int l, int d, int i) {
  int N = g.nb[l][d] * BS;
  if (g.bc == 1) {
    i %= N;
    if (i < 0) i += N;
    return i;
  }
  return i < 0 ? 0 : (i >= N ? N - 1 : i);
}

// neighbouring block coordinate with the boundary rule, -1 outside a transmissive domain
__device__ __forceinline__ int bc_block(const Geo &g, int l, int d, int b) {
  if (d >= g.dim) return b == 0 ? 0 : -1;
  int N = g.nb[l][d];
  if (g.bc == 1) {
    b %= N;
    if (b < 0) b += N;
    return b;
  }
  return (b < 0 || b >= N) ? -1 : b;
}

// needed-block marks: the 3^d-1 neighbours (boundary rule) and the children of a block
__device__ __forceinline__ void mark_nbrs(const Geo &g, uint8_t *need, int l, int bx, int by, int bz) {
  int z0 = g.dim == 3 ? -1 : 0, z1 = g.dim == 3 ? 1 : 0;
  for (int c = z0; c <= z1; c++)
    for (int b = -1; b <= 1; b++)
      for (int a = -1; a <= 1; a++) {
        int x = bc_block(g, l, 0, bx + a), y = bc_block(g, l, 1, by + b), z = bc_block(g, l, 2, bz + c);
        if (x < 0 || y < 0 || z < 0) continue;
        need[map_index(g, l, x, y, z)] = 1;
      }
}
__device__ __forceinline__ void mark_children(const Geo &g, uint8_t *need, int l, int bx, int by, int bz) {
  int kz = g.dim == 3 ? 2 : 1;
  for (int c = 0; c < kz; c++)
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++)
        need[map_index(g, l + 1, 2 * bx + a, 2 * by + b, g.dim == 3 ? 2 * bz + c : 0)] = 1;
}

// Range [begin, end) of list `kind` over levels l0..l1.
__device__ __forceinline__ void list_range(const Geo &g, int kind, int l0, int l1, int &b, int &e) {
  b = g.loff[kind * (MAXL + 2) + l0];
  e = g.loff[kind * (MAXL + 2) + l1 + 1];
}

__device__ __forceinline__ void set_err(const Geo &g, int bits) { atomicOr(g.err, bits); }

// Gather the coarse cells [o_d, o_d + EXT) (per dimension, level lc) of the
// buffer A into patch[v][p], p = x + EXT*(y + EXT*z).  With A0 != null the
// value is the linear time interpolation A0 + theta*(A - A0).  A coarse cell
// whose block does not exist marks the tree error and reads NaN.
template <typename T, int D, int EXT>
__device__ void gather_patch(const Geo &g, int lc, const T *__restrict__ A, const T *__restrict__ A0, T theta,
                             int o0, int o1, int o2, T *patch, int tid, int nthr) {
  constexpr int NP = (D == 2) ? EXT * EXT : EXT * EXT * EXT;
  constexpr int NB = (D == 2) ? 64 : 512;
  const long long cap = g.cap;
  for (int p = tid; p < NP; p += nthr) {
    int x = p % EXT, y = (p / EXT) % EXT, z = (D == 3) ? p / (EXT * EXT) : 0;
    int cx = bc_cell(g, lc, 0, o0 + x), cy = bc_cell(g, lc, 1, o1 + y), cz = (D == 3) ? bc_cell(g, lc, 2, o2 + z) : 0;
    int32_t s = g.idx[map_index(g, lc, cx >> 3, cy >> 3, cz >> 3)];
    int c = (cx & 7) + 8 * (cy & 7) + (D == 3 ? 64 * (cz & 7) : 0);
    for (int v = 0; v < D + 2; v++) {
      T val;
      if (s < 0) {
        val = T(__int_as_float(0x7fc00000));
        if (v == 0) set_err(g, EB_TREE);
      } else {
        long long off = ((long long)v * cap + s) * NB + c;
        val = A[off];
        if (A0) {
          T a0 = A0[off];
          val = a0 + theta * (val - a0);
        }
      }
      patch[v * NP + p] = val;
    }
  }
}

// gather_patch for the ghost strips between the stages of the MR step: a coarse
// cell whose block is refined takes the projection of its 2^d children (the sums
// of the level projection, in its order), read from level lc+1, in place of its
// stored value, which is projected only later.  (A coarse cell over a refined
// child is projected from that child's stale values; the prediction never reads
// such a cell: in a graded tree the blocks next to an absent position are leaves.)
template <typename T, int D, int EXT>
__device__ void gather_patch_proj(const Geo &g, int lc, const T *__restrict__ A, int o0, int o1, int o2, T *patch,
                                  int tid, int nthr) {
  constexpr int NP = (D == 2) ? EXT * EXT : EXT * EXT * EXT;
  constexpr int NB = (D == 2) ? 64 : 512;
  const long long cap = g.cap;
  for (int p = tid; p < NP; p += nthr) {
    int x = p % EXT, y = (p / EXT) % EXT, z = (D == 3) ? p / (EXT * EXT) : 0;
    int cx = bc_cell(g, lc, 0, o0 + x), cy = bc_cell(g, lc, 1, o1 + y), cz = (D == 3) ? bc_cell(g, lc, 2, o2 + z) : 0;
    int32_t s = g.idx[map_index(g, lc, cx >> 3, cy >> 3, cz >> 3)];
    // the child of level lc+1 holding this cell's children (absent under a leaf)
    int32_t cs = g.idx[map_index(g, lc + 1, cx >> 2, cy >> 2, cz >> 2)];
    int c = (cx & 7) + 8 * (cy & 7) + (D == 3 ? 64 * (cz & 7) : 0);
    int f = 2 * (cx & 3) + 16 * (cy & 3) + (D == 3 ? 128 * (cz & 3) : 0);
    for (int v = 0; v < D + 2; v++) {
      T val;
      if (s < 0) {
        val = T(__int_as_float(0x7fc00000));
        if (v == 0) set_err(g, EB_TREE);
      } else if (cs >= 0) {
        const T *C = A + ((long long)v * cap + cs) * NB + f;
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
        val = sum * T(D == 2 ? 0.25 : 0.125);
      } else {
        val = A[((long long)v * cap + s) * NB + c];
      }
      patch[v * NP + p] = val;
    }
  }
}

// Third-order prediction of the fine cell whose parent is patch cell
// (x, y, z): tensor product of the 1D rule Q_k +/- (Q_{k-1} - Q_{k+1})/8 (+ for
// the even child).  Evaluation order: Q_k, the first-order terms in direction
// order, the mixed pairs 12, 13, 23, then the triple term; each difference is
// formed left to right as written.  P points at one variable of the patch.
template <typename T, int D, int EXT>
__device__ __forceinline__ T predict(const T *P, int x, int y, int z, T si, T sj, T sk) {
  auto at = [&](int a, int b, int c) -> T {
    return (D == 2) ? P[(x + a) + EXT * (y + b)] : P[(x + a) + EXT * ((y + b) + EXT * (z + c))];
  };
  const T e1 = T(0.125), e2 = T(0.015625), e3 = T(0.001953125);
  if (D == 2) {
    T q = at(0, 0, 0);
    T d1 = at(-1, 0, 0) - at(1, 0, 0);
    T d2 = at(0, -1, 0) - at(0, 1, 0);
    T d12 = ((at(-1, -1, 0) - at(1, -1, 0)) - at(-1, 1, 0)) + at(1, 1, 0);
    T r = q + (si * e1) * d1;
    r = r + (sj * e1) * d2;
    r = r + ((si * sj) * e2) * d12;
    return r;
  } else {
    T q = at(0, 0, 0);
    T d1 = at(-1, 0, 0) - at(1, 0, 0);
    T d2 = at(0, -1, 0) - at(0, 1, 0);
    T d3 = at(0, 0, -1) - at(0, 0, 1);
    T d12 = ((at(-1, -1, 0) - at(1, -1, 0)) - at(-1, 1, 0)) + at(1, 1, 0);
    T d13 = ((at(-1, 0, -1) - at(1, 0, -1)) - at(-1, 0, 1)) + at(1, 0, 1);
    T d23 = ((at(0, -1, -1) - at(0, 1, -1)) - at(0, -1, 1)) + at(0, 1, 1);
    T elo = ((at(-1, -1, -1) - at(1, -1, -1)) - at(-1, 1, -1)) + at(1, 1, -1);
    T ehi = ((at(-1, -1, 1) - at(1, -1, 1)) - at(-1, 1, 1)) + at(1, 1, 1);
    T d123 = elo - ehi;
    T r = q + (si * e1) * d1;
    r = r + (sj * e1) * d2;
    r = r + (sk * e1) * d3;
    r = r + ((si * sj) * e2) * d12;
    r = r + ((si * sk) * e2) * d13;
    r = r + ((sj * sk) * e2) * d23;
    r = r + (((si * sj) * sk) * e3) * d123;
    return r;
  }
}

// Per-level step table (computed once per step, in double): dt_l = dt (global) or
// dt * 2^(L-l) (level-dependent steps); for each stage coefficient c (1/2, 1)
// (c dt_l) / dx_{l,n}; and its single-precision copy.
// One entry (level l, stage st) of the table.
__device__ inline void level_params_entry(const Geo &g, double dt, int lts, double *lev, float *levf, int l, int st) {
  double dtl = lts ? ldexp(dt, g.L - l) : dt;
  double coef = st == 0 ? 0.5 : 1.0;
  for (int n = 0; n < 3; n++) lev[lev_index(st, l, n)] = (coef * dtl) / g.dx[l][n];
  lev[lev_index(st, l, 3)] = dtl;
  for (int k = 0; k < 4; k++) levf[lev_index(st, l, k)] = (float)lev[lev_index(st, l, k)];
}
__device__ inline void level_params_dev(const Geo &g, double dt, int lts, double *lev, float *levf) {
  for (int l = 0; l <= g.L; l++)
    for (int st = 0; st < 2; st++) level_params_entry(g, dt, lts, lev, levf, l, st);
}

template <typename T>
__device__ __forceinline__ T nan_val() {
  return T(__int_as_float(0x7fc00000));
}

}  // namespace mrfv
