// Fused finite-volume stage kernel: MUSCL reconstruction with the van Albada
// limiter, the AUSM+ flux and the conservative RK2 stage update
// (arXiv:1603.05211, Section 2), one flux per face of each 8^d block, plus the
// CFL time-step reduction.
//
// A CTA stages BPC blocks in shared memory: each block's interior and the two
// cell layers beyond each face, read straight from the same-level neighbour's
// interior (nbr >= 0), from the block's ghost strip (coarse-fine face, filled by
// the prediction kernel) or, at a transmissive wall, from the block's own edge
// cells.  Conservative -> primitive once per staged cell; then, direction by
// direction: limited slopes -> face states, AUSM+ on every face, and the
// residual of each interior cell accumulates in registers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"

namespace mrfv {


// van Albada slope with the TVD clip: a b (a + b) / (a^2 + b^2) when a b > 0, else 0.
template <typename T>
__device__ __forceinline__ T van_albada(T a, T b) {
  T ab = a * b;
  if (ab > T(0)) return (ab * (a + b)) / ((a * a) + (b * b));
  return T(0);
}

// AUSM+ split Mach numbers (beta = 1/8) and pressures (alpha = 3/16), Liou 1996.
template <typename T>
__device__ __forceinline__ T mach4_plus(T M) {
  if (fabs(M) >= T(1)) return T(0.5) * (M + fabs(M));
  T t = M + T(1), u = (M * M) - T(1);
  return (T(0.25) * (t * t)) + (T(0.125) * (u * u));
}
template <typename T>
__device__ __forceinline__ T mach4_minus(T M) {
  if (fabs(M) >= T(1)) return T(0.5) * (M - fabs(M));
  T t = M - T(1), u = (M * M) - T(1);
  return (T(-0.25) * (t * t)) - (T(0.125) * (u * u));
}
template <typename T>
__device__ __forceinline__ T pres5_plus(T M) {
  if (fabs(M) >= T(1)) return M > T(0) ? T(1) : T(0);
  T t = M + T(1), u = (M * M) - T(1);
  return ((T(0.25) * (t * t)) * (T(2) - M)) + ((T(0.1875) * M) * (u * u));
}
template <typename T>
__device__ __forceinline__ T pres5_minus(T M) {
  if (fabs(M) >= T(1)) return M < T(0) ? T(1) : T(0);
  T t = M - T(1), u = (M * M) - T(1);
  return ((T(0.25) * (t * t)) * (T(2) + M)) - ((T(0.1875) * M) * (u * u));
}

// AUSM+ flux across a face with normal n from primitive face states
// (rho, v_1..v_D, p); interface sound speed = arithmetic mean.
template <typename T, int D>
__device__ __forceinline__ void ausm_plus(int n, const T *wl, const T *wr, T g, T goverg1, T *F) {
  T cl = sqrt((g * wl[D + 1]) / wl[0]);
  T cr = sqrt((g * wr[D + 1]) / wr[0]);
  T ch = T(0.5) * (cl + cr);
  T ml = wl[1 + n] / ch;
  T mr = wr[1 + n] / ch;
  T m = mach4_plus(ml) + mach4_minus(mr);
  T ph = (pres5_plus(ml) * wl[D + 1]) + (pres5_minus(mr) * wr[D + 1]);
  T a = ch * m;
  const T *wu = (m >= T(0)) ? wl : wr;
  T vv = (wu[1] * wu[1]) + (wu[2] * wu[2]);
  if (D == 3) vv = vv + (wu[3] * wu[3]);
  T rhoH = (goverg1 * wu[D + 1]) + ((T(0.5) * wu[0]) * vv);
  T fr = a * wu[0];
  F[0] = fr;
#pragma unroll
  for (int d = 0; d < D; d++) {
    T f = fr * wu[1 + d];
    if (d == n) f = f + ph;
    F[1 + d] = f;
  }
  F[D + 1] = a * rhoH;
}

template <typename T, int D>
__device__ __forceinline__ void cons_to_prim(const T *Q, T gm1, T *w) {
  T rho = Q[0];
  T v[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int d = 0; d < D; d++) v[d] = Q[1 + d] / rho;
  T vv = (v[0] * v[0]) + (v[1] * v[1]);
  if (D == 3) vv = vv + (v[2] * v[2]);
  w[0] = rho;
#pragma unroll
  for (int d = 0; d < D; d++) w[1 + d] = v[d];
  w[D + 1] = gm1 * (Q[D + 1] - ((T(0.5) * rho) * vv));
}

template <int D>
struct FVShape {
  static constexpr int B = (D == 2) ? 64 : 512;        // interior cells
  static constexpr int TF = (D == 2) ? 8 : 64;         // cells of one face layer
  static constexpr int NV = D + 2;
  static constexpr int TILE = (D == 2) ? 144 : 1728;   // 12^d staging box (corners unused)
  static constexpr int NF = 9 * TF;                    // faces per direction
  static constexpr int STRIP = 2 * D * 2 * TF;         // ghost cells (two layers per face)
  static constexpr int BPC = (D == 2) ? 4 : 1;         // blocks per CTA
  static constexpr int NT = B * BPC;                   // threads per CTA
};

template <typename T, int D>
constexpr size_t fv_smem_bytes() {
  using S = FVShape<D>;
  return (size_t)S::BPC * (S::NV * S::TILE + 3 * S::NV * S::NF) * sizeof(T);
}

__device__ __forceinline__ int tile_pos(int D, int x, int y, int z) {
  return (D == 2) ? (x + 2) + 12 * (y + 2) : (x + 2) + 12 * ((y + 2) + 12 * (z + 2));
}

template <typename T, int D>
__global__ void __launch_bounds__(FVShape<D>::NT) k_fv(Geo g, FVArgs<T> a) {
  using S = FVShape<D>;
  constexpr int B = S::B, TF = S::TF, NV = S::NV, TILE = S::TILE, NF = S::NF, BPC = S::BPC;
  extern __shared__ unsigned char smem_raw[];
  const int sub = threadIdx.x / B, tid = threadIdx.x % B;
  T *tile = reinterpret_cast<T *>(smem_raw) + (size_t)sub * (NV * TILE + 3 * NV * NF);
  T *WL = tile + NV * TILE;
  T *WR = WL + NV * NF;
  T *FX = WR + NV * NF;
  const long long cap = g.cap;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0), goverg1 = T(g.gamma / (g.gamma - 1.0));
  const int cx = tid & 7, cy = (tid >> 3) & 7, cz = (D == 3) ? (tid >> 6) : 0;
  const double dtf = *a.dt;
  int lb, le;
  list_range(g, a.kind, a.l0, a.l1, lb, le);
  if (a.bytes && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(a.bytes, (unsigned long long)(le - lb) * B * a.words * sizeof(T));

  for (int i0 = lb + blockIdx.x * BPC; i0 < le; i0 += gridDim.x * BPC) {
    const int i = i0 + sub;
    const bool active = i < le;
    const int s = active ? g.lists[a.kind * cap + i] : 0;
    const int l = active ? g.slot_level[s] : 0;
    const double dtl = a.lts ? ldexp(dtf, g.L - l) : dtf;
    __syncthreads();
    // ---- stage the block and its face layers as primitive variables
    if (active) {
      for (int it = tid; it < B + S::STRIP; it += B) {
        T Q[NV], w[NV];
        int pos;
        if (it < B) {
          int x = it & 7, y = (it >> 3) & 7, z = (D == 3) ? (it >> 6) : 0;
          pos = tile_pos(D, x, y, z);
#pragma unroll
          for (int v = 0; v < NV; v++) Q[v] = a.Uin[((long long)v * cap + s) * B + it];
        } else {
          int q = it - B;
          int f = q / (2 * TF), dd = (q / TF) & 1, t = q % TF;
          int n = f >> 1, side = f & 1;
          int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
          int rel[3], src[3];
          rel[t1] = t & 7;
          rel[t2] = (D == 3) ? (t >> 3) : 0;
          src[t1] = rel[t1];
          src[t2] = rel[t2];
          rel[n] = side ? 8 + dd : -1 - dd;
          pos = tile_pos(D, rel[0], rel[1], rel[2]);
          int nb = g.nbr[6 * s + f];
          if (nb == NBR_MISSING) {
#pragma unroll
            for (int v = 0; v < NV; v++) Q[v] = a.G[((long long)v * cap + s) * S::STRIP + q];
          } else {
            int from;
            if (nb >= 0) {
              src[n] = side ? dd : 7 - dd;
              from = nb;
            } else {  // transmissive wall: the block's own edge cell
              src[n] = side ? 7 : 0;
              from = s;
            }
            int c = src[0] + 8 * src[1] + (D == 3 ? 64 * src[2] : 0);
#pragma unroll
            for (int v = 0; v < NV; v++) Q[v] = a.Uin[((long long)v * cap + from) * B + c];
          }
        }
        cons_to_prim<T, D>(Q, gm1, w);
#pragma unroll
        for (int v = 0; v < NV; v++) tile[v * TILE + pos] = w[v];
      }
    }
    __syncthreads();

    T r[NV];
#pragma unroll
    for (int n = 0; n < D; n++) {
      const int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
      const int stride = (n == 0) ? 1 : (n == 1 ? 12 : 144);
      // ---- limited slopes -> face states; pencil cell p in [-1, 8] along n
      if (active) {
        for (int it = tid; it < 10 * TF; it += B) {
          int p = it % 10 - 1, t = it / 10;
          int c3[3];
          c3[n] = p;
          c3[t1] = t & 7;
          c3[t2] = (D == 3) ? (t >> 3) : 0;
          int pos = tile_pos(D, c3[0], c3[1], c3[2]);
#pragma unroll
          for (int v = 0; v < NV; v++) {
            T wm = tile[v * TILE + pos - stride], w0 = tile[v * TILE + pos], wp = tile[v * TILE + pos + stride];
            T sl = van_albada<T>(w0 - wm, wp - w0);
            if (p >= 0) WR[v * NF + p + 9 * t] = w0 - T(0.5) * sl;
            if (p <= 7) WL[v * NF + (p + 1) + 9 * t] = w0 + T(0.5) * sl;
          }
        }
      }
      __syncthreads();
      // ---- AUSM+ on every face of direction n; face k lies between cells k-1 and k
      if (active) {
        for (int it = tid; it < NF; it += B) {
          T wl[NV], wr[NV], F[NV];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            wl[v] = WL[v * NF + it];
            wr[v] = WR[v * NF + it];
          }
          ausm_plus<T, D>(n, wl, wr, gam, goverg1, F);
#pragma unroll
          for (int v = 0; v < NV; v++) FX[v * NF + it] = F[v];
          int k = it % 9;
          if (a.record && (k == 0 || k == 8)) {
            int f = 2 * n + (k == 8 ? 1 : 0), t = it / 9;
            bool fine = g.nbr[6 * s + f] == NBR_MISSING;
            bool coarse = (g.cmask[s] >> f) & 1;
            if (fine || coarse) {
              T dtT = T(dtl);
              T *R = a.FR + (long long)f * TF + t;
              bool add = fine && a.record == 2;
#pragma unroll
              for (int v = 0; v < NV; v++) {
                long long o = ((long long)v * cap + s) * (2 * D * TF);
                T val = dtT * F[v];
                R[o] = add ? R[o] + val : val;
              }
            }
          }
        }
      }
      __syncthreads();
      // ---- residual of this thread's cell: lambda_n (F_{k+1} - F_k)
      if (active) {
        const T lam = T((a.coef * dtl) / g.dx[l][n]);
        int c3[3] = {cx, cy, cz};
        int p = c3[n];
        int t = c3[t1] + ((D == 3) ? 8 * c3[t2] : 0);
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T dF = FX[v * NF + (p + 1) + 9 * t] - FX[v * NF + p + 9 * t];
          r[v] = (n == 0) ? lam * dF : r[v] + lam * dF;
        }
      }
    }
    if (active) {
#pragma unroll
      for (int v = 0; v < NV; v++) {
        long long o = ((long long)v * cap + s) * B + tid;
        a.Uout[o] = a.U0[o] - r[v];
      }
    }
  }
}

// CFL limit over the leaves: min over cells and directions of dx_{l,n} / (|v_n| + c),
// scaled by 2^(l-L) with level-dependent steps; rho <= 0, p <= 0 or NaN flags an error.
template <typename T, int D>
__global__ void k_dt(Geo g, const T *__restrict__ A, int lts, unsigned long long *red) {
  constexpr int B = (D == 2) ? 64 : 512;
  int b, e;
  list_range(g, LK_LEAF, 0, g.L, b, e);
  const long long cap = g.cap;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0);
  T best = T(INFINITY);
  bool bad = false;
  for (long long t = (long long)b * B + blockIdx.x * blockDim.x + threadIdx.x; t < (long long)e * B;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[LK_LEAF * cap + i];
    int l = g.slot_level[s];
    T Q[D + 2], w[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; v++) Q[v] = A[((long long)v * cap + s) * B + c];
    cons_to_prim<T, D>(Q, gm1, w);
    if (!(w[0] > T(0)) || !(w[D + 1] > T(0))) {
      bad = true;
      continue;
    }
    T cs = sqrt((gam * w[D + 1]) / w[0]);
#pragma unroll
    for (int d = 0; d < D; d++) {
      T rr = T(g.dx[l][d]) / (fabs(w[1 + d]) + cs);
      if (lts) rr = ldexp(rr, l - g.L);
      if (rr < best) best = rr;
    }
  }
  if (bad) set_err(g, EB_NONPHYS);
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(0xffffffffu, best, o);
    if (x < best) best = x;
  }
  if ((threadIdx.x & 31) == 0 && best < T(INFINITY))
    atomicMin(red, (unsigned long long)__double_as_longlong((double)best));
}

}  // namespace mrfv
