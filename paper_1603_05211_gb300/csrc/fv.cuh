// Finite-volume stage kernel of the MR scheme: MUSCL reconstruction of the
// primitive variables with the van Albada limiter, the AUSM+ flux and the
// conservative stage update of the explicit midpoint rule (arXiv:1603.05211,
// Section 2), one flux per face of each 8^d block; and the CFL time-step
// reduction.
//
// A CTA takes BPC blocks.  Each thread walks one line of cells of a block along
// one direction (the direction is a compile-time parameter of the walk), with
// the two cells beyond each face read from the same-level neighbour, the ghost
// strip of a coarse-fine face or, at a transmissive wall, the block's own edge
// cell; the flux differences of the lines go to shared memory, and a second
// pass sums them per cell in direction order into the update.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"

namespace mrfv {


// ---------------------------------------------------------------- arithmetic helpers
// Branches of the flux functions are written as selects of both sides, which
// give the same values as the branches.
template <typename L>
__device__ __forceinline__ L lsel(bool m, L a, L b) { return m ? a : b; }
__device__ __forceinline__ float labs(float a) { return fabsf(a); }
__device__ __forceinline__ double labs(double a) { return fabs(a); }
__device__ __forceinline__ float lsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double lsqrt(double a) { return sqrt(a); }
// a * b + c written as the product then the sum (the double-precision units are
// compiled without contraction, so both round as the oracle's expression does)
template <typename L>
__device__ __forceinline__ L lfma(L a, L b, L c) { return (a * b) + c; }

// van Albada slope with the TVD clip: a b (a + b) / (a^2 + b^2) when a b > 0, else 0.
template <typename L>
__device__ __forceinline__ L van_albada(L a, L b) {
  L ab = a * b;
  L r = (ab * (a + b)) / lfma(a, a, b * b);
  return lsel(ab > L(0.0f), r, L(0.0f));
}

// AUSM+ split Mach numbers (beta = 1/8) and pressures (alpha = 3/16), Liou 1996;
// |M| >= 1 takes the supersonic form.
template <typename L>
__device__ __forceinline__ L mach4_plus(L M) {
  L aM = labs(M);
  L sup = L(0.5f) * (M + aM);
  L t = M + L(1.0f), u = lfma(M, M, L(-1.0f));
  L sub = lfma(L(0.25f), t * t, L(0.125f) * (u * u));
  return lsel(aM >= L(1.0f), sup, sub);
}
template <typename L>
__device__ __forceinline__ L mach4_minus(L M) {
  L aM = labs(M);
  L sup = L(0.5f) * (M - aM);
  L t = M - L(1.0f), u = lfma(M, M, L(-1.0f));
  L sub = (L(-0.25f) * (t * t)) - (L(0.125f) * (u * u));
  return lsel(aM >= L(1.0f), sup, sub);
}
template <typename L>
__device__ __forceinline__ L pres5_plus(L M) {
  L aM = labs(M);
  L sup = lsel(M > L(0.0f), L(1.0f), L(0.0f));
  L t = M + L(1.0f), u = lfma(M, M, L(-1.0f));
  L sub = lfma((L(0.25f) * (t * t)), (L(2.0f) - M), (L(0.1875f) * M) * (u * u));
  return lsel(aM >= L(1.0f), sup, sub);
}
template <typename L>
__device__ __forceinline__ L pres5_minus(L M) {
  L aM = labs(M);
  L sup = lsel(M < L(0.0f), L(1.0f), L(0.0f));
  L t = M - L(1.0f), u = lfma(M, M, L(-1.0f));
  L sub = ((L(0.25f) * (t * t)) * (L(2.0f) + M)) - ((L(0.1875f) * M) * (u * u));
  return lsel(aM >= L(1.0f), sup, sub);
}

// AUSM+ flux across a face with normal n from primitive face states
// (rho, v_1..v_D, p); interface sound speed = arithmetic mean.
template <typename L, int D>
__device__ __forceinline__ void ausm_plus(int n, const L *wl, const L *wr, L g, L goverg1, L *F) {
  L cl = lsqrt((g * wl[D + 1]) / wl[0]);
  L cr = lsqrt((g * wr[D + 1]) / wr[0]);
  L ch = L(0.5f) * (cl + cr);
  L ml = wl[1 + n] / ch;
  L mr = wr[1 + n] / ch;
  L m = mach4_plus(ml) + mach4_minus(mr);
  L ph = lfma(pres5_plus(ml), wl[D + 1], pres5_minus(mr) * wr[D + 1]);
  L a = ch * m;
  const auto up = m >= L(0.0f);
  L wu[D + 2];
#pragma unroll
  for (int v = 0; v < D + 2; v++) wu[v] = lsel(up, wl[v], wr[v]);
  L vv = lfma(wu[1], wu[1], wu[2] * wu[2]);
  if (D == 3) vv = lfma(wu[3], wu[3], vv);
  L rhoH = lfma(goverg1, wu[D + 1], (L(0.5f) * wu[0]) * vv);
  L fr = a * wu[0];
  F[0] = fr;
#pragma unroll
  for (int d = 0; d < D; d++) F[1 + d] = (d == n) ? lfma(fr, wu[1 + d], ph) : fr * wu[1 + d];
  F[D + 1] = a * rhoH;
}

template <typename L, int D>
__device__ __forceinline__ void cons_to_prim(const L *Q, L gm1, L *w) {
  L rho = Q[0];
  L v[3] = {L(0.0f), L(0.0f), L(0.0f)};
#pragma unroll
  for (int d = 0; d < D; d++) v[d] = Q[1 + d] / rho;
  L vv = lfma(v[0], v[0], v[1] * v[1]);
  if (D == 3) vv = lfma(v[2], v[2], vv);
  w[0] = rho;
#pragma unroll
  for (int d = 0; d < D; d++) w[1 + d] = v[d];
  w[D + 1] = gm1 * (Q[D + 1] - ((L(0.5f) * rho) * vv));
}

// Launch shape of the stage kernel for state type T in dimension D: BPC blocks per
// CTA, one thread per line of a block along each direction (SPLIT threads per
// line).
template <typename T, int D, int SPLIT = 1>
struct FVShape {
  static constexpr int B = (D == 2) ? 64 : 512;        // interior cells
  static constexpr int TF = (D == 2) ? 8 : 64;         // cells of one face layer = pencils per direction
  static constexpr int NV = D + 2;
  static constexpr int STRIP = 2 * D * 2 * TF;         // ghost cells (two layers per face)
  static constexpr int BPC = (D == 2) ? 16 : 1;       // blocks per CTA
  static constexpr int TPD = TF;                       // lines per block and direction
  static constexpr int NT = D * TPD * BPC * SPLIT;     // threads per CTA (SPLIT threads per pencil group)
  static constexpr int NK = SPLIT == 1 ? 9 : 5;        // faces per thread (the middle face twice when split)
  static constexpr int PY = (D == 2) ? 9 : 8;          // padded shared-memory cell index x + PY y + PZ z
  static constexpr int PZ = (D == 2) ? 0 : 69;         // (bank-conflict free pencil stores in 2D, 2-way in 3D)
  static constexpr int RS = (D == 2) ? 74 : 552;       // padded cells per (block, variable) in shared memory
};

// CTAs per SM the register allocation must allow (overridable for tuning)
#ifndef MRFV_FV_MINB32
#define MRFV_FV_MINB32 4
#endif
#ifndef MRFV_FV_MINB64
#define MRFV_FV_MINB64 2
#endif
template <typename T>
struct FVMinBlocks {
  static constexpr int value = sizeof(T) == 4 ? MRFV_FV_MINB32 : MRFV_FV_MINB64;
};

// step-table entry in the kernel's precision (no double -> float conversion per cell)
template <typename T>
__device__ __forceinline__ T lev_at(const FVArgs<T> &a, int i) {
  if constexpr (sizeof(T) == 4) return a.levf[i];
  else return a.lev[i];
}

template <typename T, int D, int SPLIT = 1>
constexpr size_t fv_smem_bytes() {
  using S = FVShape<T, D, SPLIT>;
  return (size_t)D * S::BPC * S::NV * S::RS * sizeof(T);
}

// One pencil pass along direction N (compile-time: strides and the normal
// component are constants) for half HALF of the line (SPLIT = 2: faces 0..4 or
// 4..8, the middle face evaluated by both halves) or the whole line (SPLIT = 1).
// The line's cells come from the block itself, from beyond each face the
// same-level neighbour's cells, the ghost strip (coarse-fine face) or, at a
// transmissive wall, the block's own edge cell; each source is resolved once per
// line.  Primitives move through a sliding window; each cell's limited slope is
// formed once, then the two face states and the AUSM+ flux of each face; the
// flux difference F_{k+1} - F_k of every interior cell goes to shared memory
// (and dt_l F to the flux registers on the faces the correction needs).
template <typename T, int D, int SPLIT, int N, int HALF>
__device__ __forceinline__ void fv_pencil(const Geo &g, const FVArgs<T> &a, int s, int l, int t0, T *dF, T gam,
                                          T gm1, T goverg1) {
  using S = FVShape<T, D, SPLIT>;
  constexpr int B = S::B, TF = S::TF, NV = S::NV, RS = S::RS, NK = S::NK;
  constexpr int KB = HALF * 4;                                        // first face of this thread
  constexpr int STRIDE = (N == 0) ? 1 : (N == 1 ? 8 : 64);            // cell stride along N
  constexpr int SSTR = (N == 0) ? 1 : (N == 1 ? S::PY : S::PZ);       // shared-memory stride along N
  const long long cap = g.cap;
  const long long vsU = cap * B, vsG = cap * S::STRIP;
  const int t1 = t0 & 7, t2 = t0 >> 3;
  const int base = (N == 0) ? (8 * t1 + 64 * t2) : (N == 1 ? (t1 + 64 * t2) : (t1 + 8 * t2));
  const int sbase = (N == 0) ? (S::PY * t1 + S::PZ * t2) : (N == 1 ? (t1 + S::PZ * t2) : (t1 + S::PY * t2));
  const int nb_lo = g.nbr[6 * s + 2 * N], nb_hi = g.nbr[6 * s + 2 * N + 1];
  // sources: position p in 0..7 at mid + p STRIDE; position -1-dd at lo + dd lo_step;
  // position 8+dd at hi + dd hi_step (variable v one plane stride further)
  const T *mid = a.Uin + (long long)s * B + base;
  const T *lo, *hi;
  long long lo_vs = vsU, hi_vs = vsU;
  int lo_step, hi_step;
  if (nb_lo == NBR_MISSING) {
    lo = a.G + (long long)s * S::STRIP + (2 * N) * 2 * TF + t0;
    lo_vs = vsG;
    lo_step = TF;
  } else if (nb_lo >= 0) {
    lo = a.Uin + (long long)nb_lo * B + base + 7 * STRIDE;
    lo_step = -STRIDE;
  } else {
    lo = mid;
    lo_step = 0;
  }
  if (nb_hi == NBR_MISSING) {
    hi = a.G + (long long)s * S::STRIP + (2 * N + 1) * 2 * TF + t0;
    hi_vs = vsG;
    hi_step = TF;
  } else if (nb_hi >= 0) {
    hi = a.Uin + (long long)nb_hi * B + base;
    hi_step = STRIDE;
  } else {
    hi = mid + 7 * STRIDE;
    hi_step = 0;
  }
  auto load = [&](int p, T *w) {
    const T *q;
    long long vs;
    if (p < 0) {
      q = lo + (-1 - p) * lo_step;
      vs = lo_vs;
    } else if (p > 7) {
      q = hi + (p - 8) * hi_step;
      vs = hi_vs;
    } else {
      q = mid + p * STRIDE;
      vs = vsU;
    }
    T Q[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) Q[v] = q[v * vs];
    cons_to_prim<T, D>(Q, gm1, w);
  };
  const bool rec_lo = a.record && KB == 0 && (nb_lo == NBR_MISSING || ((g.cmask[s] >> (2 * N)) & 1));
  const bool rec_hi = a.record && KB + NK == 9 && (nb_hi == NBR_MISSING || ((g.cmask[s] >> (2 * N + 1)) & 1));
  const bool add_lo = a.record == 2 && nb_lo == NBR_MISSING;
  const bool add_hi = a.record == 2 && nb_hi == NBR_MISSING;
  const T dtT = lev_at(a, lev_index(a.stage, l, 3));
  // sliding window of primitives: wb = cell k-1, wc = cell k (face k lies between them)
  T wb[NV], wc[NV], slo[NV], Fprev[NV];
  {
    T wa[NV];
    load(KB - 2, wa);
    load(KB - 1, wb);
    load(KB, wc);
#pragma unroll
    for (int v = 0; v < NV; v++) slo[v] = van_albada<T>(wb[v] - wa[v], wc[v] - wb[v]);
  }
#pragma unroll
  for (int kk = 0; kk < NK; kk++) {
    const int k = KB + kk;
    T wd[NV], wl[NV], wr[NV], shi[NV], F[NV];
    load(k + 1, wd);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      shi[v] = van_albada<T>(wc[v] - wb[v], wd[v] - wc[v]);
      wl[v] = lfma(T(0.5), slo[v], wb[v]);
      wr[v] = wc[v] - T(0.5) * shi[v];
    }
    ausm_plus<T, D>(N, wl, wr, gam, goverg1, F);
    if ((k == 0 && rec_lo) || (k == 8 && rec_hi)) {
      const int side = k == 8 ? 1 : 0;
      const bool add = side ? add_hi : add_lo;
      T *R = a.FR + (long long)s * (2 * D * TF) + (2 * N + side) * TF + t0;
      const long long vsR = cap * (2 * D * TF);
#pragma unroll
      for (int v = 0; v < NV; v++) {
        T val = dtT * F[v];
        R[v * vsR] = add ? R[v * vsR] + val : val;
      }
    }
    if (kk > 0) {
#pragma unroll
      for (int v = 0; v < NV; v++) dF[v * RS + sbase + (k - 1) * SSTR] = F[v] - Fprev[v];
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      Fprev[v] = F[v];
      slo[v] = shi[v];
      wb[v] = wc[v];
      wc[v] = wd[v];
    }
  }
}

// Finite-volume stage over the blocks of a work list: one thread per line of a
// block along each direction (SPLIT = 2: two threads per line), then a second
// pass applies Q_out = Q_0 - (lambda_1 dF_1 + lambda_2 dF_2 [+ lambda_3 dF_3]),
// summed in direction order, to every cell.
template <typename T, int D, int SPLIT>
__global__ void __launch_bounds__(FVShape<T, D, SPLIT>::NT,
                                  (FVMinBlocks<T>::value / SPLIT > 0 ? FVMinBlocks<T>::value / SPLIT : 1))
    k_fv(Geo g, FVArgs<T> a) {
  using S = FVShape<T, D, SPLIT>;
  constexpr int B = S::B, NV = S::NV, BPC = S::BPC, RS = S::RS, NT = S::NT, TPD = S::TPD;
  extern __shared__ unsigned char smem_raw[];
  T *dFs = reinterpret_cast<T *>(smem_raw);  // [dir][block][v][RS]
  __shared__ int sslot[BPC];
  __shared__ T slam[BPC][3];
  const long long cap = g.cap;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0), goverg1 = T(g.gamma / (g.gamma - 1.0));
  // line of this thread: direction-major so a warp shares one direction
  const int n = threadIdx.x / (TPD * BPC * SPLIT);
  const int j = (threadIdx.x / (TPD * SPLIT)) % BPC;
  const int half = (threadIdx.x / TPD) % SPLIT;
  const int t0 = threadIdx.x % TPD;
  int lb, le;
  list_range(g, a.kind, a.l0, a.l1, lb, le);
  if (a.bytes && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(a.bytes, (unsigned long long)(le - lb) * B * a.words * sizeof(T));

  for (int i0 = lb + blockIdx.x * BPC; i0 < le; i0 += gridDim.x * BPC) {
    // ---------------- pencil pass
    {
      const int i = i0 + j;
      if (i < le) {
        const int s = g.lists[a.kind * cap + i];
        const int l = g.slot_level[s];
        if (n == 0 && half == 0 && t0 == 0) {
          sslot[j] = s;
#pragma unroll
          for (int d = 0; d < 3; d++) slam[j][d] = lev_at(a, lev_index(a.stage, l, d));
        }
        T *dF = dFs + ((size_t)(n * BPC + j) * NV) * RS;
        if (n == 0) {
          if (SPLIT == 2 && half) fv_pencil<T, D, SPLIT, 0, (SPLIT == 2 ? 1 : 0)>(g, a, s, l, t0, dF, gam, gm1, goverg1);
          else fv_pencil<T, D, SPLIT, 0, 0>(g, a, s, l, t0, dF, gam, gm1, goverg1);
        } else if (n == 1) {
          if (SPLIT == 2 && half) fv_pencil<T, D, SPLIT, 1, (SPLIT == 2 ? 1 : 0)>(g, a, s, l, t0, dF, gam, gm1, goverg1);
          else fv_pencil<T, D, SPLIT, 1, 0>(g, a, s, l, t0, dF, gam, gm1, goverg1);
        } else if constexpr (D == 3) {
          if (SPLIT == 2 && half) fv_pencil<T, D, SPLIT, 2, (SPLIT == 2 ? 1 : 0)>(g, a, s, l, t0, dF, gam, gm1, goverg1);
          else fv_pencil<T, D, SPLIT, 2, 0>(g, a, s, l, t0, dF, gam, gm1, goverg1);
        }
      }
    }
    __syncthreads();
    // ---------------- update pass
    const long long vsU = cap * B;
    for (int q = threadIdx.x; q < BPC * B; q += NT) {
      const int jj = q / B, c = q % B;
      if (i0 + jj >= le) break;
      const int s = sslot[jj];
      const int cp = (c & 7) + S::PY * ((c >> 3) & 7) + S::PZ * (c >> 6);
      const T lam0 = slam[jj][0], lam1 = slam[jj][1], lam2 = slam[jj][2];
      const long long o = (long long)s * B + c;
#pragma unroll
      for (int v = 0; v < NV; v++) {
        T r = lam0 * dFs[((size_t)(0 * BPC + jj) * NV + v) * RS + cp];
        r = r + lam1 * dFs[((size_t)(1 * BPC + jj) * NV + v) * RS + cp];
        if (D == 3) r = r + lam2 * dFs[((size_t)(2 * BPC + jj) * NV + v) * RS + cp];
        a.Uout[o + v * vsU] = a.U0[o + v * vsU] - r;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- staged-primitive pencil kernel
// The same stage with the primitives staged first: all threads of a CTA load the
// interiors and the face halos of its blocks (independent, coalesced loads; one
// conversion per cell) into a 12^d tile per block in shared memory, then each
// thread walks one line per direction out of shared memory, and a last pass
// applies the update.  Same arithmetic, so the same results as k_fv.
template <typename T, int D>
struct FVPShape {
  static constexpr int NV = D + 2;
  static constexpr int B = (D == 2) ? 64 : 512;
  static constexpr int TF = (D == 2) ? 8 : 64;
  static constexpr int STRIP = 2 * D * 2 * TF;
  static constexpr int BPC = (D == 2) ? 8 : 1;        // blocks per CTA
  static constexpr int NT = D * TF * BPC;              // one thread per line and direction
  static constexpr int WX = 13;                         // padded row of the 12-wide tile
  static constexpr int WY = 12 * WX;
  static constexpr int WN = (D == 2) ? WY : 12 * WY;    // tile values per variable
  static constexpr int PY = FVShape<T, D, 1>::PY, PZ = FVShape<T, D, 1>::PZ, RS = FVShape<T, D, 1>::RS;
  // CTAs per SM the shared memory allows in single precision (the register budget
  // is set to match)
  static constexpr int MINB = sizeof(T) == 4 ? (D == 2 ? 5 : 3) : 1;
};
template <typename T, int D>
constexpr size_t fvp_smem_bytes() {
  using S = FVPShape<T, D>;
  return (size_t)S::BPC * S::NV * (S::WN + D * S::RS) * sizeof(T);
}
// index of cell (x, y, z) (-2..9 each, relative to the block) in the padded tile
template <int D>
__device__ __forceinline__ int fvp_tile(int x, int y, int z) {
  return (D == 2) ? (x + 2) + 13 * (y + 2) : (x + 2) + 13 * ((y + 2) + 12 * (z + 2));
}

template <typename T, int D, int N>
__device__ __forceinline__ void fvp_line(const FVArgs<T> &a, int s, int l, int nb_lo, int nb_hi, int cm, int t0,
                                         long long cap, const T *W, T *dF, T gam, T goverg1) {
  using S = FVPShape<T, D>;
  constexpr int NV = S::NV, RS = S::RS, TF = S::TF;
  constexpr int SW = (N == 0) ? 1 : (N == 1 ? S::WX : S::WY);   // tile stride along N
  constexpr int SSTR = (N == 0) ? 1 : (N == 1 ? S::PY : S::PZ);  // dF stride along N
  const int t1 = t0 & 7, t2 = t0 >> 3;
  // tile index of position 0 of the line; dF index of its cell 0
  const int wbase = (N == 0) ? fvp_tile<D>(0, t1, t2) : (N == 1 ? fvp_tile<D>(t1, 0, t2) : fvp_tile<D>(t1, t2, 0));
  const int sbase = (N == 0) ? (S::PY * t1 + S::PZ * t2) : (N == 1 ? (t1 + S::PZ * t2) : (t1 + S::PY * t2));
  auto load = [&](int p, T *w) {
#pragma unroll
    for (int v = 0; v < NV; v++) w[v] = W[v * S::WN + wbase + p * SW];
  };
  const bool rec_lo = a.record && (nb_lo == NBR_MISSING || ((cm >> (2 * N)) & 1));
  const bool rec_hi = a.record && (nb_hi == NBR_MISSING || ((cm >> (2 * N + 1)) & 1));
  const bool add_lo = a.record == 2 && nb_lo == NBR_MISSING;
  const bool add_hi = a.record == 2 && nb_hi == NBR_MISSING;
  const T dtT = lev_at(a, lev_index(a.stage, l, 3));
  T wb[NV], wc[NV], slo[NV], Fprev[NV];
  {
    T wa[NV];
    load(-2, wa);
    load(-1, wb);
    load(0, wc);
#pragma unroll
    for (int v = 0; v < NV; v++) slo[v] = van_albada<T>(wb[v] - wa[v], wc[v] - wb[v]);
  }
#pragma unroll
  for (int k = 0; k < 9; k++) {
    T wd[NV], wl[NV], wr[NV], shi[NV], F[NV];
    load(k + 1, wd);
#pragma unroll
    for (int v = 0; v < NV; v++) {
      shi[v] = van_albada<T>(wc[v] - wb[v], wd[v] - wc[v]);
      wl[v] = lfma(T(0.5), slo[v], wb[v]);
      wr[v] = wc[v] - T(0.5) * shi[v];
    }
    ausm_plus<T, D>(N, wl, wr, gam, goverg1, F);
    if ((k == 0 && rec_lo) || (k == 8 && rec_hi)) {
      const int side = k == 8 ? 1 : 0;
      const bool add = side ? add_hi : add_lo;
      T *R = a.FR + (long long)s * (2 * D * TF) + (2 * N + side) * TF + t0;
      const long long vsR = cap * (2 * D * TF);
#pragma unroll
      for (int v = 0; v < NV; v++) {
        T val = dtT * F[v];
        R[v * vsR] = add ? R[v * vsR] + val : val;
      }
    }
    if (k > 0) {
#pragma unroll
      for (int v = 0; v < NV; v++) dF[v * RS + sbase + (k - 1) * SSTR] = F[v] - Fprev[v];
    }
#pragma unroll
    for (int v = 0; v < NV; v++) {
      Fprev[v] = F[v];
      slo[v] = shi[v];
      wb[v] = wc[v];
      wc[v] = wd[v];
    }
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(FVPShape<T, D>::NT, FVPShape<T, D>::MINB) k_fvp(Geo g, FVArgs<T> a) {
  using S = FVPShape<T, D>;
  constexpr int B = S::B, TF = S::TF, NV = S::NV, BPC = S::BPC, NT = S::NT, RS = S::RS;
  constexpr int NH = 2 * D * 2 * TF;                  // halo cells per block
  constexpr int NI = (BPC * B + NT - 1) / NT;         // interior cells per thread
  constexpr int NHT = (BPC * NH + NT - 1) / NT;       // halo cells per thread
  extern __shared__ unsigned char smem_raw[];
  T *Wt = reinterpret_cast<T *>(smem_raw);               // [block][v][WN] primitives
  T *dFs = Wt + (size_t)BPC * NV * S::WN;                // [dir][block][v][RS]
  __shared__ int sslot[BPC], slev[BPC], scm[BPC], snb[BPC][6];
  __shared__ T slam[BPC][3];
  const long long cap = g.cap, vsU = cap * B, vsG = cap * S::STRIP;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0), goverg1 = T(g.gamma / (g.gamma - 1.0));
  const int tid = threadIdx.x;
  int lb, le;
  list_range(g, a.kind, a.l0, a.l1, lb, le);
  if (a.bytes && blockIdx.x == 0 && tid == 0)
    atomicAdd(a.bytes, (unsigned long long)(le - lb) * B * a.words * sizeof(T));
  // slot of this thread's block in the next iteration (threads < BPC), read one
  // iteration ahead
  int s_next = -1;
  if (tid < BPC && lb + (int)blockIdx.x * BPC + tid < le) s_next = g.lists[a.kind * cap + lb + blockIdx.x * BPC + tid];
  for (int i0 = lb + blockIdx.x * BPC; i0 < le; i0 += gridDim.x * BPC) {
    if (tid < BPC) {
      const int s = s_next;
      const int in = i0 + gridDim.x * BPC + tid;
      s_next = in < le ? g.lists[a.kind * cap + in] : -1;
      if (i0 + tid < le) {
        const int l = g.slot_level[s];
        sslot[tid] = s;
        slev[tid] = l;
        scm[tid] = g.cmask[s];
#pragma unroll
        for (int f = 0; f < 2 * D; f++) snb[tid][f] = g.nbr[6 * s + f];
#pragma unroll
        for (int d = 0; d < 3; d++) slam[tid][d] = lev_at(a, lev_index(a.stage, l, d));
      }
    }
    __syncthreads();
    // ---------------- staging: all loads of this thread first, then the conversions
    {
      T Qi[NI][NV], Qh[NHT][NV];
      int ti[NI], th[NHT];
#pragma unroll
      for (int it = 0; it < NI; it++) {
        const int q = tid + it * NT;
        const int jj = q / B, c = q % B;
        const bool ok = q < BPC * B && i0 + jj < le;
        const T *src = a.Uin + (long long)sslot[ok ? jj : 0] * B + c;
        ti[it] = ok ? jj * NV * S::WN + fvp_tile<D>(c & 7, (c >> 3) & 7, c >> 6) : -1;
#pragma unroll
        for (int v = 0; v < NV; v++) Qi[it][v] = ok ? src[v * vsU] : T(1);
      }
#pragma unroll
      for (int it = 0; it < NHT; it++) {
        const int q = tid + it * NT;
        const int jj = q / NH, r = q % NH;
        const bool ok = q < BPC * NH && i0 + jj < le;
        const int j = ok ? jj : 0;
        const int s = sslot[j];
        const int f = r / (2 * TF), dd = (r / TF) & 1, t = r % TF;  // face, depth (0 touches), tangential
        const int n = f >> 1, side = f & 1;
        const int t1 = n == 0 ? 1 : 0, t2 = n == 2 ? 1 : 2;
        int cc[3] = {0, 0, 0};
        cc[t1] = t & 7;
        cc[t2] = (D == 3) ? t >> 3 : 0;
        int pc[3] = {cc[0], cc[1], cc[2]};
        pc[n] = side ? 8 + dd : -1 - dd;
        const int nb = snb[j][f];
        const T *src;
        long long vs = vsU;
        if (nb == NBR_MISSING) {
          src = a.G + (long long)s * S::STRIP + f * 2 * TF + dd * TF + t;
          vs = vsG;
        } else {
          int from = s;
          if (nb >= 0) {
            from = nb;
            cc[n] = side ? dd : 7 - dd;
          } else {
            cc[n] = side ? 7 : 0;
          }
          src = a.Uin + (long long)from * B + cc[0] + 8 * cc[1] + 64 * cc[2];
        }
        th[it] = ok ? j * NV * S::WN + fvp_tile<D>(pc[0], pc[1], (D == 3) ? pc[2] : 0) : -1;
#pragma unroll
        for (int v = 0; v < NV; v++) Qh[it][v] = ok ? src[v * vs] : T(1);
      }
#pragma unroll
      for (int it = 0; it < NI; it++) {
        T w[NV];
        cons_to_prim<T, D>(Qi[it], gm1, w);
        if (ti[it] >= 0) {
#pragma unroll
          for (int v = 0; v < NV; v++) Wt[ti[it] + v * S::WN] = w[v];
        }
      }
#pragma unroll
      for (int it = 0; it < NHT; it++) {
        T w[NV];
        cons_to_prim<T, D>(Qh[it], gm1, w);
        if (th[it] >= 0) {
#pragma unroll
          for (int v = 0; v < NV; v++) Wt[th[it] + v * S::WN] = w[v];
        }
      }
    }
    __syncthreads();
    // ---------------- lines
    {
      const int n = tid / (TF * BPC), j = (tid / TF) % BPC, t0 = tid % TF;
      if (i0 + j < le) {
        const int s = sslot[j], l = slev[j], cm = scm[j];
        const T *W = Wt + (size_t)j * NV * S::WN;
        T *dF = dFs + ((size_t)(n * BPC + j) * NV) * RS;
        if (n == 0) fvp_line<T, D, 0>(a, s, l, snb[j][0], snb[j][1], cm, t0, cap, W, dF, gam, goverg1);
        else if (n == 1) fvp_line<T, D, 1>(a, s, l, snb[j][2], snb[j][3], cm, t0, cap, W, dF, gam, goverg1);
        else if constexpr (D == 3) fvp_line<T, D, 2>(a, s, l, snb[j][4], snb[j][5], cm, t0, cap, W, dF, gam, goverg1);
      }
    }
    __syncthreads();
    // ---------------- update: the old states of this thread's cells first, then the stores
    {
      T Q0[NI][NV];
      long long o[NI];
#pragma unroll
      for (int it = 0; it < NI; it++) {
        const int q = tid + it * NT;
        const int jj = q / B, c = q % B;
        const bool ok = q < BPC * B && i0 + jj < le;
        o[it] = ok ? (long long)sslot[jj] * B + c : -1;
#pragma unroll
        for (int v = 0; v < NV; v++) Q0[it][v] = ok ? a.U0[o[it] + v * vsU] : T(0);
      }
#pragma unroll
      for (int it = 0; it < NI; it++) {
        if (o[it] < 0) continue;
        const int q = tid + it * NT;
        const int jj = q / B, c = q % B;
        const int cp = (c & 7) + S::PY * ((c >> 3) & 7) + S::PZ * (c >> 6);
        const T lam0 = slam[jj][0], lam1 = slam[jj][1], lam2 = slam[jj][2];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T r = lam0 * dFs[((size_t)(0 * BPC + jj) * NV + v) * RS + cp];
          r = r + lam1 * dFs[((size_t)(1 * BPC + jj) * NV + v) * RS + cp];
          if (D == 3) r = r + lam2 * dFs[((size_t)(2 * BPC + jj) * NV + v) * RS + cp];
          a.Uout[o[it] + v * vsU] = Q0[it][v] - r;
        }
      }
    }
    __syncthreads();
  }
}

// CFL limit over the leaves: min over cells and directions of dx_{l,n} / (|v_n| + c),
// scaled by 2^(l-L) with level-dependent steps; rho <= 0, p <= 0 or NaN flags an
// error.  The last CTA to finish sets dt = cfl * min (clipped to t_end - t) and
// fills the per-level step table.
template <typename T, int D>
__global__ void k_dt(Geo g, const T *__restrict__ A, int lts, unsigned long long *red, unsigned *done, double cfl,
                     double t_end, double *dsc, double *lev, float *levf) {
  constexpr int B = (D == 2) ? 64 : 512;
  int b, e;
  list_range(g, LK_LEAF, 0, g.L, b, e);
  const long long cap = g.cap;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0);
  T best = T(INFINITY);
  bool bad = false;
  // the time the last CTA clips dt against, read now so it is not a read of its own
  // at the end of the reduction (nothing writes it while this kernel runs)
  const double tnow = (threadIdx.x == 0 && t_end > 0.0) ? dsc[1] : 0.0;
  auto cell = [&](long long t) {
    int i = (int)(t / B), c = (int)(t % B);
    int s = g.lists[LK_LEAF * cap + i];
    int l = g.slot_level[s];
    T Q[D + 2], w[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; v++) Q[v] = A[((long long)v * cap + s) * B + c];
    cons_to_prim<T, D>(Q, gm1, w);
    if (!(w[0] > T(0)) || !(w[D + 1] > T(0))) {
      bad = true;
      return;
    }
    T cs = sqrt((gam * w[D + 1]) / w[0]);
#pragma unroll
    for (int d = 0; d < D; d++) {
      T rr = T(g.dx[l][d]) / (fabs(w[1 + d]) + cs);
      if (lts) rr = ldexp(rr, l - g.L);
      if (rr < best) best = rr;
    }
  };
  // two cells per pass, so their reads are in flight together
  const long long stride = (long long)gridDim.x * blockDim.x, end = (long long)e * B;
  for (long long t = (long long)b * B + blockIdx.x * blockDim.x + threadIdx.x; t < end; t += 2 * stride) {
    cell(t);
    if (t + stride < end) cell(t + stride);
  }
  if (bad) set_err(g, EB_NONPHYS);
  // warp minima, then the CTA minimum: one atomic per CTA on the shared word
  __shared__ T wmin[32];
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(0xffffffffu, best, o);
    if (x < best) best = x;
  }
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
  __shared__ int last;
  __shared__ double dsh;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++)
      if (wmin[w] < best) best = wmin[w];
    if (best < T(INFINITY)) atomicMin(red, (unsigned long long)__double_as_longlong((double)best));
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
    if (last) {
      __threadfence();
      double m = __longlong_as_double((long long)atomicAdd(red, 0ull));
      // ready for the next reduction (no memset before each launch)
      atomicExch(red, 0x7f7f7f7f7f7f7f7full);
      atomicExch(done, 0u);
      double d = cfl * m;
      if (t_end > 0.0) {
        double rest = t_end - tnow;
        if (rest < d) d = rest;
      }
      dsc[0] = d;
      dsh = d;
    }
  }
  __syncthreads();
  // the last CTA fills the per-level step table, one (level, stage) entry per thread
  if (last)
    for (int k = threadIdx.x; k < 2 * (g.L + 1); k += blockDim.x) level_params_entry(g, dsh, lts, lev, levf, k >> 1, k & 1);
}

}  // namespace mrfv
