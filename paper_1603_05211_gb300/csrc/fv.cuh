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


// ---------------------------------------------------------------- lanes
// The stage arithmetic is written once for a "lane" type L: a scalar (float,
// double: one pencil per thread) or vf2 (two single-precision pencils per
// thread in the packed FP32x2 instructions of sm_100+).  Branches are written as
// selects of both sides, which gives the same values as the branches.
struct vf2 {
  float2 v;
  __device__ __forceinline__ vf2() {}
  __device__ __forceinline__ vf2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ vf2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit vf2(float2 x) : v(x) {}
};
struct mask2 {
  bool x, y;
};
__device__ __forceinline__ vf2 operator+(vf2 a, vf2 b) { return vf2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ vf2 operator-(vf2 a, vf2 b) { return vf2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ vf2 operator*(vf2 a, vf2 b) { return vf2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ vf2 operator/(vf2 a, vf2 b) { return vf2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ mask2 operator>(vf2 a, vf2 b) { return {a.v.x > b.v.x, a.v.y > b.v.y}; }
__device__ __forceinline__ mask2 operator>=(vf2 a, vf2 b) { return {a.v.x >= b.v.x, a.v.y >= b.v.y}; }
__device__ __forceinline__ mask2 operator<(vf2 a, vf2 b) { return {a.v.x < b.v.x, a.v.y < b.v.y}; }
__device__ __forceinline__ vf2 lsel(mask2 m, vf2 a, vf2 b) { return vf2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }
__device__ __forceinline__ vf2 labs(vf2 a) { return vf2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ vf2 lsqrt(vf2 a) { return vf2(sqrtf(a.v.x), sqrtf(a.v.y)); }
// a * b + c: fused for vf2; for scalars written as the product then the sum (the
// double-precision unit is built without contraction, so it rounds both)
__device__ __forceinline__ vf2 lfma(vf2 a, vf2 b, vf2 c) { return vf2(__ffma2_rn(a.v, b.v, c.v)); }

template <typename L>
__device__ __forceinline__ L lsel(bool m, L a, L b) { return m ? a : b; }
__device__ __forceinline__ float labs(float a) { return fabsf(a); }
__device__ __forceinline__ double labs(double a) { return fabs(a); }
__device__ __forceinline__ float lsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double lsqrt(double a) { return sqrt(a); }
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

// Launch shape of the stage kernel for state type T in dimension D: P pencils per
// thread, BPC blocks per CTA.  Two single-precision pencils per thread in packed
// FP32x2 lanes (MRFV_FV_PPT32=1) measured slower on GB300 than one pencil per
// thread (fewer warps to hide latency), so one is the default.
#ifndef MRFV_FV_PPT32
#define MRFV_FV_PPT32 0
#endif
template <typename T, int D, int SPLIT = 1>
struct FVShape {
  static constexpr int B = (D == 2) ? 64 : 512;        // interior cells
  static constexpr int TF = (D == 2) ? 8 : 64;         // cells of one face layer = pencils per direction
  static constexpr int NV = D + 2;
  static constexpr int STRIP = 2 * D * 2 * TF;         // ghost cells (two layers per face)
  static constexpr int P = MRFV_FV_PPT32 && sizeof(T) == 4 ? 2 : 1;  // pencils per thread
  static constexpr int BPC = (D == 2) ? (P == 2 ? 32 : 16) : (P == 2 ? 2 : 1);  // blocks per CTA
  static constexpr int TPD = TF / P;                   // pencil groups per block and direction
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

template <typename T, int P>
struct Lane;
template <typename T>
struct Lane<T, 1> {
  using type = T;
};
template <>
struct Lane<float, 2> {
  using type = vf2;
};

// Conservative state of pencil position p (-2..9) of the P pencils (n, t0 .. t0+P-1)
// of block s: own cells, the same-level neighbour's cells, the ghost strip, or the
// block's own edge cell at a transmissive wall.
template <typename T, int D, int P>
__device__ __forceinline__ void pencil_load(const Geo &g, const T *__restrict__ U, const T *__restrict__ G, int s,
                                            int n, int t0, int nb_lo, int nb_hi, int p,
                                            typename Lane<T, P>::type *Q) {
  using S = FVShape<T, D>;
  constexpr int B = S::B, TF = S::TF, NV = S::NV;
  const long long cap = g.cap;
  const int stride = (n == 0) ? 1 : (n == 1 ? 8 : 64);
  const int t1 = t0 & 7, t2 = t0 >> 3;
  // cell index of tangential position t0 with coordinate 0 along n; the next
  // pencil of the thread is one cell further in the first tangential direction
  const int base = (n == 0) ? (8 * t1 + 64 * t2) : (n == 1 ? (t1 + 64 * t2) : (t1 + 8 * t2));
  const int tstep = (n == 0) ? 8 : 1;
  int from = s, c;
  if (p >= 0 && p <= 7) {
    c = base + p * stride;
  } else {
    const int side = p > 7 ? 1 : 0;
    const int dd = side ? p - 8 : -1 - p;  // 0 touches the block
    const int nb = side ? nb_hi : nb_lo;
    if (nb == NBR_MISSING) {
      const T *Gp = G + (long long)s * S::STRIP + (2 * n + side) * 2 * TF + dd * TF + t0;
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const T *q = Gp + (long long)v * cap * S::STRIP;
        if constexpr (P == 2) Q[v] = vf2(*reinterpret_cast<const float2 *>(q));
        else Q[v] = q[0];
      }
      return;
    }
    if (nb >= 0) {
      from = nb;
      c = base + (side ? dd : 7 - dd) * stride;
    } else {
      c = base + (side ? 7 : 0) * stride;
    }
  }
  const T *Up = U + (long long)from * B + c;
#pragma unroll
  for (int v = 0; v < NV; v++) {
    const T *q = Up + (long long)v * cap * B;
    if constexpr (P == 2) {
      if (tstep == 1) Q[v] = vf2(*reinterpret_cast<const float2 *>(q));
      else Q[v] = vf2(q[0], q[8]);
    } else {
      Q[v] = q[0];
    }
  }
}

// One thread per group of P pencils (SPLIT = 1) or two threads per group, each
// taking one half of the line (SPLIT = 2: faces 0..4 and 4..8, the middle face
// evaluated by both; twice the threads and half the dependency chain, for
// hierarchies too small to fill the GPU).  The cells of a line along direction n
// (two beyond each face of the block) are converted to primitives in a sliding
// window; each cell's limited slope is formed once, then the two face states
// and the AUSM+ flux of each face, and the flux difference F_{k+1} - F_k of every
// interior cell goes to shared memory.  A second pass applies
// Q_out = Q_0 - (lambda_1 dF_1 + lambda_2 dF_2 [+ lambda_3 dF_3]), summed in
// direction order, to every cell.
template <typename T, int D, int SPLIT>
__global__ void __launch_bounds__(FVShape<T, D, SPLIT>::NT,
                                  (FVMinBlocks<T>::value / SPLIT > 0 ? FVMinBlocks<T>::value / SPLIT : 1))
    k_fv(Geo g, FVArgs<T> a) {
  using S = FVShape<T, D, SPLIT>;
  constexpr int B = S::B, TF = S::TF, NV = S::NV, BPC = S::BPC, RS = S::RS, NT = S::NT, P = S::P, TPD = S::TPD;
  constexpr int NK = S::NK;
  using L = typename Lane<T, P>::type;
  extern __shared__ unsigned char smem_raw[];
  T *dFs = reinterpret_cast<T *>(smem_raw);  // [dir][block][v][RS]
  const long long cap = g.cap;
  const L gam = L(T(g.gamma)), gm1 = L(T(g.gamma - 1.0)), goverg1 = L(T(g.gamma / (g.gamma - 1.0)));
  const int stage = a.stage;
  // pencil group of this thread: direction-major so a warp shares one direction
  const int n = threadIdx.x / (TPD * BPC * SPLIT);
  const int j = (threadIdx.x / (TPD * SPLIT)) % BPC;
  const int half = (threadIdx.x / TPD) % SPLIT;
  const int t0 = (threadIdx.x % TPD) * P;
  const int kb = half * 4;  // first face of this thread
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
        const int nb_lo = g.nbr[6 * s + 2 * n], nb_hi = g.nbr[6 * s + 2 * n + 1];
        const bool rec_lo = a.record && kb == 0 && (nb_lo == NBR_MISSING || ((g.cmask[s] >> (2 * n)) & 1));
        const bool rec_hi = a.record && kb + NK == 9 && (nb_hi == NBR_MISSING || ((g.cmask[s] >> (2 * n + 1)) & 1));
        const bool add_lo = a.record == 2 && nb_lo == NBR_MISSING;
        const bool add_hi = a.record == 2 && nb_hi == NBR_MISSING;
        const T dtT = lev_at(a, lev_index(stage, l, 3));
        // padded shared-memory index of the first pencil's position 0, stride along n,
        // step to the next pencil of the thread
        const int t1 = t0 & 7, t2 = t0 >> 3;
        const int base = (n == 0) ? (S::PY * t1 + S::PZ * t2) : (n == 1 ? (t1 + S::PZ * t2) : (t1 + S::PY * t2));
        const int stride = (n == 0) ? 1 : (n == 1 ? S::PY : S::PZ);
        const int pstep = (n == 0) ? S::PY : 1;
        T *dF = dFs + ((size_t)(n * BPC + j) * NV) * RS;
        // sliding window of primitives: wb = cell k-1, wc = cell k (face k lies between them)
        L wb[NV], wc[NV], slo[NV], Fprev[NV];
        {
          L Q[NV], wa[NV];
          pencil_load<T, D, P>(g, a.Uin, a.G, s, n, t0, nb_lo, nb_hi, kb - 2, Q);
          cons_to_prim<L, D>(Q, gm1, wa);
          pencil_load<T, D, P>(g, a.Uin, a.G, s, n, t0, nb_lo, nb_hi, kb - 1, Q);
          cons_to_prim<L, D>(Q, gm1, wb);
          pencil_load<T, D, P>(g, a.Uin, a.G, s, n, t0, nb_lo, nb_hi, kb, Q);
          cons_to_prim<L, D>(Q, gm1, wc);
          // slope of cell kb - 1
#pragma unroll
          for (int v = 0; v < NV; v++) slo[v] = van_albada<L>(wb[v] - wa[v], wc[v] - wb[v]);
        }
#pragma unroll
        for (int kk = 0; kk < NK; kk++) {
          const int k = kb + kk;
          L wd[NV], wl[NV], wr[NV], shi[NV], F[NV];
          {
            L Q[NV];
            pencil_load<T, D, P>(g, a.Uin, a.G, s, n, t0, nb_lo, nb_hi, k + 1, Q);
            cons_to_prim<L, D>(Q, gm1, wd);
          }
#pragma unroll
          for (int v = 0; v < NV; v++) {
            shi[v] = van_albada<L>(wc[v] - wb[v], wd[v] - wc[v]);
            wl[v] = lfma(L(T(0.5)), slo[v], wb[v]);
            wr[v] = wc[v] - L(T(0.5)) * shi[v];
          }
          ausm_plus<L, D>(n, wl, wr, gam, goverg1, F);
          if ((k == 0 && rec_lo) || (k == 8 && rec_hi)) {
            const int side = k == 8 ? 1 : 0;
            const bool add = side ? add_hi : add_lo;
#pragma unroll
            for (int v = 0; v < NV; v++) {
              T *R = a.FR + ((long long)v * cap + s) * (2 * D * TF) + (2 * n + side) * TF + t0;
              if constexpr (P == 2) {
                float2 val = __fmul2_rn(make_float2(dtT, dtT), F[v].v);
                float2 *R2 = reinterpret_cast<float2 *>(R);
                if (add) val = __fadd2_rn(*R2, val);
                *R2 = val;
              } else {
                T val = dtT * F[v];
                *R = add ? *R + val : val;
              }
            }
          }
          if (kk > 0) {
#pragma unroll
            for (int v = 0; v < NV; v++) {
              L d = F[v] - Fprev[v];
              T *dst = dF + v * RS + base + (k - 1) * stride;
              if constexpr (P == 2) {
                dst[0] = d.v.x;
                dst[pstep] = d.v.y;
              } else {
                dst[0] = d;
              }
            }
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
    }
    __syncthreads();
    // ---------------- update pass
    for (int q = threadIdx.x; q < BPC * B; q += NT) {
      const int jj = q / B, c = q % B;
      const int i = i0 + jj;
      if (i >= le) break;
      const int s = g.lists[a.kind * cap + i];
      const int l = g.slot_level[s];
      const int cp = (c & 7) + S::PY * ((c >> 3) & 7) + S::PZ * (c >> 6);
      const T lam0 = lev_at(a, lev_index(stage, l, 0)), lam1 = lev_at(a, lev_index(stage, l, 1));
      const T lam2 = lev_at(a, lev_index(stage, l, 2));
#pragma unroll
      for (int v = 0; v < NV; v++) {
        T r = lam0 * dFs[((size_t)(0 * BPC + jj) * NV + v) * RS + cp];
        r = r + lam1 * dFs[((size_t)(1 * BPC + jj) * NV + v) * RS + cp];
        if (D == 3) r = r + lam2 * dFs[((size_t)(2 * BPC + jj) * NV + v) * RS + cp];
        long long o = ((long long)v * cap + s) * B + c;
        a.Uout[o] = a.U0[o] - r;
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
  // warp minima, then the CTA minimum: one atomic per CTA on the shared word
  __shared__ T wmin[32];
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(0xffffffffu, best, o);
    if (x < best) best = x;
  }
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++)
      if (wmin[w] < best) best = wmin[w];
    if (best < T(INFINITY)) atomicMin(red, (unsigned long long)__double_as_longlong((double)best));
    __threadfence();
    if (atomicAdd(done, 1u) == gridDim.x - 1) {
      __threadfence();
      double m = __longlong_as_double((long long)atomicAdd(red, 0ull));
      double d = cfl * m;
      if (t_end > 0.0) {
        double rest = t_end - dsc[1];
        if (rest < d) d = rest;
      }
      dsc[0] = d;
      level_params_dev(g, d, lts, lev, levf);
    }
  }
}

}  // namespace mrfv
