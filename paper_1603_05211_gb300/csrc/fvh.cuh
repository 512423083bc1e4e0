// Staged finite-volume stage kernel: one thread per cell or face of a block held
// in shared memory, for two schemes of arXiv:1603.05211 Section 2.
//
// HANCOCK = true: the scheme of the paper's AMR method: unsplit MUSCL with the
// Minmod limiter in the primitive variables rho, v, p (Section 4.2), Hancock's
// half-step predictor with the exact flux, AUSMDV numerical flux (Wada and Liou
// 1997).  One stage per step: Q^{n+1} = Q^n - dt sum_n (F_{n,+} - F_{n,-}) / dx_n.
// The predictor is unsplit: every cell's extrapolated face states w +/- s_m/2
// are advanced by one common increment
//   dQ = sum_m (dt/2)/dx_m (f_m(Q^{-m}) - f_m(Q^{+m}))     (direction order)
// so the states of a face need its two cells' slopes in every direction, and
// with them the halo cells diagonally next to the block (the edges of the halo
// at depth one).  Those come from the same-level block that holds them, or,
// where it is absent, from the third-order prediction of the coarser level
// evaluated here (the same formula and inputs as the ghost strips).
//
// HANCOCK = false: one stage of the MR scheme (van Albada MUSCL, AUSM+, stage
// of the explicit midpoint rule), the same arithmetic as the pencil kernel k_fv
// in the same order.  It trades the pencil kernel's reuse of primitives and
// slopes along a line for many more threads with short dependency chains; a
// single launch on a few thousand blocks is faster than the pencil kernel's, but
// the adaptive step as a whole is not, so it is a selectable alternative.
//
// A CTA takes BPC blocks.  Phase 1 stages primitives of the interior, the two
// face-halo layers (and for HANCOCK the halo edges) in a 12^d tile; phase 2
// (HANCOCK) forms dQ for the interior and the ring of face-halo cells next to it
// (a 10^d tile); phase 3 evaluates the numerical flux once per face; phase 4
// applies the update in the oracle's summation order.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"
#include "fv.cuh"

namespace mrfv {

template <typename T, int D, bool HANCOCK>
struct FVS {
  static constexpr int NV = D + 2;
  static constexpr int B = (D == 2) ? 64 : 512;      // interior cells
  static constexpr int TF = (D == 2) ? 8 : 64;       // cells of one face layer
  static constexpr int STRIP = 2 * D * 2 * TF;       // ghost-strip cells per block
  static constexpr int NE = (D == 2) ? 144 : 1728;   // staged tile: 12^d cells
  static constexpr int NR = HANCOCK ? ((D == 2) ? 100 : 1000) : 0;  // predictor tile: 10^d cells
  static constexpr int NF = 9 * TF;                  // faces per direction
  static constexpr int BPC = (D == 2) ? 4 : 1;       // blocks per CTA
  static constexpr int NT = (D == 2) ? 256 : 512;    // threads per CTA
  static constexpr int MINB = (D == 2 && sizeof(T) == 4) ? 4 : 1;  // CTAs per SM the registers must allow
  static constexpr int PER = (NE + NR) * NV + D * NF * NV;  // shared values per block
};

template <typename T, int D, bool HANCOCK>
constexpr size_t fvs_smem_bytes() {
  return (size_t)FVS<T, D, HANCOCK>::BPC * FVS<T, D, HANCOCK>::PER * sizeof(T);
}

// index of cell (x, y, z) (relative to the block origin) in the staged 12^d tile
// and in the predictor 10^d tile
template <int D>
__device__ __forceinline__ int fvh_te(int x, int y, int z) {
  return (D == 2) ? (x + 2) + 12 * (y + 2) : (x + 2) + 12 * ((y + 2) + 12 * (z + 2));
}
template <int D>
__device__ __forceinline__ int fvh_tr(int x, int y, int z) {
  return (D == 2) ? (x + 1) + 10 * (y + 1) : (x + 1) + 10 * ((y + 1) + 10 * (z + 1));
}

template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
  T r = fabs(a) < fabs(b) ? a : b;
  return (a * b) > T(0) ? r : T(0);
}

// primitive (rho, v_1..v_D, p) -> conservative
template <typename T, int D>
__device__ __forceinline__ void prim_to_cons(const T *w, T gm1, T *Q) {
  T vv = (w[1] * w[1]) + (w[2] * w[2]);
  if (D == 3) vv = vv + (w[3] * w[3]);
  Q[0] = w[0];
#pragma unroll
  for (int d = 0; d < D; d++) Q[1 + d] = w[0] * w[1 + d];
  Q[D + 1] = (w[D + 1] / gm1) + ((T(0.5) * w[0]) * vv);
}

// exact flux f_m of Eq. 2.2 at primitive state w with conservative state Q
template <typename T, int D>
__device__ __forceinline__ void exact_flux(int m, const T *w, const T *Q, T *F) {
  T vn = w[1 + m], p = w[D + 1];
  F[0] = Q[0] * vn;
#pragma unroll
  for (int d = 0; d < D; d++) {
    T f = Q[1 + d] * vn;
    F[1 + d] = (d == m) ? f + p : f;
  }
  F[D + 1] = (Q[D + 1] + p) * vn;
}

// AUSMDV (Wada and Liou 1997) across a face with normal n from primitive face
// states: c_m = max(c_L, c_R); pressure-weighted split velocities and split
// pressures; normal momentum flux blended between AUSMV and AUSMD with
// s = min(1, 10 |p_R - p_L| / min(p_L, p_R)) / 2; tangential momentum and
// enthalpy upwinded by the mass flux.  No entropy or shock fix.
template <typename T, int D>
__device__ __forceinline__ void ausmdv(int n, const T *wl, const T *wr, T g, T goverg1, T *F) {
  const T rl = wl[0], rr = wr[0], pl = wl[D + 1], pr = wr[D + 1], ul = wl[1 + n], ur = wr[1 + n];
  const T cl = sqrt((g * pl) / rl), cr = sqrt((g * pr) / rr);
  const T cm = cl > cr ? cl : cr;
  const T pol = pl / rl, por = pr / rr;
  const T al = (T(2) * pol) / (pol + por), ar = (T(2) * por) / (pol + por);
  const T upl = T(0.5) * (ul + fabs(ul)), umr = T(0.5) * (ur - fabs(ur));
  T ulp, urm, plp, prm;
  if (fabs(ul) <= cm) {
    T t = ul + cm;
    ulp = (al * (((t * t) / (T(4) * cm)) - upl)) + upl;
    plp = pl * (((t * t) * (T(2) - (ul / cm))) / (T(4) * (cm * cm)));
  } else {
    ulp = upl;
    plp = ul > T(0) ? pl : T(0);
  }
  if (fabs(ur) <= cm) {
    T t = ur - cm;
    urm = (ar * ((-((t * t) / (T(4) * cm))) - umr)) + umr;
    prm = pr * (((t * t) * (T(2) + (ur / cm))) / (T(4) * (cm * cm)));
  } else {
    urm = umr;
    prm = ur < T(0) ? pr : T(0);
  }
  const T mdot = (ulp * rl) + (urm * rr);
  const T am = fabs(mdot);
  const T ph = plp + prm;
  const T pmin = pl < pr ? pl : pr;
  const T sw = T(0.5) * fmin(T(1), (T(10) * fabs(pr - pl)) / pmin);
  const T fvm = (ulp * (rl * ul)) + (urm * (rr * ur));
  const T fdm = T(0.5) * ((mdot * (ul + ur)) - (am * (ur - ul)));
  const T fn = ((T(0.5) + sw) * fvm) + ((T(0.5) - sw) * fdm);
  F[0] = mdot;
#pragma unroll
  for (int d = 0; d < D; d++)
    F[1 + d] = (d == n) ? fn + ph : T(0.5) * ((mdot * (wl[1 + d] + wr[1 + d])) - (am * (wr[1 + d] - wl[1 + d])));
  T vvl = (wl[1] * wl[1]) + (wl[2] * wl[2]), vvr = (wr[1] * wr[1]) + (wr[2] * wr[2]);
  if (D == 3) {
    vvl = vvl + (wl[3] * wl[3]);
    vvr = vvr + (wr[3] * wr[3]);
  }
  const T hl = (goverg1 * pol) + (T(0.5) * vvl), hr = (goverg1 * por) + (T(0.5) * vvr);
  F[D + 1] = T(0.5) * ((mdot * (hl + hr)) - (am * (hr - hl)));
}

// Conservative state of the level-l cell at global coordinates (gx, gy, gz), as
// the scheme sees it: mapped by the boundary rule, then the value of its block
// (A) or, where that block is absent, the prediction from level l-1 (C, or
// C0 + theta (C - C0) with level-dependent steps).
template <typename T, int D>
__device__ void ext_cell(const Geo &g, int l, int gx, int gy, int gz, const T *__restrict__ A,
                         const T *__restrict__ C, const T *__restrict__ C0, T theta, T *Q) {
  constexpr int NV = D + 2, B = (D == 2) ? 64 : 512, NP = (D == 2) ? 9 : 27;
  const long long cap = g.cap;
  const int I = bc_cell(g, l, 0, gx), J = bc_cell(g, l, 1, gy), K = (D == 3) ? bc_cell(g, l, 2, gz) : 0;
  const int32_t s = g.idx[map_index(g, l, I >> 3, J >> 3, K >> 3)];
  if (s >= 0) {
    const int c = (I & 7) + 8 * (J & 7) + 64 * (K & 7);
#pragma unroll
    for (int v = 0; v < NV; v++) Q[v] = A[((long long)v * cap + s) * B + c];
    return;
  }
  if (l == 0) {  // level 0 is complete: a missing block is a broken tree
    set_err(g, EB_TREE);
#pragma unroll
    for (int v = 0; v < NV; v++) Q[v] = nan_val<T>();
    return;
  }
  T patch[NV * NP];
  gather_patch<T, D, 3>(g, l - 1, C, C0, theta, (I >> 1) - 1, (J >> 1) - 1, (K >> 1) - 1, patch, 0, 1);
  const T si = (I & 1) ? T(-1) : T(1), sj = (J & 1) ? T(-1) : T(1), sk = (K & 1) ? T(-1) : T(1);
#pragma unroll
  for (int v = 0; v < NV; v++) Q[v] = predict<T, D, 3>(patch + v * NP, 1, 1, 1, si, sj, sk);
}

template <typename T, int D, bool HANCOCK>
__global__ void __launch_bounds__(FVS<T, D, HANCOCK>::NT, FVS<T, D, HANCOCK>::MINB) k_fvs(Geo g, FVArgs<T> a) {
  using S = FVS<T, D, HANCOCK>;
  constexpr int NV = S::NV, B = S::B, TF = S::TF, NE = S::NE, NR = S::NR, NF = S::NF, BPC = S::BPC, NT = S::NT;
  extern __shared__ unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const long long cap = g.cap;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0), goverg1 = T(g.gamma / (g.gamma - 1.0));
  const T theta = T(a.theta);
  int lb, le;
  list_range(g, a.kind, a.l0, a.l1, lb, le);
  if (a.bytes && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(a.bytes, (unsigned long long)(le - lb) * B * a.words * sizeof(T));

  for (int i0 = lb + blockIdx.x * BPC; i0 < le; i0 += gridDim.x * BPC) {
    // ---------------- phase 1: primitives of the staged tile
    for (int q = threadIdx.x; q < BPC * NE; q += NT) {
      const int jj = q / NE, e = q % NE;
      const int i = i0 + jj;
      if (i >= le) break;
      const int s = g.lists[a.kind * cap + i];
      int c3[3] = {e % 12 - 2, (e / 12) % 12 - 2, (D == 3) ? e / 144 - 2 : 0};
      int nout = 0, on = 0;
      bool edge = true;
#pragma unroll
      for (int d = 0; d < D; d++)
        if (c3[d] < 0 || c3[d] > 7) {
          nout++;
          on = d;
          if (c3[d] != -1 && c3[d] != 8) edge = false;
        }
      T Q[NV];
      if (nout == 0) {
        const int c = c3[0] + 8 * c3[1] + 64 * c3[2];
#pragma unroll
        for (int v = 0; v < NV; v++) Q[v] = a.Uin[((long long)v * cap + s) * B + c];
      } else if (nout == 1) {
        const int n = on, side = c3[n] > 7 ? 1 : 0, dd = side ? c3[n] - 8 : -1 - c3[n];
        const int nb = g.nbr[6 * s + 2 * n + side];
        const int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
        const int t = c3[t1] + ((D == 3) ? 8 * c3[t2] : 0);
        if (nb == NBR_MISSING) {
#pragma unroll
          for (int v = 0; v < NV; v++)
            Q[v] = a.G[((long long)v * cap + s) * S::STRIP + (2 * n + side) * 2 * TF + dd * TF + t];
        } else {
          int cc[3] = {c3[0], c3[1], c3[2]};
          cc[n] = (nb >= 0) ? (side ? dd : 7 - dd) : (side ? 7 : 0);
          const int from = nb >= 0 ? nb : s;
          const int c = cc[0] + 8 * cc[1] + 64 * cc[2];
#pragma unroll
          for (int v = 0; v < NV; v++) Q[v] = a.Uin[((long long)v * cap + from) * B + c];
        }
      } else if (HANCOCK && nout == 2 && edge) {
        const int l = g.slot_level[s];
        const int bx = g.slot_coord[3 * s], by = g.slot_coord[3 * s + 1], bz = g.slot_coord[3 * s + 2];
        ext_cell<T, D>(g, l, 8 * bx + c3[0], 8 * by + c3[1], 8 * bz + c3[2], a.Uin, a.C, a.C0, theta, Q);
      } else {
        continue;  // never read
      }
      T w[NV];
      cons_to_prim<T, D>(Q, gm1, w);
#pragma unroll
      for (int v = 0; v < NV; v++) sm[jj * S::PER + v * NE + e] = w[v];
    }
    __syncthreads();
    // ---------------- phase 2 (HANCOCK): half-step increment of the interior and the ring
    if constexpr (HANCOCK)
    for (int q = threadIdx.x; q < BPC * NR; q += NT) {
      const int jj = q / NR, r = q % NR;
      const int i = i0 + jj;
      if (i >= le) break;
      const int c3[3] = {r % 10 - 1, (r / 10) % 10 - 1, (D == 3) ? r / 100 - 1 : 0};
      int nout = 0;
#pragma unroll
      for (int d = 0; d < D; d++) nout += (c3[d] < 0 || c3[d] > 7) ? 1 : 0;
      if (nout > 1) continue;
      const int l = g.slot_level[g.lists[a.kind * cap + i]];
      const T *W = sm + jj * S::PER;
      const int e0 = fvh_te<D>(c3[0], c3[1], c3[2]);
      T w[NV], dQ[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = W[v * NE + e0];
#pragma unroll
      for (int m = 0; m < D; m++) {
        const int st = (m == 0) ? 1 : (m == 1 ? 12 : 144);
        T wm[NV], wp[NV], Qm[NV], Qp[NV], Fm[NV], Fp[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T sl = minmod<T>(w[v] - W[v * NE + e0 - st], W[v * NE + e0 + st] - w[v]);
          wm[v] = w[v] - (T(0.5) * sl);
          wp[v] = w[v] + (T(0.5) * sl);
        }
        prim_to_cons<T, D>(wm, gm1, Qm);
        prim_to_cons<T, D>(wp, gm1, Qp);
        exact_flux<T, D>(m, wm, Qm, Fm);
        exact_flux<T, D>(m, wp, Qp, Fp);
        const T h = lev_at(a, lev_index(0, l, m));
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T inc = h * (Fm[v] - Fp[v]);
          dQ[v] = (m == 0) ? inc : dQ[v] + inc;
        }
      }
#pragma unroll
      for (int v = 0; v < NV; v++) sm[jj * S::PER + NV * NE + v * NR + r] = dQ[v];
    }
    if (HANCOCK) __syncthreads();
    // ---------------- phase 3: the numerical flux of every face, one direction at a
    // time (the direction is a constant in each copy of the loop body)
#pragma unroll
    for (int n = 0; n < D; n++)
    for (int q = threadIdx.x; q < BPC * NF; q += NT) {
      const int jj = q / NF, u = q % NF;
      const int i = i0 + jj;
      if (i >= le) break;
      const int s = g.lists[a.kind * cap + i];
      const int l = g.slot_level[s];
      // consecutive threads take neighbouring faces along x: unit-stride tile reads;
      // the flux of face f (position along n) and tangential index t is stored at
      // f + 9 t (stride 9 between threads for n >= 1: no bank conflicts)
      const int f = (n == 0) ? u % 9 : (u >> 3) % 9;
      const int t = (n == 0) ? u / 9 : (u & 7) + 8 * (u / 72);
      const int fi = f + 9 * t, ta = t & 7, tb = t >> 3;
      const int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
      int cl[3] = {0, 0, 0};
      cl[n] = f - 1;
      cl[t1] = ta;
      if (D == 3) cl[t2] = tb;
      const int st = (n == 0) ? 1 : (n == 1 ? 12 : 144);
      const T *W = sm + jj * S::PER;
      const T *DQ = W + NV * NE;
      const int el = fvh_te<D>(cl[0], cl[1], cl[2]), er = el + st;
      const int rl = fvh_tr<D>(cl[0], cl[1], cl[2]), rr = rl + ((n == 0) ? 1 : (n == 1 ? 10 : 100));
      T wl[NV], wr[NV], F[NV];
      if constexpr (!HANCOCK) {
        // van Albada slopes of the two cells along n, face states, AUSM+
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T wa = W[v * NE + el], wb = W[v * NE + er];
          T sa = van_albada<T>(wa - W[v * NE + el - st], wb - wa);
          T sb = van_albada<T>(wb - wa, W[v * NE + er + st] - wb);
          wl[v] = lfma(T(0.5), sa, wa);
          wr[v] = wb - T(0.5) * sb;
        }
        ausm_plus<T, D>(n, wl, wr, gam, goverg1, F);
      } else {
        T wq[NV], Qf[NV];
        // high face of the left cell
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T w0 = W[v * NE + el];
          T sl = minmod<T>(w0 - W[v * NE + el - st], W[v * NE + el + st] - w0);
          wq[v] = w0 + (T(0.5) * sl);
        }
        prim_to_cons<T, D>(wq, gm1, Qf);
#pragma unroll
        for (int v = 0; v < NV; v++) Qf[v] = Qf[v] + DQ[v * NR + rl];
        cons_to_prim<T, D>(Qf, gm1, wl);
        // low face of the right cell
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T w0 = W[v * NE + er];
          T sl = minmod<T>(w0 - W[v * NE + er - st], W[v * NE + er + st] - w0);
          wq[v] = w0 - (T(0.5) * sl);
        }
        prim_to_cons<T, D>(wq, gm1, Qf);
#pragma unroll
        for (int v = 0; v < NV; v++) Qf[v] = Qf[v] + DQ[v * NR + rr];
        cons_to_prim<T, D>(Qf, gm1, wr);
        ausmdv<T, D>(n, wl, wr, gam, goverg1, F);
      }
      T *FS = sm + jj * S::PER + NV * (NE + NR);
#pragma unroll
      for (int v = 0; v < NV; v++) FS[(n * NV + v) * NF + fi] = F[v];
      if (a.record && (f == 0 || f == 8)) {
        const int side = f == 8 ? 1 : 0;
        const int nb = g.nbr[6 * s + 2 * n + side];
        const bool rec = nb == NBR_MISSING || ((g.cmask[s] >> (2 * n + side)) & 1);
        if (rec) {
          const bool add = a.record == 2 && nb == NBR_MISSING;
          const T dtT = lev_at(a, lev_index(a.stage, l, 3));
#pragma unroll
          for (int v = 0; v < NV; v++) {
            T *R = a.FR + ((long long)v * cap + s) * (2 * D * TF) + (2 * n + side) * TF + t;
            T val = dtT * F[v];
            *R = add ? *R + val : val;
          }
        }
      }
    }
    __syncthreads();
    // ---------------- phase 4: update, directions summed in order
    for (int q = threadIdx.x; q < BPC * B; q += NT) {
      const int jj = q / B, c = q % B;
      const int i = i0 + jj;
      if (i >= le) break;
      const int s = g.lists[a.kind * cap + i];
      const int l = g.slot_level[s];
      const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
      const T *FS = sm + jj * S::PER + NV * (NE + NR);
      const int f0 = x + 9 * (y + 8 * z), f1 = y + 9 * (x + 8 * z), f2 = z + 9 * (x + 8 * y);
      const T lam0 = lev_at(a, lev_index(a.stage, l, 0)), lam1 = lev_at(a, lev_index(a.stage, l, 1));
      const T lam2 = lev_at(a, lev_index(a.stage, l, 2));
#pragma unroll
      for (int v = 0; v < NV; v++) {
        T r = lam0 * (FS[(0 * NV + v) * NF + f0 + 1] - FS[(0 * NV + v) * NF + f0]);
        r = r + lam1 * (FS[(1 * NV + v) * NF + f1 + 1] - FS[(1 * NV + v) * NF + f1]);
        if (D == 3) r = r + lam2 * (FS[(2 * NV + v) * NF + f2 + 1] - FS[(2 * NV + v) * NF + f2]);
        const long long o = ((long long)v * cap + s) * B + c;
        a.Uout[o] = a.U0[o] - r;
      }
    }
    __syncthreads();
  }
}

}  // namespace mrfv
