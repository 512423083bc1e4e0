// Richardson error estimate, the local error indicator the AMR code of
// arXiv:1603.05211 Section 2.2 can add to its scaled-gradient flags (the estimate
// of Berger and Oliger 1984 and Berger and Colella 1989).  On level l, with H_dt
// one step of the configured scheme over a uniform grid and R the mean of the
// 2^d children:
//     tau = (R H_dt(H_dt(E)) - H_2dt(R E)) / (2^(o+1) - 2),   o = 2,
// on the level's grid coarsened by 2 (same boundary rule), density only; E is
// the level as the scheme sees it (absent cells predicted from level l-1), dt the
// level's step in the last time step.  A block is flagged when a coarse cell of
// an existing block within one fine cell of it has |tau| > eps_r.
//
// One CTA per existing block of levels l0..L-1.  The estimate of the block's 4^d
// coarse cells depends on E only within H fine cells of the block (each stage
// reaches 2 cells; two fine steps and one coarse step: H = 8 for the MR scheme's
// two-stage steps, 4 for the AMR scheme's one-stage steps), so the CTA gathers
// that (8 + 2H)^d patch (absent cells predicted from the coarser cells under it,
// staged once), restricts it to the coarse patch, runs the coarse step of 2 dt
// and the two fine steps of dt, every stage on a region 2 cells narrower than its
// input, and compares on the block.  Each stage converts its input to primitives
// once, evaluates the numerical flux once per face of its region and applies the
// update in the order of the cell update of the stage kernels.  At a
// transmissive wall the reads are clamped to the domain, as the boundary rule
// does.  2D patches live in shared memory, 3D ones in a per-CTA area of global
// memory.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"
#include "fv.cuh"
#include "fvh.cuh"

namespace mrfv {

template <int D, bool HANCOCK>
struct RichShape {
  static constexpr int NV = D + 2;
  // fine cells around the block the estimate reads: 2 per stage, four stages of
  // the MR scheme, two of the AMR scheme
  static constexpr int H = HANCOCK ? 4 : 8;
  static constexpr int P = 8 + 2 * H;  // fine patch edge
  static constexpr int PC = P / 2;     // coarse patch edge
  static constexpr int NP = (D == 2) ? P * P : P * P * P;
  static constexpr int NPC = (D == 2) ? PC * PC : PC * PC * PC;
  static constexpr int NFACE = (D == 2) ? (P + 1) * P : (P + 1) * P * P;  // faces of one direction
  static constexpr int PP = PC + 2;  // level l-1 cells the predictions of the fine patch read (per edge)
  static constexpr int NPP = (D == 2) ? PP * PP : PP * PP * PP;
  static constexpr int NT = (D == 2) ? 128 : 256;  // threads per CTA (2D: as many per SM as the
                                                   // patch's shared memory allows; 3D: two)
  // scratch values per CTA: A, S, W, DQ [NV][NP]; CA, CS [NV][NPC]; FL [D][NV][NFACE]; CP [NV][NPP]
  static constexpr long long PER = (long long)NV * (4 * NP + 2 * NPC + NPP) + (long long)D * NV * NFACE;
};

// A box [a, b) per dimension (unused dimensions [0, 1)) walked by the CTA's threads.
struct RBox {
  int a[3], b[3];
  __device__ int count() const { return (b[0] - a[0]) * (b[1] - a[1]) * (b[2] - a[2]); }
  __device__ void at(int q, int &x, int &y, int &z) const {
    const int w0 = b[0] - a[0], w1 = b[1] - a[1];
    x = a[0] + q % w0;
    y = a[1] + (q / w0) % w1;
    z = a[2] + q / (w0 * w1);
  }
};

// One stage on a patch of edge E (buffers [NV][E^D]): out = q0 - sum_n lam_n (F_n(x + 1/2) - F_n(x - 1/2))
// (directions summed in order) on the cells of `reg`, with the fluxes from the
// stage input `in` on reg widened by 2.  dl/dh: the domain's cells of the patch
// (reads outside are clamped into it; a periodic patch has none outside).
// HANCOCK: the predictor advances the face states by dQ, h_m = (dt/2)/dx_m.
// (E is a run-time value and the direction loop is not unrolled: one copy of the
// stage serves both patches, which keeps the kernel's instruction footprint small.)
template <typename T, int D, bool HANCOCK>
__device__ __noinline__ void rich_stage(const T *in, const T *q0, T *out, T *W, T *DQ, T *FL, const RBox &reg,
                                        const int *dl, const int *dh, const T *lam, const T *h, T gam, T gm1,
                                        T goverg1, const int E, const bool w_ready, const bool w_next) {
  using S = RichShape<D, HANCOCK>;
  constexpr int NV = S::NV, NFACE = S::NFACE, NT = S::NT;
  const int NS = (D == 2) ? E * E : E * E * E;  // values per variable of the patch buffers
  auto cl = [&](int x, int d) { return x < dl[d] ? dl[d] : (x >= dh[d] ? dh[d] - 1 : x); };
  auto pidx = [&](int x, int y, int z) { return x + E * (y + E * z); };
  // primitives of the input on reg widened by 2, inside the domain (unless the
  // phase that produced the input wrote them: w_ready)
  if (!w_ready) {
    RBox wb;
    for (int d = 0; d < 3; d++) {
      wb.a[d] = d < D ? max(reg.a[d] - 2, dl[d]) : 0;
      wb.b[d] = d < D ? min(reg.b[d] + 2, dh[d]) : 1;
    }
    for (int q = threadIdx.x; q < wb.count(); q += NT) {
      int x, y, z;
      wb.at(q, x, y, z);
      const int p = pidx(x, y, z);
      T Q[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) Q[v] = in[v * NS + p];
      cons_to_prim<T, D>(Q, gm1, w);
#pragma unroll
      for (int v = 0; v < NV; v++) W[v * NS + p] = w[v];
    }
    __syncthreads();
  }
  if constexpr (HANCOCK) {
    // half-step increment of every cell a face of reg touches (the ring of ghost
    // cells at a wall included: their slopes come from clamped neighbours)
    RBox qb;
    for (int d = 0; d < 3; d++) {
      qb.a[d] = d < D ? max(reg.a[d] - 1, dl[d] - 1) : 0;
      qb.b[d] = d < D ? min(reg.b[d] + 1, dh[d] + 1) : 1;
    }
    for (int q = threadIdx.x; q < qb.count(); q += NT) {
      int c[3];
      qb.at(q, c[0], c[1], c[2]);
      const int pc = pidx(cl(c[0], 0), cl(c[1], 1), D == 3 ? cl(c[2], 2) : 0);
      T w[NV], dQ[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) w[v] = W[v * NS + pc];
#pragma unroll
      for (int m = 0; m < D; m++) {
        int lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
        lo[m] -= 1;
        hi[m] += 1;
        const int pl = pidx(cl(lo[0], 0), cl(lo[1], 1), D == 3 ? cl(lo[2], 2) : 0);
        const int ph = pidx(cl(hi[0], 0), cl(hi[1], 1), D == 3 ? cl(hi[2], 2) : 0);
        T wm[NV], wp[NV], Qm[NV], Qp[NV], Fm[NV], Fp[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T sl = minmod<T>(w[v] - W[v * NS + pl], W[v * NS + ph] - w[v]);
          wm[v] = w[v] - (T(0.5) * sl);
          wp[v] = w[v] + (T(0.5) * sl);
        }
        prim_to_cons<T, D>(wm, gm1, Qm);
        prim_to_cons<T, D>(wp, gm1, Qp);
        exact_flux<T, D>(m, wm, Qm, Fm);
        exact_flux<T, D>(m, wp, Qp, Fp);
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T inc = h[m] * (Fm[v] - Fp[v]);
          dQ[v] = (m == 0) ? inc : dQ[v] + inc;
        }
      }
      const int p = pidx(c[0], c[1], c[2]);
#pragma unroll
      for (int v = 0; v < NV; v++) DQ[v * NS + p] = dQ[v];
    }
    __syncthreads();
  }
  // numerical flux of every face of reg, all directions (face f along n lies
  // between cells f-1 and f; stored compactly over the region's faces,
  // (f - a_n) + (w_n + 1) ((t1 - a_t1) + w_t1 (t2 - a_t2)), w = the region's widths)
#pragma unroll 1
  for (int n = 0; n < D; n++) {
    const int t1 = (n == 0) ? 1 : 0, t2 = (n == 2) ? 1 : 2;
    RBox fb;
    fb.a[0] = reg.a[n];
    fb.b[0] = reg.b[n] + 1;
    fb.a[1] = reg.a[t1];
    fb.b[1] = reg.b[t1];
    fb.a[2] = D == 3 ? reg.a[t2] : 0;
    fb.b[2] = D == 3 ? reg.b[t2] : 1;
    for (int q = threadIdx.x; q < fb.count(); q += NT) {
      int f, u1, u2;
      fb.at(q, f, u1, u2);
      int c[3];
      c[n] = f - 1;
      c[t1] = u1;
      if (D == 3) c[t2] = u2;
      else c[2] = 0;
      T wl[NV], wr[NV], F[NV];
      if constexpr (!HANCOCK) {
        int cc[3] = {c[0], c[1], c[2]};
        int pk[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          cc[n] = c[n] + k - 1;  // cells f-2, f-1, f, f+1
          pk[k] = pidx(cl(cc[0], 0), cl(cc[1], 1), D == 3 ? cl(cc[2], 2) : 0);
        }
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T w0 = W[v * NS + pk[0]], wa = W[v * NS + pk[1]], wb2 = W[v * NS + pk[2]], w3 = W[v * NS + pk[3]];
          T sa = van_albada<T>(wa - w0, wb2 - wa);
          T sb = van_albada<T>(wb2 - wa, w3 - wb2);
          wl[v] = lfma(T(0.5), sa, wa);
          wr[v] = wb2 - T(0.5) * sb;
        }
        ausm_plus<T, D>(n, wl, wr, gam, goverg1, F);
      } else {
#pragma unroll
        for (int side = 0; side < 2; side++) {
          int a[3] = {c[0], c[1], c[2]};
          a[n] += side;  // the face's left (side 0) or right cell, unclamped
          int am[3] = {a[0], a[1], a[2]}, ap[3] = {a[0], a[1], a[2]};
          am[n] -= 1;
          ap[n] += 1;
          const int p0 = pidx(cl(a[0], 0), cl(a[1], 1), D == 3 ? cl(a[2], 2) : 0);
          const int pm = pidx(cl(am[0], 0), cl(am[1], 1), D == 3 ? cl(am[2], 2) : 0);
          const int pp = pidx(cl(ap[0], 0), cl(ap[1], 1), D == 3 ? cl(ap[2], 2) : 0);
          const int pd = pidx(a[0], a[1], a[2]);
          T wq[NV], Qf[NV];
#pragma unroll
          for (int v = 0; v < NV; v++) {
            T w0 = W[v * NS + p0];
            T sl = minmod<T>(w0 - W[v * NS + pm], W[v * NS + pp] - w0);
            wq[v] = side == 0 ? w0 + (T(0.5) * sl) : w0 - (T(0.5) * sl);
          }
          prim_to_cons<T, D>(wq, gm1, Qf);
#pragma unroll
          for (int v = 0; v < NV; v++) Qf[v] = Qf[v] + DQ[v * NS + pd];
          if (side == 0) cons_to_prim<T, D>(Qf, gm1, wl);
          else cons_to_prim<T, D>(Qf, gm1, wr);
        }
        ausmdv<T, D>(n, wl, wr, gam, goverg1, F);
      }
      const int fi = (f - fb.a[0]) + (fb.b[0] - fb.a[0]) * ((u1 - fb.a[1]) + (fb.b[1] - fb.a[1]) * (u2 - fb.a[2]));
#pragma unroll
      for (int v = 0; v < NV; v++) FL[(n * NV + v) * NFACE + fi] = F[v];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < reg.count(); q += NT) {
    int x, y, z;
    reg.at(q, x, y, z);
    const int p = pidx(x, y, z);
    const int rx = x - reg.a[0], ry = y - reg.a[1], rz = z - reg.a[2];
    const int w0 = reg.b[0] - reg.a[0], w1 = reg.b[1] - reg.a[1], w2 = reg.b[2] - reg.a[2];
    const int f0 = rx + (w0 + 1) * (ry + w1 * rz), f1 = ry + (w1 + 1) * (rx + w0 * rz),
              f2 = rz + (w2 + 1) * (rx + w0 * ry);
    T o[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
      T r = lam[0] * (FL[(0 * NV + v) * NFACE + f0 + 1] - FL[(0 * NV + v) * NFACE + f0]);
      r = r + lam[1] * (FL[(1 * NV + v) * NFACE + f1 + 1] - FL[(1 * NV + v) * NFACE + f1]);
      if (D == 3) r = r + lam[2] * (FL[(2 * NV + v) * NFACE + f2 + 1] - FL[(2 * NV + v) * NFACE + f2]);
      o[v] = q0[v * NS + p] - r;
      out[v * NS + p] = o[v];
    }
    if (w_next) {  // the next stage's primitives: its input region is this stage's output region
      T w[NV];
      cons_to_prim<T, D>(o, gm1, w);
#pragma unroll
      for (int v = 0; v < NV; v++) W[v * NS + p] = w[v];
    }
  }
  __syncthreads();
}

// H_dt on a patch of edge E: the stages of one step, each on the region `lo`/`hi`
// of its row (cells per dimension, clipped to the domain).  The result is in A
// (RK2: both stages; the second writes A in place) or, for the one Hancock stage,
// in `res`.
// w_ready: W already holds the primitives of A's input region; w_next: leave the
// primitives of the step's result in W for the next step.
template <typename T, int D, bool HANCOCK>
__device__ void rich_step(T *A, T *Sb, T *res, T *W, T *DQ, T *FL, int lo1, int hi1, int lo2, int hi2,
                          const int *dl, const int *dh, double dt, const double *dx, T gam, T gm1, T goverg1, int E,
                          bool w_ready, bool w_next) {
  T lam1[3], lam2[3], hh[3];
  for (int d = 0; d < 3; d++) {
    lam1[d] = T((0.5 * dt) / dx[d]);
    lam2[d] = T((1.0 * dt) / dx[d]);
    hh[d] = T((0.5 * dt) / dx[d]);
  }
  auto box = [&](int lo, int hi) {
    RBox b;
    for (int d = 0; d < 3; d++) {
      b.a[d] = d < D ? max(lo, dl[d]) : 0;
      b.b[d] = d < D ? min(hi, dh[d]) : 1;
    }
    return b;
  };
  if constexpr (HANCOCK) {
    rich_stage<T, D, true>(A, A, res, W, DQ, FL, box(lo2, hi2), dl, dh, lam2, hh, gam, gm1, goverg1, E, w_ready,
                           w_next);
  } else {
    rich_stage<T, D, false>(A, A, Sb, W, DQ, FL, box(lo1, hi1), dl, dh, lam1, hh, gam, gm1, goverg1, E, w_ready,
                            true);
    rich_stage<T, D, false>(Sb, A, A, W, DQ, FL, box(lo2, hi2), dl, dh, lam2, hh, gam, gm1, goverg1, E, true,
                            w_next);
  }
}

// Per block: rmask = bit (x + 4 y + 16 z) set for each of its coarse cells with
// |tau| > eps_r, maxdet = the largest |tau| of its coarse cells.  Levels l0..L-1;
// with A0 set, the absent cells of level l0 are predicted from level l0-1
// interpolated in time, A0 + theta (A - A0) (a remesh inside the level recursion).
template <typename T, int D, bool HANCOCK>
__global__ void __launch_bounds__(RichShape<D, HANCOCK>::NT) k_rich(Geo g, const T *__restrict__ A, const T *__restrict__ A0,
                                                           T theta, int l0, const double *__restrict__ lev,
                                                           double eps_r, unsigned long long *rmask, double *maxdet,
                                                           T *scratch, unsigned long long *nblk) {
  using S = RichShape<D, HANCOCK>;
  constexpr int NV = S::NV, P = S::P, PC = S::PC, NP = S::NP, NPC = S::NPC, NT = S::NT, H = S::H;
  constexpr int NC = (D == 2) ? 16 : 64;  // coarse cells of a block
  __shared__ T cc[NC], tau[NC];
  if (g.L < 1 || l0 > g.L - 1) return;
  int b, e;
  list_range(g, LK_EXIST, l0, g.L - 1, b, e);
  if (nblk && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(nblk, (unsigned long long)(e - b));
  const long long cap = g.cap;
  // 2D patches fit in shared memory (dynamic, S::PER values); 3D ones use the
  // CTA's area of the global scratch
  extern __shared__ __align__(16) unsigned char rich_smem[];
  T *Ab = (D == 2) ? reinterpret_cast<T *>(rich_smem) : scratch + (long long)blockIdx.x * S::PER;
  T *Sb = Ab + NV * NP, *Wb = Sb + NV * NP, *DQb = Wb + NV * NP;
  T *CA = DQb + NV * NP, *CS = CA + NV * NPC, *FL = CS + NV * NPC, *CP = FL + D * NV * S::NFACE;
  constexpr int PP = S::PP, NPP = S::NPP;
  const T gam = T(g.gamma), gm1 = T(g.gamma - 1.0), goverg1 = T(g.gamma / (g.gamma - 1.0));
  for (int it = b + blockIdx.x; it < e; it += gridDim.x) {
    const int s = g.lists[LK_EXIST * cap + it];
    const int l = g.slot_level[s];
    const int bc3[3] = {g.slot_coord[3 * s], g.slot_coord[3 * s + 1], g.slot_coord[3 * s + 2]};
    const double dtl = lev[lev_index(1, l, 3)];
    // the domain's cells of the fine and coarse patches (periodic: all)
    int dl[3], dh[3], cdl[3], cdh[3];
    for (int d = 0; d < 3; d++) {
      if (d >= D) {
        dl[d] = cdl[d] = 0;
        dh[d] = cdh[d] = 1;
      } else if (g.bc == 1) {
        dl[d] = cdl[d] = 0;
        dh[d] = P;
        cdh[d] = PC;
      } else {
        const int og = 8 * bc3[d] - H, N = g.nb[l][d] * 8;
        dl[d] = max(0, -og);
        dh[d] = min(P, N - og);
        cdl[d] = max(0, -og / 2);
        cdh[d] = min(PC, N / 2 - og / 2);
      }
    }
    // gather E on the fine patch (domain cells only): the value of the cell's block,
    // or the third-order prediction from level l-1, whose cells the patch needs
    // (coarse cells 4 bc - H/2 - 1 .. 4 bc + 4 + H/2 per dimension, by the boundary
    // rule, in time-interpolated form at level l0 with A0) are staged in CP first
    {
      const T *C0 = (l == l0) ? A0 : nullptr;
      if (l > 0) {
        RBox pb;
        for (int d = 0; d < 3; d++) {
          pb.a[d] = 0;
          pb.b[d] = d < D ? PP : 1;
        }
        for (int r = threadIdx.x; r < pb.count(); r += NT) {
          int c[3];
          pb.at(r, c[0], c[1], c[2]);
          const int q = c[0] + PP * (c[1] + PP * c[2]);
          int cg[3] = {0, 0, 0};
          for (int d = 0; d < D; d++) cg[d] = bc_cell(g, l - 1, d, 4 * bc3[d] - H / 2 - 1 + c[d]);
          const int32_t sc = g.idx[map_index(g, l - 1, cg[0] >> 3, cg[1] >> 3, cg[2] >> 3)];
          const int cin = (cg[0] & 7) + 8 * (cg[1] & 7) + (D == 3 ? 64 * (cg[2] & 7) : 0);
#pragma unroll
          for (int v = 0; v < NV; v++) {
            T val = nan_val<T>();  // an absent coarse block is never read by a prediction of the tree
            if (sc >= 0) {
              const long long off = ((long long)v * cap + sc) * (D == 2 ? 64 : 512) + cin;
              val = A[off];
              if (C0) {
                const T a0 = C0[off];
                val = a0 + theta * (val - a0);
              }
            }
            CP[v * NPP + q] = val;
          }
        }
        __syncthreads();
      }
      RBox gb;
      for (int d = 0; d < 3; d++) {
        gb.a[d] = dl[d];
        gb.b[d] = dh[d];
      }
      for (int q = threadIdx.x; q < gb.count(); q += NT) {
        int x, y, z;
        gb.at(q, x, y, z);
        const int u[3] = {8 * bc3[0] - H + x, 8 * bc3[1] - H + y, D == 3 ? 8 * bc3[2] - H + z : 0};  // unwrapped
        int f[3] = {0, 0, 0};
        for (int d = 0; d < D; d++) f[d] = bc_cell(g, l, d, u[d]);
        const int32_t sf = g.idx[map_index(g, l, f[0] >> 3, f[1] >> 3, f[2] >> 3)];
        const int p = x + P * (y + P * z);
        if (sf >= 0) {
          const int c = (f[0] & 7) + 8 * (f[1] & 7) + (D == 3 ? 64 * (f[2] & 7) : 0);
#pragma unroll
          for (int v = 0; v < NV; v++) Ab[v * NP + p] = A[((long long)v * cap + sf) * (D == 2 ? 64 : 512) + c];
        } else if (l == 0) {  // level 0 is complete: a missing block is a broken tree
          set_err(g, EB_TREE);
#pragma unroll
          for (int v = 0; v < NV; v++) Ab[v * NP + p] = nan_val<T>();
        } else {
          // parent of the cell in CP: (u >> 1) - (4 bc - H/2 - 1), i.e. 1..PC
          const int px = (x >> 1) + 1, py = (y >> 1) + 1, pz = D == 3 ? (z >> 1) + 1 : 0;
          const T si = (f[0] & 1) ? T(-1) : T(1), sj = (f[1] & 1) ? T(-1) : T(1), sk = (f[2] & 1) ? T(-1) : T(1);
#pragma unroll
          for (int v = 0; v < NV; v++) Ab[v * NP + p] = predict<T, D, PP>(CP + v * NPP, px, py, pz, si, sj, sk);
        }
      }
    }
    __syncthreads();
    // R E on the coarse patch: children summed in lexicographic order (x fastest)
    {
      RBox cb;
      for (int d = 0; d < 3; d++) {
        cb.a[d] = cdl[d];
        cb.b[d] = cdh[d];
      }
      for (int q = threadIdx.x; q < cb.count(); q += NT) {
        int x, y, z;
        cb.at(q, x, y, z);
        const int pc = x + PC * (y + PC * z);
        T Q[NV], w[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
          T sum = T(0);
#pragma unroll
          for (int k = 0; k < (D == 3 ? 8 : 4); k++) {
            const int p = (2 * x + (k & 1)) + P * ((2 * y + ((k >> 1) & 1)) + P * (D == 3 ? 2 * z + (k >> 2) : 0));
            const T val = Ab[v * NP + p];
            sum = k == 0 ? val : sum + val;
          }
          Q[v] = sum * T(D == 3 ? 0.125 : 0.25);
          CA[v * NPC + pc] = Q[v];
        }
        cons_to_prim<T, D>(Q, gm1, w);  // the first coarse stage's primitives (its input region)
#pragma unroll
        for (int v = 0; v < NV; v++) Wb[v * NPC + pc] = w[v];
      }
    }
    __syncthreads();
    // coarse step of 2 dt (MR scheme: cells 2..PC-2 then 4..PC-4 of the coarse
    // patch; AMR scheme: its one stage on 2..PC-2, the block's coarse cells)
    double dxc[3], dxf[3];
    for (int d = 0; d < 3; d++) {
      dxf[d] = g.dx[l][d];
      dxc[d] = 2.0 * g.dx[l][d];
    }
    rich_step<T, D, HANCOCK>(CA, CS, CS, Wb, DQb, FL, 2, PC - 2, HANCOCK ? 2 : 4, HANCOCK ? PC - 2 : PC - 4, cdl, cdh,
                             2.0 * dtl, dxc, gam, gm1, goverg1, PC, true, false);
    const T *Cres = HANCOCK ? CS : CA;
    for (int q = threadIdx.x; q < NC; q += NT) {
      const int x = q & 3, y = (q >> 2) & 3, z = q >> 4;
      cc[q] = Cres[(H / 2 + x) + PC * ((H / 2 + y) + PC * (D == 3 ? H / 2 + z : 0))];
    }
    // two fine steps of dt (regions 2..P-2, 4..P-4, 6..P-6, 8..P-8; AMR scheme 2..P-2, 4..P-4)
    if constexpr (HANCOCK) {
      rich_step<T, D, true>(Ab, Sb, Sb, Wb, DQb, FL, 0, 0, 2, P - 2, dl, dh, dtl, dxf, gam, gm1, goverg1, P, false,
                            true);
      rich_step<T, D, true>(Sb, Ab, Ab, Wb, DQb, FL, 0, 0, 4, P - 4, dl, dh, dtl, dxf, gam, gm1, goverg1, P, true,
                            false);
    } else {
      rich_step<T, D, false>(Ab, Sb, Ab, Wb, DQb, FL, 2, P - 2, 4, P - 4, dl, dh, dtl, dxf, gam, gm1, goverg1, P,
                             false, true);
      rich_step<T, D, false>(Ab, Sb, Ab, Wb, DQb, FL, 6, P - 6, 8, P - 8, dl, dh, dtl, dxf, gam, gm1, goverg1, P,
                             true, false);
    }
    // restrict the fine result on the block and compare
    for (int q = threadIdx.x; q < NC; q += NT) {
      const int x = q & 3, y = (q >> 2) & 3, z = q >> 4;
      T sum = T(0);
#pragma unroll
      for (int k = 0; k < (D == 3 ? 8 : 4); k++) {
        const int p = (H + 2 * x + (k & 1)) + P * ((H + 2 * y + ((k >> 1) & 1)) + P * (D == 3 ? H + 2 * z + (k >> 2) : 0));
        const T val = Ab[p];
        sum = k == 0 ? val : sum + val;
      }
      tau[q] = (sum * T(D == 3 ? 0.125 : 0.25) - cc[q]) / T(6);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // warp 0: mask by ballot, maximum by shuffles
      const int ln = threadIdx.x;
      const T t0 = ln < NC ? fabs(tau[ln]) : T(0), t1 = ln + 32 < NC ? fabs(tau[ln + 32]) : T(0);
      const unsigned lo = __ballot_sync(0xffffffffu, t0 > T(eps_r)), hi = __ballot_sync(0xffffffffu, t1 > T(eps_r));
      double m = (double)(t0 > t1 ? t0 : t1);
      for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, m, o);
        m = u > m ? u : m;
      }
      if (ln == 0) {
        const long long mi = map_index(g, l, bc3[0], bc3[1], bc3[2]);
        rmask[mi] = (unsigned long long)lo | ((unsigned long long)hi << 32);
        maxdet[mi] = m;
      }
    }
    __syncthreads();
  }
}

// Richardson block flags: a block of levels l0..L-1 is flagged (gflag |= 1) when
// its own mask or the mask of an existing same-level neighbour has a coarse cell
// within one fine cell of it (the neighbour's coarse layer next to the shared
// face, edge or corner).
template <int D>
__global__ void k_rich_flags(Geo g, int l0, const unsigned long long *__restrict__ rmask, uint8_t *gflag) {
  if (g.L < 1 || l0 > g.L - 1) return;
  int b, e;
  list_range(g, LK_EXIST, l0, g.L - 1, b, e);
  const long long cap = g.cap;
  for (int it = b + blockIdx.x * blockDim.x + threadIdx.x; it < e; it += gridDim.x * blockDim.x) {
    const int s = g.lists[LK_EXIST * cap + it];
    const int l = g.slot_level[s];
    const int bc3[3] = {g.slot_coord[3 * s], g.slot_coord[3 * s + 1], g.slot_coord[3 * s + 2]};
    const long long self = map_index(g, l, bc3[0], bc3[1], bc3[2]);
    bool hit = rmask[self] != 0;
    for (int o = 0; o < (D == 3 ? 27 : 9) && !hit; o++) {
      const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, D == 3 ? o / 9 - 1 : 0};
      if (off[0] == 0 && off[1] == 0 && off[2] == 0) continue;
      int nb[3];
      bool in = true;
      for (int d = 0; d < 3; d++) {
        nb[d] = bc3[d] + off[d];
        if (d >= D) continue;
        const int N = g.nb[l][d];
        if (nb[d] < 0 || nb[d] >= N) {
          if (g.bc == 1) nb[d] = (nb[d] + N) % N;
          else in = false;
        }
      }
      if (!in) continue;
      const long long mi = map_index(g, l, nb[0], nb[1], nb[2]);
      if (g.idx[mi] < 0) continue;
      const unsigned long long m = rmask[mi];
      // coarse cells of the neighbour next to this block: layer 3 (neighbour below),
      // layer 0 (above) or every layer (same position) in each direction
      for (int q = 0; q < (D == 3 ? 64 : 16); q++) {
        const int c[3] = {q & 3, (q >> 2) & 3, q >> 4};
        bool adj = true;
        for (int d = 0; d < D; d++)
          if ((off[d] < 0 && c[d] != 3) || (off[d] > 0 && c[d] != 0)) adj = false;
        if (adj && ((m >> q) & 1ull)) hit = true;
      }
    }
    if (hit) gflag[self] = 1;
  }
}

}  // namespace mrfv
