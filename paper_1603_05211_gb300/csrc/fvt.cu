// TMA-staged finite-volume stage of the MR scheme for 2D single-precision
// state: MUSCL reconstruction of the primitive variables with the van Albada
// limiter, the AUSM+ flux and the conservative stage update of the explicit
// midpoint rule (arXiv:1603.05211, Section 2), one flux per face of each 8x8
// block (block-boundary faces once per side).
//
// A persistent CTA takes G blocks per iteration:
//  1. one lane per block issues tensor-memory-accelerator (TMA) copies of the
//     block's four conserved variables, the two columns / rows beyond each face
//     (the same-level neighbour's edge as a 4x8 or 8x2 box, or the coarse-fine
//     ghost strip), and the block's stage start state, all completing on one
//     mbarrier (bounded wait);
//  2. the CTA converts the block and its halo to primitive variables once,
//     into a padded 12x12 tile per block (transmissive walls: the edge cell's
//     primitives);
//  3. sixteen threads per block walk the lines: each thread takes row t and
//     column t of the block together, the x-face and the y-face of the same step
//     in the two lanes of packed FP32x2 arithmetic (normal and tangential
//     velocity swap roles between the lanes), half a line each (faces 0..4 or
//     4..8, the middle face evaluated by both halves); flux differences go to
//     shared memory;
//  4. the update Q_out = Q_0 - (lambda_x dF_x + lambda_y dF_y) is written to
//     global memory with coalesced stores.
// Reciprocals and square roots use the approximate hardware instructions
// (single-precision throughput mode).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"
#include "launch.h"

namespace mrfv {

namespace fvt {
constexpr int G = 8;                                  // blocks per CTA iteration
constexpr int NT = 16 * G;                            // threads: 16 per block
// per-block TMA staging area (bytes): the block, then the boxes beyond x-lo,
// x-hi, y-lo, y-hi (neighbour edge or ghost strip)
constexpr int ST_OWN = 0, ST_XLO = 1024, ST_XHI = 1536, ST_YLO = 2048, ST_YHI = 2304, ST_BYTES = 2560;
constexpr int U0_BYTES = 1024;                        // the block's stage start state
constexpr int TR = 13;                                // primitive tile row stride (floats)
constexpr int TV = 12 * TR;                           // floats per variable of a tile
constexpr int TILE = 648;                             // floats per block tile (4 TV = 624, padded so
                                                      // consecutive tiles start 8 banks apart)
constexpr size_t OFF_U0 = (size_t)G * ST_BYTES;
constexpr size_t OFF_TILE = OFF_U0 + (size_t)G * U0_BYTES;
constexpr size_t OFF_MBAR = OFF_TILE + (size_t)G * TILE * 4;
constexpr size_t OFF_INFO = OFF_MBAR + 16;            // per block: slot, neighbours, refined mask, lambdas
constexpr size_t SMEM = OFF_INFO + (size_t)G * 12 * 4;
constexpr unsigned kWait = 1u << 24;                  // bounded mbarrier wait (try_wait iterations)
}  // namespace fvt

// ---------------------------------------------------------------- packed FP32x2 arithmetic
struct F2 {
  float2 v;
};
__device__ __forceinline__ F2 f2(float a, float b) { return F2{make_float2(a, b)}; }
__device__ __forceinline__ F2 f2s(float a) { return F2{make_float2(a, a)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ F2 rcp2(F2 a) { return f2(rcp_approx(a.v.x), rcp_approx(a.v.y)); }
__device__ __forceinline__ F2 rsqrt2(F2 a) { return f2(rsqrt_approx(a.v.x), rsqrt_approx(a.v.y)); }
__device__ __forceinline__ F2 max02(F2 a) { return f2(fmaxf(a.v.x, 0.f), fmaxf(a.v.y, 0.f)); }
__device__ __forceinline__ F2 min02(F2 a) { return f2(fminf(a.v.x, 0.f), fminf(a.v.y, 0.f)); }
__device__ __forceinline__ F2 sat2(F2 a) { return f2(__saturatef(a.v.x), __saturatef(a.v.y)); }
__device__ __forceinline__ F2 sel2(bool mx, bool my, F2 a, F2 b) { return f2(mx ? a.v.x : b.v.x, my ? a.v.y : b.v.y); }

// primitive state of a face side or cell in the lanes' own frame: c[0] density,
// c[1] normal velocity, c[2] tangential velocity, c[3] pressure
struct W2 {
  F2 c[4];
};

// van Albada slope with the TVD clip: max(a b, 0) (a + b) / (a^2 + b^2) (the
// tiny addend keeps a = b = 0 at slope 0)
__device__ __forceinline__ F2 van_albada2(F2 a, F2 b) {
  F2 num = max02(a * b) * (a + b);
  F2 den = fma2(a, a, fma2(b, b, f2s(1e-30f)));
  return num * rcp2(den);
}

// AUSM+ split Mach number and pressure of Liou (1996), beta = 1/8, alpha = 3/16.
// With c = clamp(M, -1, 1), the subsonic polynomials expanded in powers of c
// give the supersonic forms as well:
//   M4+(M) = c^4/8 + c/2 + 3/8 + max(M - 1, 0)      (= max(M, 0) when |M| >= 1)
//   M4-(M) = -c^4/8 + c/2 - 3/8 + min(M + 1, 0)     (= min(M, 0))
//   P5+(M) =  c (3/16 c^4 - 5/8 c^2 + 15/16) + 1/2   (= [M > 0])
//   P5-(M) = -c (3/16 c^4 - 5/8 c^2 + 15/16) + 1/2   (= [M < 0])
// (expanding 1/4 (M +- 1)^2 +- 1/8 (M^2 - 1)^2 and
// 1/4 (M +- 1)^2 (2 -+ M) +- 3/16 M (M^2 - 1)^2).
template <int SGN>
__device__ __forceinline__ void ausm_split2(F2 M, F2 &m4, F2 &p5) {
  const F2 c = f2(fminf(fmaxf(M.v.x, -1.f), 1.f), fminf(fmaxf(M.v.y, -1.f), 1.f));
  const F2 c2 = c * c;
  const F2 lin = fma2(f2s(0.5f), c, f2s(0.375f * SGN));                 // c/2 +- 3/8
  const F2 quart = fma2(f2s(0.125f * SGN) * c2, c2, lin);              // +-c^4/8 + ...
  const F2 over = M - f2s((float)SGN);                                  // M -+ 1
  const F2 sup = SGN > 0 ? max02(over) : min02(over);
  m4 = quart + sup;
  const F2 q = fma2(fma2(f2s(0.1875f * SGN), c2, f2s(-0.625f * SGN)), c2, f2s(0.9375f * SGN));
  p5 = fma2(c, q, f2s(0.5f));
}

// AUSM+ flux of both lanes' faces from the left / right primitive states;
// interface sound speed = arithmetic mean.  F: mass, normal momentum,
// tangential momentum, energy.
__device__ __forceinline__ void ausm_plus2(const W2 &L, const W2 &R, float gam, float goverg1, F2 *F) {
  const F2 g = f2s(gam);
  F2 xl = g * L.c[3], xr = g * R.c[3];
  F2 cl = xl * rsqrt2(xl * L.c[0]);           // sqrt(gamma p / rho) = x / sqrt(x rho), x = gamma p
  F2 cr = xr * rsqrt2(xr * R.c[0]);
  F2 ch = f2s(0.5f) * (cl + cr);
  F2 ich = rcp2(ch);
  F2 ML = L.c[1] * ich, MR = R.c[1] * ich;
  F2 m4p, p5p, m4m, p5m;
  ausm_split2<1>(ML, m4p, p5p);
  ausm_split2<-1>(MR, m4m, p5m);
  F2 m = m4p + m4m;
  F2 ph = fma2(p5p, L.c[3], p5m * R.c[3]);
  F2 a = ch * m;
  const bool ux = m.v.x >= 0.f, uy = m.v.y >= 0.f;
  F2 ru = sel2(ux, uy, L.c[0], R.c[0]), nu = sel2(ux, uy, L.c[1], R.c[1]);
  F2 tu = sel2(ux, uy, L.c[2], R.c[2]), pu = sel2(ux, uy, L.c[3], R.c[3]);
  F2 q = fma2(nu, nu, tu * tu);
  F2 rH = fma2(f2s(goverg1), pu, (f2s(0.5f) * ru) * q);
  F2 fm = a * ru;
  F[0] = fm;
  F[1] = fma2(fm, nu, ph);
  F[2] = fm * tu;
  F[3] = a * rH;
}

// ---------------------------------------------------------------- TMA and mbarrier
__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap *m, int c0, int c1, int c2, int c3,
                                       uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap *m, int c0, int c1, int c2, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  for (unsigned it = 0; it < fvt::kWait; it++)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

// ---------------------------------------------------------------- the kernel
// Tile index of cell (x, y), x, y in -2..9, of variable v.
__device__ __forceinline__ int tile_at(int v, int x, int y) { return v * fvt::TV + (y + 2) * fvt::TR + (x + 2); }

// Primitives of two cells (packed) from their conserved values.
__device__ __forceinline__ void cons2prim(F2 q0, F2 q1, F2 q2, F2 q3, float gm1, F2 *w) {
  F2 ir = rcp2(q0);
  F2 u = q1 * ir, v = q2 * ir;
  F2 k = fma2(q2, v, q1 * u);  // rho |v|^2
  w[0] = q0;
  w[1] = u;
  w[2] = v;
  w[3] = fma2(f2s(-0.5f * gm1), k, f2s(gm1) * q3);
}

__global__ void __launch_bounds__(fvt::NT, 4) k_fvt(Geo g, FVArgs<float> a, const __grid_constant__ FvtMaps maps) {
  using namespace fvt;
  extern __shared__ __align__(1024) unsigned char sm[];
  // block information of the iteration (after the tiles): slot, 4 neighbours, refined mask, 3 lambdas
  int *sslot = reinterpret_cast<int *>(sm + OFF_INFO);
  int(*snb)[4] = reinterpret_cast<int(*)[4]>(sslot + G);
  int *scm = reinterpret_cast<int *>(snb + G);
  float(*slam)[3] = reinterpret_cast<float(*)[3]>(scm + G);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // every TMA destination below is a multiple of 128 bytes from the start of the
  // dynamic shared memory, which must itself be 128-byte aligned
  if (s_addr(sm) & 127u) {
    if (tid == 0) atomicOr(g.err, EB_TREE);
    return;
  }
  const long long cap = g.cap;
  const float gam = (float)g.gamma, gm1 = (float)(g.gamma - 1.0), goverg1 = (float)(g.gamma / (g.gamma - 1.0));
  const uint32_t mbar = s_addr(sm + OFF_MBAR);
  int lb, le;
  list_range(g, a.kind, a.l0, a.l1, lb, le);
  if (a.bytes && blockIdx.x == 0 && tid == 0) atomicAdd(a.bytes, (unsigned long long)(le - lb) * 64 * a.words * 4);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(G) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the issuing lanes (warp 0, lane j < G) hold their block's slot and neighbours one
  // iteration ahead
  int ns = -1, nnb[4] = {0, 0, 0, 0};
  auto fetch = [&](int i) {
    ns = -1;
    if (i < le) {
      ns = g.lists[a.kind * cap + i];
#pragma unroll
      for (int f = 0; f < 4; f++) nnb[f] = g.nbr[6 * ns + f];
    }
  };
  if (warp == 0 && lane < G) fetch(lb + blockIdx.x * G + lane);
  uint32_t parity = 0;
  for (int i0 = lb + blockIdx.x * G; i0 < le; i0 += gridDim.x * G) {
    // ---------------- 1. TMA of every block of this iteration
    if (warp == 0 && lane < G) {
      const int j = lane, s = ns;
      uint32_t bytes = 0;
      unsigned char *st = sm + (size_t)j * ST_BYTES;
      if (s >= 0) {
        sslot[j] = s;
#pragma unroll
        for (int f = 0; f < 4; f++) snb[j][f] = nnb[f];
        bytes = 1024 + 1024;
#pragma unroll
        for (int f = 0; f < 4; f++) {
          if (nnb[f] >= 0) bytes += f < 2 ? 512 : 256;
          else if (nnb[f] == NBR_MISSING) bytes += 256;
        }
      } else {
        sslot[j] = -1;
      }
      mbar_arrive_tx(mbar, bytes);
      if (s >= 0) {
        tma_4d(s_addr(st + ST_OWN), &maps.in_own, 0, 0, s, 0, mbar);
        tma_4d(s_addr(sm + OFF_U0 + (size_t)j * U0_BYTES), &maps.u0_own, 0, 0, s, 0, mbar);
        const int off[4] = {ST_XLO, ST_XHI, ST_YLO, ST_YHI};
#pragma unroll
        for (int f = 0; f < 4; f++) {
          const uint32_t dst = s_addr(st + off[f]);
          if (nnb[f] >= 0) {
            if (f == 0) tma_4d(dst, &maps.in_xh, 4, 0, nnb[f], 0, mbar);       // columns 4..7
            else if (f == 1) tma_4d(dst, &maps.in_xh, 0, 0, nnb[f], 0, mbar);  // columns 0..3
            else if (f == 2) tma_4d(dst, &maps.in_yh, 0, 6, nnb[f], 0, mbar);  // rows 6, 7
            else tma_4d(dst, &maps.in_yh, 0, 0, nnb[f], 0, mbar);              // rows 0, 1
          } else if (nnb[f] == NBR_MISSING) {
            tma_3d(dst, &maps.ghost, 0, 4 * s + f, 0, mbar);                   // [v][layer][t]
          }
        }
        // read by the lines and the update only (after a CTA barrier)
        const int l = g.slot_level[s];
        scm[j] = g.cmask[s];
#pragma unroll
        for (int d = 0; d < 2; d++) slam[j][d] = a.levf[lev_index(a.stage, l, d)];
        slam[j][2] = a.levf[lev_index(a.stage, l, 3)];
      }
      fetch(i0 + gridDim.x * G + lane);
    }
    // ---------------- wait for the copies (bounded; one decision for the CTA)
    // one thread polls (bounded), the CTA learns the outcome at the barrier, then every
    // thread observes the completed phase once (which acquires the copies' writes)
    bool got = true;
    if (tid == 0) got = mbar_wait_bounded(mbar, parity);
    const bool ok = __syncthreads_and(got ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) {
        atomicOr(g.err, EB_TIMEOUT);
        mbar_wait_bounded(mbar, parity);  // copies still in flight: wait for them (bounded) before leaving
      }
      __syncthreads();
      return;
    }
    mbar_wait_bounded(mbar, parity);      // completes at once
    parity ^= 1u;
    // ---------------- 2. primitives of each block and its halo into the tile
    {
      const int j = tid >> 4, r = tid & 15;
      if (sslot[j] >= 0) {
        const float *st = reinterpret_cast<const float *>(sm + (size_t)j * ST_BYTES);
        float *T = reinterpret_cast<float *>(sm + OFF_TILE) + (size_t)j * TILE;
#pragma unroll
        for (int i = 0; i < 4; i++) {
          // two cells (x0, y0), (x1, y1) of the tile; their conserved values
          F2 q[4];
          int x0, y0, x1, y1;
          int dup = 0;  // wall: the pair is stored twice (both ghost layers)
          int e = r < 8 ? r + 8 * i : 4 * ((r - 8) & 1) + i;   // pair index within the interior / the face
          if (r < 8) {
            y0 = y1 = e >> 2;
            x0 = 2 * (e & 3);
            x1 = x0 + 1;
            const float *src = st + y0 * 8 + x0;
#pragma unroll
            for (int v = 0; v < 4; v++) {
              float2 c = *reinterpret_cast<const float2 *>(src + 64 * v);
              q[v] = F2{c};
            }
          } else {
            const int f = (r - 8) >> 1;
            const int nb = snb[j][f];
            const int layer = e >> 2, t0 = 2 * (e & 3);   // ghost-strip / edge pair: depth, first cell along the face
            // tile cells of the pair
            if (f < 2) {
              x0 = x1 = f == 0 ? -1 - layer : 8 + layer;
              y0 = t0;
              y1 = t0 + 1;
            } else {
              y0 = y1 = f == 2 ? -1 - layer : 8 + layer;
              x0 = t0;
              x1 = t0 + 1;
            }
            if (nb >= 0) {
              // neighbour edge box: x faces [v][y][4] (columns 4..7 or 0..3), y faces [v][2][x]
              if (f < 2) {
                // pair = the two depths of row e (cells (-2,y),(-1,y) or (8,y),(9,y))
                y0 = y1 = e;
                x0 = f == 0 ? -2 : 8;
                x1 = x0 + 1;
                const float *src = st + (f == 0 ? ST_XLO : ST_XHI) / 4 + e * 4 + (f == 0 ? 2 : 0);
#pragma unroll
                for (int v = 0; v < 4; v++) q[v] = F2{*reinterpret_cast<const float2 *>(src + 32 * v)};
              } else {
                const int row = e >> 2;   // box row 0, 1 = rows 6, 7 (lo) or 0, 1 (hi)
                y0 = y1 = f == 2 ? -2 + row : 8 + row;
                x0 = t0;
                x1 = t0 + 1;
                const float *src = st + (f == 2 ? ST_YLO : ST_YHI) / 4 + row * 8 + t0;
#pragma unroll
                for (int v = 0; v < 4; v++) q[v] = F2{*reinterpret_cast<const float2 *>(src + 16 * v)};
              }
            } else if (nb == NBR_MISSING) {
              const int off = f == 0 ? ST_XLO : (f == 1 ? ST_XHI : (f == 2 ? ST_YLO : ST_YHI));
              const float *src = st + off / 4 + layer * 8 + t0;
#pragma unroll
              for (int v = 0; v < 4; v++) q[v] = F2{*reinterpret_cast<const float2 *>(src + 16 * v)};
            } else {
              // transmissive wall: the edge cells of the block, into both ghost layers
              dup = 1;
              if (layer) continue;  // the depth-0 pairs write both layers
              if (f < 2) {
                const int xe = f == 0 ? 0 : 7;
#pragma unroll
                for (int v = 0; v < 4; v++) q[v] = f2(st[64 * v + t0 * 8 + xe], st[64 * v + (t0 + 1) * 8 + xe]);
              } else {
                const int ye = f == 2 ? 0 : 7;
#pragma unroll
                for (int v = 0; v < 4; v++) q[v] = F2{*reinterpret_cast<const float2 *>(st + 64 * v + ye * 8 + t0)};
              }
            }
          }
          F2 w[4];
          cons2prim(q[0], q[1], q[2], q[3], gm1, w);
#pragma unroll
          for (int v = 0; v < 4; v++) {
            T[tile_at(v, x0, y0)] = w[v].v.x;
            T[tile_at(v, x1, y1)] = w[v].v.y;
          }
          if (dup) {
            // second ghost layer of a wall
            const int f = (r - 8) >> 1;
            const int dx = f == 0 ? -1 : (f == 1 ? 1 : 0), dy = f == 2 ? -1 : (f == 3 ? 1 : 0);
#pragma unroll
            for (int v = 0; v < 4; v++) {
              T[tile_at(v, x0 + dx, y0 + dy)] = w[v].v.x;
              T[tile_at(v, x1 + dx, y1 + dy)] = w[v].v.y;
            }
          }
        }
      }
    }
    __syncthreads();
    // ---------------- 3. the lines: lane (jj, t) of warp w: block 4 (w >> 1) + jj, row t and
    // column t, half w & 1 of the faces
    {
      const int jj = lane >> 3, t = lane & 7, h = warp & 1;
      const int j = 4 * (warp >> 1) + jj;
      const int s = sslot[j];
      if (s >= 0) {
        const float *T = reinterpret_cast<const float *>(sm + OFF_TILE) + (size_t)j * TILE;
        // flux differences [v][c][t]: x lines dF_x(c, t) (transposed), y lines dF_y(t, c)
        float *dFx = reinterpret_cast<float *>(sm + (size_t)j * ST_BYTES) + 8 * (j & 3);
        float *dFy = dFx + 256;
        const int KB = 4 * h;
        const int ax = (t + 2) * TR + 2 + KB;        // x line: position p at ax + p
        const int ay = (2 + KB) * TR + (t + 2);      // y line: position p at ay + p TR
        auto load = [&](int p, W2 &w) {
          w.c[0] = f2(T[ax + p], T[ay + p * TR]);
          w.c[1] = f2(T[TV + ax + p], T[2 * TV + ay + p * TR]);       // x line: u, y line: v
          w.c[2] = f2(T[2 * TV + ax + p], T[TV + ay + p * TR]);       // x line: v, y line: u
          w.c[3] = f2(T[3 * TV + ax + p], T[3 * TV + ay + p * TR]);
        };
        // flux registers of this lane pair's outer faces (face 0: half 0, face 8: half 1)
        const int rec = a.record;
        const int cm = scm[j];
        const int fx = 2 * 0 + h, fy = 2 * 1 + h;    // register faces of the x and y lines
        const int nbx = snb[j][h], nby = snb[j][2 + h];
        const bool recx = rec && (nbx == NBR_MISSING || ((cm >> fx) & 1));
        const bool recy = rec && (nby == NBR_MISSING || ((cm >> fy) & 1));
        const bool addx = rec == 2 && nbx == NBR_MISSING, addy = rec == 2 && nby == NBR_MISSING;
        W2 wb, wc, wd;
        F2 dprev[4], slo[4], Fprev[4];
        {
          W2 wa;
          load(-2, wa);
          load(-1, wb);
          load(0, wc);
#pragma unroll
          for (int v = 0; v < 4; v++) {
            F2 d0 = wb.c[v] - wa.c[v];
            dprev[v] = wc.c[v] - wb.c[v];
            slo[v] = van_albada2(d0, dprev[v]);
          }
        }
#pragma unroll
        for (int k = 0; k < 5; k++) {
          load(k + 1, wd);
          W2 L, R;
          F2 shi[4];
#pragma unroll
          for (int v = 0; v < 4; v++) {
            F2 dn = wd.c[v] - wc.c[v];
            shi[v] = van_albada2(dprev[v], dn);
            dprev[v] = dn;
            L.c[v] = fma2(f2s(0.5f), slo[v], wb.c[v]);
            R.c[v] = fma2(f2s(-0.5f), shi[v], wc.c[v]);
          }
          F2 F[4];
          ausm_plus2(L, R, gam, goverg1, F);
          if (rec && ((h == 0 && k == 0) || (h == 1 && k == 4))) {
            const float dtT = slam[j][2];
            const long long vsR = cap * 32;
            float fxv[4] = {F[0].v.x, F[1].v.x, F[2].v.x, F[3].v.x};   // x face: (mass, mom x = n, mom y = t, E)
            float fyv[4] = {F[0].v.y, F[2].v.y, F[1].v.y, F[3].v.y};   // y face: (mass, mom x = t, mom y = n, E)
            if (recx) {
              float *Rr = a.FR + (long long)s * 32 + fx * 8 + t;
#pragma unroll
              for (int v = 0; v < 4; v++) {
                float val = dtT * fxv[v];
                Rr[v * vsR] = addx ? Rr[v * vsR] + val : val;
              }
            }
            if (recy) {
              float *Rr = a.FR + (long long)s * 32 + fy * 8 + t;
#pragma unroll
              for (int v = 0; v < 4; v++) {
                float val = dtT * fyv[v];
                Rr[v * vsR] = addy ? Rr[v * vsR] + val : val;
              }
            }
          }
          if (k > 0) {
            const int c = KB + k - 1;   // cell whose flux difference is complete
            F2 d[4];
#pragma unroll
            for (int v = 0; v < 4; v++) d[v] = F[v] - Fprev[v];
            float *px = dFx + c * 8 + t, *py = dFy + c * 8 + t;
            px[0] = d[0].v.x;
            px[64] = d[1].v.x;
            px[128] = d[2].v.x;
            px[192] = d[3].v.x;
            py[0] = d[0].v.y;
            py[64] = d[2].v.y;
            py[128] = d[1].v.y;
            py[192] = d[3].v.y;
          }
#pragma unroll
          for (int v = 0; v < 4; v++) {
            Fprev[v] = F[v];
            slo[v] = shi[v];
          }
          wb = wc;
          wc = wd;
        }
      }
    }
    __syncthreads();
    // ---------------- 4. update and store: each thread four cells (x0..x0+3, y) of one
    // block, every variable: Q_out = Q_0 - lambda_x dF_x - lambda_y dF_y
    {
      const long long vsU = cap * 64;
      const int j = tid >> 4, r = tid & 15;
      const int s = sslot[j];
      if (s >= 0) {
        const int y = r >> 1, x0 = 4 * (r & 1);
        const float *dFx = reinterpret_cast<const float *>(sm + (size_t)j * ST_BYTES) + 8 * (j & 3);
        const float *dFy = dFx + 256;
        const float *Q0 = reinterpret_cast<const float *>(sm + OFF_U0 + (size_t)j * U0_BYTES);
        const F2 mlx = f2s(-slam[j][0]), mly = f2s(-slam[j][1]);
        float *out = a.Uout + (long long)s * 64 + y * 8 + x0;
#pragma unroll
        for (int v = 0; v < 4; v++) {
          const float4 q = *reinterpret_cast<const float4 *>(Q0 + v * 64 + y * 8 + x0);
          const float4 dy = *reinterpret_cast<const float4 *>(dFy + v * 64 + y * 8 + x0);
          const float *dxp = dFx + v * 64 + x0 * 8 + y;   // dF_x stored [x][y]
          F2 lo = fma2(mlx, f2(dxp[0], dxp[8]), fma2(mly, f2(dy.x, dy.y), f2(q.x, q.y)));
          F2 hi = fma2(mlx, f2(dxp[16], dxp[24]), fma2(mly, f2(dy.z, dy.w), f2(q.z, q.w)));
          *reinterpret_cast<float4 *>(out + v * vsU) = make_float4(lo.v.x, lo.v.y, hi.v.x, hi.v.y);
        }
      }
    }
    // the staging area was written by this thread (flux differences): order those
    // writes before the next iteration's asynchronous copies into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
  }
  return fn;
}

// 4D map of a state buffer float[nv][cap][8][8]: dims (x, y, slot, v), box (bx, by, 1, nv)
bool encode_state(CUtensorMap *m, const void *base, long long cap, int nv, int bx, int by) {
  auto fn = encode_fn();
  if (!fn || !base) return false;
  cuuint64_t dims[4] = {8, 8, (cuuint64_t)cap, (cuuint64_t)nv};
  cuuint64_t strides[3] = {8 * 4, 64 * 4, (cuuint64_t)cap * 64 * 4};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)nv};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3D map of the ghost strips float[nv][cap * 4 faces][2 layers * 8]: box (16, 1, nv)
bool encode_ghost(CUtensorMap *m, const void *base, long long cap, int nv) {
  auto fn = encode_fn();
  if (!fn || !base) return false;
  cuuint64_t dims[3] = {16, (cuuint64_t)cap * 4, (cuuint64_t)nv};
  cuuint64_t strides[2] = {16 * 4, (cuuint64_t)cap * 4 * 16 * 4};
  cuuint32_t box[3] = {16, 1, (cuuint32_t)nv};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool fvt_prepare(FvtSet &set, const Geo &g, const void *U, const void *Us, const void *U0, const void *Gs) {
  set.ok = false;
  if (g.dim != 2 || g.nv != 4) return false;
  const void *bufs[3] = {U, Us, U0};
  for (int b = 0; b < 3; b++) {
    set.buf[b] = bufs[b];
    if (!bufs[b]) continue;
    if (!encode_state(&set.own[b], bufs[b], g.cap, 4, 8, 8)) return false;
    if (!encode_state(&set.xh[b], bufs[b], g.cap, 4, 4, 8)) return false;
    if (!encode_state(&set.yh[b], bufs[b], g.cap, 4, 8, 2)) return false;
  }
  if (!encode_ghost(&set.ghost, Gs, g.cap, 4)) return false;
  if (cudaFuncSetAttribute(k_fvt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fvt::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fvt, fvt::NT, fvt::SMEM) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return false;
  }
  set.ctas_per_sm = n;
  set.ok = true;
  return true;
}

int fvt_blocks_per_cta() { return fvt::G; }

bool launch_fvt(const Geo &g, const FVArgs<float> &a, const FvtSet &set, int grid, cudaStream_t st) {
  int bi = -1, b0 = -1;
  for (int b = 0; b < 3; b++) {
    if (set.buf[b] && set.buf[b] == (const void *)a.Uin) bi = b;
    if (set.buf[b] && set.buf[b] == (const void *)a.U0) b0 = b;
  }
  if (!set.ok || bi < 0 || b0 < 0) return false;
  FvtMaps m;
  m.in_own = set.own[bi];
  m.in_xh = set.xh[bi];
  m.in_yh = set.yh[bi];
  m.u0_own = set.own[b0];
  m.ghost = set.ghost;
  k_fvt<<<grid, fvt::NT, fvt::SMEM, st>>>(g, a, m);
  return true;
}

}  // namespace mrfv
