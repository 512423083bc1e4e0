// Learned refinement proposer: a 3-layer 3D convolutional net over per-block
// features of every level (16 channels, 3^3 kernels, zero padding, ReLU between
// layers; BF16 weights and activations, FP32 accumulation) whose logits mark
// the blocks to add before the next step.  It replaces the safety zone of the
// MR refinement rule; the MR thresholding at the next analysis still keeps and
// refines every significant block, so a missed block is re-refined one step
// later.  No counterpart in the paper (its refinement is Section 2.1's
// heuristic).
//
// Inference: implicit-GEMM convolution on the 5th-generation tensor cores.  A
// CTA takes 128 output positions (rows, M = 128) x 16 output channels
// (N = 16) x K = Cin * 27 taps; the im2col rows and the weights are staged in
// shared memory in the no-swizzle K-major core-matrix layout (8 x 16 B core
// matrices), one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32)
// per K = 16 slice into a TMEM accumulator of 128 lanes x 16 columns, commits
// to an mbarrier, and the four warps read the accumulator back with tcgen05.ld.
// Every wait is bounded; on expiry the kernel records EB_TIMEOUT, frees its TMEM
// and returns.
//
// Training: the same tensor-core convolutions for the forward pass and, with the
// taps mirrored, for the gradients of the layer inputs; weight gradients from the
// BF16 rows summed in double on the CUDA cores; Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"
#include "launch.h"

namespace mrfv {

// ---------------------------------------------------------------- geometry of positions
// Positions are the block positions of every level (dense maps, levels
// concatenated); a 3^3 neighbourhood stays inside the level (zero outside).
__device__ __forceinline__ int pos_level(const Geo &g, long long p) {
  int l = 0;
  while (l < g.L && p >= g.mapoff[l + 1]) l++;
  return l;
}
__device__ __forceinline__ long long pos_neighbour(const Geo &g, int l, long long p, int dx, int dy, int dz) {
  long long u = p - g.mapoff[l];
  int nx = g.nb[l][0], ny = g.nb[l][1], nz = g.nb[l][2];
  int x = (int)(u % nx) + dx, y = (int)((u / nx) % ny) + dy, z = (int)(u / ((long long)nx * ny)) + dz;
  if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return -1;
  return g.mapoff[l] + x + (long long)nx * (y + (long long)ny * z);
}

// ---------------------------------------------------------------- features
// Per position of level l: block-mean density / s_rho, block-mean pressure /
// ((gamma-1) s_E), and min(max normalised detail / eps, 8) / 8.  An absent block
// takes its means from the octant (quadrant) of its parent that covers it, and
// detail 0; without a parent all three are 0.
template <typename T, int D>
__global__ void k_prop_features(Geo g, const T *__restrict__ U, const double *__restrict__ maxdet,
                                const T *__restrict__ scale, double eps, float *__restrict__ feat) {
  constexpr int B = (D == 2) ? 64 : 512;
  const long long n = g.mapoff[g.L + 1];
  const long long cap = g.cap;
  const float srho = (float)scale[0], sp = (float)((g.gamma - 1.0) * (double)scale[D + 1]);
  const float gm1 = (float)(g.gamma - 1.0);
  const int lane = threadIdx.x & 31;
  const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
  // one warp per position: the lanes share the block's cells, then reduce
  for (long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nwarp) {
    int l = pos_level(g, p);
    long long u = p - g.mapoff[l];
    int bx = (int)(u % g.nb[l][0]), by = (int)((u / g.nb[l][0]) % g.nb[l][1]);
    int bz = (int)(u / ((long long)g.nb[l][0] * g.nb[l][1]));
    int32_t s = g.idx[p];
    int c0[3] = {0, 0, 0}, ext = 8;
    float f2 = 0.f;
    if (s < 0 && l > 0) {
      s = g.idx[map_index(g, l - 1, bx >> 1, by >> 1, bz >> 1)];
      c0[0] = 4 * (bx & 1);
      c0[1] = 4 * (by & 1);
      c0[2] = (D == 3) ? 4 * (bz & 1) : 0;
      ext = 4;
    } else if (s >= 0) {
      float m = (float)(maxdet[p] / eps);
      f2 = fminf(m, 8.f) / 8.f;
    }
    float sr = 0.f, spp = 0.f;
    const int ncell = (D == 3) ? ext * ext * ext : ext * ext;
    if (s >= 0) {
      for (int q = lane; q < ncell; q += 32) {
        int i = q % ext, j = (q / ext) % ext, k = q / (ext * ext);
        int c = (c0[0] + i) + 8 * (c0[1] + j) + ((D == 3) ? 64 * (c0[2] + k) : 0);
        float rho = (float)U[((long long)0 * cap + s) * B + c];
        float vv = 0.f;
        for (int d = 0; d < D; d++) {
          float m = (float)U[((long long)(1 + d) * cap + s) * B + c];
          vv += m * m;
        }
        float E = (float)U[((long long)(D + 1) * cap + s) * B + c];
        sr += rho;
        spp += gm1 * (E - 0.5f * vv / rho);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      spp += __shfl_xor_sync(0xffffffffu, spp, o);
    }
    if (lane == 0) {
      float f0 = 0.f, f1 = 0.f;
      if (s >= 0) {
        f0 = (sr / (float)ncell) / srho;
        f1 = (spp / (float)ncell) / sp;
      }
      feat[p] = f0;
      feat[n + p] = f1;
      feat[2 * n + p] = f2;
    }
  }
}

// features (FP32 [3][n]) -> layer-1 input rows (BF16 [n][8], channels 3..7 zero)
__global__ void k_feat_rows(const float *__restrict__ feat, uint4 *__restrict__ rows, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    __nv_bfloat162 a = __floats2bfloat162_rn(feat[p], feat[n + p]);
    __nv_bfloat162 c = __floats2bfloat162_rn(feat[2 * n + p], 0.f);
    rows[p] = make_uint4(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&c), 0u, 0u);
  }
}

// ---------------------------------------------------------------- tcgen05 helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading-dimension byte offset
// (between core matrices adjacent along K), stride byte offset (between 8-row
// groups along M or N), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a K-major tile with KP columns, core-matrix layout
__device__ __forceinline__ uint32_t cm_offset(int r, int k, int KP) {
  return (uint32_t)((((r >> 3) * (KP >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

constexpr unsigned kWaitLimit = 1u << 24;

// bounded wait for the mbarrier phase `parity`; false on expiry
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned limit = kWaitLimit) {
  for (unsigned it = 0; it < limit; it++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---------------------------------------------------------------- convolution layer on tensor cores
// Activations are channel-last BF16 rows, one per position: the layer-1 input
// has 8 channels (the 3 features, zero padded; 16 B per position), the hidden
// layers 16 (32 B).  The GEMM's K index is tap-major, k = tap * CIN + channel
// (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)), so one tap of one row is one or two
// 16-byte rows of core matrices and is gathered with vector loads.
// Wcm: the 16 x KP BF16 weight operand, already in the shared-memory
// core-matrix byte order (k_pack_weights); bias FP32 [16].
// MODE kHidden: out[p][n] = bf16(relu(acc + bias)); kLogit: logits[p] = acc[0] + bias[0];
// kBackData (training, the gradient of a layer input): out[p][n] = bf16(acc) where the
// forward activation act[p][n] > 0, else 0 (the ReLU's derivative); no bias.
constexpr int kHidden = 0, kLogit = 1, kBackData = 2;
constexpr int kConvThreads = 256;  // two threads per tile row: taps 0..13 and 14..26

// tneed (may be null: every tile): per 128-position tile, nonzero when some position
// of the tile is needed by the layer; other tiles are skipped (their outputs stay as
// they were: only needed positions are read downstream).
template <int CIN, int KP, int MODE>
__global__ void __launch_bounds__(kConvThreads) k_prop_conv_tc(Geo g, const __nv_bfloat16 *__restrict__ in,
                                                               const uint4 *__restrict__ Wcm,
                                                               const float *__restrict__ bias,
                                                               __nv_bfloat16 *__restrict__ out,
                                                               float *__restrict__ logits,
                                                               const uint8_t *__restrict__ tneed,
                                                               const __nv_bfloat16 *__restrict__ act) {
  constexpr bool LAST = MODE == kLogit;
  constexpr int M = 128, N = 16;
  constexpr int KREAL = CIN * 27;
  static_assert(CIN == 8 || CIN == 16, "channel-last rows of 16 or 32 bytes");
  static_assert(KP % 16 == 0 && KP >= KREAL && KP - KREAL < 16, "K padding");
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *sA = sm;                       // M x KP bf16
  unsigned char *sB = sm + M * KP * 2;          // N x KP bf16
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + (M + N) * KP * 2);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (M - 1), half = tid >> 7;
  const int t0 = half ? 14 : 0, t1 = half ? 27 : 14;
  const long long npos = g.mapoff[g.L + 1];
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(32)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1) : "memory");
  }
  for (int i = tid; i < N * KP * 2 / 16; i += kConvThreads) reinterpret_cast<uint4 *>(sB)[i] = Wcm[i];
  if (KP > KREAL && half == 0) *reinterpret_cast<uint4 *>(sA + cm_offset(row, KREAL, KP)) = zero;
  float b[8];
#pragma unroll
  for (int n = 0; n < 8; n++) b[n] = MODE == kBackData ? 0.f : bias[8 * (warp >> 2) + n];
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
  constexpr uint32_t LBO = 128, SBO = (KP / 8) * 128;
  constexpr uint32_t IDESC = idesc_bf16(M, N);
  uint32_t phase = 0;
  bool ok = true;

  const long long ntiles = (npos + M - 1) / M;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    if (tneed && !tneed[tile]) continue;  // the same decision for the whole CTA
    // this row's position, level and block coordinates
    const long long p = tile * M + row;
    int x = 0, y = 0, z = 0, nx = 0, ny = 0, nz = 0;
    long long base = 0;
    if (p < npos) {
      int l = pos_level(g, p);
      long long u = p - g.mapoff[l];
      nx = g.nb[l][0];
      ny = g.nb[l][1];
      nz = g.nb[l][2];
      x = (int)(u % nx);
      y = (int)((u / nx) % ny);
      z = (int)(u / ((long long)nx * ny));
      base = g.mapoff[l];
    }
    // im2col of this row's taps (zero outside the level), in batches of 7 taps
#pragma unroll 1
    for (int tb = t0; tb < t1; tb += 7) {
      uint4 v[7][CIN / 8];
#pragma unroll
      for (int j = 0; j < 7; j++) {
        int t = tb + j;
        int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        int xx = x + dx, yy = y + dy, zz = z + dz;
        bool inside = t < t1 && xx >= 0 && yy >= 0 && zz >= 0 && xx < nx && yy < ny && zz < nz;
        long long qn = inside ? base + xx + (long long)nx * (yy + (long long)ny * zz) : 0;
        const uint4 *src = reinterpret_cast<const uint4 *>(in) + qn * (CIN / 8);
#pragma unroll
        for (int h = 0; h < CIN / 8; h++) v[j][h] = inside ? src[h] : zero;
      }
#pragma unroll
      for (int j = 0; j < 7; j++) {
        int t = tb + j;
        if (t < t1) {
#pragma unroll
          for (int h = 0; h < CIN / 8; h++)
            *reinterpret_cast<uint4 *>(sA + cm_offset(row, t * CIN + 8 * h, KP)) = v[j][h];
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll 1
      for (int ks = 0; ks < KP / 16; ks++) {
        uint64_t ad = smem_desc(aaddr + ks * 256, LBO, SBO);
        uint64_t bd = smem_desc(baddr + ks * 256, LBO, SBO);
        uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    __syncwarp();
    ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;  // one decision for the whole CTA
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
      if (tid == 0) atomicOr(g.err, EB_TIMEOUT);
      break;
    }
    // warp w reads accumulator lanes 32*(w%4) .. +31 (one row per lane), columns 8*(w/4) .. +7
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(8 * (warp >> 2))));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const long long q = tile * M + 32 * (warp & 3) + lane;
    if (q < npos) {
      if (LAST) {
        if (warp < 4) logits[q] = __uint_as_float(r[0]) + b[0];
      } else if (MODE == kBackData) {
        const uint4 fa = reinterpret_cast<const uint4 *>(act)[q * 2 + (warp >> 2)];  // 8 forward activations
        const uint32_t fw[4] = {fa.x, fa.y, fa.z, fa.w};
        uint32_t pk[4];
#pragma unroll
        for (int n = 0; n < 4; n++) {
          // a bfloat16 is positive when its sign bit is clear and it is not zero
          const bool plo = (fw[n] & 0x8000u) == 0 && (fw[n] & 0x7FFFu) != 0;
          const bool phi = (fw[n] & 0x80000000u) == 0 && (fw[n] & 0x7FFF0000u) != 0;
          __nv_bfloat162 h2 = __floats2bfloat162_rn(plo ? __uint_as_float(r[2 * n]) : 0.f,
                                                    phi ? __uint_as_float(r[2 * n + 1]) : 0.f);
          pk[n] = *reinterpret_cast<uint32_t *>(&h2);
        }
        reinterpret_cast<uint4 *>(out)[q * 2 + (warp >> 2)] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      } else {
        uint32_t pk[4];
#pragma unroll
        for (int n = 0; n < 4; n++) {
          float lo = __uint_as_float(r[2 * n]) + b[2 * n], hi = __uint_as_float(r[2 * n + 1]) + b[2 * n + 1];
          __nv_bfloat162 h2 = __floats2bfloat162_rn(lo > 0.f ? lo : 0.f, hi > 0.f ? hi : 0.f);
          pk[n] = *reinterpret_cast<uint32_t *>(&h2);
        }
        reinterpret_cast<uint4 *>(out)[q * 2 + (warp >> 2)] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
  }
}

template <int KP>
constexpr size_t conv_smem() {
  return (size_t)(128 + 16) * KP * 2 + 16;
}
constexpr int kKP1 = 224;  // layer 1: 27 taps x 8 channels = 216, padded to a multiple of 16
constexpr int kKP2 = 432;  // layers 2, 3: 27 taps x 16 channels

// ---------------------------------------------------------------- tiles the marking needs
// A logit is used only at positions of level >= 1 whose parent block exists: the
// 2^d children positions of every existing block below the finest level.  Layer 3
// is needed there, layer 2 within one position of them (its 3^d stencil), layer 1
// within two.  flags[k * ntp + tile] = 1 for every 128-position tile that holds a
// position layer k + 1 needs (k = 0: distance 2, 1: distance 1, 2: the children).
__global__ void k_prop_tiles(Geo g, uint8_t *__restrict__ flags, long long ntp) {
  int b, e;
  list_range(g, LK_EXIST, 0, g.L - 1, b, e);
  const long long cap = g.cap;
  for (int i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
    const int s = g.lists[LK_EXIST * cap + i];
    const int l = g.slot_level[s] + 1;  // the children's level
    const int c0 = 2 * g.slot_coord[3 * s], c1 = 2 * g.slot_coord[3 * s + 1], c2 = 2 * g.slot_coord[3 * s + 2];
    const int nx = g.nb[l][0], ny = g.nb[l][1], nz = g.nb[l][2];
    for (int k = 0; k < 3; k++) {
      const int r = 2 - k;
      const int x0 = max(c0 - r, 0), x1 = min(c0 + 1 + r, nx - 1);
      const int y0 = max(c1 - r, 0), y1 = min(c1 + 1 + r, ny - 1);
      const int z0 = g.dim == 3 ? max(c2 - r, 0) : 0, z1 = g.dim == 3 ? min(c2 + 1 + r, nz - 1) : 0;
      for (int z = z0; z <= z1; z++)
        for (int y = y0; y <= y1; y++) {
          const long long row = g.mapoff[l] + (long long)nx * (y + (long long)ny * z);
          for (long long t = (row + x0) >> 7; t <= (row + x1) >> 7; t++) flags[k * ntp + t] = 1;
        }
    }
  }
}
// tiles flagged per layer, added to cnt[3] (profiling)
__global__ void k_prop_tile_count(const uint8_t *__restrict__ flags, long long ntp, unsigned long long *cnt) {
  for (int k = 0; k < 3; k++) {
    unsigned long long c = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntp; t += (long long)gridDim.x * blockDim.x)
      c += flags[k * ntp + t] ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt + k, c);
  }
}

// ---------------------------------------------------------------- marking
// Positions of level >= 1 whose parent exists and whose logit is positive are
// needed (the closure then adds their siblings, parents and grading).
__global__ void k_prop_mark(Geo g, const float *__restrict__ logits, uint8_t *need) {
  const long long n = g.mapoff[g.L + 1];
  for (long long p = g.mapoff[1] + blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    if (!(logits[p] > 0.f)) continue;
    int l = pos_level(g, p);
    long long u = p - g.mapoff[l];
    int bx = (int)(u % g.nb[l][0]), by = (int)((u / g.nb[l][0]) % g.nb[l][1]);
    int bz = (int)(u / ((long long)g.nb[l][0] * g.nb[l][1]));
    if (g.idx[map_index(g, l - 1, bx >> 1, by >> 1, bz >> 1)] < 0) continue;
    need[p] = 1;
  }
}

// ---------------------------------------------------------------- training: loss, Adam
// binary cross-entropy with logits, averaged over positions of level >= 1
// whose parent exists and whose target is not 255 (excluded): dL/dz = (sigmoid(z) - y) / count
__global__ void k_bce_grad(Geo g, const float *__restrict__ z, const uint8_t *__restrict__ target,
                           float *__restrict__ dz, double *loss, float inv_count) {
  const long long n = g.mapoff[g.L + 1];
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    float d = 0.f;
    int l = pos_level(g, p);
    bool use = l > 0 && target[p] != 255;
    if (use) {
      long long u = p - g.mapoff[l];
      int bx = (int)(u % g.nb[l][0]), by = (int)((u / g.nb[l][0]) % g.nb[l][1]);
      int bz = (int)(u / ((long long)g.nb[l][0] * g.nb[l][1]));
      use = g.idx[map_index(g, l - 1, bx >> 1, by >> 1, bz >> 1)] >= 0;
    }
    if (use) {
      float x = z[p], y = target[p] ? 1.f : 0.f;
      float s = 1.f / (1.f + expf(-x));
      d = (s - y) * inv_count;
      acc += (double)(fmaxf(x, 0.f) - x * y + log1pf(expf(-fabsf(x)))) * inv_count;
    }
    dz[p] = d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// Adam on the FP32 master weights (beta1 0.9, beta2 0.999, eps 1e-8), step t; the
// bias corrections 1 - beta^t are formed in double precision (in single precision
// 1 - 0.999f loses five digits to cancellation)
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ grad, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, int t) {
  const float b1t = (float)(1.0 - pow(0.9, (double)t)), b2t = (float)(1.0 - pow(0.999, (double)t));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = grad[i];
    m[i] = 0.9f * m[i] + 0.1f * gi;
    v[i] = 0.999f * v[i] + 0.001f * gi * gi;
    w[i] -= lr * (m[i] / b1t) / (sqrtf(v[i] / b2t) + 1e-8f);
  }
}

// FP32 master weights (host blob order, [co][ci][tap]) -> the BF16 weight operands
// in shared-memory core-matrix byte order with the tap-major K index of
// k_prop_conv_tc (layer 1: 16 x kKP1, channels padded to 8; layers 2, 3:
// 16 x kKP2, layer 3's output channels 1..15 zero) and FP32 biases [16].
__global__ void k_pack_weights(const float *__restrict__ blob, __nv_bfloat16 *w1, float *b1, __nv_bfloat16 *w2,
                               float *b2, __nv_bfloat16 *w3, float *b3) {
  const float *W1 = blob, *B1 = W1 + 16 * 81, *W2 = B1 + 16, *B2 = W2 + 16 * 432, *W3 = B2 + 16, *B3 = W3 + 432;
  for (int i = threadIdx.x; i < 16 * kKP1; i += blockDim.x) {
    int n = i / kKP1, k = i % kKP1, t = k / 8, ci = k % 8;
    float v = (t < 27 && ci < 3) ? W1[(n * 3 + ci) * 27 + t] : 0.f;
    w1[cm_offset(n, k, kKP1) / 2] = __float2bfloat16_rn(v);
  }
  for (int i = threadIdx.x; i < 16 * kKP2; i += blockDim.x) {
    int n = i / kKP2, k = i % kKP2, t = k / 16, ci = k % 16;
    w2[cm_offset(n, k, kKP2) / 2] = __float2bfloat16_rn(W2[(n * 16 + ci) * 27 + t]);
    w3[cm_offset(n, k, kKP2) / 2] = __float2bfloat16_rn(n == 0 ? W3[ci * 27 + t] : 0.f);
  }
  for (int i = threadIdx.x; i < 16; i += blockDim.x) {
    b1[i] = B1[i];
    b2[i] = B2[i];
    b3[i] = i == 0 ? B3[0] : 0.f;
  }
}

// ---------------------------------------------------------------- training on the tensor cores
// The gradient of a layer's input is the correlation of the output gradient with
// the taps mirrored (tap t -> 26 - t) and the channel roles swapped:
//   dIn[ci](q) = sum_{co,t} W[co][ci][26 - t] dOut[co](q + off(t)).
// These operands, in the core-matrix byte order of k_prop_conv_tc: layer 3 (one
// output channel; input rows of 8 channels, channel 0 = dz): w3t[ci][t*8 + 0] =
// W3[0][ci][26 - t]; layer 2: w2t[ci][t*16 + co] = W2[co][ci][26 - t].
__global__ void k_pack_weights_back(const float *__restrict__ blob, __nv_bfloat16 *w3t, __nv_bfloat16 *w2t) {
  const float *W1 = blob, *B1 = W1 + 16 * 81, *W2 = B1 + 16, *B2 = W2 + 16 * 432, *W3 = B2 + 16;
  for (int i = threadIdx.x; i < 16 * kKP1; i += blockDim.x) {
    int n = i / kKP1, k = i % kKP1, t = k / 8, c = k % 8;
    float v = (t < 27 && c == 0) ? W3[n * 27 + (26 - t)] : 0.f;
    w3t[cm_offset(n, k, kKP1) / 2] = __float2bfloat16_rn(v);
  }
  for (int i = threadIdx.x; i < 16 * kKP2; i += blockDim.x) {
    int n = i / kKP2, k = i % kKP2, t = k / 16, co = k % 16;
    w2t[cm_offset(n, k, kKP2) / 2] = __float2bfloat16_rn(W2[(co * 16 + n) * 27 + (26 - t)]);
  }
}

// dL/dz (FP32 [n]) -> BF16 rows [n][8], channel 0 = dz
__global__ void k_dz_rows(const float *__restrict__ dz, uint4 *__restrict__ rows, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    __nv_bfloat162 a = __floats2bfloat162_rn(dz[p], 0.f);
    rows[p] = make_uint4(*reinterpret_cast<uint32_t *>(&a), 0u, 0u, 0u);
  }
}

// Weight (and bias) gradient from channel-last BF16 rows: x rows [n][XS] (channels
// 0..cin-1 used), output gradient either FP32 [n] (dzf, one channel) or BF16 rows
// [n][16] (dyr).  dW[co][ci][t] += sum_p dy[co][p] x[ci][p + off(t)], summed in double;
// db[co] += sum_p dy[co][p] (on ci == 0, t == 13).  One CTA per weight.
template <int XS>
__global__ void k_conv_dw_rows(Geo g, const __nv_bfloat16 *__restrict__ x, int cin, const float *__restrict__ dzf,
                               const __nv_bfloat16 *__restrict__ dyr, int cout, float *__restrict__ dw,
                               float *__restrict__ db) {
  const long long n = g.mapoff[g.L + 1];
  const int dim3d = g.dim == 3;
  const int wi = blockIdx.x;  // (co * cin + ci) * 27 + t
  const int t = wi % 27, ci = (wi / 27) % cin, co = wi / (27 * cin);
  const int dz = t / 9 - 1, dy_ = (t / 3) % 3 - 1, dx = t % 3 - 1;
  __shared__ double red[2][32];
  double acc = 0.0, accb = 0.0;
  if (dim3d || dz == 0) {
    for (long long p = threadIdx.x; p < n; p += blockDim.x) {
      const float d = dzf ? dzf[p] : __bfloat162float(dyr[p * 16 + co]);
      if (d == 0.f) continue;
      const long long q = pos_neighbour(g, pos_level(g, p), p, dx, dy_, dz);
      if (q >= 0) acc += (double)d * (double)__bfloat162float(x[q * XS + ci]);
      accb += d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    accb += __shfl_xor_sync(0xffffffffu, accb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc;
    red[1][threadIdx.x >> 5] = accb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sw = 0, sb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sw += red[0][w];
      sb += red[1][w];
    }
    dw[wi] += (float)sw;
    if (ci == 0 && t == 13) db[co] += (float)sb;
  }
}

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_prop_features(const Geo &g, const T *U, const double *maxdet, const T *scale, double eps, float *feat,
                          int grid, cudaStream_t st) {
  if (g.dim == 2) k_prop_features<T, 2><<<grid, 256, 0, st>>>(g, U, maxdet, scale, eps, feat);
  else k_prop_features<T, 3><<<grid, 256, 0, st>>>(g, U, maxdet, scale, eps, feat);
}
template void launch_prop_features<float>(const Geo &, const float *, const double *, const float *, double, float *,
                                          int, cudaStream_t);
template void launch_prop_features<double>(const Geo &, const double *, const double *, const double *, double,
                                           float *, int, cudaStream_t);

void prop_setup() {
  cudaFuncSetAttribute(k_prop_conv_tc<8, kKP1, kBackData>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)conv_smem<kKP1>());
  cudaFuncSetAttribute(k_prop_conv_tc<16, kKP2, kBackData>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)conv_smem<kKP2>());
  cudaFuncSetAttribute(k_prop_conv_tc<8, kKP1, kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)conv_smem<kKP1>());
  cudaFuncSetAttribute(k_prop_conv_tc<16, kKP2, kHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)conv_smem<kKP2>());
  cudaFuncSetAttribute(k_prop_conv_tc<16, kKP2, kLogit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)conv_smem<kKP2>());
}

// features (float [3][n]) -> logits (float [n]) through the three layers on tensor
// cores; a0: BF16 [n][8], a1, a2: BF16 [n][16]
// Self-test of the failure path of the bounded waits: one warp initialises an
// mbarrier expecting one arrival, arrives on it only when `arrive` is set, and
// waits for its first phase with the tensor-core kernel's bounded wait (limit
// iterations); an expired wait records EB_TIMEOUT, as the real kernels do.
__global__ void k_wait_selftest(int *err, unsigned limit, int arrive) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t mb = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (threadIdx.x == 0 && arrive) {
    uint64_t state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(mb) : "memory");
    (void)state;
  }
  __syncwarp();
  const bool ok = mbar_wait(mb, 0, limit);
  if (threadIdx.x == 0 && !ok) atomicOr(err, EB_TIMEOUT);
}

void launch_wait_selftest(int *err, unsigned limit, int arrive, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err, limit, arrive);
}

void launch_prop_tiles(const Geo &g, uint8_t *flags, long long ntp, unsigned long long *count, int grid,
                       cudaStream_t st) {
  cudaMemsetAsync(flags, 0, 3 * (size_t)ntp, st);
  if (g.L >= 1) k_prop_tiles<<<grid, 256, 0, st>>>(g, flags, ntp);
  if (count) k_prop_tile_count<<<64, 256, 0, st>>>(flags, ntp, count);
}

void launch_prop_infer(const Geo &g, const float *feat, __nv_bfloat16 *a0, __nv_bfloat16 *a1, __nv_bfloat16 *a2,
                       const __nv_bfloat16 *w1, const float *b1, const __nv_bfloat16 *w2, const float *b2,
                       const __nv_bfloat16 *w3, const float *b3, float *logits, int nsm, cudaEvent_t conv_begin,
                       cudaEvent_t conv_end, const uint8_t *tneed, cudaStream_t st) {
  long long n = g.mapoff[g.L + 1];
  long long tiles = (n + 127) / 128;
  const uint8_t *t1 = tneed, *t2 = tneed ? tneed + tiles : nullptr, *t3 = tneed ? tneed + 2 * tiles : nullptr;
  // layer 1 fits three CTAs per SM in shared memory, layers 2 and 3 one
  int grid1 = (int)(tiles < 3 * nsm ? tiles : 3 * nsm), grid2 = (int)(tiles < nsm ? tiles : nsm);
  long long fb = (n + 255) / 256;
  k_feat_rows<<<(int)(fb < 4 * nsm ? fb : 4 * nsm), 256, 0, st>>>(feat, reinterpret_cast<uint4 *>(a0), n);
  if (conv_begin) cudaEventRecord(conv_begin, st);
  k_prop_conv_tc<8, kKP1, kHidden><<<grid1, kConvThreads, conv_smem<kKP1>(), st>>>(
      g, a0, reinterpret_cast<const uint4 *>(w1), b1, a1, nullptr, t1, nullptr);
  k_prop_conv_tc<16, kKP2, kHidden><<<grid2, kConvThreads, conv_smem<kKP2>(), st>>>(
      g, a1, reinterpret_cast<const uint4 *>(w2), b2, a2, nullptr, t2, nullptr);
  k_prop_conv_tc<16, kKP2, kLogit><<<grid2, kConvThreads, conv_smem<kKP2>(), st>>>(
      g, a2, reinterpret_cast<const uint4 *>(w3), b3, nullptr, logits, t3, nullptr);
  if (conv_end) cudaEventRecord(conv_end, st);
}

void launch_prop_mark(const Geo &g, const float *logits, uint8_t *need, int grid, cudaStream_t st) {
  k_prop_mark<<<grid, 256, 0, st>>>(g, logits, need);
}

void launch_pack_weights(const float *blob, __nv_bfloat16 *w1, float *b1, __nv_bfloat16 *w2, float *b2,
                         __nv_bfloat16 *w3, float *b3, cudaStream_t st) {
  k_pack_weights<<<1, 256, 0, st>>>(blob, w1, b1, w2, b2, w3, b3);
}

// One Adam step on a batch of snapshots, on the tensor cores: per snapshot the
// BF16 forward pass of inference (layer inputs rounded to BF16, FP32 accumulation),
// the binary cross-entropy gradient dz (FP32), the gradients of the layer inputs by
// the mirrored-tap convolutions (BF16 operands, FP32 accumulation, rounded to BF16
// and masked by the forward ReLU), and the weight gradients from the BF16 rows
// (summed in double on the CUDA cores); then Adam on the FP32 master weights and
// the re-packing of the BF16 operands.  feat: [ns][3][n] floats, target: [ns][n]
// bytes (device).  work: kPropWorkPerPos floats per position (z, dz, and the BF16
// rows of dz, dL/dh2, dL/dh1).
void launch_prop_train_step(const Geo &g, const float *feat, const uint8_t *target, int ns, float *blob, float *grad,
                            float *m1, float *m2, int t, float lr, float *work, double *loss, int adam,
                            __nv_bfloat16 *a0, __nv_bfloat16 *a1, __nv_bfloat16 *a2, __nv_bfloat16 *w1,
                            float *b1, __nv_bfloat16 *w2, float *b2, __nv_bfloat16 *w3, float *b3,
                            __nv_bfloat16 *w3t, __nv_bfloat16 *w2t, int nsm, cudaStream_t st) {
  long long n = g.mapoff[g.L + 1];
  const int NW = 16 * 81 + 16 + 16 * 432 + 16 + 432 + 1;
  float *gW1 = grad, *gB1 = gW1 + 16 * 81, *gW2 = gB1 + 16, *gB2 = gW2 + 16 * 432, *gW3 = gB2 + 16, *gB3 = gW3 + 432;
  const long long n4 = (n + 3) & ~3LL;                             // 16-byte aligned rows below
  float *z = work, *dz = z + n4;
  __nv_bfloat16 *dzr = reinterpret_cast<__nv_bfloat16 *>(dz + n4);  // [n][8]
  __nv_bfloat16 *d2r = dzr + 8 * n;                                 // [n][16]
  __nv_bfloat16 *d1r = d2r + 16 * n;                                // [n][16]
  cudaMemsetAsync(grad, 0, NW * sizeof(float), st);
  launch_pack_weights(blob, w1, b1, w2, b2, w3, b3, st);
  k_pack_weights_back<<<1, 256, 0, st>>>(blob, w3t, w2t);
  // the loss is normalised by the positions of levels >= 1 times the snapshots (a
  // fixed scale; the positions entering it are selected inside k_bce_grad)
  float inv = 1.f / (float)((n - g.mapoff[1]) * (long long)ns);
  const int grid = 1024;
  const long long tiles = (n + 127) / 128;
  const int grid1 = (int)(tiles < 3 * nsm ? tiles : 3 * nsm), grid2 = (int)(tiles < nsm ? tiles : nsm);
  for (int k = 0; k < ns; k++) {
    const float *x = feat + (long long)k * 3 * n;
    launch_prop_infer(g, x, a0, a1, a2, w1, b1, w2, b2, w3, b3, z, nsm, nullptr, nullptr, nullptr, st);
    k_bce_grad<<<grid, 256, 0, st>>>(g, z, target + (long long)k * n, dz, loss, inv);
    k_dz_rows<<<grid, 256, 0, st>>>(dz, reinterpret_cast<uint4 *>(dzr), n);
    k_conv_dw_rows<16><<<432, 256, 0, st>>>(g, a2, 16, dz, nullptr, 1, gW3, gB3);
    k_prop_conv_tc<8, kKP1, kBackData><<<grid1, kConvThreads, conv_smem<kKP1>(), st>>>(
        g, dzr, reinterpret_cast<const uint4 *>(w3t), nullptr, d2r, nullptr, nullptr, a2);
    k_conv_dw_rows<16><<<16 * 432, 256, 0, st>>>(g, a1, 16, nullptr, d2r, 16, gW2, gB2);
    k_prop_conv_tc<16, kKP2, kBackData><<<grid2, kConvThreads, conv_smem<kKP2>(), st>>>(
        g, d2r, reinterpret_cast<const uint4 *>(w2t), nullptr, d1r, nullptr, nullptr, a1);
    k_conv_dw_rows<8><<<16 * 81, 256, 0, st>>>(g, a0, 3, nullptr, d1r, 16, gW1, gB1);
  }
  if (adam) {
    k_adam<<<64, 256, 0, st>>>(blob, grad, m1, m2, NW, lr, t);
    launch_pack_weights(blob, w1, b1, w2, b2, w3, b3, st);
  }
}

}  // namespace mrfv
