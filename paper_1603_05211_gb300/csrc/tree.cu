// Tree update kernels (integer work): the block reading of the refinement,
// safety-zone, gradedness and coarsening rules of arXiv:1603.05211 Section 2.1,
// row clustering of gradient flags (Section 2.2), pool allocation, and the
// prefix-scan compaction that rebuilds the neighbour tables and the work lists
// in level-major Morton order.
#include <cuda_runtime.h>

#include <algorithm>
#include <limits.h>
#include <stdint.h>

#include "common.h"
#include "dev.cuh"
#include "launch.h"

namespace mrfv {

__device__ __forceinline__ int level_of_map(const Geo &g, long long t) {
  int l = 0;
  while (l < g.L && t >= g.mapoff[l + 1]) l++;
  return l;
}
// (32-bit arithmetic: a level holds fewer than 2^31 block positions)
__device__ __forceinline__ void map_coords(const Geo &g, int l, long long t, int &bx, int &by, int &bz) {
  const int u = (int)(t - g.mapoff[l]);
  const int nx = g.nb[l][0], ny = g.nb[l][1];
  const int r = u / nx;
  bx = u - r * nx;
  by = r % ny;
  bz = r / ny;
}


// MR: a significant block of level >= 1 is kept with its 3^d-1 neighbours and,
// below the finest level, its children are added.  GRAD: the children of every
// flagged block are added.  MR with the proposer (crit 2): as MR without the
// neighbours.
// lkeep: a remesh keeps the levels <= lkeep as they are, so a significant block
// there only asks for its children.
__device__ __forceinline__ void k_need_mark_dev(Geo g, const uint8_t *sig, uint8_t *need, int crit, int lkeep) {
  long long total = g.mapoff[g.L + 1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    if (g.idx[t] < 0 || !sig[t]) continue;
    int l = level_of_map(g, t), bx, by, bz;
    map_coords(g, l, t, bx, by, bz);
    if (crit == 0 || crit == 2) {  // MR (crit 2: without the safety zone, which the proposer replaces)
      if (l == 0) continue;
      if (l > lkeep) {
        need[t] = 1;
        if (crit == 0) mark_nbrs(g, need, l, bx, by, bz);
      }
    }
    if (l < g.L) mark_children(g, need, l, bx, by, bz);
  }
}

// Closure on level l (run from the finest level down): a needed block needs its
// siblings, its parent and the 3^d-1 neighbours of its parent (gradedness).
__device__ __forceinline__ void k_need_close_dev(Geo g, int l, uint8_t *need, int parents) {
  long long n = g.mapoff[l + 1] - g.mapoff[l];
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    long long t = g.mapoff[l] + u;
    if (!need[t]) continue;
    int bx, by, bz;
    map_coords(g, l, t, bx, by, bz);
    int px = bx >> 1, py = by >> 1, pz = bz >> 1;
    mark_children(g, need, l - 1, px, py, pz);  // siblings (children of the parent)
    if (!parents) continue;                     // remesh: level l-1 is kept as it is
    need[map_index(g, l - 1, px, py, pz)] = 1;
    mark_nbrs(g, need, l - 1, px, py, pz);
  }
}

__device__ __forceinline__ void k_free_dev(Geo g, const uint8_t *need, int32_t *freestack, int *freetop) {
  long long total = g.mapoff[g.L + 1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int32_t s = g.idx[t];
    if (s < 0 || need[t]) continue;
    int pos = atomicAdd(freetop, 1);
    freestack[pos] = s;
    g.idx[t] = -1;
    g.slot_level[s] = -1;
  }
}

__device__ __forceinline__ void k_alloc_dev(Geo g, const uint8_t *need, int32_t *freestack, int *freetop, int32_t *newlist, int *nnew) {
  long long total = g.mapoff[g.L + 1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    if (g.idx[t] >= 0 || !need[t]) continue;
    int pos = atomicSub(freetop, 1) - 1;
    if (pos < 0) {  // pool exhausted: give the count back so the stack top never stays negative
      atomicAdd(freetop, 1);
      set_err(g, EB_POOL);
      continue;
    }
    int32_t s = freestack[pos];
    int l = level_of_map(g, t), bx, by, bz;
    map_coords(g, l, t, bx, by, bz);
    g.idx[t] = s;
    g.slot_level[s] = l;
    g.slot_coord[3 * s] = bx;
    g.slot_coord[3 * s + 1] = by;
    g.slot_coord[3 * s + 2] = bz;
    newlist[g.mapoff[l] + atomicAdd(nnew + l, 1)] = s;  // per-level segment of the new-block list
  }
}

__global__ void k_init_freestack(int32_t *freestack, int *freetop, long long cap) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cap; i += (long long)gridDim.x * blockDim.x)
    freestack[i] = (int32_t)(cap - 1 - i);
  if (blockIdx.x == 0 && threadIdx.x == 0) *freetop = (int)cap;
}

// ---------------------------------------------------------------- classification
__device__ __forceinline__ unsigned compact_bits(unsigned long long m, int stride, int off, int nbits) {
  unsigned r = 0;
  for (int b = 0; b < nbits; b++) r |= (unsigned)((m >> (b * stride + off)) & 1ull) << b;
  return r;
}

__device__ __forceinline__ bool morton_block(const Geo &g, long long m, int &l, int &bx, int &by, int &bz) {
  l = 0;
  while (l < g.L && m >= g.moff[l + 1]) l++;
  unsigned long long u = (unsigned long long)(m - g.moff[l]);
  int nb = g.mbits[l];
  if (g.dim == 2) {
    bx = compact_bits(u, 2, 0, nb);
    by = compact_bits(u, 2, 1, nb);
    bz = 0;
  } else {
    bx = compact_bits(u, 3, 0, nb);
    by = compact_bits(u, 3, 1, nb);
    bz = compact_bits(u, 3, 2, nb);
  }
  return bx < g.nb[l][0] && by < g.nb[l][1] && bz < g.nb[l][2];
}

__device__ __forceinline__ bool has_children(const Geo &g, int l, int bx, int by, int bz) {
  if (l >= g.L) return false;
  return g.idx[map_index(g, l + 1, 2 * bx, 2 * by, g.dim == 3 ? 2 * bz : 0)] >= 0;
}

// One thread per Morton position of every level: kind bits of the block there
// (exist / leaf / refined / needs ghost strips / needs flux correction), its face
// neighbour table and its refined-neighbour mask.
__device__ __forceinline__ uint8_t classify_position(const Geo &g, long long m) {
  {
    int l, bx, by, bz;
    uint8_t bits = 0;
    if (morton_block(g, m, l, bx, by, bz)) {
      int32_t s = g.idx[map_index(g, l, bx, by, bz)];
      if (s >= 0) {
        bits = 1u << LK_EXIST;
        bool leaf = !has_children(g, l, bx, by, bz);
        bits |= leaf ? (1u << LK_LEAF) : (1u << LK_INTERNAL);
        if (!leaf) {
          const int nk = g.dim == 3 ? 8 : 4;
          for (int q = 0; q < nk; q++)
            g.kids[8 * s + q] =
                g.idx[map_index(g, l + 1, 2 * bx + (q & 1), 2 * by + ((q >> 1) & 1), g.dim == 3 ? 2 * bz + (q >> 2) : 0)];
        }
        uint8_t cm = 0;
        bool missing = false;
        for (int f = 0; f < 2 * g.dim; f++) {
          int n = f >> 1, side = f & 1;
          int c[3] = {bx, by, bz};
          c[n] += side ? 1 : -1;
          int w = bc_block(g, l, n, c[n]);
          int32_t nb;
          if (w < 0) {
            nb = NBR_WALL;
          } else {
            c[n] = w;
            int32_t ns = g.idx[map_index(g, l, c[0], c[1], c[2])];
            if (ns >= 0) {
              nb = ns;
              if (has_children(g, l, c[0], c[1], c[2])) cm |= (uint8_t)(1u << f);
            } else {
              nb = NBR_MISSING;
              missing = true;
            }
          }
          g.nbr[6 * s + f] = nb;
        }
        g.cmask[s] = cm;
        if (missing) bits |= 1u << LK_GHOST;
        if (leaf && cm) bits |= 1u << LK_REFLUX;
      }
    }
    return bits;
  }
}
__device__ __forceinline__ void k_classify_dev(Geo g, uint8_t *kbits) {
  long long total = g.moff[g.L + 1];
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total; m += (long long)gridDim.x * blockDim.x)
    kbits[m] = classify_position(g, m);
}

constexpr int SCAN_NT = 256;
constexpr int SCAN_PER = 1;  // one Morton position per thread: no serial chain of table reads per thread
constexpr int SCAN_TILE = SCAN_NT * SCAN_PER;
constexpr int kFusedScanTiles = 1024;  // up to this many tiles each scatter CTA sums the counts before it

// per tile: number of entries of each kind
__device__ __forceinline__ void k_tile_count_dev(Geo g, const uint8_t *kbits, int32_t *tcount, int ntiles) {
  __shared__ int32_t red[LK_NUM][SCAN_NT / 32];
  long long total = g.moff[g.L + 1];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int cnt[LK_NUM] = {0, 0, 0, 0, 0};
    long long base = (long long)tile * SCAN_TILE + threadIdx.x * SCAN_PER;
    for (int j = 0; j < SCAN_PER; j++) {
      long long m = base + j;
      if (m < total) {
        uint8_t b = kbits[m];
        for (int k = 0; k < LK_NUM; k++) cnt[k] += (b >> k) & 1;
      }
    }
    for (int k = 0; k < LK_NUM; k++) {
      int c = cnt[k];
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < LK_NUM) {
      int s = 0;
      for (int w = 0; w < SCAN_NT / 32; w++) s += red[threadIdx.x][w];
      tcount[threadIdx.x * ntiles + tile] = s;
    }
    __syncthreads();
  }
}

// Classification and tile counts in one pass (each thread classifies its
// SCAN_PER consecutive Morton positions, then the CTA counts the tile).
__global__ void k_classify_count(Geo g, uint8_t *kbits, int32_t *tcount, int ntiles) {
  __shared__ int32_t red[LK_NUM][SCAN_NT / 32];
  long long total = g.moff[g.L + 1];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int cnt[LK_NUM] = {0, 0, 0, 0, 0};
    long long base = (long long)tile * SCAN_TILE + threadIdx.x * SCAN_PER;
    for (int j = 0; j < SCAN_PER; j++) {
      long long m = base + j;
      if (m < total) {
        uint8_t b = classify_position(g, m);
        kbits[m] = b;
        for (int k = 0; k < LK_NUM; k++) cnt[k] += (b >> k) & 1;
      }
    }
    for (int k = 0; k < LK_NUM; k++) {
      int c = cnt[k];
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < LK_NUM) {
      int sum = 0;
      for (int w = 0; w < SCAN_NT / 32; w++) sum += red[threadIdx.x][w];
      tcount[threadIdx.x * ntiles + tile] = sum;
    }
    __syncthreads();
  }
}

// single CTA (1024 threads): exclusive scan of the tile counts of each kind;
// totals -> loff[kind][L+1].  Each thread sums a run of tiles, the runs are
// scanned with warp shuffles, then each thread writes its tiles' offsets.
__device__ __forceinline__ void k_tile_scan_dev(Geo g, const int32_t *tcount, int32_t *toff, int ntiles) {
  __shared__ int32_t wsum[LK_NUM][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (ntiles + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(ntiles, b + per);
  int run[LK_NUM];
  for (int k = 0; k < LK_NUM; k++) {
    int x = 0;
    for (int t = b; t < e; t++) x += tcount[k * ntiles + t];
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[k][warp] = incl;
    run[k] = incl - x;
  }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < LK_NUM; k++) {
      int x = lane < nw ? wsum[k][lane] : 0;
      int incl = x;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane < nw) wsum[k][lane] = incl - x;
      if (lane == 31) g.loff[k * (MAXL + 2) + g.L + 1] = incl;
    }
  }
  __syncthreads();
  for (int k = 0; k < LK_NUM; k++) {
    int r = run[k] + wsum[k][warp];
    for (int t = b; t < e; t++) {
      toff[k * ntiles + t] = r;
      r += tcount[k * ntiles + t];
    }
  }
}

// per tile: local exclusive scan, scatter slots into the lists; the thread that
// owns the first Morton position of a level writes that level's list offsets.
// toff == null: each CTA forms its tile's exclusive prefix from the tile counts
// itself (few tiles), and CTA 0 writes the totals.
__device__ __forceinline__ void k_scatter_dev(Geo g, const uint8_t *kbits, const int32_t *toff, int ntiles,
                                             const int32_t *tcount = nullptr) {
  __shared__ int32_t pre[LK_NUM][SCAN_NT / 32], alls[LK_NUM][SCAN_NT / 32];
  __shared__ int32_t wsum[LK_NUM][SCAN_NT / 32];
  long long total = g.moff[g.L + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    long long base = (long long)tile * SCAN_TILE + threadIdx.x * SCAN_PER;
    uint8_t b[SCAN_PER];
    int cnt[LK_NUM] = {0, 0, 0, 0, 0};
    for (int j = 0; j < SCAN_PER; j++) {
      long long m = base + j;
      b[j] = (m < total) ? kbits[m] : 0;
      for (int k = 0; k < LK_NUM; k++) cnt[k] += (b[j] >> k) & 1;
    }
    int excl[LK_NUM];
    for (int k = 0; k < LK_NUM; k++) {
      int x = cnt[k];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[k][warp] = x;
      excl[k] = x - cnt[k];
    }
    if (!toff) {
      // counts of the tiles before this one (and, for tile 0, of all tiles)
      int part[LK_NUM] = {0, 0, 0, 0, 0}, all[LK_NUM] = {0, 0, 0, 0, 0};
      for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        for (int k = 0; k < LK_NUM; k++) {
          int c = tcount[k * ntiles + t];
          if (t < tile) part[k] += c;
          all[k] += c;
        }
      for (int k = 0; k < LK_NUM; k++) {
        for (int o = 16; o > 0; o >>= 1) {
          part[k] += __shfl_xor_sync(0xffffffffu, part[k], o);
          all[k] += __shfl_xor_sync(0xffffffffu, all[k], o);
        }
      }
      if (lane == 0)
        for (int k = 0; k < LK_NUM; k++) {
          pre[k][warp] = part[k];
          alls[k][warp] = all[k];
        }
      __syncthreads();
      if (tile == 0 && threadIdx.x < LK_NUM) {  // the totals of every kind
        int sum = 0;
        for (int w = 0; w < SCAN_NT / 32; w++) sum += alls[threadIdx.x][w];
        g.loff[threadIdx.x * (MAXL + 2) + g.L + 1] = sum;
      }
    }
    __syncthreads();
    for (int k = 0; k < LK_NUM; k++) {
      int add = 0;
      if (toff) {
        add = toff[k * ntiles + tile];
      } else {
        for (int w = 0; w < SCAN_NT / 32; w++) add += pre[k][w];
      }
      for (int w = 0; w < warp; w++) add += wsum[k][w];
      excl[k] += add;
    }
    for (int j = 0; j < SCAN_PER; j++) {
      long long m = base + j;
      if (m >= total) break;
      for (int l = 0; l <= g.L; l++)
        if (g.moff[l] == m)
          for (int k = 0; k < LK_NUM; k++) g.loff[k * (MAXL + 2) + l] = excl[k];
      if (b[j]) {
        int l, bx, by, bz;
        morton_block(g, m, l, bx, by, bz);
        int32_t s = g.idx[map_index(g, l, bx, by, bz)];
        for (int k = 0; k < LK_NUM; k++)
          if ((b[j] >> k) & 1) g.lists[(long long)k * g.cap + excl[k]++] = s;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- kernels
__global__ void k_need_mark(Geo g, const uint8_t *sig, uint8_t *need, int crit, int lkeep) {
  k_need_mark_dev(g, sig, need, crit, lkeep);
}
__global__ void k_need_close(Geo g, int l, uint8_t *need, int parents) { k_need_close_dev(g, l, need, parents); }
// Levels lhi..1 closed by one CTA, finest first: the need map of levels 0..lhi
// (at most kTailNeedBytes) is read into shared memory once, closed there level by
// level and written back.  Each level is closed by gathering instead of
// scattering: with any(q) = "some child of q (level l-1) is needed", the rule of
// k_need_close_dev (parents included) marks on level l every child of a q with
// any(q), and on level l-1 every position p with any(q) for some q among p and its
// 3^d-1 neighbours (the neighbour relation is symmetric, boundary rule included).
// Two passes over the positions of level l-1 per level, no scattered writes.
__global__ void k_need_close_tail(Geo g, int lhi, uint8_t *need) {
  __shared__ __align__(16) uint8_t sn[kTailNeedBytes];
  __shared__ uint8_t anyc[kTailThreads];
  const int total = (int)g.mapoff[lhi + 1];
#pragma unroll 4
  for (int i = threadIdx.x; i < total; i += blockDim.x) sn[i] = need[i];
  __syncthreads();
  const bool d3 = g.dim == 3;
  for (int l = lhi; l >= 1; l--) {
    const int lp = l - 1;
    const int nx = g.nb[lp][0], ny = g.nb[lp][1];
    const int n = (int)(g.mapoff[l] - g.mapoff[lp]);  // positions of level l-1 (at most kTailThreads)
    const int cx = g.nb[l][0], cxy = g.nb[l][0] * g.nb[l][1];
    uint8_t *fine = sn + g.mapoff[l];
    uint8_t *coarse = sn + g.mapoff[lp];
    int qx = 0, qy = 0, qz = 0;
    const int u = threadIdx.x;
    if (u < n) {
      qy = u / nx;
      qx = u - qy * nx;
      qz = qy / ny;
      qy -= qz * ny;
      const int f = 2 * qx + cx * (2 * qy) + cxy * (2 * qz);
      uint8_t a = fine[f] | fine[f + 1] | fine[f + cx] | fine[f + cx + 1];
      if (d3) a |= fine[f + cxy] | fine[f + cxy + 1] | fine[f + cxy + cx] | fine[f + cxy + cx + 1];
      anyc[u] = a;
    }
    __syncthreads();
    if (u < n) {
      if (anyc[u]) {  // the children of q, the siblings of its needed child
        const int f = 2 * qx + cx * (2 * qy) + cxy * (2 * qz);
        fine[f] = fine[f + 1] = fine[f + cx] = fine[f + cx + 1] = 1;
        if (d3) fine[f + cxy] = fine[f + cxy + 1] = fine[f + cxy + cx] = fine[f + cxy + cx + 1] = 1;
      }
      uint8_t m = 0;
      for (int c = d3 ? -1 : 0; c <= (d3 ? 1 : 0); c++) {
        const int z = bc_block(g, lp, 2, qz + c);
        if (z < 0) continue;
        for (int b = -1; b <= 1; b++) {
          const int y = bc_block(g, lp, 1, qy + b);
          if (y < 0) continue;
          for (int a = -1; a <= 1; a++) {
            const int x = bc_block(g, lp, 0, qx + a);
            if (x >= 0) m |= anyc[x + nx * (y + ny * z)];
          }
        }
      }
      if (m) coarse[u] = 1;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < total; i += blockDim.x) need[i] = sn[i];
}

// Remesh(l0) inside the level recursion (Fig. 2): flags cleared, the tree of
// levels <= l0 kept as needed, the levels above it to be rebuilt from flags.
__global__ void k_remesh_begin(Geo g, long long total, uint8_t *sig, uint8_t *gflag, uint8_t *need, int *nnew,
                               int l0) {
  const long long keep = g.mapoff[l0 + 1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    sig[t] = 0;
    gflag[t] = 0;
    need[t] = (t < keep && g.idx[t] >= 0) ? 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x < MAXL) nnew[threadIdx.x] = 0;
}

// Nesting of a remesh: a needed block of level l stays only where its parent and
// the parent's 3^d-1 neighbours are needed (run coarse to fine, so a dropped
// block takes its descendants along).
__global__ void k_need_prune(Geo g, int l, uint8_t *need) {
  long long n = g.mapoff[l + 1] - g.mapoff[l];
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    long long t = g.mapoff[l] + u;
    if (!need[t]) continue;
    int bx, by, bz;
    map_coords(g, l, t, bx, by, bz);
    const int px = bx >> 1, py = by >> 1, pz = bz >> 1;
    bool ok = need[map_index(g, l - 1, px, py, pz)] != 0;
    const int z0 = g.dim == 3 ? -1 : 0, z1 = g.dim == 3 ? 1 : 0;
    for (int c = z0; c <= z1 && ok; c++)
      for (int b = -1; b <= 1 && ok; b++)
        for (int a = -1; a <= 1 && ok; a++) {
          int x = bc_block(g, l - 1, 0, px + a), y = bc_block(g, l - 1, 1, py + b), z = bc_block(g, l - 1, 2, pz + c);
          if (x < 0 || y < 0 || z < 0) continue;
          if (!need[map_index(g, l - 1, x, y, z)]) ok = false;
        }
    if (!ok) need[t] = 0;
  }
}
__global__ void k_free(Geo g, const uint8_t *need, int32_t *fs, int *ft) { k_free_dev(g, need, fs, ft); }
__global__ void k_alloc(Geo g, const uint8_t *need, int32_t *fs, int *ft, int32_t *nl, int *nn) {
  k_alloc_dev(g, need, fs, ft, nl, nn);
}
__global__ void k_classify(Geo g, uint8_t *kbits) { k_classify_dev(g, kbits); }
__global__ void k_tile_count(Geo g, const uint8_t *kbits, int32_t *tcount, int ntiles) {
  k_tile_count_dev(g, kbits, tcount, ntiles);
}
__global__ void k_tile_scan(Geo g, const int32_t *tcount, int32_t *toff, int ntiles) {
  k_tile_scan_dev(g, tcount, toff, ntiles);
}
__global__ void k_scatter(Geo g, const uint8_t *kbits, const int32_t *toff, int ntiles) {
  k_scatter_dev(g, kbits, toff, ntiles);
}
__global__ void k_scatter_prefix(Geo g, const uint8_t *kbits, const int32_t *tcount, int ntiles) {
  k_scatter_dev(g, kbits, nullptr, ntiles, tcount);
}

// ---------------------------------------------------------------- gradient flags: row clustering
// Per row of a level's block grid (first direction), runs of at most 8 blocks
// whose flagged fraction stays >= eta; every block of a run is flagged.
__global__ void k_cluster(Geo g, const uint8_t *gflag, uint8_t *sig, double eta) {
  long long rows = 0;
  for (int l = 0; l < g.L; l++) rows += (long long)g.nb[l][1] * g.nb[l][2];
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
    long long u = r;
    int l = 0;
    while (u >= (long long)g.nb[l][1] * g.nb[l][2]) {
      u -= (long long)g.nb[l][1] * g.nb[l][2];
      l++;
    }
    int by = (int)(u % g.nb[l][1]), bz = (int)(u / g.nb[l][1]);
    int nx = g.nb[l][0];
    int x = 0;
    while (x < nx) {
      if (!gflag[map_index(g, l, x, by, bz)]) {
        x++;
        continue;
      }
      int best = x, cnt = 0;
      for (int e = x; e < nx && e - x < 8; e++) {
        if (gflag[map_index(g, l, e, by, bz)]) {
          cnt++;
          if ((double)cnt >= eta * (double)(e - x + 1)) best = e;
        }
      }
      for (int e = x; e <= best; e++) sig[map_index(g, l, e, by, bz)] = 1;
      x = best + 1;
    }
  }
}

// ---------------------------------------------------------------- Berger-Rigoutsos clustering
// The boxes of Berger and Rigoutsos (Section 2.2, the AMROC clustering) over the
// flagged blocks of each level l < L, one CTA per level.  Each box is shrunk to
// its flags; accepted at efficiency >= eta with no side above kBrMaxSide blocks
// (every block of it flagged in sig); else an efficient box is bisected across
// its longest side, and an inefficient one is cut at a hole of its signatures
// (flags per slice; first direction with one, the hole nearest the middle), else
// at the strongest inflection of the signatures (sign change of the second
// difference; ties: lower direction, nearer the middle, lower index), else
// bisected; a cut at slice i gives [lo, i] and [i+1, hi].  Boxes are processed
// breadth-first, one warp per box: the union of accepted boxes does not depend
// on the order, so it equals the depth-first recursion's.
constexpr int kBrMaxSide = 8;
constexpr int kBrMaxRounds = 4096;  // bound on the breadth-first rounds (error bit past it)
constexpr int kBrThreads = 1024;
constexpr int kBrSmemFlags = 160 * 1024;  // flags of a level held in shared memory up to this size

struct BrBox {
  int lo[3], hi[3];
};

// F: the level's flags in map order (shared memory when they fit)
__device__ __forceinline__ int br_flag(const Geo &g, const uint8_t *F, int l, int x, int y, int z) {
  return F[x + (long long)g.nb[l][0] * (y + (long long)g.nb[l][1] * z)] ? 1 : 0;
}

// Shared partial results of the warps of a CTA, reduced per group of warps.
struct BrShared {
  long long cnt[32];
  int mn[32][3], mx[32][3];
  int hd[32][3], hs[32][3];                 // best hole per direction: distance, position
  long long istr[32];                       // best inflection: strength, direction, distance, position
  int idir[32], idm[32], ipos[32];
};

// barrier of a box step: the CTA when groups span several warps, else the warp
// (the group size is the same for every thread of a round)
__device__ __forceinline__ void br_sync(int G) {
  if (G > 1) __syncthreads();
  else __syncwarp();
}

__device__ __forceinline__ bool br_better(long long s1, int d1, int m1, int p1, long long s2, int d2, int m2, int p2) {
  if (s1 != s2) return s1 > s2;
  if (d1 != d2) return d1 < d2;
  if (m1 != m2) return m1 < m2;
  return p1 < p2;
}

// One box of the round, processed by a group of G warps (warps gw0..gw0+G-1;
// tg = thread index in the group): shrink to its flags, then mark it (efficient
// and no side above kBrMaxSide) or cut it in two (a hole of the signatures, the
// strongest inflection, else the middle of the longest side) and push the parts.
// Every thread of the CTA calls this with the same control flow (the barriers);
// a group without a box passes active = false.  The decisions do not depend on
// the group size: integer counts and a total order on the candidate cuts.
__device__ void br_group_box(const Geo &g, int l, const uint8_t *F, uint8_t *sig, double eta, BrBox b, bool active,
                             int gw0, int G, int tg, BrBox *next, int *nnext, int cap, int *sigs, int maxside,
                             BrShared &sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, GT = 32 * G;
  const int D = g.dim;
  int ext[3] = {b.hi[0] - b.lo[0] + 1, b.hi[1] - b.lo[1] + 1, b.hi[2] - b.lo[2] + 1};
  long long vol = active ? (long long)ext[0] * ext[1] * ext[2] : 0;
  // ---- shrink: count and bounding box of the flags
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  long long cnt = 0;
  for (long long t = tg; t < vol; t += GT) {
    int c[3] = {b.lo[0] + (int)(t % ext[0]), b.lo[1] + (int)((t / ext[0]) % ext[1]),
                b.lo[2] + (int)(t / ((long long)ext[0] * ext[1]))};
    if (!br_flag(g, F, l, c[0], c[1], c[2])) continue;
    cnt++;
    for (int d = 0; d < 3; d++) {
      mn[d] = min(mn[d], c[d]);
      mx[d] = max(mx[d], c[d]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    for (int d = 0; d < 3; d++) {
      mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
  }
  if (lane == 0) {
    sh.cnt[warp] = cnt;
    for (int d = 0; d < 3; d++) {
      sh.mn[warp][d] = mn[d];
      sh.mx[warp][d] = mx[d];
    }
  }
  br_sync(G);
  cnt = 0;
  for (int d = 0; d < 3; d++) {
    mn[d] = INT_MAX;
    mx[d] = INT_MIN;
  }
  for (int w = gw0; w < gw0 + G; w++) {
    cnt += sh.cnt[w];
    for (int d = 0; d < 3; d++) {
      mn[d] = min(mn[d], sh.mn[w][d]);
      mx[d] = max(mx[d], sh.mx[w][d]);
    }
  }
  const bool live = active && cnt > 0;
  int longest = 0;
  bool big = false, efficient = false;
  if (live) {
    for (int d = 0; d < 3; d++) {
      b.lo[d] = mn[d];
      b.hi[d] = mx[d];
      ext[d] = mx[d] - mn[d] + 1;
    }
    vol = (long long)ext[0] * ext[1] * ext[2];
    for (int d = 0; d < D; d++) {
      if (ext[d] > kBrMaxSide) big = true;
      if (ext[d] > ext[longest]) longest = d;
    }
    efficient = (double)cnt >= eta * (double)vol;
  }
  const bool mark = live && efficient && !big;
  if (mark) {
    for (long long t = tg; t < vol; t += GT) {
      int x = b.lo[0] + (int)(t % ext[0]), y = b.lo[1] + (int)((t / ext[0]) % ext[1]);
      int z = b.lo[2] + (int)(t / ((long long)ext[0] * ext[1]));
      sig[map_index(g, l, x, y, z)] = 1;
    }
  }
  const bool split = live && !mark, search = split && !efficient;
  // ---- signatures: flags per slice along each direction (the group's threads over slices)
  if (search) {
    for (int d = 0; d < D; d++) {
      const int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;
      for (int sl = tg; sl < ext[d]; sl += GT) {
        int n = 0;
        for (int j = 0; j < ext[a2]; j++)
          for (int i = 0; i < ext[a1]; i++) {
            int c[3];
            c[d] = b.lo[d] + sl;
            c[a1] = b.lo[a1] + i;
            c[a2] = b.lo[a2] + j;
            n += br_flag(g, F, l, c[0], c[1], c[2]);
          }
        sigs[d * maxside + sl] = n;
      }
    }
  }
  br_sync(G);
  // ---- candidate cuts of this thread: per direction the hole nearest the middle
  // (lower index on ties); the strongest inflection (then lower direction, cut
  // nearer the middle, lower position)
  int bd[3] = {INT_MAX, INT_MAX, INT_MAX}, bs[3] = {INT_MAX, INT_MAX, INT_MAX};
  long long bstr = -1;
  int bdir = INT_MAX, bdm = INT_MAX, bpos = INT_MAX;
  if (search) {
    for (int d = 0; d < D; d++) {
      const int mid2 = b.lo[d] + b.hi[d];
      const int *S = sigs + d * maxside;
      for (int sidx = 1 + tg; sidx + 1 < ext[d]; sidx += GT) {
        if (S[sidx] != 0) continue;
        const int s = b.lo[d] + sidx, dist = abs(2 * s - mid2);
        if (dist < bd[d] || (dist == bd[d] && s < bs[d])) {
          bd[d] = dist;
          bs[d] = s;
        }
      }
      const int n = ext[d];
      if (n < 4) continue;
      for (int sidx = 1 + tg; sidx + 2 < n; sidx += GT) {
        long long l1 = (long long)S[sidx - 1] - 2LL * S[sidx] + S[sidx + 1];
        long long l2 = (long long)S[sidx] - 2LL * S[sidx + 1] + S[sidx + 2];
        if (!((l1 < 0 && l2 > 0) || (l1 > 0 && l2 < 0))) continue;
        long long str = l2 - l1 < 0 ? l1 - l2 : l2 - l1;
        int pos = b.lo[d] + sidx, dm = abs(2 * pos + 1 - mid2);
        if (br_better(str, d, dm, pos, bstr, bdir, bdm, bpos)) {
          bstr = str;
          bdir = d;
          bdm = dm;
          bpos = pos;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int d = 0; d < 3; d++) {
      const int od = __shfl_xor_sync(0xffffffffu, bd[d], o), os = __shfl_xor_sync(0xffffffffu, bs[d], o);
      if (od < bd[d] || (od == bd[d] && os < bs[d])) {
        bd[d] = od;
        bs[d] = os;
      }
    }
    const long long ostr = __shfl_xor_sync(0xffffffffu, bstr, o);
    const int odir = __shfl_xor_sync(0xffffffffu, bdir, o), odm = __shfl_xor_sync(0xffffffffu, bdm, o),
              opos = __shfl_xor_sync(0xffffffffu, bpos, o);
    if (br_better(ostr, odir, odm, opos, bstr, bdir, bdm, bpos)) {
      bstr = ostr;
      bdir = odir;
      bdm = odm;
      bpos = opos;
    }
  }
  if (lane == 0) {
    for (int d = 0; d < 3; d++) {
      sh.hd[warp][d] = bd[d];
      sh.hs[warp][d] = bs[d];
    }
    sh.istr[warp] = bstr;
    sh.idir[warp] = bdir;
    sh.idm[warp] = bdm;
    sh.ipos[warp] = bpos;
  }
  br_sync(G);
  if (split && tg == 0) {
    int cd = -1, cut = 0;
    if (search) {
      // holes: the first direction with one
      for (int d = 0; d < D && cd < 0; d++) {
        int hd = INT_MAX, hs = INT_MAX;
        for (int w = gw0; w < gw0 + G; w++)
          if (sh.hd[w][d] < hd || (sh.hd[w][d] == hd && sh.hs[w][d] < hs)) {
            hd = sh.hd[w][d];
            hs = sh.hs[w][d];
          }
        if (hs != INT_MAX) {
          cd = d;
          cut = hs;
        }
      }
      if (cd < 0) {
        long long s1 = -1;
        int d1 = INT_MAX, m1 = INT_MAX, p1 = INT_MAX;
        for (int w = gw0; w < gw0 + G; w++)
          if (br_better(sh.istr[w], sh.idir[w], sh.idm[w], sh.ipos[w], s1, d1, m1, p1)) {
            s1 = sh.istr[w];
            d1 = sh.idir[w];
            m1 = sh.idm[w];
            p1 = sh.ipos[w];
          }
        if (s1 >= 0) {
          cd = d1;
          cut = p1;
        }
      }
    }
    if (cd < 0) {
      cd = longest;
      cut = (b.lo[cd] + b.hi[cd]) / 2;
    }
    BrBox a = b, c = b;
    a.hi[cd] = cut;
    c.lo[cd] = cut + 1;
    int k = atomicAdd(nnext, 2);
    if (k + 1 < cap) {
      next[k] = a;
      next[k + 1] = c;
    } else {
      set_err(g, EB_TREE);  // cannot happen: live boxes are disjoint and each holds a flag
    }
  }
  br_sync(G);
}

// boxes: per level 2 lists of cap_l boxes (cap_l = blocks of the level), at
// boxes + 2 * mapoff[l]; sigs: per level and warp 3 * maxside ints
__global__ void __launch_bounds__(kBrThreads) k_br(Geo g, const uint8_t *gflag, uint8_t *sig, double eta, BrBox *boxes,
                                                   int *sigs, int maxside, int smem_flags) {
  const int l = blockIdx.x;
  if (l >= g.L) return;
  __shared__ int ncur, nnext;
  // the level's flags, read by every round of box splitting: in shared memory when they fit
  extern __shared__ uint8_t sflags[];
  const long long nlev = g.mapoff[l + 1] - g.mapoff[l];
  const uint8_t *F = gflag + g.mapoff[l];
  if (nlev <= smem_flags) {
    for (long long t = threadIdx.x; t < nlev; t += blockDim.x) sflags[t] = F[t];
    __syncthreads();
    F = sflags;
  }
  __shared__ BrShared sh;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int cap = (int)(g.mapoff[l + 1] - g.mapoff[l]);
  BrBox *A = boxes + 2 * g.mapoff[l], *B = A + cap;
  if (threadIdx.x == 0) {
    BrBox w;
    for (int d = 0; d < 3; d++) {
      w.lo[d] = 0;
      w.hi[d] = g.nb[l][d] - 1;
    }
    A[0] = w;
    ncur = 1;
  }
  __syncthreads();
  int round = 0;
  for (; round < kBrMaxRounds && ncur > 0; round++) {
    if (threadIdx.x == 0) nnext = 0;
    __syncthreads();
    // groups of G warps per box while there are fewer boxes than warps (G a power
    // of two dividing the warp count), one warp per box after that
    const int n = ncur;
    int G = 1;
    while (2 * G <= nwarps && 2 * G * n <= nwarps) G *= 2;
    const int ngroups = nwarps / G, gid = warp / G, gw0 = gid * G, tg = threadIdx.x - 32 * gw0;
    int *gsig = sigs + ((long long)l * nwarps + gw0) * 3 * maxside;
    const int iters = (n + ngroups - 1) / ngroups;
    for (int it = 0; it < iters; it++) {
      const int i = gid + it * ngroups;
      const bool active = i < n;
      br_group_box(g, l, F, sig, eta, A[active ? i : 0], active, gw0, G, tg, B, &nnext, cap, gsig, maxside, sh);
    }
    __syncthreads();
    BrBox *t = A;
    A = B;
    B = t;
    if (threadIdx.x == 0) ncur = nnext < cap ? nnext : cap;
    __syncthreads();
  }
  if (threadIdx.x == 0 && ncur > 0) set_err(g, EB_TREE);
}

// ---------------------------------------------------------------- scalars
__global__ void k_set_double(double *p, double v) { *p = v; }

// per-level step table of a preset dt (the CFL path fills it in k_dt's last CTA)
// (one (level, stage) entry per thread: a single thread's chain of double-precision
// divisions would take microseconds on this part)
__global__ void k_level_params(Geo g, const double *dt, int lts, double *lev, float *levf) {
  const double d = *dt;
  for (int k = threadIdx.x; k < 2 * (g.L + 1); k += blockDim.x) level_params_entry(g, d, lts, lev, levf, k >> 1, k & 1);
}

// t += factor * dt; cell-update counter += leaf cells (weighted per level for
// level-dependent steps: a leaf of level l takes 2^l steps per coarse step);
// the list offsets are copied to `pub` (host-mapped memory) when it is set
__global__ void k_advance(Geo g, double *t, const double *dt, double factor, long long *counter, int lts,
                          int32_t *pub) {
  if (pub)
    for (int i = threadIdx.x; i < LK_NUM * (MAXL + 2); i += blockDim.x) pub[i] = g.loff[i];
  if (threadIdx.x != 0) return;
  *t = *t + factor * *dt;
  long long cells = 0;
  int B = block_cells(g.dim);
  for (int l = 0; l <= g.L; l++) {
    long long nl = g.loff[LK_LEAF * (MAXL + 2) + l + 1] - g.loff[LK_LEAF * (MAXL + 2) + l];
    cells += (lts ? (nl << l) : nl) * B;
  }
  counter[0] += cells;
  counter[1] += 1;
}

// Start of an adaptation: significance, gradient-flag and detail maps cleared,
// the needed map set to level 0 alone, the new-block counts zeroed.  With t set,
// CTA 0 also does the step's bookkeeping of k_advance (one launch instead of
// that kernel and five memsets).
__global__ void k_adapt_begin(Geo g, long long total, uint8_t *sig, double *maxdet, uint8_t *gflag, uint8_t *need,
                              int *nnew, double *t, const double *dt, double factor, long long *counter, int lts,
                              int32_t *pub) {
  const long long lvl0 = g.mapoff[1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    sig[i] = 0;
    if (maxdet) maxdet[i] = 0.0;
    if (gflag) gflag[i] = 0;
    need[i] = i < lvl0 ? 1 : 0;
  }
  if (blockIdx.x != 0) return;
  if (threadIdx.x < MAXL) nnew[threadIdx.x] = 0;
  if (!t) return;
  if (pub)
    for (int i = threadIdx.x; i < LK_NUM * (MAXL + 2); i += blockDim.x) pub[i] = g.loff[i];
  if (threadIdx.x == 0) {
    *t = *t + factor * *dt;
    long long cells = 0;
    int B = block_cells(g.dim);
    for (int l = 0; l <= g.L; l++) {
      long long nl = g.loff[LK_LEAF * (MAXL + 2) + l + 1] - g.loff[LK_LEAF * (MAXL + 2) + l];
      cells += (lts ? (nl << l) : nl) * B;
    }
    counter[0] += cells;
    counter[1] += 1;
  }
}

// ---------------------------------------------------------------- launchers
// The tree kernels loop over fixed domains (the dense block maps, the Morton
// positions, the scan tiles): a grid larger than the domain only adds CTAs that
// find no work, and dispatching them costs time.
static int fit(long long items, int per_cta, int grid) {
  long long n = (items + per_cta - 1) / per_cta;
  if (n < 1) n = 1;
  return (int)(n < grid ? n : grid);
}

void launch_need_mark(const Geo &g, const uint8_t *sig, uint8_t *need, int crit, int grid, cudaStream_t st, int lkeep) {
  k_need_mark<<<fit(g.mapoff[g.L + 1], 256, grid), 256, 0, st>>>(g, sig, need, crit, lkeep);
}
void launch_need_close_tail(const Geo &g, int lhi, uint8_t *need, cudaStream_t st) {
  k_need_close_tail<<<1, kTailThreads, 0, st>>>(g, lhi, need);
}
void launch_need_close(const Geo &g, int l, uint8_t *need, int grid, cudaStream_t st, bool parents) {
  k_need_close<<<grid, 256, 0, st>>>(g, l, need, parents ? 1 : 0);
}
void launch_remesh_begin(const Geo &g, long long total, uint8_t *sig, uint8_t *gflag, uint8_t *need, int *nnew, int l0,
                         int grid, cudaStream_t st) {
  k_remesh_begin<<<fit(total, 256, grid), 256, 0, st>>>(g, total, sig, gflag, need, nnew, l0);
}
// every existing block of level l into level l's segment of the new-block list
// (the prolongation kernel's input), its count into nnew[l]
__global__ void k_list_level(Geo g, int l, int32_t *newlist, int *nnew) {
  int b, e;
  list_range(g, LK_EXIST, l, l, b, e);
  const long long cap = g.cap;
  for (int i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x)
    newlist[g.mapoff[l] + (i - b)] = g.lists[LK_EXIST * cap + i];
  if (blockIdx.x == 0 && threadIdx.x == 0) nnew[l] = e - b;
}
void launch_list_level(const Geo &g, int l, int32_t *newlist, int *nnew, int grid, cudaStream_t st) {
  k_list_level<<<grid, 256, 0, st>>>(g, l, newlist, nnew);
}
void launch_need_prune(const Geo &g, int l, uint8_t *need, int grid, cudaStream_t st) {
  k_need_prune<<<fit(g.mapoff[l + 1] - g.mapoff[l], 256, grid), 256, 0, st>>>(g, l, need);
}
void launch_free(const Geo &g, const uint8_t *need, int32_t *fs, int *ft, int grid, cudaStream_t st) {
  k_free<<<fit(g.mapoff[g.L + 1], 256, grid), 256, 0, st>>>(g, need, fs, ft);
}
void launch_alloc(const Geo &g, const uint8_t *need, int32_t *fs, int *ft, int32_t *nl, int *nn, int grid,
                  cudaStream_t st) {
  k_alloc<<<fit(g.mapoff[g.L + 1], 256, grid), 256, 0, st>>>(g, need, fs, ft, nl, nn);
}
void launch_init_freestack(int32_t *fs, int *ft, long long cap, int grid, cudaStream_t st) {
  k_init_freestack<<<grid, 256, 0, st>>>(fs, ft, cap);
}
void launch_rebuild_lists(const Geo &g, uint8_t *kbits, int32_t *tcount, int32_t *toff, int ntiles, int grid,
                          cudaStream_t st) {
  if (ntiles <= kFusedScanTiles) {
    // few tiles: classification fused with the counts, each scatter CTA forms its prefix
    k_classify_count<<<fit(ntiles, 1, grid), SCAN_NT, 0, st>>>(g, kbits, tcount, ntiles);
    k_scatter_prefix<<<fit(ntiles, 1, grid), SCAN_NT, 0, st>>>(g, kbits, tcount, ntiles);
    return;
  }
  k_classify<<<fit(g.moff[g.L + 1], 256, grid), 256, 0, st>>>(g, kbits);
  k_tile_count<<<fit(ntiles, 1, grid), SCAN_NT, 0, st>>>(g, kbits, tcount, ntiles);
  k_tile_scan<<<1, 1024, 0, st>>>(g, tcount, toff, ntiles);
  k_scatter<<<fit(ntiles, 1, grid), SCAN_NT, 0, st>>>(g, kbits, toff, ntiles);
}
int scan_tile_entries() { return SCAN_TILE; }
int rebuild_launches(int ntiles) { return ntiles <= kFusedScanTiles ? 2 : 4; }

void launch_cluster(const Geo &g, const uint8_t *gflag, uint8_t *sig, double eta, int grid, cudaStream_t st) {
  k_cluster<<<grid, 128, 0, st>>>(g, gflag, sig, eta);
}
// scratch of the Berger-Rigoutsos clustering: 2 boxes per block position, and
// 3 * maxside signature counts per warp and level
size_t br_scratch_bytes(const Geo &g, long long maptotal, int maxside) {
  return (size_t)2 * maptotal * sizeof(BrBox) + (size_t)(g.L + 1) * (kBrThreads / 32) * 3 * maxside * sizeof(int) + 256;
}
// opt in to the clustering kernel's shared memory (once per context, outside any capture)
void prepare_br() { cudaFuncSetAttribute(k_br, cudaFuncAttributeMaxDynamicSharedMemorySize, kBrSmemFlags); }
void launch_br(const Geo &g, const uint8_t *gflag, uint8_t *sig, double eta, void *scratch, long long maptotal,
               int maxside, cudaStream_t st) {
  if (g.L < 1) return;
  BrBox *boxes = reinterpret_cast<BrBox *>(scratch);
  int *sigs = reinterpret_cast<int *>(boxes + 2 * maptotal);
  // shared memory for the largest level's flags, up to 160 KB
  long long most = 0;
  for (int l = 0; l < g.L; l++) most = std::max(most, g.mapoff[l + 1] - g.mapoff[l]);
  const int smem = (int)std::min<long long>(most, kBrSmemFlags);
  k_br<<<g.L, kBrThreads, smem, st>>>(g, gflag, sig, eta, boxes, sigs, maxside, smem);
}
void launch_set_double(double *p, double v, cudaStream_t st) { k_set_double<<<1, 1, 0, st>>>(p, v); }
void launch_level_params(const Geo &g, const double *dt, int lts, double *lev, float *levf, cudaStream_t st) {
  k_level_params<<<1, 32, 0, st>>>(g, dt, lts, lev, levf);
}
void launch_adapt_begin(const Geo &g, long long total, uint8_t *sig, double *maxdet, uint8_t *gflag, uint8_t *need,
                        int *nnew, double *t, const double *dt, double factor, long long *counter, int lts,
                        int32_t *pub, int grid, cudaStream_t st) {
  k_adapt_begin<<<fit(total, 256, grid), 256, 0, st>>>(g, total, sig, maxdet, gflag, need, nnew, t, dt, factor,
                                                       counter, lts, pub);
}
void launch_advance(const Geo &g, double *t, const double *dt, double factor, long long *counter, int lts,
                    int32_t *pub, cudaStream_t st) {
  k_advance<<<1, 32, 0, st>>>(g, t, dt, factor, counter, lts, pub);
}

}  // namespace mrfv
