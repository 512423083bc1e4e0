// Tree update kernels (integer work): the block reading of the refinement,
// safety-zone, gradedness and coarsening rules of arXiv:1603.05211 Section 2.1,
// row clustering of gradient flags (Section 2.2), pool allocation, and the
// prefix-scan compaction that rebuilds the neighbour tables and the work lists
// in level-major Morton order.
#include <cuda_runtime.h>
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
__device__ __forceinline__ void map_coords(const Geo &g, int l, long long t, int &bx, int &by, int &bz) {
  long long u = t - g.mapoff[l];
  bx = (int)(u % g.nb[l][0]);
  by = (int)((u / g.nb[l][0]) % g.nb[l][1]);
  bz = (int)(u / ((long long)g.nb[l][0] * g.nb[l][1]));
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

__device__ void mark_nbrs(const Geo &g, uint8_t *need, int l, int bx, int by, int bz) {
  int z0 = g.dim == 3 ? -1 : 0, z1 = g.dim == 3 ? 1 : 0;
  for (int c = z0; c <= z1; c++)
    for (int b = -1; b <= 1; b++)
      for (int a = -1; a <= 1; a++) {
        int x = bc_block(g, l, 0, bx + a), y = bc_block(g, l, 1, by + b), z = bc_block(g, l, 2, bz + c);
        if (x < 0 || y < 0 || z < 0) continue;
        need[map_index(g, l, x, y, z)] = 1;
      }
}
__device__ void mark_children(const Geo &g, uint8_t *need, int l, int bx, int by, int bz) {
  int kz = g.dim == 3 ? 2 : 1;
  for (int c = 0; c < kz; c++)
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++)
        need[map_index(g, l + 1, 2 * bx + a, 2 * by + b, g.dim == 3 ? 2 * bz + c : 0)] = 1;
}

// MR: a significant block of level >= 1 is kept with its 3^d-1 neighbours and,
// below the finest level, its children are added.  GRAD: the children of every
// flagged block are added.  MR with the proposer (crit 2): as MR without the
// neighbours.
__device__ __forceinline__ void k_need_mark_dev(Geo g, const uint8_t *sig, uint8_t *need, int crit) {
  long long total = g.mapoff[g.L + 1];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    if (g.idx[t] < 0 || !sig[t]) continue;
    int l = level_of_map(g, t), bx, by, bz;
    map_coords(g, l, t, bx, by, bz);
    if (crit == 0 || crit == 2) {  // MR (crit 2: without the safety zone, which the proposer replaces)
      if (l == 0) continue;
      need[t] = 1;
      if (crit == 0) mark_nbrs(g, need, l, bx, by, bz);
    }
    if (l < g.L) mark_children(g, need, l, bx, by, bz);
  }
}

// Closure on level l (run from the finest level down): a needed block needs its
// siblings, its parent and the 3^d-1 neighbours of its parent (gradedness).
__device__ __forceinline__ void k_need_close_dev(Geo g, int l, uint8_t *need) {
  long long n = g.mapoff[l + 1] - g.mapoff[l];
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n; u += (long long)gridDim.x * blockDim.x) {
    long long t = g.mapoff[l] + u;
    if (!need[t]) continue;
    int bx, by, bz;
    map_coords(g, l, t, bx, by, bz);
    int px = bx >> 1, py = by >> 1, pz = bz >> 1;
    mark_children(g, need, l - 1, px, py, pz);  // siblings (children of the parent)
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
__device__ __forceinline__ void k_classify_dev(Geo g, uint8_t *kbits) {
  long long total = g.moff[g.L + 1];
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total; m += (long long)gridDim.x * blockDim.x) {
    int l, bx, by, bz;
    uint8_t bits = 0;
    if (morton_block(g, m, l, bx, by, bz)) {
      int32_t s = g.idx[map_index(g, l, bx, by, bz)];
      if (s >= 0) {
        bits = 1u << LK_EXIST;
        bool leaf = !has_children(g, l, bx, by, bz);
        bits |= leaf ? (1u << LK_LEAF) : (1u << LK_INTERNAL);
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
    kbits[m] = bits;
  }
}

constexpr int SCAN_NT = 256;
constexpr int SCAN_PER = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_PER;

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
// owns the first Morton position of a level writes that level's list offsets
__device__ __forceinline__ void k_scatter_dev(Geo g, const uint8_t *kbits, const int32_t *toff, int ntiles) {
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
    __syncthreads();
    for (int k = 0; k < LK_NUM; k++) {
      int add = toff[k * ntiles + tile];
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
__global__ void k_need_mark(Geo g, const uint8_t *sig, uint8_t *need, int crit) { k_need_mark_dev(g, sig, need, crit); }
__global__ void k_need_close(Geo g, int l, uint8_t *need) { k_need_close_dev(g, l, need); }
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

// ---------------------------------------------------------------- scalars
__global__ void k_set_double(double *p, double v) { *p = v; }

// per-level step table of a preset dt (the CFL path fills it in k_dt's last CTA)
__global__ void k_level_params(Geo g, const double *dt, int lts, double *lev, float *levf) {
  if (threadIdx.x == 0) level_params_dev(g, *dt, lts, lev, levf);
}

// t += factor * dt; cell-update counter += leaf cells (weighted per level for
// level-dependent steps: a leaf of level l takes 2^l steps per coarse step)
__global__ void k_advance(Geo g, double *t, const double *dt, double factor, long long *counter, int lts) {
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

// ---------------------------------------------------------------- launchers
// The tree kernels loop over fixed domains (the dense block maps, the Morton
// positions, the scan tiles): a grid larger than the domain only adds CTAs that
// find no work, and dispatching them costs time.
static int fit(long long items, int per_cta, int grid) {
  long long n = (items + per_cta - 1) / per_cta;
  if (n < 1) n = 1;
  return (int)(n < grid ? n : grid);
}

void launch_need_mark(const Geo &g, const uint8_t *sig, uint8_t *need, int crit, int grid, cudaStream_t st) {
  k_need_mark<<<fit(g.mapoff[g.L + 1], 256, grid), 256, 0, st>>>(g, sig, need, crit);
}
void launch_need_close(const Geo &g, int l, uint8_t *need, int grid, cudaStream_t st) {
  k_need_close<<<grid, 256, 0, st>>>(g, l, need);
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
  k_classify<<<fit(g.moff[g.L + 1], 256, grid), 256, 0, st>>>(g, kbits);
  k_tile_count<<<fit(ntiles, 1, grid), SCAN_NT, 0, st>>>(g, kbits, tcount, ntiles);
  k_tile_scan<<<1, 1024, 0, st>>>(g, tcount, toff, ntiles);
  k_scatter<<<fit(ntiles, 1, grid), SCAN_NT, 0, st>>>(g, kbits, toff, ntiles);
}
int scan_tile_entries() { return SCAN_TILE; }

void launch_cluster(const Geo &g, const uint8_t *gflag, uint8_t *sig, double eta, int grid, cudaStream_t st) {
  k_cluster<<<grid, 128, 0, st>>>(g, gflag, sig, eta);
}
void launch_set_double(double *p, double v, cudaStream_t st) { k_set_double<<<1, 1, 0, st>>>(p, v); }
void launch_level_params(const Geo &g, const double *dt, int lts, double *lev, float *levf, cudaStream_t st) {
  k_level_params<<<1, 32, 0, st>>>(g, dt, lts, lev, levf);
}
void launch_advance(const Geo &g, double *t, const double *dt, double factor, long long *counter, int lts,
                    cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(g, t, dt, factor, counter, lts);
}

}  // namespace mrfv
