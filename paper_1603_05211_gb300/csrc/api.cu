// C interface (include/mrfv.h): context, device arena, and the host-side
// sequencing of the kernels for the time step of arXiv:1603.05211
// (Section 2 RK2 step, Section 2.1 adaptation cycle, Fig. 2 level recursion).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.h"
#include "launch.h"
#include "mrfv.h"
#include <cuda_bf16.h>

using namespace mrfv;

// Default persistent-grid sizes, CTAs per SM: `grid` for the grid-stride kernels
// (256-thread CTAs), `bgrid` for the kernels that take one block per CTA.
// Dispatching a CTA costs time even when it finds no work, so these stay small;
// mrfv_set_launch_shape overrides them.
constexpr int kGridCtasPerSm = 8;
constexpr int kBlockCtasPerSm = 16;
// A level with at most this many CTAs of block positions per SM is projected by a
// sweep of its dense maps (two independent reads before the data, against three
// dependent ones for the list of refined blocks); a larger sweep dispatches more
// CTAs than the list needs.
constexpr int kRestrictPosCtasPerSm = 1;
// Up to this many level-0 cells every CTA of the details kernel computes the
// level-0 normalisation itself (no separate reduction launch before it).
constexpr long long kOwnScaleCells = 256;
// Below these leaf counts the MR-scheme stage runs in the staged (thread per
// face) kernel.  Measured on GB300 (FP32): per launch on uniform grids staged
// 11.7 vs pencil 13.0 us at 1024 2D blocks, 22.9 vs 19.7 us at 4096; but inside
// the adaptive 2D step (1400-3000 leaf blocks, the graph keeps the kernel of its
// capture) the pencil kernel gives the shortest step (0.152 ms against 0.157
// staged and 0.156 with two threads per line); in 3D the pencil kernel is
// faster from 512 blocks up (21 vs 34 us).  So both take the pencil kernel.
constexpr long long kStagedBelow2D = 0;
constexpr long long kStagedBelow3D = 0;
// Below these the pencil kernel runs with two threads per line (each half a
// line).  Measured (FP32 uniform, one / two threads per line): 2D 4096 blocks
// 19.9 / 16.8 us, 16384 blocks 36.4 / 36.1 us, 65536 blocks 123 / 140 us; 3D 512
// blocks 21.1 / 22.9 us.
constexpr long long kSplitBelow2D = 0;
constexpr long long kSplitBelow3D = 0;
// Below these leaf counts the single-precision MR-scheme stage runs in the pencil
// kernel that reads primitives staged in shared memory (k_fvp).  Measured on GB300
// inside the adaptive 2D step (about 1700 leaf blocks; same box, alternating runs):
// 0.1011-0.1019 ms per step against 0.1038-0.1040 with the plain pencil kernel.
// Not measured above that size nor in 3D, where the plain pencil kernel stays.
constexpr long long kStagedPrimBelow2D = 4096;
constexpr long long kStagedPrimBelow3D = 0;
// From this leaf count on (2D single precision), the TMA-staged kernel runs.
// Measured (FP32, CUDA events per launch, TMA-staged / pencil): uniform 4096^2
// (262144 blocks) 0.352 / 0.371 ms, 8192^2 1.374 / 1.433 ms; the adaptive 8-level
// workload (about 1700 leaf blocks) 14.3-15.7 / 14.0-14.2 us.
constexpr long long kFvtAbove2D = 65536;

struct mrfv_ctx {
  mrfv_config cfg;
  Geo g;
  int prec;         // MRFV_FP64 / MRFV_FP32
  size_t tsize;     // bytes per state value
  cudaStream_t st;
  int nsm, grid, bgrid, fvgrid[2], fv_occupancy[2];  // pencil kernel: [0] one thread per line, [1] two
  int fvs_occupancy[2], fvsgrid[2];  // staged stage kernel: [0] MR scheme, [1] MUSCL-Hancock
  int stage_kernel;                  // 0 by leaf count, 1 pencil, 2 staged, 3 split pencil, 4 pencil on staged primitives
  int fvpgrid, fvp_occupancy, fvp_bpc;
  int fv_kinds;                      // stage kernels launched since profiling was enabled (bit mask)
  int gkinds[2];                     // stage kernels in each captured step graph (bit mask)
  char *arena;
  size_t arena_bytes;
  bool own_arena;
  void *U, *Us, *U0, *G, *FR, *scale;
  uint8_t *sig, *need, *gflag, *kbits;
  double *maxdet;
  int32_t *freestack, *newlist, *tcount, *toff;
  int *freetop, *nnew;
  double *dsc;              // [0] dt of the finest level, [1] t
  double *lev;              // per-level step table (lev_index)
  float *levf;              // its single-precision copy
  unsigned long long *red;  // reductions
  long long *counter;       // [0] cell updates, [1] steps
  double *totals;
  int ntiles;
  long long maptotal, mtotal;
  bool initialized;
  std::string err;
  // diagnostics
  long long nlaunch;
  bool prof;
  std::vector<cudaEvent_t> evs;  // start/end pairs of timed stage launches
  size_t ev_used;
  std::vector<cudaEvent_t> pevs;  // start/end pairs around the proposer's convolution launches
  size_t pev_used;
  std::vector<cudaEvent_t> revs;  // start/end pairs around the Richardson estimate's launches
  size_t rev_used;
  unsigned long long *dbytes;
  unsigned *done;  // last-CTA counter of the CFL reduction
  // learned proposer
  float *pfeat, *plogit, *pb1, *pb2, *pb3, *pblob, *pgrad, *pm1, *pm2, *pwork;
  uint8_t *ptile;                 // tiles each layer needs (restricted inference), 3 x ptiles bytes
  long long ptiles;               // 128-position tiles
  unsigned long long *ptcount;    // tiles computed per layer while profiling
  long long pdense;               // dense inferences while profiling
  __nv_bfloat16 *pa0, *pa1, *pa2, *pw1, *pw2, *pw3, *pw3t, *pw2t;
  double *ploss;
  bool has_weights;
  int adam_t;
  // CUDA graph of one step: [0] with the CFL reduction, [1] with a preset dt
  cudaStream_t cap_st;
  // second branch of a step: work that only reads the state runs beside the main chain
  cudaStream_t st2;
  cudaEvent_t ev_step, ev_dt, ev_ghost, ev_begin;
  cudaGraphExec_t gexec[2];
  long long glaunch[2];  // kernels in each captured step
  // Launch sizing: the list offsets the current launch shapes were chosen for
  // (snap), and host-mapped memory into which every step copies the current
  // offsets (pub_host, written by the GPU through pub_dev).
  int32_t snap[LK_NUM * (MAXL + 2)];
  bool snap_valid;
  int32_t *pub_host, *pub_dev;
  int fv_bpc, fvs_bpc;  // blocks per CTA iteration of the pencil and the staged kernels
  void *brscratch;      // Berger-Rigoutsos boxes and signatures
  unsigned *rctl;       // [3]: CTAs done of the scale reduction
  int br_maxside;       // longest side, in blocks, of the levels that are clustered
  unsigned long long *rmask;  // Richardson: per block position, the coarse cells with |tau| > eps_r
  void *rscratch;       // Richardson: the patches of each CTA
  unsigned long long *rcount;  // Richardson: blocks estimated while profiling
  int rich_ctas;        // CTAs of the Richardson estimate (0: off)
  FvtSet fvt;           // TMA-staged stage kernel (2D single precision): tensor maps
  int fvtgrid;          // its persistent grid
};

// CTAs of the Richardson estimate, at most one per block below the finest level.
// 3D: two per SM of a 152-SM part, each with its own area of the global scratch
// (the arena is sized for these).  2D: an upper bound here; mrfv_create lowers it
// to the CTAs the SMs hold with the patch's shared memory.
int rich_ctas_of(const mrfv_config *cfg, const Geo &g) {
  if (!(cfg->eps_r > 0.0) || g.L < 1) return 0;
  long long n = g.mapoff[g.L];
  long long want = cfg->dim == 2 ? 1216 : 304;
  return (int)(n < want ? n : want);
}

static thread_local std::string g_create_error;

namespace {

int fail(mrfv_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return code;
}

int check_launch(mrfv_ctx *c, const char *where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, MRFV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return MRFV_OK;
}

// synchronise the stream and turn the device error word into a status
int check_device(mrfv_ctx *c, const char *where) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return fail(c, MRFV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  int bits = 0;
  e = cudaMemcpy(&bits, c->g.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(c, MRFV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  if (bits) {
    cudaMemset(c->g.err, 0, sizeof(int));
    if (bits & EB_TIMEOUT) return fail(c, MRFV_ERR_TIMEOUT, std::string(where) + ": a bounded device wait expired");
    if (bits & EB_POOL) return fail(c, MRFV_ERR_POOL_FULL, std::string(where) + ": block pool capacity exceeded");
    if (bits & EB_TREE) return fail(c, MRFV_ERR_TREE, std::string(where) + ": a kernel met a block tree that is not graded");
    if (bits & EB_NONPHYS)
      return fail(c, MRFV_ERR_NONPHYSICAL, std::string(where) + ": non-physical state (rho <= 0, p <= 0 or NaN)");
  }
  return MRFV_OK;
}

int ilog2_ceil(int x) {
  int b = 0;
  while ((1 << b) < x) b++;
  return b;
}

bool fill_geo(const mrfv_config *cfg, Geo &g, long long &maptotal, long long &mtotal, long long &full) {
  memset(&g, 0, sizeof(g));
  if (cfg->dim != 2 && cfg->dim != 3) return false;
  if (cfg->levels < 1 || cfg->levels > MAXL) return false;
  g.dim = cfg->dim;
  g.nv = cfg->dim + 2;
  g.L = cfg->levels - 1;
  g.bc = cfg->bc;
  g.gamma = cfg->gamma;
  for (int d = 0; d < 3; d++) g.lo[d] = cfg->lo[d];
  maptotal = 0;
  mtotal = 0;
  for (int l = 0; l <= g.L; l++) {
    long long nblk = 1;
    int mx = 1;
    for (int d = 0; d < 3; d++) {
      if (d < g.dim) {
        long long n = (long long)cfg->base_blocks[d] << l;
        if (cfg->base_blocks[d] < 1 || n > (1 << 20)) return false;
        g.nb[l][d] = (int)n;
        g.dx[l][d] = (cfg->hi[d] - cfg->lo[d]) / (double)(n * BS);
        if (!(g.dx[l][d] > 0.0)) return false;
        if (g.nb[l][d] > mx) mx = g.nb[l][d];
      } else {
        g.nb[l][d] = 1;
        g.dx[l][d] = 1.0;
      }
      nblk *= g.nb[l][d];
    }
    if (nblk >= (1ll << 31)) return false;  // block positions of one level are indexed in 32 bits
    g.mapoff[l] = maptotal;
    maptotal += nblk;
    g.mbits[l] = ilog2_ceil(mx);
    g.moff[l] = mtotal;
    mtotal += 1ll << (g.mbits[l] * g.dim);
  }
  g.mapoff[g.L + 1] = maptotal;
  g.moff[g.L + 1] = mtotal;
  full = maptotal;
  return true;
}

struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = (off + 255) & ~(size_t)255;
    off = o + bytes;
    return o;
  }
};

// Assign every device buffer an offset in the arena; returns the total size.
size_t layout(const mrfv_config *cfg, const Geo &g, long long cap, long long maptotal, long long mtotal, int ntiles,
              mrfv_ctx *c) {
  size_t ts = cfg->precision == MRFV_FP32 ? 4 : 8;
  int nv = g.nv, B = block_cells(g.dim), TF = face_cells(g.dim);
  Layout L;
  size_t state = (size_t)nv * cap * B * ts;
  size_t oU = L.take(state), oUs = L.take(state), oU0 = L.take(cfg->lts ? state : 0);  // U0: level-step start states (LTS)
  size_t oG = L.take((size_t)nv * cap * 2 * g.dim * 2 * TF * ts);
  size_t oFR = L.take((size_t)nv * cap * 2 * g.dim * TF * ts);
  size_t oidx = L.take(maptotal * 4), olev = L.take(cap * 4), ocoord = L.take(cap * 12), onbr = L.take(cap * 24);
  size_t ocm = L.take(cap), okids = L.take(cap * 32), oloff = L.take(LK_NUM * (MAXL + 2) * 4), olists = L.take((size_t)LK_NUM * cap * 4);
  size_t oerr = L.take(4);
  size_t osig = L.take(maptotal), oneed = L.take(maptotal), ogf = L.take(maptotal), omd = L.take(maptotal * 8);
  size_t okb = L.take(mtotal), otc = L.take((size_t)LK_NUM * ntiles * 4), oto = L.take((size_t)LK_NUM * ntiles * 4);
  size_t ofs = L.take(cap * 4), oft = L.take(4), onl = L.take(maptotal * 4), onn = L.take(MAXL * 4);
  size_t odsc = L.take(4 * 8), ored = L.take(4 * 8), ocnt = L.take(2 * 8), otot = L.take(5 * 8), osc = L.take(5 * ts);
  size_t obyt = L.take(8), olevp = L.take(2 * MAXL * 4 * 8), olevf = L.take(2 * MAXL * 4 * 4);
  size_t odone = L.take(8);
  const size_t NW = MRFV_PROPOSER_NWEIGHTS;
  size_t opf = L.take(3 * maptotal * 4), opl = L.take(maptotal * 4), opa0 = L.take(8 * maptotal * 2);
  size_t opa1 = L.take(16 * maptotal * 2), opa2 = L.take(16 * maptotal * 2);
  size_t opw1 = L.take(16 * 224 * 2), opw2 = L.take(16 * 432 * 2), opw3 = L.take(16 * 432 * 2);
  size_t opw3t = L.take(16 * 224 * 2), opw2t = L.take(16 * 432 * 2);
  size_t opb = L.take(3 * 16 * 4), opblob = L.take(4 * NW * 4), opwork = L.take((size_t)kPropWorkPerPos * maptotal * 4), oploss = L.take(8);
  const long long ptiles = (maptotal + 127) / 128;
  size_t optile = L.take(3 * (size_t)ptiles), optc = L.take(3 * 8);
  int maxside = 1;
  if (g.L >= 1)
    for (int d = 0; d < g.dim; d++) maxside = g.nb[g.L - 1][d] > maxside ? g.nb[g.L - 1][d] : maxside;
  size_t obr = L.take(br_scratch_bytes(g, maptotal, maxside));
  size_t orctl = L.take(4 * 4);
  const int rctas = rich_ctas_of(cfg, g);
  size_t ormask = L.take(rctas ? maptotal * 8 : 0), orcnt = L.take(8);
  const int hk = cfg->scheme == MRFV_SCHEME_HANCOCK ? 1 : 0;
  size_t orscr = L.take(rctas ? (size_t)rctas * (size_t)(cfg->precision == MRFV_FP32 ? rich_scratch_bytes<float>(g.dim, hk)
                                                                                  : rich_scratch_bytes<double>(g.dim, hk))
                              : 0);
  if (c) {
    c->br_maxside = maxside;
    char *a = c->arena;
    c->U = a + oU; c->Us = a + oUs; c->U0 = a + oU0; c->G = a + oG; c->FR = a + oFR;
    c->g.idx = (int32_t *)(a + oidx); c->g.slot_level = (int32_t *)(a + olev);
    c->g.slot_coord = (int32_t *)(a + ocoord); c->g.nbr = (int32_t *)(a + onbr);
    c->g.cmask = (uint8_t *)(a + ocm); c->g.kids = (int32_t *)(a + okids); c->g.loff = (int32_t *)(a + oloff); c->g.lists = (int32_t *)(a + olists);
    c->g.err = (int *)(a + oerr);
    c->sig = (uint8_t *)(a + osig); c->need = (uint8_t *)(a + oneed); c->gflag = (uint8_t *)(a + ogf);
    c->maxdet = (double *)(a + omd); c->kbits = (uint8_t *)(a + okb);
    c->tcount = (int32_t *)(a + otc); c->toff = (int32_t *)(a + oto);
    c->freestack = (int32_t *)(a + ofs); c->freetop = (int *)(a + oft);
    c->newlist = (int32_t *)(a + onl); c->nnew = (int *)(a + onn);
    c->dsc = (double *)(a + odsc); c->red = (unsigned long long *)(a + ored);
    c->counter = (long long *)(a + ocnt); c->totals = (double *)(a + otot); c->scale = a + osc;
    c->dbytes = (unsigned long long *)(a + obyt);
    c->lev = (double *)(a + olevp);
    c->levf = (float *)(a + olevf);
    c->done = (unsigned *)(a + odone);
    c->pfeat = (float *)(a + opf);
    c->plogit = (float *)(a + opl);
    c->pa0 = (__nv_bfloat16 *)(a + opa0);
    c->pa1 = (__nv_bfloat16 *)(a + opa1);
    c->pa2 = (__nv_bfloat16 *)(a + opa2);
    c->pw1 = (__nv_bfloat16 *)(a + opw1);
    c->pw2 = (__nv_bfloat16 *)(a + opw2);
    c->pw3 = (__nv_bfloat16 *)(a + opw3);
    c->pw3t = (__nv_bfloat16 *)(a + opw3t);
    c->pw2t = (__nv_bfloat16 *)(a + opw2t);
    c->pb1 = (float *)(a + opb);
    c->pb2 = c->pb1 + 16;
    c->pb3 = c->pb2 + 16;
    c->pblob = (float *)(a + opblob);
    c->pgrad = c->pblob + NW;
    c->pm1 = c->pgrad + NW;
    c->pm2 = c->pm1 + NW;
    c->pwork = (float *)(a + opwork);
    c->ploss = (double *)(a + oploss);
    c->ptile = (uint8_t *)(a + optile);
    c->ptiles = ptiles;
    c->ptcount = (unsigned long long *)(a + optc);
    c->brscratch = a + obr;
    c->rctl = (unsigned *)(a + orctl);
    c->rich_ctas = rctas;
    c->rmask = rctas ? (unsigned long long *)(a + ormask) : nullptr;
    c->rscratch = rctas ? (void *)(a + orscr) : nullptr;
    c->rcount = (unsigned long long *)(a + orcnt);
  }
  return L.off + 256;
}

long long capacity_of(const mrfv_config *cfg, long long full) {
  return cfg->pool_blocks > 0 ? (long long)cfg->pool_blocks : full;
}

int ntiles_of(long long mtotal) { return (int)((mtotal + scan_tile_entries() - 1) / scan_tile_entries()); }

long long level_blocks(const Geo &g, int l) { return g.mapoff[l + 1] - g.mapoff[l]; }
// captured step graphs hold kernel arguments and launch shapes: drop them when either changes
void drop_graphs(mrfv_ctx *c) {
  for (int v = 0; v < 2; v++)
    if (c->gexec[v]) {
      cudaGraphExecDestroy(c->gexec[v]);
      c->gexec[v] = nullptr;
    }
}

// The largest level l <= lmax whose dense map holds at most max_positions block
// positions (the levels below it hold fewer), or -1.
int tail_level(const Geo &g, long long max_positions, int lmax) {
  int lt = -1;
  for (int l = 0; l <= lmax && l <= g.L; l++)
    if (level_blocks(g, l) <= max_positions) lt = l;
    else break;
  return lt;
}

int grid_for(long long items, int per_cta, int cap_grid) {
  long long n = (items + per_cta - 1) / per_cta;
  if (n < 1) n = 1;
  return (int)(n < cap_grid ? n : cap_grid);
}

// Exact list offsets (synchronises the stream); used when a step graph is
// captured and after explicit tree changes.
void snapshot_exact(mrfv_ctx *c) {
  cudaStreamSynchronize(c->st);
  if (cudaMemcpy(c->snap, c->g.loff, sizeof(c->snap), cudaMemcpyDeviceToHost) == cudaSuccess) {
    c->snap_valid = true;
    if (c->pub_host) memcpy(c->pub_host, c->snap, sizeof(c->snap));  // nothing in flight writes it now
  } else {
    cudaGetLastError();
  }
}
// The offsets the last finished step published (no synchronisation; at most a
// step old).
void snapshot_published(mrfv_ctx *c) {
  if (!c->pub_host) return;
  memcpy(c->snap, (const void *)c->pub_host, sizeof(c->snap));
  c->snap_valid = true;
}
long long list_count(const mrfv_ctx *c, const int32_t *off, int kind, int l0, int l1) {
  return (long long)off[kind * (MAXL + 2) + l1 + 1] - off[kind * (MAXL + 2) + l0];
}
// CTAs for a kernel that loops over list `kind` on levels l0..l1: twice the
// snapshot's count (per_item work units per listed block, per_cta units per CTA
// iteration), at least one CTA per SM (launching up to that many costs no more
// than launching one), at most cap.  Every kernel loops over the device-resident
// list, so any size is correct; the size only decides how fast.
int sized(const mrfv_ctx *c, int kind, int l0, int l1, long long per_item, long long per_cta, int cap) {
  if (!c->snap_valid) return cap;
  long long n = list_count(c, c->snap, kind, l0, l1);
  long long want = (2 * n * per_item + per_cta - 1) / per_cta;
  if (want < c->nsm) want = c->nsm;
  return (int)(want < cap ? want : cap);
}
// A captured graph keeps its launch shapes; re-capture when the tree the shapes
// were sized for has grown past the headroom or shrunk well below it.
bool shapes_stale(const mrfv_ctx *c) {
  if (!c->pub_host || !c->snap_valid) return false;
  const int kinds[3] = {LK_LEAF, LK_EXIST, LK_GHOST};
  for (int k : kinds) {
    long long was = list_count(c, c->snap, k, 0, c->g.L);
    long long now = list_count(c, (const int32_t *)c->pub_host, k, 0, c->g.L);
    if (now > (was * 3) / 2 + 16 || (was > 64 && now < was / 3)) return true;
  }
  return false;
}

// ---------------------------------------------------------------- typed sequencing
template <typename T>
struct Seq {
  mrfv_ctx *c;
  T *U() { return (T *)c->U; }
  T *Us() { return (T *)c->Us; }
  T *U0() { return (T *)c->U0; }
  T *G() { return (T *)c->G; }
  T *FR() { return (T *)c->FR; }

  void restrict_level(int l, T *A) {
    // at most the blocks of level l are refined
    const int bpc = c->g.dim == 2 ? 4 : 1;
    const long long pos = level_blocks(c->g, l);
    if (pos <= (long long)kRestrictPosCtasPerSm * bpc * c->nsm) {
      // few positions: one pass over the dense maps, a shorter chain of reads
      launch_restrict_pos<T>(c->g, l, A, grid_for(pos, bpc, c->grid), c->st);
      return;
    }
    int dense = grid_for(pos, bpc, c->grid);
    launch_restrict<T>(c->g, l, A, sized(c, LK_INTERNAL, l, l, 1, bpc, dense), c->st);
  }
  // every level, finest first: one launch per level, and the coarse levels whose
  // positions one CTA covers in a pass together in one single-CTA launch
  void restrict_all(T *A) { restrict_from(c->g.L - 1, A); }
  // levels top..0
  void restrict_from(int top, T *A) {
    int lt = tail_level(c->g, kTailThreads / block_cells(c->g.dim), top);
    while (lt >= 0 && c->g.mapoff[lt + 1] > (c->g.dim == 2 ? kRestrictTailBlocks2D : kRestrictTailBlocks3D)) lt--;
    for (int l = top; l > lt; l--) restrict_level(l, A);
    if (top > lt) c->nlaunch += top - lt;
    if (lt >= 0) {
      launch_restrict_tail<T>(c->g, lt, A, c->st);
      c->nlaunch += 1;
    }
  }
  // end of a step: flux correction of levels 0..L-1, then the projection of every
  // level; where level L-1 takes the list form, its projection shares the launch
  // of the correction (neither reads what the other writes)
  void reflux_restrict_all() {
    const Geo &g = c->g;
    const int L = g.L;
    if (L < 1) return;
    const int bpc = g.dim == 2 ? 4 : 1, nt = g.dim == 2 ? 256 : 512;
    const long long pos = level_blocks(g, L - 1);
    int lt = tail_level(g, kTailThreads / block_cells(g.dim), L - 1);
    while (lt >= 0 && g.mapoff[lt + 1] > (g.dim == 2 ? kRestrictTailBlocks2D : kRestrictTailBlocks3D)) lt--;
    if (L - 1 > lt && pos > (long long)kRestrictPosCtasPerSm * bpc * c->nsm) {
      const int nr = sized(c, LK_REFLUX, 0, L - 1, block_cells(g.dim), nt, c->grid);
      const int np = sized(c, LK_INTERNAL, L - 1, L - 1, 1, bpc, grid_for(pos, bpc, c->grid));
      launch_reflux_restrict<T>(g, U(), FR(), nr, np, c->st);
      c->nlaunch += 1;
      restrict_from(L - 2, U());
      return;
    }
    launch_reflux<T>(g, 0, L - 1, U(), FR(), sized(c, LK_REFLUX, 0, L - 1, block_cells(g.dim), 256, c->grid), c->st);
    c->nlaunch += 1;
    restrict_all(U());
  }
  // between the two stages: the ghost strips and the projection of restrict_edge_dev
  // in one launch (the strips project their coarse cells on the fly)
  void ghost_edge(T *A) {
    if (c->g.L < 1) return;
    const int ng = sized(c, LK_GHOST, 1, c->g.L, 1, 1, c->bgrid);
    int dense = grid_for(c->g.mapoff[c->g.L + 1] - c->g.mapoff[1], 4, c->grid);
    const int ne = sized(c, LK_LEAF, 1, c->g.L, 1, 4, dense);
    launch_ghost_edge<T>(c->g, A, G(), ng, ne, c->st);
    c->nlaunch += 1;
  }
  void fv(int kind, int l0, int l1, const T *Uin, const T *U0b, T *Uout, double coef, int lts, int record) {
    FVArgs<T> a;
    a.Uin = Uin; a.U0 = U0b; a.Uout = Uout; a.G = G(); a.FR = FR();
    a.kind = kind; a.l0 = l0; a.l1 = l1; a.coef = coef; a.lev = c->lev; a.levf = c->levf; a.record = record;
    (void)lts;
    a.stage = coef == 0.5 ? 0 : 1;
    a.words = (coef == 0.5 ? 2 : 3) * c->g.nv;
    a.C = nullptr; a.C0 = nullptr; a.theta = 0.0;
    timed_fv(a, false);
  }
  // one MUSCL-Hancock stage (Section 2, AMR scheme): Uout = Uin - dt F(Uin); halo
  // edges that need prediction read level l-1 of Uin (or its time interpolation
  // from C0 at theta)
  void fvh(int kind, int l0, int l1, const T *Uin, T *Uout, const T *C0, double theta, int record) {
    FVArgs<T> a;
    a.Uin = Uin; a.U0 = Uin; a.Uout = Uout; a.G = G(); a.FR = FR();
    a.kind = kind; a.l0 = l0; a.l1 = l1; a.coef = 1.0; a.lev = c->lev; a.levf = c->levf; a.record = record;
    a.stage = 1;
    a.words = 2 * c->g.nv;
    a.C = Uin; a.C0 = C0; a.theta = theta;
    timed_fv(a, true);
  }
  // MR-scheme stage: the pencil kernel, or the staged kernel while the list is
  // too short for the pencil kernel's one thread per line to fill the GPU
  bool use_staged(const FVArgs<T> &a) const {
    if (c->stage_kernel != 0) return c->stage_kernel == 2;
    if (!c->snap_valid) return false;
    long long n = list_count(c, c->snap, a.kind, a.l0, a.l1);
    return n < (c->g.dim == 2 ? kStagedBelow2D : kStagedBelow3D);
  }
  // pencil kernel reading primitives staged in shared memory
  bool use_fvp(const FVArgs<T> &a) const {
    if (c->stage_kernel != 0) return c->stage_kernel == 4;
    if (sizeof(T) != 4 || !c->snap_valid) return false;
    long long n = list_count(c, c->snap, a.kind, a.l0, a.l1);
    return n < (c->g.dim == 2 ? kStagedPrimBelow2D : kStagedPrimBelow3D);
  }
  // pencil kernel with two threads per line while the list is short
  bool use_split(const FVArgs<T> &a) const {
    if (c->stage_kernel != 0) return c->stage_kernel == 3;
    if (!c->snap_valid) return false;
    long long n = list_count(c, c->snap, a.kind, a.l0, a.l1);
    return n < (c->g.dim == 2 ? kSplitBelow2D : kSplitBelow3D);
  }
  // TMA-staged stage kernel (2D single precision, every buffer of the launch mapped)
  bool use_fvt(const FVArgs<T> &a) const {
    if constexpr (sizeof(T) != 4) {
      return false;
    } else {
      if (!c->fvt.ok) return false;
      if (c->stage_kernel != 0 && c->stage_kernel != 5) return false;
      if (c->stage_kernel == 0) {
        if (!c->snap_valid) return false;
        if (list_count(c, c->snap, a.kind, a.l0, a.l1) < kFvtAbove2D) return false;
      }
      bool in = false, u0 = false;
      for (int b = 0; b < 3; b++) {
        in = in || (c->fvt.buf[b] && c->fvt.buf[b] == (const void *)a.Uin);
        u0 = u0 || (c->fvt.buf[b] && c->fvt.buf[b] == (const void *)a.U0);
      }
      return in && u0;
    }
  }
  // launch a finite-volume stage kernel, bracketed by events when profiling
  void timed_fv(FVArgs<T> &a, bool hancock) {
    a.bytes = c->prof ? c->dbytes : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
      if (c->ev_used + 2 > c->evs.size()) {
        for (int k = 0; k < 64; k++) {
          cudaEvent_t e;
          cudaEventCreate(&e);
          c->evs.push_back(e);
        }
      }
      e0 = c->evs[c->ev_used];
      e1 = c->evs[c->ev_used + 1];
      c->ev_used += 2;
      cudaEventRecord(e0, c->st);
    }
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (!hancock && use_fvt(a)) {
        done = launch_fvt(c->g, a, c->fvt, sized(c, a.kind, a.l0, a.l1, 1, fvt_blocks_per_cta(), c->fvtgrid), c->st);
        if (done) c->fv_kinds |= 32;
      }
    }
    if (done) {
    } else if (!hancock && use_fvp(a)) {
      launch_fvp<T>(c->g, a, sized(c, a.kind, a.l0, a.l1, 1, c->fvp_bpc, c->fvpgrid), c->st);
      c->fv_kinds |= 8;
    } else if (hancock || use_staged(a)) {
      int h = hancock ? 1 : 0;
      launch_fvs<T>(c->g, a, hancock, sized(c, a.kind, a.l0, a.l1, 1, c->fvs_bpc, c->fvsgrid[h]), c->st);
      c->fv_kinds |= hancock ? 16 : 2;
    } else {
      int sp = use_split(a) ? 1 : 0;
      launch_fv<T>(c->g, a, sp == 1, sized(c, a.kind, a.l0, a.l1, 1, c->fv_bpc, c->fvgrid[sp]), c->st);
      c->fv_kinds |= sp ? 4 : 1;
    }
    if (c->prof) cudaEventRecord(e1, c->st);
    c->nlaunch += 1;
  }
  void ghost(int l0, int l1, const T *A, const T *A0, double theta) {
    if (l1 < 1) return;
    int a0 = l0 < 1 ? 1 : l0;
    launch_ghost<T>(c->g, a0, l1, A, A0, theta, G(), sized(c, LK_GHOST, a0, l1, 1, 1, c->bgrid), c->st);
    c->nlaunch += 1;
  }
  // one midpoint-RK2 step of every leaf with the same dt (Section 2)
  // (ghost_done: the first ghost strips were filled on the step's second branch)
  void step_global(bool ghost_done = false) {
    int L = c->g.L;
    if (c->cfg.scheme == MRFV_SCHEME_HANCOCK) {
      // one stage into Us, leaves copied back, then the correction and projection
      if (!ghost_done) ghost(1, L, U(), nullptr, 0.0);
      fvh(LK_LEAF, 0, L, U(), Us(), nullptr, 0.0, 1);
      launch_copy_level<T>(c->g, LK_LEAF, 0, L, Us(), U(), sized(c, LK_LEAF, 0, L, block_cells(c->g.dim), 256, c->grid), c->st);
      c->nlaunch += 1;
      reflux_restrict_all();
      return;
    }
    if (!ghost_done) ghost(1, L, U(), nullptr, 0.0);
    fv(LK_LEAF, 0, L, U(), U(), Us(), 0.5, 0, 0);
    ghost_edge(Us());
    fv(LK_LEAF, 0, L, Us(), U(), U(), 1.0, 0, 1);
    reflux_restrict_all();
  }
  // Fig. 2 recursion: level l takes one step of dt_l = 2^(L-l) dt (all its blocks),
  // then level l+1 two steps, then projection and flux correction of level l.
  void advance(int l, int sub) {
    int L = c->g.L;
    // Fig. 2: Remesh(l) before the update; at the first sub-step it would repeat
    // the parent's Remesh(l-1), which regenerated these levels from the same data
    if (sub == 1 && l >= 1 && l < L && c->cfg.adapt && c->cfg.lts_remesh) remesh(l);
    double th1 = 0.5 * sub, th2 = th1 + 0.25;
    launch_copy_level<T>(c->g, LK_EXIST, l, l, U(), U0(), sized(c, LK_EXIST, l, l, block_cells(c->g.dim), 256, c->grid), c->st);
    c->nlaunch += 1;
    if (l >= 1) ghost(l, l, U(), U0(), th1);
    if (c->cfg.scheme == MRFV_SCHEME_HANCOCK) {
      // one stage from the sub-step start, halo at its start time
      fvh(LK_EXIST, l, l, U(), Us(), U0(), th1, sub == 1 ? 2 : 1);
      launch_copy_level<T>(c->g, LK_EXIST, l, l, Us(), U(), sized(c, LK_EXIST, l, l, block_cells(c->g.dim), 256, c->grid), c->st);
      c->nlaunch += 1;
    } else {
      fv(LK_EXIST, l, l, U(), U(), Us(), 0.5, 1, 0);
      if (l >= 1) ghost(l, l, U(), U0(), th2);
      fv(LK_EXIST, l, l, Us(), U(), U(), 1.0, 1, sub == 1 ? 2 : 1);
    }
    if (l < L) {
      advance(l + 1, 0);
      advance(l + 1, 1);
      restrict_level(l, U());
      launch_reflux<T>(c->g, l, l, U(), FR(), sized(c, LK_REFLUX, l, l, block_cells(c->g.dim), 256, c->grid), c->st);
      c->nlaunch += 2;
    }
  }
  // cleared: the maps were cleared by the adaptation's first kernel; l0, A0: a
  // remesh's analysis of levels l0..L, level l0 against level l0-1 halfway
  // through its step (A0 + (A - A0)/2)
  // marks: the MR criterion's needed-block marks made by the details kernel (the
  // adaptation of a step, without the proposer)
  void analyse(double eps, bool cleared = false, int l0 = 1, const T *A0 = nullptr, bool marks = false) {
    // a level 0 of a few blocks: every details CTA computes the normalisation itself
    const bool own = level_blocks(c->g, 0) * block_cells(c->g.dim) <= kOwnScaleCells;
    if (!own) {
      launch_scales<T>(c->g, U(), c->red + 0, c->rctl + 3, (T *)c->scale,
                       grid_for(level_blocks(c->g, 0) * block_cells(c->g.dim), 256, c->grid), c->st);
      c->nlaunch += 1;
    }
    if (!cleared) {
      cudaMemsetAsync(c->sig, 0, c->maptotal, c->st);
      cudaMemsetAsync(c->maxdet, 0, c->maptotal * 8, c->st);
    }
    launch_details<T>(c->g, U(), (const T *)c->scale, eps, c->sig, c->maxdet, l0, A0, 0.5,
                      sized(c, LK_EXIST, l0, c->g.L, 1, 1, c->bgrid), c->st, own ? (T *)c->scale : nullptr,
                      marks ? c->need : nullptr);
    c->nlaunch += 1;
  }
  // new blocks of levels lfrom..lto (default L; a remesh above l0 creates none below l0+1)
  void prolong_new(int lfrom = 1, int lto = -1) {
    // at most two CTAs per SM: an adaptation adds few blocks per level, and a
    // level that gets none costs the dispatch of every CTA of the grid
    const int top = lto < 0 ? c->g.L : lto;
    int l = lfrom;
    if (lfrom == 1) {
      // the coarse levels, where a new block is rare (at most 64 positions in 2D,
      // 8 in 3D), in one single-CTA launch that takes the new blocks one by one
      const int lt = tail_level(c->g, c->g.dim == 2 ? 64 : 8, top);
      if (lt >= 2) {
        launch_prolong_tail<T>(c->g, lt, c->newlist, c->nnew, U(), c->st);
        c->nlaunch += 1;
        l = lt + 1;
      }
    }
    for (; l <= top; l++) {
      launch_prolong<T>(c->g, l, c->newlist, c->nnew, U(),
                        sized(c, LK_EXIST, l, l, 1, 1, grid_for(level_blocks(c->g, l), 1, 2 * c->nsm)), c->st);
      c->nlaunch += 1;
    }
  }
  // CFL reduction; its last CTA sets dt and the per-level step table
  void compute_dt(int lts) {
    launch_dt<T>(c->g, U(), lts, c->red + 3, c->done, c->cfg.cfl, c->cfg.t_end, c->dsc, c->lev, c->levf,
                 sized(c, LK_LEAF, 0, c->g.L, block_cells(c->g.dim), 1024, c->grid),
                 c->st);
    c->nlaunch += 1;
  }
  void init_level(const ICParams &ic) {
    launch_init<T>(c->g, ic, c->cfg.hi, U(), c->grid, c->st);
    c->nlaunch += 1;
    restrict_all(U());
  }
  void prop_features() {
    launch_prop_features<T>(c->g, U(), c->maxdet, (const T *)c->scale, c->cfg.eps, c->pfeat, c->grid, c->st);
    c->nlaunch += 1;
  }
  // Remesh(l0) of Fig. 2 at the second sub-step of level l0: gradient flags of
  // levels l0..L-1 (level l0's absent cells from level l0-1 halfway through its
  // step) and clustering, or the MR analysis of levels l0..L (level l0 against
  // level l0-1 halfway through its step); the marks above l0 (children of
  // flagged or significant blocks, the safety zone above l0), closure above l0
  // only, nesting, then the tree update of the levels above l0
  void remesh(int l0);
  // Richardson estimate of levels l0..L-1 (level l0's absent cells from level
  // l0-1 halfway through its step when A0 is set) and gflag |= its block flags
  void rich(int l0, const T *A0) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
      if (c->rev_used + 2 > c->revs.size())
        for (int k = 0; k < 16; k++) {
          cudaEvent_t e;
          cudaEventCreate(&e);
          c->revs.push_back(e);
        }
      e0 = c->revs[c->rev_used];
      e1 = c->revs[c->rev_used + 1];
      c->rev_used += 2;
      cudaEventRecord(e0, c->st);
    }
    launch_rich<T>(c->g, c->cfg.scheme, U(), A0, 0.5, l0, c->lev, c->cfg.eps_r, c->rmask, c->maxdet, c->gflag,
                   (T *)c->rscratch, c->rich_ctas, c->grid, c->prof ? c->rcount : nullptr, c->st);
    if (c->prof) cudaEventRecord(e1, c->st);
    c->nlaunch += 2;
  }
  void gradflags(bool cleared = false) {
    if (!cleared) {
      cudaMemsetAsync(c->gflag, 0, c->maptotal, c->st);
      cudaMemsetAsync(c->sig, 0, c->maptotal, c->st);
    }
    launch_gradflags<T>(c->g, U(), c->cfg.eps_w, c->cfg.eps_p, c->gflag, 0, (const T *)nullptr, 0.0, c->bgrid, c->st);
    if (c->rich_ctas) rich(0, nullptr);
    if (c->cfg.clustering == MRFV_CLUSTER_BR)
      launch_br(c->g, c->gflag, c->sig, c->cfg.eta_tol, c->brscratch, c->maptotal, c->br_maxside, c->st);
    else
      launch_cluster(c->g, c->gflag, c->sig, c->cfg.eta_tol, c->grid, c->st);
    c->nlaunch += 2;
  }
};

template <typename F>
void dispatch(mrfv_ctx *c, F f) {
  if (c->prec == MRFV_FP32) {
    Seq<float> s{c};
    f(s);
  } else {
    Seq<double> s{c};
    f(s);
  }
}

// free, allocate, rebuild neighbour tables and lists, optionally predict new blocks
void apply_need(mrfv_ctx *c, bool prolong, bool cleared = false, int lfrom = 1) {
  if (!cleared) cudaMemsetAsync(c->nnew, 0, MAXL * sizeof(int), c->st);
  launch_free(c->g, c->need, c->freestack, c->freetop, c->grid, c->st);
  launch_alloc(c->g, c->need, c->freestack, c->freetop, c->newlist, c->nnew, c->grid, c->st);
  launch_rebuild_lists(c->g, c->kbits, c->tcount, c->toff, c->ntiles, c->grid, c->st);
  c->nlaunch += 2 + rebuild_launches(c->ntiles);
  if (prolong) dispatch(c, [&](auto &s) { s.prolong_new(lfrom); });
}

template <typename T>
void Seq<T>::remesh(int l0) {
  const Geo &g = c->g;
  const int L = g.L;
  launch_remesh_begin(g, c->maptotal, c->sig, c->gflag, c->need, c->nnew, l0, c->grid, c->st);
  if (c->cfg.criterion == MRFV_CRIT_GRAD) {
    launch_gradflags<T>(g, U(), c->cfg.eps_w, c->cfg.eps_p, c->gflag, l0, U0(), 0.5, c->bgrid, c->st);
    if (c->rich_ctas) rich(l0, U0());
    if (c->cfg.clustering == MRFV_CLUSTER_BR)
      launch_br(g, c->gflag, c->sig, c->cfg.eta_tol, c->brscratch, c->maptotal, c->br_maxside, c->st);
    else
      launch_cluster(g, c->gflag, c->sig, c->cfg.eta_tol, c->grid, c->st);
  } else {
    // the MR analysis of levels l0..L (the safety zone, not the proposer, inside the recursion)
    analyse(c->cfg.eps, true, l0, U0());
  }
  launch_need_mark(g, c->sig, c->need, c->cfg.criterion, c->grid, c->st, l0);
  for (int m = L; m >= l0 + 1; m--)
    launch_need_close(g, m, c->need, grid_for(level_blocks(g, m), 256, c->grid), c->st, m - 1 > l0);
  for (int m = l0 + 1; m <= L; m++) launch_need_prune(g, m, c->need, c->grid, c->st);
  c->nlaunch += 5 + 2 * (L - l0);
  apply_need(c, true, true, l0 + 1);
}

// restricted: only the tiles whose logits can add a block (the adaptation's use);
// otherwise every position (mrfv_proposer_infer, and cfg.proposer_dense)
void prop_infer(mrfv_ctx *c, bool restricted) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (restricted) {
    launch_prop_tiles(c->g, c->ptile, c->ptiles, c->prof ? c->ptcount : nullptr, c->grid, c->st);
    c->nlaunch += c->prof ? 2 : 1;
  } else if (c->prof) {
    c->pdense += 1;
  }
  if (c->prof) {
    if (c->pev_used + 2 > c->pevs.size())
      for (int k = 0; k < 16; k++) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->pevs.push_back(e);
      }
    e0 = c->pevs[c->pev_used];
    e1 = c->pevs[c->pev_used + 1];
    c->pev_used += 2;
  }
  launch_prop_infer(c->g, c->pfeat, c->pa0, c->pa1, c->pa2, c->pw1, c->pb1, c->pw2, c->pb2, c->pw3, c->pb3, c->plogit,
                    c->nsm, e0, e1, restricted ? c->ptile : nullptr, c->st);
  c->nlaunch += 4;
}

// analysis / flags -> needed blocks -> closure -> apply
// the first kernel of an adaptation (step: with the step's time and counter bookkeeping)
void adapt_begin(mrfv_ctx *c, bool step) {
  const int lts = c->cfg.lts;
  launch_adapt_begin(c->g, c->maptotal, c->sig, c->maxdet, c->gflag, c->need, c->nnew, step ? c->dsc + 1 : nullptr,
                     c->dsc, lts ? ldexp(1.0, c->g.L) : 1.0, c->counter, lts, c->pub_dev, c->grid, c->st);
  c->nlaunch += 1;
}
// (begun: adapt_begin already ran, on the step's second branch)
void adapt_tree(mrfv_ctx *c, bool step = false, bool begun = false) {
  const Geo &g = c->g;
  bool use_prop = c->cfg.proposer && c->has_weights && c->cfg.criterion == MRFV_CRIT_MR;
  if (!begun) adapt_begin(c, step);
  // MR without the proposer: the details kernel makes the needed-block marks
  const bool fused_marks = c->cfg.criterion == MRFV_CRIT_MR && !use_prop;
  if (c->cfg.criterion == MRFV_CRIT_MR) dispatch(c, [&](auto &s) { s.analyse(c->cfg.eps, true, 1, nullptr, fused_marks); });
  else dispatch(c, [&](auto &s) { s.gradflags(true); });
  if (use_prop) {
    dispatch(c, [&](auto &s) { s.prop_features(); });
    prop_infer(c, !c->cfg.proposer_dense);
  }
  if (!fused_marks) {
    launch_need_mark(g, c->sig, c->need, use_prop ? 2 : c->cfg.criterion, c->grid, c->st);
    c->nlaunch += 1;
  }
  if (use_prop) {
    launch_prop_mark(g, c->plogit, c->need, c->grid, c->st);
    c->nlaunch += 1;
  }
  // finest first; the levels whose positions one CTA covers in a pass together
  // (and whose need maps fit in its shared memory)
  int lt = tail_level(g, kTailThreads, g.L);
  while (lt >= 1 && g.mapoff[lt + 1] > kTailNeedBytes) lt--;
  for (int l = g.L; l >= 1 && l > lt; l--) {
    launch_need_close(g, l, c->need, grid_for(level_blocks(g, l), 256, c->grid), c->st);
    c->nlaunch += 1;
  }
  if (lt >= 1) {
    launch_need_close_tail(g, lt, c->need, c->st);
    c->nlaunch += 1;
  }
  apply_need(c, true, true);
}

bool valid_tree(const mrfv_ctx *c, const uint8_t *ex) {
  const Geo &g = c->g;
  auto at = [&](int l, int x, int y, int z) -> bool {
    return ex[g.mapoff[l] + x + (long long)g.nb[l][0] * (y + (long long)g.nb[l][1] * z)] != 0;
  };
  for (long long t = 0; t < g.mapoff[1]; t++)
    if (!ex[t]) return false;
  for (int l = 1; l <= g.L; l++)
    for (int z = 0; z < g.nb[l][2]; z++)
      for (int y = 0; y < g.nb[l][1]; y++)
        for (int x = 0; x < g.nb[l][0]; x++) {
          if (!at(l, x, y, z)) continue;
          int px = x >> 1, py = y >> 1, pz = g.dim == 3 ? z >> 1 : 0;
          for (int cz = 0; cz < (g.dim == 3 ? 2 : 1); cz++)
            for (int cy = 0; cy < 2; cy++)
              for (int cx = 0; cx < 2; cx++)
                if (!at(l, 2 * px + cx, 2 * py + cy, g.dim == 3 ? 2 * pz + cz : 0)) return false;
          for (int c3 = (g.dim == 3 ? -1 : 0); c3 <= (g.dim == 3 ? 1 : 0); c3++)
            for (int b = -1; b <= 1; b++)
              for (int a = -1; a <= 1; a++) {
                int q[3] = {px + a, py + b, pz + c3};
                bool in = true;
                for (int d = 0; d < g.dim; d++) {
                  int N = g.nb[l - 1][d];
                  if (q[d] < 0 || q[d] >= N) {
                    if (g.bc == MRFV_BC_PERIODIC) q[d] = (q[d] % N + N) % N;
                    else in = false;
                  }
                }
                if (in && !at(l - 1, q[0], q[1], q[2])) return false;
              }
        }
  return true;
}

long long level_cells(const Geo &g, int l) {
  long long n = 1;
  for (int d = 0; d < g.dim; d++) n *= (long long)g.nb[l][d] * BS;
  return n;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int mrfv_config_default(mrfv_config *cfg) {
  if (!cfg) return MRFV_ERR_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->dim = 2;
  cfg->precision = MRFV_FP64;
  cfg->levels = 1;
  cfg->base_blocks[0] = cfg->base_blocks[1] = cfg->base_blocks[2] = 1;
  cfg->hi[0] = cfg->hi[1] = cfg->hi[2] = 1.0;
  cfg->bc = MRFV_BC_TRANSMISSIVE;
  cfg->gamma = 1.4;
  cfg->cfl = 0.5;
  cfg->eps = 1e-3;
  cfg->eps_w = 0.05;
  cfg->eta_tol = 0.8;
  cfg->use_graph = 1;
  cfg->lts_remesh = 1;
  return MRFV_OK;
}

size_t mrfv_arena_bytes(const mrfv_config *cfg) {
  if (!cfg) return 0;
  Geo g;
  long long mt, mo, full;
  if (!fill_geo(cfg, g, mt, mo, full)) return 0;
  return layout(cfg, g, capacity_of(cfg, full), mt, mo, ntiles_of(mo), nullptr);
}

int mrfv_create(const mrfv_config *cfg, mrfv_ctx **out) {
  if (!cfg || !out) return fail(nullptr, MRFV_ERR_ARG, "null argument");
  *out = nullptr;
  if (cfg->precision != MRFV_FP32 && cfg->precision != MRFV_FP64) return fail(nullptr, MRFV_ERR_ARG, "precision");
  if (cfg->bc != MRFV_BC_TRANSMISSIVE && cfg->bc != MRFV_BC_PERIODIC) return fail(nullptr, MRFV_ERR_ARG, "bc");
  if (cfg->criterion != MRFV_CRIT_MR && cfg->criterion != MRFV_CRIT_GRAD) return fail(nullptr, MRFV_ERR_ARG, "criterion");
  if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return fail(nullptr, MRFV_ERR_ARG, "gamma/cfl");
  if (cfg->pool_blocks < 0) return fail(nullptr, MRFV_ERR_ARG, "pool_blocks");
  if (cfg->scheme != MRFV_SCHEME_MUSCL_RK2 && cfg->scheme != MRFV_SCHEME_HANCOCK)
    return fail(nullptr, MRFV_ERR_ARG, "scheme");
  if (cfg->clustering != MRFV_CLUSTER_ROWS && cfg->clustering != MRFV_CLUSTER_BR)
    return fail(nullptr, MRFV_ERR_ARG, "clustering");
  if (!(cfg->eps_p >= 0.0)) return fail(nullptr, MRFV_ERR_ARG, "eps_p");
  if (!(cfg->eps_r >= 0.0) || !(cfg->eps_r < INFINITY)) return fail(nullptr, MRFV_ERR_ARG, "eps_r");
  if (cfg->eps_r > 0.0 && cfg->criterion != MRFV_CRIT_GRAD)
    return fail(nullptr, MRFV_ERR_ARG, "eps_r: the Richardson estimate adds to the gradient criterion");
  if (cfg->lts_remesh != 0 && cfg->lts_remesh != 1) return fail(nullptr, MRFV_ERR_ARG, "lts_remesh");
  if (cfg->proposer_dense != 0 && cfg->proposer_dense != 1) return fail(nullptr, MRFV_ERR_ARG, "proposer_dense");
  {
    Geo gg;
    long long a, b, f;
    if (!fill_geo(cfg, gg, a, b, f)) return fail(nullptr, MRFV_ERR_ARG, "dim/levels/base_blocks/domain");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(nullptr, MRFV_ERR_CUDA, "no CUDA device: this library has no CPU path");
  }
  mrfv_ctx *c = new mrfv_ctx();
  c->cfg = *cfg;
  c->prec = cfg->precision;
  c->tsize = c->prec == MRFV_FP32 ? 4 : 8;
  c->st = (cudaStream_t)cfg->stream;
  long long full;
  fill_geo(cfg, c->g, c->maptotal, c->mtotal, full);
  c->g.cap = capacity_of(cfg, full);
  if (c->g.cap > (1ll << 30)) {
    delete c;
    return fail(nullptr, MRFV_ERR_ARG, "pool capacity too large");
  }
  c->ntiles = ntiles_of(c->mtotal);
  if (c->ntiles > 65535) {
    delete c;
    return fail(nullptr, MRFV_ERR_ARG, "hierarchy too large");
  }
  size_t bytes = layout(cfg, c->g, c->g.cap, c->maptotal, c->mtotal, c->ntiles, nullptr);
  if (cfg->device_arena) {
    if (cfg->arena_bytes < bytes) {
      delete c;
      return fail(nullptr, MRFV_ERR_ARG, "device_arena smaller than mrfv_arena_bytes()");
    }
    c->arena = (char *)cfg->device_arena;
    c->own_arena = false;
  } else {
    if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return fail(nullptr, MRFV_ERR_CUDA, "cudaMalloc of the device arena failed");
    }
    c->own_arena = true;
  }
  c->arena_bytes = bytes;
  layout(cfg, c->g, c->g.cap, c->maptotal, c->mtotal, c->ntiles, c);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
  for (int sp = 0; sp < 2; sp++)
    c->fv_occupancy[sp] =
        c->prec == MRFV_FP32 ? fv_ctas_per_sm<float>(cfg->dim, sp == 1) : fv_ctas_per_sm<double>(cfg->dim, sp == 1);
  c->grid = c->nsm * kGridCtasPerSm;
  c->bgrid = c->nsm * kBlockCtasPerSm;
  for (int sp = 0; sp < 2; sp++) c->fvgrid[sp] = c->nsm * c->fv_occupancy[sp];
  for (int h = 0; h < 2; h++) {
    c->fvs_occupancy[h] =
        c->prec == MRFV_FP32 ? fvs_ctas_per_sm<float>(cfg->dim, h == 1) : fvs_ctas_per_sm<double>(cfg->dim, h == 1);
    c->fvsgrid[h] = c->nsm * c->fvs_occupancy[h];
  }
  c->stage_kernel = 0;
  c->fv_kinds = 0;
  c->gkinds[0] = c->gkinds[1] = 0;
  prepare_br();
  if (c->rich_ctas) {
    int per_sm = 0;
    const int h = cfg->scheme == MRFV_SCHEME_HANCOCK ? 1 : 0;
    cudaError_t e = c->prec == MRFV_FP32 ? prepare_rich<float>(cfg->dim, h, &per_sm)
                                         : prepare_rich<double>(cfg->dim, h, &per_sm);
    if (e != cudaSuccess) {
      std::string msg = std::string("Richardson estimate: shared-memory set-up failed: ") + cudaGetErrorString(e);
      cudaGetLastError();
      mrfv_destroy(c);
      return fail(nullptr, MRFV_ERR_CUDA, msg);
    }
    // 2D: the CTAs the SMs hold at once with the patch in shared memory
    if (cfg->dim == 2 && per_sm > 0 && (long long)per_sm * c->nsm < c->rich_ctas) c->rich_ctas = per_sm * c->nsm;
  }
  c->fvp_occupancy = c->prec == MRFV_FP32 ? fvp_ctas_per_sm<float>(cfg->dim) : fvp_ctas_per_sm<double>(cfg->dim);
  c->fvpgrid = c->nsm * c->fvp_occupancy;
  c->fvp_bpc = c->prec == MRFV_FP32 ? fvp_blocks_per_cta<float>(cfg->dim) : fvp_blocks_per_cta<double>(cfg->dim);
  c->fv_bpc = c->prec == MRFV_FP32 ? fv_blocks_per_cta<float>(cfg->dim, false) : fv_blocks_per_cta<double>(cfg->dim, false);
  c->fvs_bpc = c->prec == MRFV_FP32 ? fv_blocks_per_cta<float>(cfg->dim, true) : fv_blocks_per_cta<double>(cfg->dim, true);
  // the TMA-staged stage kernel for 2D single precision (tensor maps of the state
  // buffers and the ghost strips); without it the pencil kernel runs
  c->fvt.ok = false;
  c->fvtgrid = 0;
  if (c->prec == MRFV_FP32 && cfg->dim == 2 && fvt_prepare(c->fvt, c->g, c->U, c->Us, c->U0, c->G))
    c->fvtgrid = c->nsm * c->fvt.ctas_per_sm;
  cudaGetLastError();
  c->snap_valid = false;
  c->pub_host = c->pub_dev = nullptr;
  if (cudaHostAlloc((void **)&c->pub_host, sizeof(c->snap), cudaHostAllocMapped) == cudaSuccess) {
    memset(c->pub_host, 0, sizeof(c->snap));
    if (cudaHostGetDevicePointer((void **)&c->pub_dev, c->pub_host, 0) != cudaSuccess) {
      cudaFreeHost(c->pub_host);
      c->pub_host = c->pub_dev = nullptr;
    }
  }
  cudaGetLastError();  // without mapped memory the shapes are sized from exact snapshots only
  cudaMemsetAsync(c->g.idx, 0xff, c->maptotal * 4, c->st);
  cudaMemsetAsync(c->g.slot_level, 0xff, c->g.cap * 4, c->st);
  cudaMemsetAsync(c->g.loff, 0, LK_NUM * (MAXL + 2) * 4, c->st);
  cudaMemsetAsync(c->g.err, 0, 4, c->st);
  cudaMemsetAsync(c->dsc, 0, 4 * 8, c->st);
  cudaMemsetAsync(c->counter, 0, 2 * 8, c->st);
  cudaMemsetAsync(c->rctl, 0, 4 * 4, c->st);
  cudaMemsetAsync(c->red, 0, 4 * 8, c->st);
  cudaMemsetAsync(c->red + 3, 0x7f, 8, c->st);  // the CFL minimum's start value, a huge positive double
  cudaMemsetAsync(c->done, 0, 4, c->st);
  // step table zero until the first step (the Richardson estimate of an adaptation
  // before any step is then zero)
  cudaMemsetAsync(c->lev, 0, 2 * MAXL * 4 * 8, c->st);
  cudaMemsetAsync(c->levf, 0, 2 * MAXL * 4 * 4, c->st);
  launch_init_freestack(c->freestack, c->freetop, c->g.cap, c->grid, c->st);
  if (cfg->use_graph && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) c->cap_st = nullptr;
  if (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess) c->st2 = nullptr;
  for (cudaEvent_t *e : {&c->ev_step, &c->ev_dt, &c->ev_ghost, &c->ev_begin})
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) *e = nullptr;
  prop_setup();
  int rc = check_launch(c, "mrfv_create");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_create");
  if (rc != MRFV_OK) {
    g_create_error = c->err;
    mrfv_destroy(c);
    return rc;
  }
  *out = c;
  return MRFV_OK;
}

int mrfv_destroy(mrfv_ctx *c) {
  if (!c) return MRFV_OK;
  cudaStreamSynchronize(c->st);
  for (cudaEvent_t e : c->evs) cudaEventDestroy(e);
  for (cudaEvent_t e : c->pevs) cudaEventDestroy(e);
  for (cudaEvent_t e : c->revs) cudaEventDestroy(e);
  for (int v = 0; v < 2; v++)
    if (c->gexec[v]) cudaGraphExecDestroy(c->gexec[v]);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  if (c->st2) cudaStreamDestroy(c->st2);
  for (cudaEvent_t e : {c->ev_step, c->ev_dt, c->ev_ghost, c->ev_begin})
    if (e) cudaEventDestroy(e);
  if (c->pub_host) cudaFreeHost(c->pub_host);
  if (c->own_arena && c->arena) cudaFree(c->arena);
  delete c;
  return MRFV_OK;
}

const char *mrfv_last_error(const mrfv_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int mrfv_init_state(mrfv_ctx *c, int kind, const double *params, int n) {
  if (!c || n < 0 || n > 16 || (n > 0 && !params) || kind < 0 || kind > 5) return fail(c, MRFV_ERR_ARG, "init: arguments");
  if (c->g.cap < c->maptotal) return fail(c, MRFV_ERR_POOL_FULL, "init needs a pool that holds every block of every level");
  ICParams ic;
  memset(&ic, 0, sizeof(ic));
  ic.kind = kind;
  for (int i = 0; i < n; i++) ic.p[i] = params[i];
  drop_graphs(c);
  c->snap_valid = false;
  cudaMemsetAsync(c->need, 1, c->maptotal, c->st);
  apply_need(c, false);
  dispatch(c, [&](auto &s) { s.init_level(ic); });
  cudaMemsetAsync(c->dsc, 0, 4 * 8, c->st);
  cudaMemsetAsync(c->counter, 0, 2 * 8, c->st);
  if (c->cfg.adapt) adapt_tree(c);
  int rc = check_launch(c, "mrfv_init_state");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_init_state");
  c->initialized = rc == MRFV_OK;
  if (rc == MRFV_OK) snapshot_exact(c);
  return rc;
}

int mrfv_analyse(mrfv_ctx *c, double eps, int64_t *n_sig) {
  if (!c) return MRFV_ERR_ARG;
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "analyse before init");
  dispatch(c, [&](auto &s) {
    s.restrict_all(s.U());
    s.analyse(eps);
  });
  int rc = check_launch(c, "mrfv_analyse");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_analyse");
  if (rc != MRFV_OK) return rc;
  if (n_sig) {
    std::vector<uint8_t> h(c->maptotal);
    cudaMemcpy(h.data(), c->sig, c->maptotal, cudaMemcpyDeviceToHost);
    int64_t k = 0;
    for (uint8_t b : h) k += b;
    *n_sig = k;
  }
  return MRFV_OK;
}

int mrfv_adapt(mrfv_ctx *c, int use_proposer, int64_t *n_blocks) {
  if (!c || (use_proposer != 0 && use_proposer != 1)) return fail(c, MRFV_ERR_ARG, "adapt: use_proposer is 0 or 1");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "adapt before init");
  if (use_proposer && !c->has_weights) return fail(c, MRFV_ERR_STATE, "adapt: proposer without weights");
  int saved = c->cfg.proposer;
  c->cfg.proposer = use_proposer;
  adapt_tree(c);
  c->cfg.proposer = saved;
  int rc = check_launch(c, "mrfv_adapt");
  if (rc != MRFV_OK) return rc;
  snapshot_exact(c);
  if (n_blocks) {
    rc = check_device(c, "mrfv_adapt");
    if (rc != MRFV_OK) return rc;
    int32_t e = 0;
    cudaMemcpy(&e, c->g.loff + LK_EXIST * (MAXL + 2) + c->g.L + 1, 4, cudaMemcpyDeviceToHost);
    *n_blocks = e;
  }
  return MRFV_OK;
}

int mrfv_compute_dt(mrfv_ctx *c, double *dt_out) {
  if (!c) return MRFV_ERR_ARG;
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "dt before init");
  dispatch(c, [&](auto &s) { s.compute_dt(c->cfg.lts); });
  int rc = check_launch(c, "mrfv_compute_dt");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_compute_dt");
  if (rc == MRFV_OK && dt_out) cudaMemcpy(dt_out, c->dsc, 8, cudaMemcpyDeviceToHost);
  return rc;
}

int mrfv_fill_ghosts(mrfv_ctx *c, int level, int buffer) {
  if (!c || level < 1 || level > c->g.L || buffer < 0 || buffer > 1) return fail(c, MRFV_ERR_ARG, "fill_ghosts: arguments");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "fill_ghosts before init");
  dispatch(c, [&](auto &s) { s.ghost(level, level, buffer ? s.Us() : s.U(), nullptr, 0.0); });
  return check_launch(c, "mrfv_fill_ghosts");
}

}  // extern "C"

namespace {
// Every launch of one step after dt is set (preset) or with the CFL reduction;
// nothing here synchronises, so the sequence can be captured into a graph.
void issue_step(mrfv_ctx *c, bool preset) {
  int lts = c->cfg.lts;
  // With global steps two branches: the first ghost strips and, once dt is known,
  // the adaptation's first kernel (it clears maps the stages do not touch) run
  // beside the CFL reduction and the stages.
  const bool fork = !lts && c->st2 && c->ev_step && c->ev_dt && c->ev_ghost && c->ev_begin;
  const bool fork_begin = fork && c->cfg.adapt;
  dispatch(c, [&](auto &s) {
    if (fork) {
      cudaEventRecord(c->ev_step, c->st);
      cudaStreamWaitEvent(c->st2, c->ev_step, 0);
      cudaStream_t main = c->st;
      c->st = c->st2;
      s.ghost(1, c->g.L, s.U(), nullptr, 0.0);
      c->st = main;
      cudaEventRecord(c->ev_ghost, c->st2);
    }
    if (!preset) {
      s.compute_dt(lts);
    } else {
      launch_level_params(c->g, c->dsc, lts, c->lev, c->levf, c->st);
      c->nlaunch += 1;
    }
    if (fork_begin) {
      cudaEventRecord(c->ev_dt, c->st);
      cudaStreamWaitEvent(c->st2, c->ev_dt, 0);
      cudaStream_t main = c->st;
      c->st = c->st2;
      adapt_begin(c, true);
      c->st = main;
      cudaEventRecord(c->ev_begin, c->st2);
    }
    if (fork) cudaStreamWaitEvent(c->st, c->ev_ghost, 0);
    if (lts) s.advance(0, 0);
    else s.step_global(fork);
  });
  if (fork_begin) cudaStreamWaitEvent(c->st, c->ev_begin, 0);
  if (c->cfg.adapt) {
    adapt_tree(c, true, fork_begin);
  } else {
    launch_advance(c->g, c->dsc + 1, c->dsc, lts ? ldexp(1.0, c->g.L) : 1.0, c->counter, lts, c->pub_dev, c->st);
    c->nlaunch += 1;
  }
}

// Capture one step into graph variant v (once per context: every kernel argument
// is a fixed device pointer or a configuration constant, and every work-list
// length is read on the device).
int capture_step(mrfv_ctx *c, int v) {
  snapshot_exact(c);  // the graph's launch shapes are sized for the tree of now
  cudaStream_t user = c->st;
  c->st = c->cap_st;
  long long before = c->nlaunch;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal);
  const int kinds = c->fv_kinds;
  c->fv_kinds = 0;
  if (e == cudaSuccess) {
    issue_step(c, v == 1);
    e = cudaStreamEndCapture(c->cap_st, &graph);
  }
  c->gkinds[v] = c->fv_kinds;
  c->fv_kinds = kinds;
  c->st = user;
  c->glaunch[v] = c->nlaunch - before;
  c->nlaunch = before;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec[v], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->gexec[v] = nullptr;
    return fail(c, MRFV_ERR_CUDA, std::string("mrfv_step: graph capture: ") + cudaGetErrorString(e));
  }
  return MRFV_OK;
}
}  // namespace

extern "C" {

int mrfv_step(mrfv_ctx *c, double dt, double *dt_out) {
  if (!c) return MRFV_ERR_ARG;
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "step before init");
  bool preset = dt > 0.0;
  if (preset) {
    launch_set_double(c->dsc, dt, c->st);
    c->nlaunch += 1;
  }
  if (c->cfg.use_graph && c->cap_st && !c->prof) {
    int v = preset ? 1 : 0;
    if (shapes_stale(c)) drop_graphs(c);
    if (!c->gexec[v]) {
      int rc = capture_step(c, v);
      if (rc != MRFV_OK) return rc;
    }
    if (cudaGraphLaunch(c->gexec[v], c->st) != cudaSuccess) return check_launch(c, "mrfv_step: graph launch");
    c->nlaunch += c->glaunch[v];
  } else {
    snapshot_published(c);
    issue_step(c, preset);
  }
  int rc = check_launch(c, "mrfv_step");
  if (rc != MRFV_OK) return rc;
  if (dt_out) {
    rc = check_device(c, "mrfv_step");
    if (rc != MRFV_OK) return rc;
    cudaMemcpy(dt_out, c->dsc, 8, cudaMemcpyDeviceToHost);
  }
  return MRFV_OK;
}

int mrfv_step_level(mrfv_ctx *c, int level, double dt) {
  if (!c || level < 0 || level > c->g.L || !(dt > 0.0)) return fail(c, MRFV_ERR_ARG, "step_level: arguments");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "step_level before init");
  if (!c->cfg.lts) return fail(c, MRFV_ERR_STATE, "step_level needs cfg.lts (the level-step start states)");
  launch_set_double(c->dsc, dt, c->st);
  launch_level_params(c->g, c->dsc, 1, c->lev, c->levf, c->st);
  c->nlaunch += 2;
  dispatch(c, [&](auto &s) { s.advance(level, 0); });
  return check_launch(c, "mrfv_step_level");
}

int mrfv_restrict(mrfv_ctx *c, int fine_level) {
  if (!c || fine_level > c->g.L) return fail(c, MRFV_ERR_ARG, "restrict: level");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "restrict before init");
  dispatch(c, [&](auto &s) {
    if (fine_level <= 0) s.restrict_all(s.U());
    else s.restrict_level(fine_level - 1, s.U());
  });
  return check_launch(c, "mrfv_restrict");
}

int mrfv_prolong(mrfv_ctx *c, int coarse_level) {
  if (!c || coarse_level < 0 || coarse_level >= c->g.L) return fail(c, MRFV_ERR_ARG, "prolong: level");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "prolong before init");
  const int l = coarse_level + 1;
  launch_list_level(c->g, l, c->newlist, c->nnew, c->grid, c->st);
  c->nlaunch += 1;
  dispatch(c, [&](auto &s) { s.prolong_new(l, l); });
  cudaMemsetAsync(c->nnew, 0, MAXL * sizeof(int), c->st);  // no stale count for the next adaptation
  int rc = check_launch(c, "mrfv_prolong");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_prolong");
  return rc;
}

int mrfv_conserved_totals(mrfv_ctx *c, double *out, int n) {
  if (!c || !out || n < c->g.nv) return fail(c, MRFV_ERR_ARG, "totals: buffer");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "totals before init");
  dispatch(c, [&](auto &s) { launch_totals(c->g, s.U(), c->totals, c->grid, c->st); });
  c->nlaunch += 1;
  int rc = check_launch(c, "mrfv_conserved_totals");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_conserved_totals");
  if (rc == MRFV_OK) cudaMemcpy(out, c->totals, c->g.nv * 8, cudaMemcpyDeviceToHost);
  return rc;
}

int mrfv_get_stats(mrfv_ctx *c, mrfv_stats *o) {
  if (!c || !o) return MRFV_ERR_ARG;
  int rc = check_device(c, "mrfv_get_stats");
  if (rc != MRFV_OK) return rc;
  memset(o, 0, sizeof(*o));
  std::vector<int32_t> loff(LK_NUM * (MAXL + 2));
  cudaMemcpy(loff.data(), c->g.loff, loff.size() * 4, cudaMemcpyDeviceToHost);
  double d[2];
  long long cnt[2];
  cudaMemcpy(d, c->dsc, 16, cudaMemcpyDeviceToHost);
  cudaMemcpy(cnt, c->counter, 16, cudaMemcpyDeviceToHost);
  o->levels = c->g.L + 1;
  for (int l = 0; l <= c->g.L; l++) {
    o->blocks[l] = loff[LK_EXIST * (MAXL + 2) + l + 1] - loff[LK_EXIST * (MAXL + 2) + l];
    o->leaves[l] = loff[LK_LEAF * (MAXL + 2) + l + 1] - loff[LK_LEAF * (MAXL + 2) + l];
    o->total_blocks += o->blocks[l];
    o->total_leaves += o->leaves[l];
  }
  o->leaf_cells = o->total_leaves * block_cells(c->g.dim);
  o->pool_capacity = c->g.cap;
  o->last_dt = d[0];
  o->t = d[1];
  o->cell_updates = cnt[0];
  o->steps = cnt[1];
  return check_launch(c, "mrfv_get_stats");
}

int mrfv_download_level(mrfv_ctx *c, int level, double *host, int64_t n, uint8_t *exist) {
  if (!c || level < 0 || level > c->g.L || !host) return fail(c, MRFV_ERR_ARG, "download: arguments");
  long long nc = level_cells(c->g, level);
  if (n != nc * c->g.nv) return fail(c, MRFV_ERR_ARG, "download: n must be nv * cells(level)");
  double *buf = nullptr;
  if (cudaMalloc(&buf, n * 8) != cudaSuccess) return fail(c, MRFV_ERR_CUDA, "download: staging allocation");
  dispatch(c, [&](auto &s) { launch_gather(c->g, level, s.U(), buf, c->st); });
  int rc = check_launch(c, "mrfv_download_level");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_download_level");
  if (rc == MRFV_OK) cudaMemcpy(host, buf, n * 8, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (rc == MRFV_OK && exist) rc = mrfv_get_tree(c, level, exist, c->g.mapoff[level + 1] - c->g.mapoff[level]);
  return rc;
}

int mrfv_download_var(mrfv_ctx *c, int level, int var, int coarsen, double *host, int64_t n) {
  if (!c || level < 0 || level > c->g.L || !host || var < 0 || var >= c->g.nv)
    return fail(c, MRFV_ERR_ARG, "download_var: arguments");
  if (coarsen != 1 && coarsen != 2 && coarsen != 4 && coarsen != 8)
    return fail(c, MRFV_ERR_ARG, "download_var: coarsen is 1, 2, 4 or 8");
  long long nc = level_cells(c->g, level);
  long long per = c->g.dim == 3 ? (long long)coarsen * coarsen * coarsen : (long long)coarsen * coarsen;
  if (n != nc / per) return fail(c, MRFV_ERR_ARG, "download_var: n must be cells(level) / coarsen^d");
  double *buf = nullptr;
  if (cudaMalloc(&buf, n * 8) != cudaSuccess) return fail(c, MRFV_ERR_CUDA, "download_var: staging allocation");
  dispatch(c, [&](auto &s) { launch_gather_var(c->g, level, var, coarsen, s.U(), buf, c->st); });
  int rc = check_launch(c, "mrfv_download_var");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_download_var");
  if (rc == MRFV_OK) cudaMemcpy(host, buf, n * 8, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  return rc;
}

int mrfv_upload_level(mrfv_ctx *c, int level, const double *host, int64_t n) {
  if (!c || level < 0 || level > c->g.L || !host) return fail(c, MRFV_ERR_ARG, "upload: arguments");
  long long nc = level_cells(c->g, level);
  if (n != nc * c->g.nv) return fail(c, MRFV_ERR_ARG, "upload: n must be nv * cells(level)");
  double *buf = nullptr;
  if (cudaMalloc(&buf, n * 8) != cudaSuccess) return fail(c, MRFV_ERR_CUDA, "upload: staging allocation");
  cudaMemcpy(buf, host, n * 8, cudaMemcpyHostToDevice);
  dispatch(c, [&](auto &s) { launch_scatter(c->g, level, buf, s.U(), c->st); });
  int rc = check_launch(c, "mrfv_upload_level");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_upload_level");
  cudaFree(buf);
  return rc;
}

int mrfv_project_finest(mrfv_ctx *c, double *host, int64_t n) {
  if (!c || !host) return fail(c, MRFV_ERR_ARG, "project_finest: arguments");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "project_finest before init");
  const int L = c->g.L;
  if (n != level_cells(c->g, L) * c->g.nv) return fail(c, MRFV_ERR_ARG, "project_finest: n = nv * cells(finest)");
  double *bufs[2] = {nullptr, nullptr};
  size_t big = (size_t)n * 8;
  if (cudaMalloc(&bufs[0], big) != cudaSuccess || cudaMalloc(&bufs[1], big) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(bufs[0]);
    return fail(c, MRFV_ERR_CUDA, "project_finest: staging allocation");
  }
  for (int l = 0; l <= L; l++) {
    double *out = bufs[l & 1], *coarse = l > 0 ? bufs[(l - 1) & 1] : nullptr;
    dispatch(c, [&](auto &s) { launch_project_level(c->g, l, s.U(), coarse, out, c->st); });
  }
  int rc = check_launch(c, "mrfv_project_finest");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_project_finest");
  if (rc == MRFV_OK) cudaMemcpy(host, bufs[L & 1], big, cudaMemcpyDeviceToHost);
  cudaFree(bufs[0]);
  cudaFree(bufs[1]);
  return rc;
}

int mrfv_get_tree(mrfv_ctx *c, int level, uint8_t *exist, int64_t n) {
  if (!c || level < 0 || level > c->g.L || !exist) return fail(c, MRFV_ERR_ARG, "get_tree: arguments");
  long long nb = c->g.mapoff[level + 1] - c->g.mapoff[level];
  if (n != nb) return fail(c, MRFV_ERR_ARG, "get_tree: n must be the number of blocks of the level");
  int rc = check_device(c, "mrfv_get_tree");
  if (rc != MRFV_OK) return rc;
  std::vector<int32_t> h(nb);
  cudaMemcpy(h.data(), c->g.idx + c->g.mapoff[level], nb * 4, cudaMemcpyDeviceToHost);
  for (long long i = 0; i < nb; i++) exist[i] = h[i] >= 0;
  return check_launch(c, "mrfv_get_tree");
}

int mrfv_set_tree(mrfv_ctx *c, const uint8_t *ex, int64_t n) {
  if (!c || !ex || n != c->maptotal) return fail(c, MRFV_ERR_ARG, "set_tree: n must be the total number of block positions");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "set_tree before init");
  if (!valid_tree(c, ex)) return fail(c, MRFV_ERR_ARG, "set_tree: tree is not complete, nested and graded");
  drop_graphs(c);
  c->snap_valid = false;
  cudaMemcpyAsync(c->need, ex, n, cudaMemcpyHostToDevice, c->st);
  apply_need(c, true);
  int rc = check_launch(c, "mrfv_set_tree");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_set_tree");
  if (rc == MRFV_OK) snapshot_exact(c);
  return rc;
}

int mrfv_get_flags(mrfv_ctx *c, int level, uint8_t *flags, double *maxdet, int64_t n) {
  if (!c || level < 0 || level > c->g.L || !flags) return fail(c, MRFV_ERR_ARG, "get_flags: arguments");
  long long nb = c->g.mapoff[level + 1] - c->g.mapoff[level];
  if (n != nb) return fail(c, MRFV_ERR_ARG, "get_flags: n must be the number of blocks of the level");
  int rc = check_device(c, "mrfv_get_flags");
  if (rc != MRFV_OK) return rc;
  cudaMemcpy(flags, c->sig + c->g.mapoff[level], nb, cudaMemcpyDeviceToHost);
  if (maxdet) cudaMemcpy(maxdet, c->maxdet + c->g.mapoff[level], nb * 8, cudaMemcpyDeviceToHost);
  return check_launch(c, "mrfv_get_flags");
}

int mrfv_synchronize(mrfv_ctx *c) {
  if (!c) return MRFV_ERR_ARG;
  return check_device(c, "mrfv_synchronize");
}

int mrfv_wait_selftest(mrfv_ctx *c, int64_t iterations, int complete) {
  if (!c || iterations < 1 || iterations > (1 << 24) || (complete != 0 && complete != 1))
    return fail(c, MRFV_ERR_ARG, "wait_selftest: arguments");
  int rc = check_device(c, "wait_selftest: before");  // earlier errors are not this test's
  if (rc != MRFV_OK) return rc;
  launch_wait_selftest(c->g.err, (unsigned)iterations, complete, c->st);
  rc = check_launch(c, "mrfv_wait_selftest");
  if (rc != MRFV_OK) return rc;
  return check_device(c, "mrfv_wait_selftest");
}

int mrfv_proposer_set_weights(mrfv_ctx *c, const float *w, int64_t n) {
  if (!c || !w || n != MRFV_PROPOSER_NWEIGHTS) return fail(c, MRFV_ERR_ARG, "proposer_set_weights: n");
  const size_t NW = MRFV_PROPOSER_NWEIGHTS;
  cudaMemcpyAsync(c->pblob, w, NW * 4, cudaMemcpyHostToDevice, c->st);
  cudaMemsetAsync(c->pm1, 0, 2 * NW * 4, c->st);
  launch_pack_weights(c->pblob, c->pw1, c->pb1, c->pw2, c->pb2, c->pw3, c->pb3, c->st);
  int rc = check_launch(c, "mrfv_proposer_set_weights");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_proposer_set_weights");
  if (rc == MRFV_OK) {
    c->has_weights = true;
    c->adam_t = 0;
    drop_graphs(c);  // a captured step graph does not contain the proposer path yet
  }
  return rc;
}

int mrfv_proposer_get_weights(mrfv_ctx *c, float *w, int64_t n) {
  if (!c || !w || n != MRFV_PROPOSER_NWEIGHTS) return fail(c, MRFV_ERR_ARG, "proposer_get_weights: n");
  int rc = check_device(c, "mrfv_proposer_get_weights");
  if (rc == MRFV_OK) cudaMemcpy(w, c->pblob, n * 4, cudaMemcpyDeviceToHost);
  return rc;
}

int mrfv_proposer_features(mrfv_ctx *c, float *feat, int64_t n) {
  if (!c || !feat || n != 3 * c->maptotal) return fail(c, MRFV_ERR_ARG, "proposer_features: n = 3 * positions");
  if (!c->initialized) return fail(c, MRFV_ERR_STATE, "proposer_features before init");
  dispatch(c, [&](auto &s) { s.prop_features(); });
  int rc = check_launch(c, "mrfv_proposer_features");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_proposer_features");
  if (rc == MRFV_OK) cudaMemcpy(feat, c->pfeat, n * 4, cudaMemcpyDeviceToHost);
  return rc;
}

int mrfv_proposer_infer(mrfv_ctx *c, float *logits, int64_t n) {
  if (!c || !logits || n != c->maptotal) return fail(c, MRFV_ERR_ARG, "proposer_infer: n = positions");
  if (!c->initialized || !c->has_weights) return fail(c, MRFV_ERR_STATE, "proposer_infer before init / weights");
  dispatch(c, [&](auto &s) { s.prop_features(); });
  prop_infer(c, false);
  int rc = check_launch(c, "mrfv_proposer_infer");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_proposer_infer");
  if (rc == MRFV_OK) cudaMemcpy(logits, c->plogit, n * 4, cudaMemcpyDeviceToHost);
  return rc;
}

int mrfv_proposer_train(mrfv_ctx *c, const float *feat, const uint8_t *target, int nsnap, int steps, float lr,
                        double *loss) {
  if (!c || !feat || !target || nsnap < 1 || steps < 0 || !(lr > 0.f))
    return fail(c, MRFV_ERR_ARG, "proposer_train: arguments");
  if (!c->initialized || !c->has_weights) return fail(c, MRFV_ERR_STATE, "proposer_train before init / weights");
  long long n = c->maptotal;
  float *df = nullptr;
  uint8_t *dt = nullptr;
  if (cudaMalloc(&df, (size_t)nsnap * 3 * n * 4) != cudaSuccess || cudaMalloc(&dt, (size_t)nsnap * n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(df);
    return fail(c, MRFV_ERR_CUDA, "proposer_train: staging allocation");
  }
  cudaMemcpy(df, feat, (size_t)nsnap * 3 * n * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dt, target, (size_t)nsnap * n, cudaMemcpyHostToDevice);
  double last = 0.0;
  int rc = MRFV_OK;
  for (int k = 0; k < steps && rc == MRFV_OK; k++) {
    cudaMemsetAsync(c->ploss, 0, 8, c->st);
    launch_prop_train_step(c->g, df, dt, nsnap, c->pblob, c->pgrad, c->pm1, c->pm2, ++c->adam_t, lr, c->pwork,
                           c->ploss, 1, c->pa0, c->pa1, c->pa2, c->pw1, c->pb1, c->pw2, c->pb2, c->pw3, c->pb3,
                           c->pw3t, c->pw2t, c->nsm, c->st);
    rc = check_launch(c, "mrfv_proposer_train");
    if (rc == MRFV_OK && k == steps - 1) {
      rc = check_device(c, "mrfv_proposer_train");
      cudaMemcpy(&last, c->ploss, 8, cudaMemcpyDeviceToHost);
    }
  }
  launch_pack_weights(c->pblob, c->pw1, c->pb1, c->pw2, c->pb2, c->pw3, c->pb3, c->st);
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_proposer_train");
  cudaFree(df);
  cudaFree(dt);
  if (loss) *loss = last;
  return rc;
}

int mrfv_proposer_grad(mrfv_ctx *c, const float *feat, const uint8_t *target, int nsnap, float *grad, int64_t n,
                       double *loss) {
  if (!c || !feat || !target || !grad || nsnap < 1 || n != MRFV_PROPOSER_NWEIGHTS)
    return fail(c, MRFV_ERR_ARG, "proposer_grad: arguments");
  if (!c->initialized || !c->has_weights) return fail(c, MRFV_ERR_STATE, "proposer_grad before init / weights");
  long long np = c->maptotal;
  float *df = nullptr;
  uint8_t *dt = nullptr;
  if (cudaMalloc(&df, (size_t)nsnap * 3 * np * 4) != cudaSuccess || cudaMalloc(&dt, (size_t)nsnap * np) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(df);
    return fail(c, MRFV_ERR_CUDA, "proposer_grad: staging allocation");
  }
  cudaMemcpy(df, feat, (size_t)nsnap * 3 * np * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dt, target, (size_t)nsnap * np, cudaMemcpyHostToDevice);
  cudaMemsetAsync(c->ploss, 0, 8, c->st);
  launch_prop_train_step(c->g, df, dt, nsnap, c->pblob, c->pgrad, c->pm1, c->pm2, c->adam_t, 0.f, c->pwork, c->ploss,
                         0, c->pa0, c->pa1, c->pa2, c->pw1, c->pb1, c->pw2, c->pb2, c->pw3, c->pb3, c->pw3t, c->pw2t,
                         c->nsm, c->st);
  int rc = check_launch(c, "mrfv_proposer_grad");
  if (rc == MRFV_OK) rc = check_device(c, "mrfv_proposer_grad");
  if (rc == MRFV_OK) {
    cudaMemcpy(grad, c->pgrad, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (loss) cudaMemcpy(loss, c->ploss, 8, cudaMemcpyDeviceToHost);
  }
  cudaFree(df);
  cudaFree(dt);
  return rc;
}

int mrfv_proposer_activations(mrfv_ctx *c, float *h1, float *h2, int64_t n) {
  if (!c || !h1 || !h2 || n != 16 * c->maptotal) return fail(c, MRFV_ERR_ARG, "proposer_activations: n = 16 * positions");
  if (!c->initialized || !c->has_weights) return fail(c, MRFV_ERR_STATE, "proposer_activations before init / weights");
  int rc = check_device(c, "mrfv_proposer_activations");
  if (rc != MRFV_OK) return rc;
  std::vector<uint16_t> raw((size_t)n);
  for (int k = 0; k < 2 && rc == MRFV_OK; k++) {
    if (cudaMemcpy(raw.data(), k == 0 ? (void *)c->pa1 : (void *)c->pa2, (size_t)n * 2, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      rc = check_device(c, "mrfv_proposer_activations");
    float *out = k == 0 ? h1 : h2;
    for (int64_t i = 0; i < n && rc == MRFV_OK; i++) {
      uint32_t b = (uint32_t)raw[(size_t)i] << 16;  // bfloat16 = the high half of a float
      memcpy(out + i, &b, 4);
    }
  }
  return rc;
}

int mrfv_set_launch_shape(mrfv_ctx *c, int grid_ctas_per_sm, int block_ctas_per_sm, int fv_ctas_per_sm,
                          int stage_kernel) {
  if (!c) return MRFV_ERR_ARG;
  if (stage_kernel < 0 || stage_kernel > 5) return fail(c, MRFV_ERR_ARG, "set_launch_shape: stage_kernel is 0..5");
  if (stage_kernel == 5 && !c->fvt.ok)
    return fail(c, MRFV_ERR_ARG, "set_launch_shape: stage kernel 5 (TMA-staged) needs 2D single-precision state");
  if (grid_ctas_per_sm < 0 || grid_ctas_per_sm > 32 || block_ctas_per_sm < 0 || block_ctas_per_sm > 32 ||
      fv_ctas_per_sm < 0 || fv_ctas_per_sm > 32)
    return fail(c, MRFV_ERR_ARG, "set_launch_shape: CTAs per SM outside 0..32");
  int rc = check_device(c, "mrfv_set_launch_shape");
  if (rc != MRFV_OK) return rc;
  c->grid = c->nsm * (grid_ctas_per_sm ? grid_ctas_per_sm : kGridCtasPerSm);
  c->bgrid = c->nsm * (block_ctas_per_sm ? block_ctas_per_sm : kBlockCtasPerSm);
  for (int sp = 0; sp < 2; sp++) c->fvgrid[sp] = c->nsm * (fv_ctas_per_sm ? fv_ctas_per_sm : c->fv_occupancy[sp]);
  for (int h = 0; h < 2; h++) c->fvsgrid[h] = c->nsm * (fv_ctas_per_sm ? fv_ctas_per_sm : c->fvs_occupancy[h]);
  c->stage_kernel = stage_kernel;
  c->fvpgrid = c->nsm * (fv_ctas_per_sm ? fv_ctas_per_sm : c->fvp_occupancy);
  if (c->fvt.ok) {
    const int n = fv_ctas_per_sm && fv_ctas_per_sm < c->fvt.ctas_per_sm ? fv_ctas_per_sm : c->fvt.ctas_per_sm;
    c->fvtgrid = c->nsm * n;
  }
  drop_graphs(c);
  return MRFV_OK;
}

int mrfv_profile_enable(mrfv_ctx *c, int enable) {
  if (!c) return MRFV_ERR_ARG;
  int rc = check_device(c, "mrfv_profile_enable");
  if (rc != MRFV_OK) return rc;
  c->prof = enable != 0;
  c->ev_used = 0;
  c->pev_used = 0;
  c->rev_used = 0;
  c->nlaunch = 0;
  cudaMemsetAsync(c->rcount, 0, 8, c->st);
  cudaMemsetAsync(c->ptcount, 0, 3 * 8, c->st);
  c->pdense = 0;
  c->fv_kinds = 0;
  cudaMemsetAsync(c->dbytes, 0, 8, c->st);
  return check_launch(c, "mrfv_profile_enable");
}

int mrfv_profile_read(mrfv_ctx *c, mrfv_profile *o) {
  if (!c || !o) return MRFV_ERR_ARG;
  int rc = check_device(c, "mrfv_profile_read");
  if (rc != MRFV_OK) return rc;
  memset(o, 0, sizeof(*o));
  o->launches = c->nlaunch;
  o->fv_launches = (int64_t)(c->ev_used / 2);
  double ms = 0.0;
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->evs[k], c->evs[k + 1]) == cudaSuccess) ms += t;
  }
  o->fv_ms = ms;
  unsigned long long b = 0;
  cudaMemcpy(&b, c->dbytes, 8, cudaMemcpyDeviceToHost);
  o->fv_bytes = (double)b;
  double pms = 0.0;
  for (size_t k = 0; k + 1 < c->pev_used; k += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->pevs[k], c->pevs[k + 1]) == cudaSuccess) pms += t;
  }
  o->prop_launches = (int64_t)(3 * (c->pev_used / 2));
  o->prop_ms = pms;
  // algorithmic flops of the positions the convolutions covered: every position for a
  // dense inference, the flagged tiles' positions for a restricted one
  unsigned long long tc[3] = {0, 0, 0};
  cudaMemcpy(tc, c->ptcount, sizeof(tc), cudaMemcpyDeviceToHost);
  o->prop_flops = 2.0 * ((double)c->pdense * (double)c->maptotal * (16.0 * 81 + 16.0 * 432 + 432.0) +
                         128.0 * ((double)tc[0] * 16.0 * 81 + (double)tc[1] * 16.0 * 432 + (double)tc[2] * 432.0));
  double rms = 0.0;
  for (size_t k = 0; k + 1 < c->rev_used; k += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->revs[k], c->revs[k + 1]) == cudaSuccess) rms += t;
  }
  o->rich_launches = (int64_t)(c->rev_used / 2);
  o->rich_ms = rms;
  unsigned long long rb = 0;
  cudaMemcpy(&rb, c->rcount, 8, cudaMemcpyDeviceToHost);
  o->rich_blocks = (double)rb;
  o->fv_kernels = c->fv_kinds;
  o->graph_fv_kernels = (c->gexec[0] ? c->gkinds[0] : 0) | (c->gexec[1] ? c->gkinds[1] : 0);
  return check_launch(c, "mrfv_profile_read");
}

}  // extern "C"
