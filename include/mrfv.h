/*
 * mrfv.h -- C interface of the GB300 (sm_103a) adaptive multiresolution
 * finite-volume solver for the compressible Euler equations.
 *
 * Method (arXiv:1603.05211): cell averages Q = (rho, rho v, rho e) of the Euler
 * equations (Section 2, Eqs. 2.1-2.3) advanced by dQ/dt = -F(Q) with MUSCL
 * reconstruction (van Albada limiter), the AUSM+ flux and the explicit midpoint
 * RK2 rule (Section 2), on the leaves of a graded tree of 8^d-cell blocks that a
 * multiresolution analysis (projection, third-order prediction, details,
 * eps-thresholding; Section 2.1) or a scaled-gradient criterion (Section 2.2)
 * adapts every step; coarse-fine faces are made conservative by flux
 * correction (Section 2.1 virtual leaves, Section 2.2 / Fig. 2), and levels can
 * advance with their own step 2^(L-l) dt (Section 2.1 MRLT, Fig. 2).
 *
 * Conventions for every entry point:
 *   - return value: MRFV_OK (0) or a negative MRFV_ERR_* code; the text of the
 *     last error of a context is given by mrfv_last_error();
 *   - host pointers are owned by the caller and only read or written during the
 *     call; the library keeps no reference to them;
 *   - all device state is owned by the context (allocated by the library with
 *     cudaMalloc, or placed in a caller-provided device arena that must outlive
 *     the context);
 *   - work is issued on the configured CUDA stream.  Entry points that return
 *     host data synchronise that stream; the others only enqueue work;
 *   - after MRFV_ERR_CUDA, MRFV_ERR_POOL_FULL or MRFV_ERR_TIMEOUT the context's
 *     state is undefined and it must be destroyed;
 *   - there is no CPU fallback: without a usable GPU mrfv_create fails.
 *
 * Dense level layout used by download/upload: level l has N_l = base_blocks*8*2^l
 * cells per dimension; a level array is [v][k][j][i] (i fastest), nv = dim+2
 * conserved variables (rho, rho v_1..rho v_d, rho e), always in double.
 * Block maps are [bk][bj][bi] bytes, base_blocks*2^l blocks per dimension.
 */
#ifndef MRFV_H
#define MRFV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRFV_OK 0
#define MRFV_ERR_ARG (-1)         /* invalid argument or configuration */
#define MRFV_ERR_POOL_FULL (-2)   /* block pool capacity exceeded */
#define MRFV_ERR_NONPHYSICAL (-3) /* rho <= 0, p <= 0 or NaN met by the time-step reduction */
#define MRFV_ERR_TIMEOUT (-4)     /* a bounded device wait expired */
#define MRFV_ERR_CUDA (-5)        /* CUDA runtime error */
#define MRFV_ERR_STATE (-6)       /* call out of order (e.g. step before init) */
#define MRFV_ERR_TREE (-7)        /* a kernel met a tree that is not graded */

enum { MRFV_FP64 = 0, MRFV_FP32 = 1 };
enum { MRFV_BC_TRANSMISSIVE = 0, MRFV_BC_PERIODIC = 1 };
enum { MRFV_CRIT_MR = 0, MRFV_CRIT_GRAD = 1 };
/* initial data (parameter lists as in the Python module mrfv_inputs) */
enum {
  MRFV_IC_QUADRANTS = 0,         /* 16: (rho, v1, v2, p) of quadrants I, II, III, IV (Table 1 order) */
  MRFV_IC_ELLIPSOID = 1,         /* 10: cx, cy, cz, a, b, c, rho_in, p_in, rho_out, p_out */
  MRFV_IC_SHOCKTUBE = 2,         /* 8: axis, x0, rho_L, u_L, p_L, rho_R, u_R, p_R */
  MRFV_IC_UNIFORM = 3,           /* 5: rho, v1, v2, v3, p */
  MRFV_IC_WAVE = 4,              /* 5: amp, v1, v2, v3, p; rho = 1 + amp sin(2 pi sum x) */
  MRFV_IC_ROTATED_ELLIPSOID = 5  /* 10: a, b, c, r_c, theta, phi, rho_in, rhoe_in, rho_out, rhoe_out */
};

/* Finite-volume schemes of Section 2.  MUSCL_RK2: MUSCL reconstruction of the
   primitive variables with the van Albada limiter, AUSM+ flux, explicit
   midpoint rule (two stages per step; the scheme of the paper's MR method).
   HANCOCK: unsplit MUSCL-Hancock, Minmod limiter on rho, v, p, AUSMDV flux (one
   stage per step: face states advanced half a step with the exact flux of every
   direction; the scheme of the paper's AMR method). */
enum { MRFV_SCHEME_MUSCL_RK2 = 0, MRFV_SCHEME_HANCOCK = 1 };

/* Clustering of the gradient flags into the blocks to refine (Section 2.2).
   ROWS: runs of at most 8 blocks along the first direction whose flagged
   fraction stays >= eta_tol.  BR: Berger-Rigoutsos boxes (AMROC's clustering):
   a box shrunk to its flags is accepted at efficiency >= eta_tol with sides of
   at most 8 blocks, else cut at a hole of the flag signatures, else at their
   strongest inflection, else bisected across its longest side. */
enum { MRFV_CLUSTER_ROWS = 0, MRFV_CLUSTER_BR = 1 };

#define MRFV_MAX_LEVELS 12

/* Solver configuration; plain data, copied by mrfv_create. */
typedef struct {
  int dim;              /* 2 or 3 */
  int precision;        /* MRFV_FP64 (parity mode) or MRFV_FP32 (state and flux in single precision) */
  int levels;           /* number of levels L+1 (1..MRFV_MAX_LEVELS); level l has base_blocks*2^l blocks per dim */
  int base_blocks[3];   /* blocks of 8 cells per dimension on level 0 (unused dimensions: 1) */
  double lo[3], hi[3];  /* domain box */
  int bc;               /* MRFV_BC_TRANSMISSIVE (outflow, Section 4) or MRFV_BC_PERIODIC */
  double gamma;         /* ratio of specific heats (1.4, Section 2) */
  double cfl;           /* CFL number of the time-step rule */
  double t_end;         /* > 0: steps with a CFL-computed dt are clipped to end at t_end */
  int adapt;            /* 1: analyse and adapt the tree after every (coarse) step */
  int criterion;        /* MRFV_CRIT_MR (details vs eps) or MRFV_CRIT_GRAD (density gradient vs eps_w,
                           and pressure gradient vs eps_p when eps_p > 0) */
  double eps;           /* MR threshold, the same on every level (Section 2.1) */
  double eps_w;         /* gradient threshold (Section 2.2) */
  double eta_tol;       /* clustering efficiency (Section 2.2) */
  int lts;              /* 1: level-dependent time steps 2^(L-l) dt (Section 2.1 MRLT, Fig. 2) */
  int64_t pool_blocks;  /* block pool capacity; 0 = every block of every level (never full) */
  void *stream;         /* cudaStream_t to issue work on; NULL = the legacy default stream */
  void *device_arena;   /* optional device memory for all state (e.g. from a PyTorch tensor) */
  size_t arena_bytes;   /* its size; must be >= mrfv_arena_bytes(config) */
  int use_graph;        /* 1 (default): the first mrfv_step captures the step's launch sequence into a
                           CUDA graph (on a private stream) and every step replays it on `stream` */
  int proposer;         /* 1: MR adaptation takes the learned proposer's blocks instead of the safety
                           zone, once weights are set (mrfv_proposer_set_weights) */
  int scheme;           /* MRFV_SCHEME_MUSCL_RK2 (default) or MRFV_SCHEME_HANCOCK (Section 2) */
  int clustering;       /* gradient criterion: MRFV_CLUSTER_ROWS (default) or MRFV_CLUSTER_BR */
  double eps_p;         /* gradient criterion: > 0 also flags |p(Q_{i+alpha}) - p(Q_i)| > eps_p, with p from
                           the cell's (predicted, where its block is absent) conserved state; 0 (default):
                           density only.  The 3D case of Section 4.2 tests density and pressure. */
  int lts_remesh;       /* with adapt and lts: 1 (default) regenerates the levels above l at the second
                           sub-step of every level l >= 1 inside the level recursion (Remesh(l) of Fig. 2,
                           with the configured criterion on data at one time; the MR criterion uses its
                           safety zone there, not the proposer); 0 adapts once per coarse step */
  double eps_r;         /* gradient criterion: > 0 also flags by the Richardson estimate (Section 2.2: the local
                           error indicator AMROC can add; Berger-Oliger 1984, Berger-Colella 1989):
                           tau = (R H_dt(H_dt(E)) - H_2dt(R E)) / 6 on each level l < L coarsened by 2, H one
                           step of the configured scheme over the level's uniform grid (absent cells predicted),
                           R the mean of the 2^d children, dt the level's step in the last time step (zero
                           before the first step); a block is flagged when |tau| of density exceeds eps_r on
                           a coarse cell of an existing block within one fine cell of it.  0 (default): off.
                           With the MR criterion it must be 0. */
  int proposer_dense;   /* with the proposer: 0 (default) computes its convolutions only on the 128-position
                           tiles whose logits can add a block (children of existing blocks, and the one- and
                           two-position neighbourhoods the second and first layer feed them from); 1: on every
                           block position of every level (the same blocks are added) */
} mrfv_config;

typedef struct {
  int levels;
  int64_t blocks[MRFV_MAX_LEVELS];  /* existing blocks per level */
  int64_t leaves[MRFV_MAX_LEVELS];  /* leaf blocks per level */
  int64_t total_blocks, total_leaves;
  int64_t leaf_cells;               /* cells advanced per step (leaves x 8^d) */
  int64_t pool_capacity;
  double t;                         /* simulated time */
  double last_dt;                   /* last (finest-level) time step */
  int64_t steps;                    /* steps taken */
  int64_t cell_updates;             /* sum over steps of the leaf cells advanced */
} mrfv_stats;

typedef struct mrfv_ctx mrfv_ctx;

/* Fill *cfg with defaults: 2D, FP64, one level of 1x1 blocks on [0,1]^2,
   transmissive, gamma 1.4, CFL 0.5, eps 1e-3, eps_w 0.05, eta_tol 0.8,
   CUDA graph replay on. */
int mrfv_config_default(mrfv_config *cfg);

/* Device bytes the context needs for cfg (pool, maps, lists, scratch). */
size_t mrfv_arena_bytes(const mrfv_config *cfg);

/* Create a context on the current CUDA device.  Validates cfg (MRFV_ERR_ARG)
   and allocates the block pool (MRFV_ERR_CUDA when memory is short). */
int mrfv_create(const mrfv_config *cfg, mrfv_ctx **out);
int mrfv_destroy(mrfv_ctx *ctx);
/* Text of the last error of ctx (valid until the next call on ctx); for a NULL
   ctx, the last error of mrfv_create on this thread. */
const char *mrfv_last_error(const mrfv_ctx *ctx);

/* Initial data (Section 4.1 / 4.2 set-ups): every block of every level is
   created, the finest level is sampled at cell centres, coarser levels are its
   projections (Section 2.1), t = 0.  With cfg.adapt the tree is then adapted
   (analysis + thresholding), so only the blocks the threshold keeps remain. */
int mrfv_init_state(mrfv_ctx *ctx, int ic_kind, const double *params, int n_params);

/* MR analysis (Section 2.1): projection onto refined blocks, details of every
   block of level >= 1 against the third-order prediction from its parent level,
   normalised by the level-0 maxima, thresholded with eps (strict >).
   *n_significant (may be NULL) = significant blocks.  Synchronises. */
int mrfv_analyse(mrfv_ctx *ctx, double eps, int64_t *n_significant);

/* Tree update from the current flags/state with cfg.criterion: refinement by
   one level and safety zone (MR) or gradient flags + clustering (GRAD),
   gradedness closure, removal of blocks that are no longer needed, prediction
   of new blocks from their parent level, rebuild of neighbour tables and work
   lists.  use_proposer = 1 takes the learned proposer's blocks instead of the MR
   safety zone (weights must be set).  *n_blocks (may be NULL) receives the
   number of existing blocks (synchronises when non-NULL). */
int mrfv_adapt(mrfv_ctx *ctx, int use_proposer, int64_t *n_blocks);

/* CFL time step over the leaves: cfl * min over leaf cells and directions of
   dx_{l,n} / (|v_n| + c); with cfg.lts the finest step (each leaf's limit scaled
   by 2^(l-L)).  Returns MRFV_ERR_NONPHYSICAL on rho <= 0, p <= 0 or NaN. */
int mrfv_compute_dt(mrfv_ctx *ctx, double *dt_out);

/* Ghost strips of level l (Section 2.2 ghost cells; Section 2.1 virtual
   leaves): every face of a leaf block of level l whose same-level neighbour is
   absent gets its two cell layers predicted (third order) from level l-1 of the
   chosen buffer (0 = state Q^n, 1 = RK stage Q*).  Same-level neighbours and
   domain boundaries need no strip: the flux kernel reads them directly. */
int mrfv_fill_ghosts(mrfv_ctx *ctx, int level, int buffer);

/* One step.  dt > 0: that (finest-level) step; dt <= 0: the CFL step, clipped
   to cfg.t_end when set.  Global stepping: one midpoint-RK2 step of every leaf
   (stage fluxes at coarse-fine faces corrected as in Fig. 2).  cfg.lts: one
   coarse step of the level recursion of Fig. 2 (2^L finest sub-steps).  With
   cfg.adapt the tree is adapted after the step.  *dt_out (may be NULL; then
   nothing synchronises) receives the finest-level dt used. */
int mrfv_step(mrfv_ctx *ctx, double dt, double *dt_out);

/* The level recursion of Fig. 2 from level l (levels l..L advance by one step
   of level l, dt_l = 2^(L-l) dt_finest), without adaptation.  Needs cfg.lts
   (only then does the arena hold the level-step start states): MRFV_ERR_STATE
   otherwise. */
int mrfv_step_level(mrfv_ctx *ctx, int level, double dt_finest);

/* Projection (Section 2.1) of level fine_level onto the refined blocks of
   fine_level-1; fine_level <= 0 restricts every level, finest first. */
int mrfv_restrict(mrfv_ctx *ctx, int fine_level);

/* Prediction (Section 2.1, third order) of every existing block of level
   coarse_level+1 from level coarse_level, overwriting those blocks (0 <=
   coarse_level < L).  The tree's own prolongation fills only the blocks an
   adaptation creates; this call applies the operator to a whole level (tests,
   re-initialisation of a level from its parent). */
int mrfv_prolong(mrfv_ctx *ctx, int coarse_level);

/* Conserved totals: sum over leaf cells of Q_v times the cell volume, in double
   (nv values).  Synchronises. */
int mrfv_conserved_totals(mrfv_ctx *ctx, double *out, int n);

int mrfv_get_stats(mrfv_ctx *ctx, mrfv_stats *out);

/* Dense copy of level l into host[nv * cells(l)] (double; NaN in absent
   blocks); exist (may be NULL) receives the block map of level l. */
int mrfv_download_level(mrfv_ctx *ctx, int level, double *host, int64_t n, uint8_t *exist);
/* One conserved variable of a dense level, averaged over cubes of coarsen^d
   cells (coarsen 1, 2, 4 or 8; cell means, as the projection of Section 2.1);
   host[(k*n1 + j)*n0 + i] with n = cells(level) / coarsen^d; NaN where a block is
   absent.  For measuring errors against a fine reference without moving every
   variable of it (no counterpart in the paper). */
int mrfv_download_var(mrfv_ctx *ctx, int level, int var, int coarsen, double *host, int64_t n);
/* Write host[nv * cells(l)] into the existing blocks of level l. */
int mrfv_upload_level(mrfv_ctx *ctx, int level, const double *host, int64_t n);

/* Leaf representation projected to the finest level (Section 3, error
   assessment for MR): existing cells as stored, every other cell predicted
   (third order) from the level below, level by level; host[nv * cells(L)]
   (double, dense layout as above). */
int mrfv_project_finest(mrfv_ctx *ctx, double *host, int64_t n);

/* Block map of level l (1 = block exists). */
int mrfv_get_tree(mrfv_ctx *ctx, int level, uint8_t *exist, int64_t n);
/* Replace the tree: exist_all = the block maps of levels 0..L concatenated.
   The tree must hold every level-0 block, complete child sets, parents and the
   gradedness rule (MRFV_ERR_ARG otherwise).  New blocks are predicted from
   their parent level; removed blocks are dropped. */
int mrfv_set_tree(mrfv_ctx *ctx, const uint8_t *exist_all, int64_t n);

/* Last analysis of level l: flags[b] = 1 when block b was significant (MR) or
   flagged for refinement (GRAD); maxdet[b] (may be NULL) = its largest
   normalised detail (MR) or, with eps_r > 0, its largest |tau| of the Richardson
   estimate (GRAD, levels below the finest), in the state precision widened to
   double. */
int mrfv_get_flags(mrfv_ctx *ctx, int level, uint8_t *flags, double *maxdet, int64_t n);

/* Wait for all work issued on the context's stream. */
int mrfv_synchronize(mrfv_ctx *ctx);

/* Failure-path self-test of the bounded device waits (no counterpart in the
   paper).  Launches one warp that waits, with the same bounded mbarrier wait the
   tensor-core kernels use (at most `iterations` tries, 1..2^24), on a phase that
   completes only when `complete` = 1.  Returns MRFV_OK when the phase
   completed, MRFV_ERR_TIMEOUT when the bound expired; either way nothing is left
   waiting and the context stays usable.  Errors pending before the call are
   returned first. */
int mrfv_wait_selftest(mrfv_ctx *ctx, int64_t iterations, int complete);

/* Diagnostics (no counterpart in the paper, which profiled its CPU codes with
   perf, Section 4.1 Table 5): kernel launch count and CUDA-event timing of the
   finite-volume stage launches. */
typedef struct {
  int64_t launches;     /* kernels this context launched since profiling was enabled */
  int64_t fv_launches;  /* finite-volume stage launches timed */
  double fv_ms;         /* sum of their CUDA-event durations on the context stream */
  double fv_bytes;      /* algorithmic bytes of those launches: per cell, stage 1 reads
                           Q^n and writes Q* (2 nv words), stage 2 reads Q^n and Q* and
                           writes Q^{n+1} (3 nv words) */
  int64_t prop_launches; /* tensor-core convolution launches of the proposer timed (3 per inference) */
  double prop_ms;        /* their CUDA-event time */
  double prop_flops;     /* their algorithmic flops: 2 x (16*81 + 16*432 + 432) per position covered (every
                            position for mrfv_proposer_infer; in the adaptation, the positions of the tiles
                            each layer needs, unless cfg.proposer_dense) */
  int fv_kernels;        /* stage kernels those launches used (bit mask): 1 pencil, 2 staged (MR scheme),
                            4 pencil with two threads per line, 8 pencil on staged primitives,
                            16 staged MUSCL-Hancock, 32 TMA-staged */
  int graph_fv_kernels;  /* the same bit mask for the stage kernels in the step graphs captured now */
  int64_t rich_launches; /* Richardson estimates timed (the estimate and its block flags, two kernels each) */
  double rich_ms;        /* their CUDA-event time */
  double rich_blocks;    /* blocks they estimated */
} mrfv_profile;
/* enable != 0: reset the counters and bracket every finite-volume stage launch
   with CUDA events on the context stream (steps then launch eagerly instead of
   replaying the captured graph); 0: stop. */
int mrfv_profile_enable(mrfv_ctx *ctx, int enable);
/* Read the counters (synchronises the stream). */
int mrfv_profile_read(mrfv_ctx *ctx, mrfv_profile *out);

/* Launch shape (no counterpart in the paper): CTAs per SM of the persistent
   grids, for the grid-stride kernels (256-thread CTAs), the kernels that take
   one block per CTA, and the finite-volume stage kernels.  0 keeps the default
   (the stage kernels' default is their occupancy limit); each value is 0..32.
   stage_kernel picks the MR-scheme stage kernel: 0 by leaf count, 1 the pencil
   kernel (one thread per line of cells), 2 the staged kernel (one thread per
   face), 3 the pencil kernel with two threads per line, 4 the pencil kernel
   reading primitives staged in shared memory, 5 the TMA-staged kernel (2D
   single-precision state only: each block and its halo copied into shared
   memory by the tensor memory accelerator, x and y lines walked together in
   packed FP32x2 arithmetic; the automatic choice there from 65536 leaf blocks).  Out-of-range values, and 5 for
   another configuration, give MRFV_ERR_ARG.  The TMA-staged kernel holds at most
   its occupancy limit of CTAs per SM (a larger fv_ctas_per_sm is capped).  Every kernel loops over its
   device-resident work list, so any shape gives the same results; captured
   step graphs are dropped and re-captured at the next step. */
int mrfv_set_launch_shape(mrfv_ctx *ctx, int grid_ctas_per_sm, int block_ctas_per_sm, int fv_ctas_per_sm,
                          int stage_kernel);

/* Learned refinement proposer (no counterpart in the paper, which refines by
   the heuristic of Section 2.1): a 3-layer 3D convolutional net (16 channels,
   3^3 kernels, zero padding, ReLU between layers; BF16 weights and activations,
   FP32 accumulation, inference on the tensor cores) over three features of every
   block position of every level (block-mean density / s_rho, block-mean pressure
   / ((gamma-1) s_E), min(max normalised detail / eps, 8) / 8; absent blocks take
   the means of their parent's covering octant).  A position of level >= 1 with a
   positive logit and an existing parent is added to the tree; with cfg.proposer
   this replaces the safety zone of the MR rule, and the MR thresholding of the
   next analysis re-refines anything it missed.
   "positions" = sum over levels of the level's block count.
   Weight layout (FP32): W1[16][3][27], b1[16], W2[16][16][27], b2[16],
   W3[1][16][27], b3[1]; tap index (dz+1)*9 + (dy+1)*3 + (dx+1). */
#define MRFV_PROPOSER_NWEIGHTS 8673
/* Set the FP32 master weights (n = MRFV_PROPOSER_NWEIGHTS) and reset the Adam state. */
int mrfv_proposer_set_weights(mrfv_ctx *ctx, const float *w, int64_t n);
int mrfv_proposer_get_weights(mrfv_ctx *ctx, float *w, int64_t n);
/* Features of the current state and last analysis: feat[3][positions] (n = 3 * positions). */
int mrfv_proposer_features(mrfv_ctx *ctx, float *feat, int64_t n);
/* Logits of the current features (n = positions), through the tensor-core kernels. */
int mrfv_proposer_infer(mrfv_ctx *ctx, float *logits, int64_t n);
/* `steps` Adam steps (learning rate lr) on nsnap snapshots: feat[nsnap][3][positions],
   target[nsnap][positions] (1 = block needed at the next step, 0 = not, 255 =
   left out of the loss); binary cross-entropy over positions of level >= 1 with
   an existing parent (in the current tree) and a target other than 255.  With a
   full tree (cfg.adapt = 0) the 255 entries alone select the positions, so
   snapshots of different trees (255 where the snapshot's parent block was
   absent) train together.  *loss = loss of the last step. */
int mrfv_proposer_train(mrfv_ctx *ctx, const float *feat, const uint8_t *target, int nsnap, int steps, float lr,
                        double *loss);
/* The gradient the next Adam step of mrfv_proposer_train would take, without
   taking it: the same forward and backward kernels on the same snapshots
   (feat[nsnap][3][positions], target[nsnap][positions]), the loss summed over
   the snapshots and over the positions of level >= 1 with an existing parent
   (current tree), divided by nsnap * (positions of levels >= 1).  grad: host,
   n = MRFV_PROPOSER_NWEIGHTS floats in the weight layout above; *loss (host,
   optional) its loss.  Weights and Adam state are left unchanged. */
int mrfv_proposer_grad(mrfv_ctx *ctx, const float *feat, const uint8_t *target, int nsnap, float *grad, int64_t n,
                       double *loss);
/* The BF16 layer inputs of the second and third convolution of the last
   mrfv_proposer_infer (the ReLU outputs of layers 1 and 2, rounded to
   bfloat16), widened to float: h1, h2 host [positions][16] (n = 16 * positions). */
int mrfv_proposer_activations(mrfv_ctx *ctx, float *h1, float *h2, int64_t n);

/* Allocation-free CFL time step of a caller-owned dense array of cells (no
   counterpart in the paper).  Some callers cannot call cudaMalloc: work issued
   while a CUDA stream is being captured into a graph may not allocate, some host
   frameworks own all device memory through their own pool, and latency-critical
   loops cannot afford cudaMalloc's implicit device synchronisation.  This entry
   point allocates nothing; its scratch (one partial minimum per tile of
   MRFV_NOALLOC_DT_TILE_CELLS cells) is a file-scope device array of
   MRFV_NOALLOC_DT_MAX_TILES doubles (512 KiB), held by every GPU that loads the
   library until the process exits.
     state   device pointer, [v][k][j][i] with nv = dim+2 conserved variables
             (rho, rho v_1..rho v_d, rho e), float (MRFV_FP32) or double (MRFV_FP64);
     n0,n1,n2 cells per dimension (n2 = 1 in 2D); at most MRFV_NOALLOC_DT_MAX_CELLS
             cells in total, larger arrays return MRFV_ERR_ARG;
     dx      host pointer to the 3 cell widths;
     dt_out  device pointer to one double: cfl * min over cells and directions of
             dx_n / (|v_n| + c) (the rule of mrfv_compute_dt on one uniform level),
             or -1.0 when a cell has rho <= 0, p <= 0 or NaN;
     stream  cudaStream_t (NULL = legacy default stream); the call only enqueues.
   The first call on a device looks up the scratch array's device address (with
   that device current) and caches it: make that first call before any stream
   capture.  The cached address does not survive cudaDeviceReset or any other
   teardown of the device's primary context: do not call this entry point after
   one in the same process.  Every call shares the scratch array, which keeps the last call's
   contents; calls that overlap on the GPU (on different streams, or from several
   threads) race on it and must be serialised by the caller. */
#define MRFV_NOALLOC_DT_TILE_CELLS 4096
#define MRFV_NOALLOC_DT_MAX_TILES 65536
#define MRFV_NOALLOC_DT_MAX_CELLS ((int64_t)MRFV_NOALLOC_DT_TILE_CELLS * MRFV_NOALLOC_DT_MAX_TILES)
int mrfv_cfl_dt_noalloc(int dim, int precision, const void *state, int64_t n0, int64_t n1, int64_t n2,
                        const double *dx, double gamma, double cfl, double *dt_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MRFV_H */
