// Internal definitions shared by the host orchestration and the kernels.
//
// Device data layout (all in one arena, see api.cu):
//   state buffers  U, Us, U0     : T[nv][cap][8^d]      (SoA per conserved variable; a block's
//                                  8^d cells are contiguous, 256 B per variable in 2D fp32)
//   ghost strips   G             : T[nv][cap][2d][2][8^(d-1)]  (two cell layers per face; only
//                                  faces whose same-level neighbour is absent are ever written)
//   flux registers FR            : T[nv][cap][2d][8^(d-1)] (dt*F on the block's boundary faces)
//   dense maps     idx           : int32 per block position of every level (slot or -1),
//                                  levels concatenated at mapoff[l], [bk][bj][bi]
//   per slot       slot_level, slot_coord[3], nbr[6] (slot | NBR_MISSING | NBR_WALL), cmask
//   work lists     lists[kind]   : slots in level-major Morton order, level ranges in loff
#pragma once
#include <stdint.h>

namespace mrfv {

constexpr int BS = 8;        // cells per block edge
constexpr int MAXL = 12;     // maximum number of levels
// block positions the single-CTA projection of the coarse levels holds in shared
// memory (levels 0..lhi together), 2D and 3D
constexpr int kRestrictTailBlocks2D = 22;
constexpr int kRestrictTailBlocks3D = 2;
constexpr int NBR_MISSING = -1;  // same-level neighbour absent: read the ghost strip
constexpr int NBR_WALL = -2;     // outside a transmissive domain: zero-gradient copy

enum ListKind { LK_EXIST = 0, LK_LEAF = 1, LK_INTERNAL = 2, LK_GHOST = 3, LK_REFLUX = 4, LK_NUM = 5 };
enum ErrBits { EB_TREE = 1, EB_NONPHYS = 2, EB_POOL = 4, EB_TIMEOUT = 8 };

// Geometry and tree pointers, passed to kernels by value.
struct Geo {
  int dim, nv, L, bc;
  int nb[MAXL][3];          // blocks per dimension (1 in unused ones)
  int mbits[MAXL];          // Morton bits per dimension on level l
  double dx[MAXL][3];
  double lo[3];
  double gamma;
  long long cap;            // pool capacity in blocks
  long long mapoff[MAXL + 1];   // offsets of the dense maps
  long long moff[MAXL + 1];     // offsets of the (padded) Morton enumeration
  int32_t *idx;
  int32_t *slot_level;
  int32_t *slot_coord;      // [slot*3 + d]
  int32_t *nbr;             // [slot*6 + face], face = 2*dir + side
  uint8_t *cmask;           // [slot]: bit f = neighbour across face f exists and is refined
  int32_t *kids;            // [slot*8 + q]: slots of a refined block's children, q = x + 2y + 4z
                            // (child offsets); written with the lists, read only for refined blocks
  int32_t *loff;            // [kind*(MAXL+2) + l] start of level l in list kind; [L+1] = end
  int32_t *lists;           // [kind*cap + i]
  int *err;                 // error bits (ErrBits)
};

template <typename T>
struct FVArgs {
  const T *Uin;   // state the fluxes are computed from
  const T *U0;    // state the stage update starts from
  T *Uout;        // stage result (may alias U0: each block reads only its own U0 cells)
  const T *G;     // ghost strips
  T *FR;          // flux registers (dt_l * F on block faces)
  int kind;       // work list
  int l0, l1;     // level range of the list
  double coef;    // stage coefficient: 1/2 (stage 1) or 1 (stage 2)
  int stage;      // 0 (coef 1/2) or 1 (coef 1): row of the step table
  const double *lev;  // per-level step table: [(stage*MAXL + l)*4 + n] = (coef dt_l)/dx_{l,n}, [.. + 3] = dt_l
  const float *levf;  // the same table rounded to single precision (read by the single-precision kernel)
  int record;     // 0: no registers; 1: store dt_l F on marked faces; 2: add on fine-role faces
  int words;      // algorithmic state words moved per cell (for the byte counter)
  unsigned long long *bytes;  // optional: += algorithmic bytes of this launch
  // coarse source of halo cells predicted inside the MUSCL-Hancock kernel: level
  // l-1 of C, or C0 + theta (C - C0) with level-dependent steps (C0 null: C)
  const T *C;
  const T *C0;
  double theta;
};

// training scratch of the learned proposer, in floats per block position: logits z
// and dL/dz (FP32), and the BF16 rows of dL/dz (8 channels), dL/dh2 and dL/dh1 (16
// each), i.e. 2 + 4 + 8 + 8 floats, and two for the 16-byte alignment of the rows
constexpr long long kPropWorkPerPos = 2 + 4 + 8 + 8 + 2;

// rows of the per-level step table (see FVArgs::lev): stage 0 has coef 1/2, stage 1 coef 1
__host__ __device__ inline int lev_index(int stage, int l, int k) { return (stage * MAXL + l) * 4 + k; }

struct ICParams {
  int kind;
  double p[16];
};

__host__ __device__ inline int block_cells(int dim) { return dim == 2 ? 64 : 512; }
__host__ __device__ inline int face_cells(int dim) { return dim == 2 ? 8 : 64; }

}  // namespace mrfv
