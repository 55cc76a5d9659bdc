// Internal types of libbats shared by the host code (bats_host.cu) and the
// kernels (bats_stage.cu).  Device layout of a state buffer: block-major
// [n_blocks_total][8 variables][512 cells] (k, j, i; i fastest), so that one
// block's state is one contiguous 32 KB (FP64) or 16 KB (FP32) run that a
// single bulk copy per variable stages into shared memory.
#pragma once
#include <cstdint>
#include <cuda.h>  // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

namespace batsk {

constexpr int NV = 8;          // conserved variables
constexpr int NC = 8;          // cells per block per axis
constexpr int NCELL = 512;     // cells per block
constexpr int NFACE = 576;     // faces per block per direction (9 x 8 x 8)
constexpr int NGHOST = 768;    // face-slab ghost cells (6 x 2 x 64)
constexpr int NTILE = 1280;    // interior + face-slab ghosts
constexpr int MAXLEV = 14;
constexpr int FACE_THREADS = 384;   // face phase: two threads per grid line, three directions
// stage CTA threads per form: 384 both (2 CTAs per SM at 80 registers in the
// mixed form, 1 at 168 in FP64).  512 threads (one per cell in the cell phase)
// measured slower in the mixed form: 64 registers spill in the face phase.
constexpr int STAGE_THREADS_MIXED = 384, STAGE_THREADS_FP64 = 384;

// Mixed-form tile of the plain stage kernel (FP32 primitives, floats):
//  * interior [8 v][8 k][8 j][8 i] in the 32-byte TMA swizzle: the two
//    16-byte halves of each 8-cell row are exchanged in rows with j >= 4, so
//    that cell (i, j, k) of variable v sits at
//    v * 512 + 64 k + 8 j + (i ^ (4 * ((j >> 2) & 1)));
//  * the six face slabs in the layouts that tensor copies of the neighbour's
//    cells nearest the face produce, in the neighbour's own cell order:
//    -x / +x [8 v][8 k][8 j][4 i] (the neighbour's cells 4-7 / 0-3 along x:
//    ghost cells -2, -1 at positions 2, 3, ghost cells 8, 9 at 0, 1), -y / +y
//    [8 v][8 k][2 j][8 i] and -z / +z [8 v][2 k][8 j][8 i] (the neighbour's
//    cells 6, 7 / 0, 1: ghost cells -2, -1 and 8, 9 at positions 0, 1).
constexpr int MX_GX0 = 4096, MX_GX1 = 6144, MX_GY0 = 8192, MX_GY1 = 9216, MX_GZ0 = 10240, MX_GZ1 = 11264;
constexpr int MX_TILE = 12288;
constexpr int GSLOT = 2048;    // floats per ghost-slab buffer slot (either layout)

enum FaceType : int32_t { FACE_SAME = 0, FACE_COARSER = 1, FACE_FINER = 2, FACE_OUTFLOW = 3, FACE_INFLOW = 4 };
enum B0Mode : int32_t { B0_NONE = 0, B0_UNIFORM = 1, B0_DIPOLE = 2, B0_LINEAR = 3 };
enum ErrBits : int32_t { ERR_NONPHYSICAL = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 4 };

struct GridDev {
  double lo[3], hi[3];
  int32_t root[3];
  int32_t bc[6];
  int32_t maxlev;
  int32_t block0, nb;
  int64_t map_off[MAXLEV + 1];   // offset of each level's block map in levmap
  double body_r;
  double Winflow[8], Wbody[8];   // primitive, as given
  double Uinflow[8], Ubody[8];   // conservative, computed on the device at create
  float Winflow32[8];            // mixed-form primitive of Uinflow
  // per-level geometry, computed once on the host: dx = (hi - lo) / cells
  double dx[MAXLEV + 1][3], idx[MAXLEV + 1][3];
  float dxf[MAXLEV + 1][3], idxf[MAXLEV + 1][3];
  float lof[3];
};

struct BlockDev {
  int32_t grid, level, bi, bj, bk;
  int32_t ftype[6];              // FaceType per face (-x, +x, -y, +y, -z, +z)
  int32_t fnb[6];                // neighbour block (global index) for SAME / COARSER
  int32_t amr;                   // 1 if any face is COARSER or FINER
  int32_t body;                  // 1 if some cell centre lies inside the inner body
  int32_t rslot[6];              // refluxing: flux-register slot of a COARSER/FINER face, else -1
  int32_t pad_[2];
};

struct PhysDev {
  double gamma, gm1, inv_gm1;
  float gammaf, gm1f, inv_gm1f, padf_;
  int32_t limiter, rk, precision, b0, powell, learned;  // limiter 2: first order; rk 2: one stage
  int32_t flux, padi_;                                  // FLUX_RUSANOV, FLUX_HLL or FLUX_LINDE
  double b0p[12];
};
enum { FLUX_RUSANOV = 0, FLUX_HLL = 1, FLUX_LINDE = 2 };

// Learned flux correction: network sizes and the device weight set (BF16
// pairs in the layouts the tensor-core kernels read, FP32 biases).
constexpr int MLP_IN = 40, MLP_H = 64, MLP_OUT = 8;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;
struct MlpDev {
  uint32_t *w1, *w2, *w3, *w2t, *w3t;  // [64][24], [64][32], [8][32], [64][32], [64][8]
  float *b1, *b2, *b3;
  // the inference kernel's layouts, biases folded into the products: each
  // row's bias as a BF16 pair (hi, lo = b - hi) at K 40, 41 (layer 1, K =
  // 48) or 64, 65 (layers 2 and 3, K = 80, weights halved: that kernel's
  // hidden activations are twice the GELU).  w1b [64][24], w2b [64][40],
  // w3b [16][40] (rows 8..15 zero)
  uint32_t *w1b, *w2b, *w3b;
};

// Refluxing: one coarse face that borders a refined region.  The register
// slot cslot holds the coarse block's own 8 x 8 face fluxes, fslot[q] those of
// the fine block in transverse quadrant q (= q1 + 2 q2) on its opposite face.
struct RefluxTask {
  int32_t blk, s, cslot, fslot[4];
};

// Mixed form: one face of a block at a resolution change (COARSER or FINER),
// whose face-slab ghosts are computed ahead of the stage into slot `slot` of
// the ghost-slab buffer.
struct GhostTask {
  int32_t blk, s, slot;
};

// Arguments of one stage launch.
struct StageArgs {
  const double* Uin;      // stage input, block-major FP64
  const double* Ubase;    // base state of the stage (U^n)
  double* Uout;           // output (may alias Ubase: each CTA reads its own cells first)
  const float* Win;       // mixed form: FP32 primitives of Uin
  float* Wout;            // mixed form: FP32 primitives of Uout
  const GridDev* grids;
  const BlockDev* blocks;
  const int32_t* levmap;
  const double* dt;       // per grid
  unsigned long long* smax_next;  // per grid, bit pattern of a positive double
  int32_t* err;           // [0] error bits, [1] first bad block
  int32_t nblocks;
  int32_t blocks_per_item;
  int32_t kind;           // 0: Uout = Ubase + c R;  1: Uout = 0.5 Ubase + 0.5 (Uin + c R);
                          // 2: Uout = R (debug);  3: face features only (Xb);
                          // 4: features and plain fluxes only (Xf, Fd)
  int32_t last;           // 1: reduce the CFL bound of Uout into smax_next
  int32_t write_u_all;    // mixed: 1 = write Uout (FP64) too, 0 = only the FP32 primitives Wout
  double beta;            // c = beta * dt[grid], or beta * dtc[cell] with local time steps
  double* dtc;            // local time stepping: per-cell dt (read), rewritten from the new
                          // state by the last stage (nullptr: global dt)
  double cfl;             // CFL number for dtc
  double* freg;           // refluxing: flux register [slot][64][8] (nullptr: off)
  float* gbuf;            // mixed form: ghost slabs of faces at resolution changes [slot][8][128]
  int32_t nslots;         // slots of freg and gbuf (index checks of the checked build)
  PhysDev ph;
  // learned form; face index ((blk * 3 + d) * 576 + line * 9 + f)
  int32_t learned;        // kinds 0-2: add the clipped, rescaled correction Y
  uint32_t* Xb;           // kind 3: BF16 features, 24 words (48 columns) per face
  float* Xf;              // kind 4: FP32 features, 40 per face
  double* Fd;             // kind 4: plain Rusanov flux (8, x/y/z components), rho_ref, c_ref per face
  const float* Y;         // normalised correction in the face frame, 8 per face
  // mixed form, plain stage kernel: tensor maps of Win (interior box
  // 8x8x8x8 with the 32-byte swizzle; face-slab boxes 4x8x8x8, 8x2x8x8,
  // 8x8x2x8 over the dims (i, j, k, 8 * block + v)), and the staging layout:
  // 1 = same-level face slabs by tensor copies, 0 = gathered by the threads
  int32_t stage_tma;
  int32_t gbuf_mx;        // ghost-slab buffer in the mixed tile's slab layouts (1) or the generic one (0)
  MlpDev mlp;             // mixed learned stage: the network, run fused in the stage kernel
  CUtensorMap tm[4];
};

}  // namespace batsk
