// Launch arguments of the GEMM form of a fused bucket launch (gemm.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace qt {

enum { GEMM_SIMT = 0, GEMM_TC_TF32 = 1, GEMM_TC_BF16 = 2, GEMM_TC_3XTF32 = 3, GEMM_TILE = 4,
       GEMM_UMMA_TF32 = 5, GEMM_UMMA_3XTF32 = 6 };

constexpr int GEMM_MAXOP = 12;

struct GMeta {
  unsigned int maxabs;
  int E;
};

struct GOp {
  long long base, slice_stride, meta;
  unsigned long long smask;  // slice-id bits fixed into the operand
  unsigned int umask;
  int sshift, meta_per_slice, side;
  unsigned int xmask;  // GEMM_TILE: the operand's indices in the bit numbering of its side's big operand
  int tfold;           // triangle form: 0 large, 1 folded into C, 2 weight over K
};

struct GemmArgs {
  int m, nsum;
  unsigned int mK, mSA, mSB, mM, mN, mBt;
  long long nslices, slice_first;
  long long out_base, out_slice_stride, out_meta;
  int out_meta_per_slice;
  int fold_in;              // streaming GEMM: the small side is folded inside the kernel
  long long scratch_a, scratch_b, scratch_stride;  // elements (complex64 units)
  // GEMM_TILE: big operands, output indices per tile, which sides are folded
  int gA, gB, tb, fold_a, fold_b;
  unsigned int tile_inner;  // high output indices (above tb) visited innermost
  int reg_a, reg_b;         // register-blocking bits of the tile (-1: none)
  int reg_a2, reg_b2;       // second A-only / B-only bits (-1: none)
  int wide;                 // k_gemm_tma block: 0 2 x 2, 1 2 x 4 (reg_b2), 2 4 x 2 (reg_a2)
  int tA, tB, tC;           // triangle form: the large operands
  unsigned int tK, tX, tY;  // triangle form: summed bits of each class
  int use_tma;              // GEMM_TILE: stage the blocks with tensor copies (TMA)
  int stay;                 // GEMM_TILE: 0 the tiles of a group share A's block, 1 B's
  int use_stream;           // GEMM_TILE: the streaming kernel (gemm_stream_ok) instead
  long long ws_elems;       // workspace size (complex): the extent of the tensor maps
  int umma_shape;           // tcgen05 tiles: 0 the longest output runs, 1 the widest products (default)
  int umma_kc_max;          // tcgen05 work units: at most 2^this summed values (0: as many as fit)
  int* err;                 // device status word: set to 1 when a bounded wait gives up
  GOp op[GEMM_MAXOP];
};

// Output indices per tile of the GEMM_TILE kernel for a launch (0: the launch
// does not take that form: a one-sided summed index, or too little shared memory).
int gemm_tile_bits(const GemmArgs& a, int u);
// Tile visiting order of the GEMM_TILE kernel for a launch with tile bits a.tb:
// the high output indices visited innermost (those only the smaller operand has),
// and the side whose block the tiles differing only in them share (0 A, 1 B).
unsigned int gemm_tile_inner(const GemmArgs& a, int u);
int gemm_tile_stay(const GemmArgs& a);
// The streaming GEMM kernel applies: the smaller operand (at most 12 indices, nothing
// folded into the larger one) is staged whole per slice, one thread per row of the other.
bool gemm_stream_ok(const GemmArgs& a);
// Register-blocking bits of the GEMM_TILE kernels (an A-only and a B-only output bit
// inside the tile, or -1, -1; second bits for the wider blocks) and the block shape
// of k_gemm_tma (fewest shared-memory wavefronts per output).
// block_mode: 0 chosen by shared-memory wavefronts, 1 always 2 x 2, 2 (3) 2 x 4 (4 x 2)
// whenever that side has a second bit, else the other wide block, else 2 x 2.
void gemm_tile_regs(GemmArgs& a, int block_mode = 0);

// Triangle form (three large operands): output indices per tile (0: not taken)
// and the launch (one kernel).
int tri_tile_bits(const GemmArgs& a, int u);
// Tile visiting order of the triangle form for tiles of a.tb bits.
unsigned int tri_tile_inner(const GemmArgs& a, int u);
int tri_launch(const GemmArgs& a, float* data, GMeta* meta, cudaStream_t s, int sms,
               bool* used_tma = nullptr);

// GEMM_TILE: fold A', fold B' (when the side has small operands), tiled GEMM
// (tensor-copy staging when a.use_tma and the blocks allow it: *used_tma);
// other modes: pack A', pack B', GEMM. Returns the number of kernels launched.
int gemm_launch(const GemmArgs& a, int mode, float* data, GMeta* meta, cudaStream_t s, int sms,
                bool* used_tma = nullptr);

// GEMM form on the tcgen05 tensor cores (umma.cu). A tile: one slice, 128 rows of
// the lane side (its 7 lowest only-indices: the MMA's M), 2^cb rows of the column side
// (the MMA's N is twice that: re and im rows) and 2^gb values of batch indices, all
// chosen by walking the output indices from the lowest so that the tile covers as
// long a prefix of them as tensor memory allows (contiguous output runs). A work unit
// is one group value and one chunk of the summed values (all of them unless the rows do
// not fit shared memory; the chunks of a group accumulate in the same tensor-memory
// columns): its lane-side and column-side rows, one TMA box each. Masks are over the
// launch's U bits.
struct UmmaPlan {
  int lside;                 // 0: A gives the lanes (M), B the columns; 1: the reverse
  int nsum, cb, gb;          // summed indices; column bits (Nt = 2^cb); group bits (G = 2^gb)
  int passes;                // 1 TF32, 3 split TF32 (hi.hi + hi.lo + lo.hi)
  int sraw, splane;          // units of raw rows and of split planes in shared memory
  int tmem_cols;             // tensor-memory columns allocated per block
  unsigned int mlane, mcol, mgrp;
  int nrest;                 // U bits that enumerate the tiles, in tile order
  int rest[32];
  // a unit's rows in each operand's row index: runs of consecutive row bits
  int nlrun, lrun_start[3], lrun_len[3];
  int ncrun, crun_start[3], crun_len[3];
  int cwb;                   // epilogue chunk: 2^cwb columns x G groups x 32 lanes of a warp
  int rb;                    // contiguous output runs of 2^rb complex inside a chunk
  unsigned int chunk_out;    // the chunk's output bits (the run index takes those above rb)
  int prefix;                // output indices from the lowest that the tile covers
  int kc;                    // a work unit carries 2^kc of the 2^nsum summed values (kc <= nsum)
};
// The launch takes the form (false: it does not; the caller keeps another kernel).
bool umma_plan(const GemmArgs& a, int passes, UmmaPlan& p);
size_t umma_smem(const UmmaPlan& p);
// Launches k_gemm_umma (the folds of A', B' must have run); false if the operand rows
// or the output are not aligned as the kernel needs, or a tensor map does not encode.
bool umma_launch(const GemmArgs& a, const UmmaPlan& p, float* data, GMeta* meta, cudaStream_t s,
                 int sms);

}  // namespace qt
