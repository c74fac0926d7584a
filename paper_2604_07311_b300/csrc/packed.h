// Packing kernels that feed the TMA tensor-core product (see k_pack.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "device.h"

namespace famlies {

enum { PACK_BF16 = 0, PACK_TF32 = 1, PACK_F64 = 2 };

// Digit width b of the fp64 split (emulated precision, Sec. 1.5): each
// slice holds b-bit balanced digits, exact in bf16 (8 significant bits).
// At most 7 slices: the scaled integer F < 2^(b s) must fit in int64.
constexpr int kSplitBits = 8;
constexpr int kMaxSplitSlices = 7;

// One operand to pack: rows x k (batch l) read through offset tables.
struct PackOp {
  const void* x;        // source operand (strided)
  const int64_t* roff;  // row offsets (rows entries)
  const int64_t* koff;  // k offsets (k entries)
  const int64_t* loff;  // batch offsets (l entries)
  int64_t rows;
  int contig;           // 1: unit stride along rows, 2: along k, 0: neither
  void* out;            // slices [S][l][rows][kp]
  int32_t* e;           // fp64 split: row exponents [l][rows] (pre-set to INT_MIN)
  int32_t* flag;        // fp64 split: non-finite row flags [l][rows] (pre-set to 0)
  int32_t* list;        // fp64 split: list[0] = count, list[1..] = flagged l*rows + r
  // When a class fused to at most one mode its offsets are affine:
  // affine bit 0 -> row offset = r * rs, bit 1 -> k offset = k * ks
  // (the tables are then not read).
  int affine;
  int64_t rs, ks;
  // > 0: the operand is the lower triangle of a symmetric sym_n x sym_n
  // matrix, column by column; rows and k index the two sides (packed by
  // k_rowexp_sym / k_pack_sym, not by the generic kernels).
  int64_t sym_n;
  // gen != 0: the operand is generated as it is packed (k_rowexp_gen /
  // k_pack_gen): 1 = its affine source with a tridiagonal factor along k
  // (band), 2 = a Khatri-Rao product of factor matrices (krp).
  int gen;
  Band band;
  Krp krp;
};

// Sets the affine fields of a pack operand from its row and k classes
// (which: 0 = the plan's row operand, 1 = its column operand).
void set_affine(PackOp& o, const ClassModes& R, const ClassModes& K, int which);

struct PackArgs {
  PackOp op[2];
  int64_t k, kp, l;
  int slices;
};

// fp64 split, pass 1: row exponent bounds and non-finite flags (both operands).
cudaError_t launch_rowexp(const PackArgs& pa, cudaStream_t s);
// Writes the slices of both operands.
cudaError_t launch_pack(int pmode, const PackArgs& pa, cudaStream_t s);
// fp64 split in one pass over operand pa.op[side] (row exponents, flags and
// slices) when its k is one unit-stride mode and kRowPackMinK <= k <=
// kRowPackMaxK (each row is then held in registers while it is split).
constexpr int64_t kRowPackMinK = 512;
constexpr int64_t kRowPackMaxK = 16384;
cudaError_t launch_rowpack(const PackArgs& pa, int side, cudaStream_t s);
// Symmetric packed operand pa.op[side] (fp64 split): row exponents and flags
// (every stored element bounds its row and, by symmetry, its column) and its
// slices, both from one read of the lower triangle.
// scr: sym_scratch_bytes(sym_n) of workspace for the per-tile maxima.
cudaError_t launch_rowexp_sym(const PackArgs& pa, int side, int32_t* scr, cudaStream_t s);
int64_t sym_scratch_bytes(int64_t n);
cudaError_t launch_pack_sym(const PackArgs& pa, int side, cudaStream_t s);
// Generated operand pa.op[side] (banded or Khatri-Rao, see PackOp::gen):
// row exponents and flags (fp64 split) and its slices (PACK_F64 or
// PACK_TF32), the values computed as each tile is staged.
cudaError_t launch_rowexp_gen(const PackArgs& pa, int side, cudaStream_t s);
cudaError_t launch_pack_gen(int pmode, const PackArgs& pa, int side, cudaStream_t s);
// fp64 split: recomputes in native fp64 the outputs of flagged rows/columns.
cudaError_t launch_fixup(const GemmArgs& g, const PackArgs& pa, cudaStream_t s);

// Grouped forms: n problems' PackArgs / GemmArgs in device memory, one launch
// each.  off[2n+1] (device) numbers the tiles of segment s = 2*problem +
// operand from off[s]; off[2n] = total.  The tile counts per segment come
// from rowexp_tiles / pack_tiles.
int64_t rowexp_tiles(int64_t rows, int64_t k, int64_t l);
int64_t pack_tiles(int64_t rows, int64_t k, int64_t l);
cudaError_t launch_rowexp_grouped(const PackArgs* pas, const int64_t* off, int n, int64_t total,
                                  cudaStream_t s);
cudaError_t launch_pack_grouped(int pmode, const PackArgs* pas, const int64_t* off, int n,
                                int64_t total, cudaStream_t s);
cudaError_t launch_fixup_grouped(const GemmArgs* gs, const PackArgs* pas, int n, cudaStream_t s);

}  // namespace famlies
