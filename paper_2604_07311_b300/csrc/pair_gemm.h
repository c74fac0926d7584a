// The packed tensor-core product (k_pair_gemm, csrc/k_pack_gemm.cu): the
// per-problem descriptor, the unit schedule, and the launchers shared by the
// single-problem path and the grouped (many-problem) path.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "device.h"

namespace famlies {

constexpr int kPairBM = 128;      // rows of an output tile
constexpr int kPairMaxDiag = 10;

enum { PAIR_KIND_BF16 = 0, PAIR_KIND_TF32 = 1 };
// fp32 output; fp64 split with one int64 sum per output; fp64 split with a
// second, exact sum for the fine diagonals (Sched::nlow > 0)
enum { PAIR_MODE_F32OUT = 0, PAIR_MODE_EMU = 1, PAIR_MODE_EMU_FINE = 2 };

// The unit schedule of one output tile (identical for every tile of a launch).
struct Sched {
  int ndiag;
  int slices;
  int shift[kPairMaxDiag];        // diagonal weight 2^-shift (fp64 split)
  int kcb[kPairMaxDiag];          // k-blocks per unit
  int flush_every[kPairMaxDiag];  // units between flushes of the int32 sums
  int npairs[kPairMaxDiag];
  int8_t pa[kPairMaxDiag][8], pb[kPairMaxDiag][8];  // slice of A and B in each pair
  // fp64 split: int64 sums per output in units of 2^-xunit (as fine as K
  // allows without overflow) and, when nlow > 0, a second one in units of
  // 2^-xlo for the nlow diagonals finer than 2^-xunit (di < nlow: the walk
  // starts from the least significant).  A diagonal's int32 sums enter its
  // sum shifted by xshift: left (exact), or right with rounding for a fine
  // diagonal folded into the coarse sum (nlow = 0).
  int xunit, xlo, nlow;
  int xshift[kPairMaxDiag];
};

// What the product needs to know about one problem.
struct Prob {
  const CUtensorMap* map_a;  // grouped launches: maps in global memory (64-byte aligned)
  const CUtensorMap* map_b;
  void* c;
  const int64_t* cm;
  const int64_t* cn;
  const int64_t* cl;
  const int32_t* ea;  // fp64 split: row exponents and non-finite flags
  const int32_t* eb;
  const int32_t* fa;
  const int32_t* fb;
  int64_t m, n, k, l;
  double alpha, beta;
  int bn;  // grouped launches: this problem's tile width (64, 128 or 256, <= the launch's)
  // Single problems restricted to a triangle of C (tri 1: row >= col, 2:
  // row <= col; no batch): the tiles that meet it, listed row tile by row
  // tile (tri_list[i] = {tm, tn}), tri_tiles of them.
  int tri;
  const int2* tri_list;
  int64_t tri_tiles;
  // Single problems in a network (fp64 split): the finish folds every
  // output into the consuming step's row exponents and flags (see Plan).
  int emit_mode;
  int32_t* emit_e;
  int32_t* emit_flag;
  int32_t* emit_list;
};

// One entry of a grouped launch's tile list: problem, row tile, column tile, batch.
struct TileEntry {
  int32_t p, tm, tn, il;
};

// k: the largest contracted extent the schedule serves (bounds the tile sums);
// parts: the work items that share one tile's sums (its K splits).
Sched make_pair_sched(int kernel, int slices, int bits, int64_t k, int64_t parts = 1);
int pair_bn_for(int64_t n, int request);
// 3-D map over slices [z][rows][kp] (k innermost), box {box_k, box_rows, 1}.
bool make_slice_map(CUtensorMap* map, void* base, bool f32, int64_t k, int64_t kp, int64_t rows,
                    int64_t z, int box_k, int box_rows);
// Grouped product over a device tile list; probs/tiles are device arrays.
// slots (fp64 split, may be null): every tile leaves its int64 sums in its
// slot [tile][bn][BM] (two sums per element with the fine diagonals) for
// launch_group_finish instead of finishing inside the product.
cudaError_t launch_pair_grouped(int kind, int mode, int bn, const Prob* probs,
                                const TileEntry* tiles, int64_t ntiles, const Sched& sc,
                                double* G, int64_t* slots, int grid, int* status, int64_t wait_limit,
                                cudaStream_t s);
// C of every tile of the list from its slot (after a product with slots).
cudaError_t launch_group_finish(bool fine, const int64_t* X, const Prob* probs, const TileEntry* tiles,
                                int64_t ntiles, int bn, int xunit, int xlo, cudaStream_t s);
// k per ring stage.  bf16 stages hold rows of kBf16StageK values (64 bytes at
// 32, read through the 64-byte swizzle; 128 bytes at 64, the 128-byte one);
// tf32 stages rows of 32 values (128 bytes).  Smaller stages of the same
// total size let the ring hold more of them.
constexpr int kBf16StageK = 64;
constexpr int pair_stage_k(int kind) { return kind == PAIR_KIND_BF16 ? kBf16StageK : 32; }
constexpr int pair_row_bytes(int kind) { return kind == PAIR_KIND_BF16 ? 2 * kBf16StageK : 128; }
// Stages per unit of the fp32-output schedule: 1024 k (bf16) or 512 k (tf32)
// summed in tensor memory before each fp32 register update.
constexpr int f32out_unit_stages(int kind) { return (kind == PAIR_KIND_BF16 ? 1024 : 512) / pair_stage_k(kind); }

}  // namespace famlies
