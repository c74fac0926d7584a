// Host-side plan of one contraction: label classes after index fusion.
//
// The kernels see every contraction as a batched product
//     C[m, n] (batch l) = alpha * sum_k A[m, k] * B[n, k] + beta * C[m, n]
// where m, n, k, l are flat indices over the (fused) modes of each label
// class.  Element offsets are affine per mode, so each operand's offset is
// a sum of per-class offsets ("block-scatter" vectors: one offset table per
// operand and class, Sec. 2.3 of the paper, TBLIS item).  No operand is
// ever transposed or copied into a matrix layout.
#pragma once

#include <cstdint>

#include "../../include/famlies.h"

namespace famlies {

constexpr int kMaxModes = FAMLIES_MAX_NDIM;

// One mode of a label class: its extent and its stride in the kernel's row
// operand (sa), column operand (sb) and output (sc).  A stride is 0 when
// the operand does not hold the label.
struct Mode {
  int64_t ext;
  int64_t sa, sb, sc;
};

struct ClassModes {
  int n = 0;
  Mode m[kMaxModes];
  int64_t total() const {
    int64_t t = 1;
    for (int i = 0; i < n; ++i) t *= m[i].ext;
    return t;
  }
};

// A tridiagonal factor applied along k to one operand (the sandwiched
// product C := beta C + alpha A T A^T, famlies_gemmt_tridiag): element
// (r, p) of the operand the kernels see is
//   sub[p-1] x(r, p-1) + diag[p] x(r, p) + sup[p] x(r, p+1)
// of its strided source x, terms outside 0..k-1 left out (a band: entries
// of T off its three diagonals are not multiplied).  diag == null: no
// diagonal term; sup == null: sup[p] = -sub[p] (T skew-symmetric).
struct Band {
  const void* sub = nullptr;
  const void* diag = nullptr;
  const void* sup = nullptr;
};

// A Khatri-Rao operand (famlies_mttkrp): element (r, k) is the product,
// factor by factor in order, of U_f[i_f, r] (element (i, r) of factor f at
// u[f] + i * rs[f] + r * cs[f]), where i_f = (o / st[f]) % ext[f] are the
// digits of k's offset o in the operand's dense layout.
struct Krp {
  int nf = 0;
  const void* u[kMaxModes] = {};
  int64_t rs[kMaxModes] = {}, cs[kMaxModes] = {};
  int64_t ext[kMaxModes] = {}, st[kMaxModes] = {};
};

struct Plan {
  famlies_dtype_t dtype;
  ClassModes M, N, K, L;   // after role swap: M belongs to the row operand
  int64_t m = 0, n = 0, k = 0, l = 0;
  bool swapped = false;    // row operand is the caller's B
  bool c_empty = false;    // C has no entries: nothing to do
  bool scale_only = false; // alpha == 0 or an empty K: C := beta*C
  const void* a = nullptr; // row operand data (after swap)
  const void* b = nullptr; // column operand data
  void* c = nullptr;
  int es_a = 8, es_b = 8, es_c = 8;  // element sizes in bytes
  int a_contig = 0, b_contig = 0, c_contig = 0;
  int64_t span_a = 0, span_b = 0, span_c = 0;  // reachable elements (max offset + 1)
  int kernel = FAMLIES_KERNEL_NONE;
  int slices = 6;
  int tile_n = 0;  // tensor-core tile width request (0 = automatic)
  int cta_pair = 0;  // fp64 split: run the product on CTA pairs where it supports them
  int force_gather = 0;  // direct bf16 kernel: operands staged by gather warps (bit 0 row, bit 1 column)
  // Symmetric packed operand (famlies_contract_sym): n > 0 when the row
  // (side 0) or column (side 1) operand is stored as the lower triangle of
  // a symmetric n x n matrix; its classes are then one mode each (rows and
  // k of extent n) and its tables hold the offsets of the dense layout.
  int64_t sym_n = 0;
  int sym_side = -1;
  // Sandwiched product: operand band_side (0 row, 1 column) carries the
  // tridiagonal factor band; tri != 0 restricts the update to a triangle of
  // C in the kernel's indices (1: row >= col, 2: row <= col; no batch).
  Band band;
  int band_side = -1;
  int tri = 0;
  // Matricised tensor times Khatri-Rao product: operand krp_side is the
  // Khatri-Rao product krp, generated while it is packed.
  Krp krp;
  int krp_side = -1;
  // Contraction networks (fp64 split): exponents, non-finite flags and the
  // flagged-row list of operand side w computed by the step that produced
  // it (null: this call's exponent pass computes them) ...
  int32_t* pre_e[2] = {nullptr, nullptr};
  int32_t* pre_flag[2] = {nullptr, nullptr};
  int32_t* pre_list[2] = {nullptr, nullptr};
  // ... and, on that producing step, where its finish records them for the
  // consumer: emit_mode 1 = the consumer's row index is this call's row
  // index, 2 = its column index (0: nothing recorded).
  int emit_mode = 0;
  int32_t* emit_e = nullptr;
  int32_t* emit_flag = nullptr;
  int32_t* emit_list = nullptr;
};

// Validates and plans; returns FAMLIES_OK or a FAMLIES_ERR_* code.  Never
// touches the device.  `alpha` decides scale_only (alpha == 0 => A and B
// are not read and need not alias-check).
int make_plan(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
              const famlies_tensor_t* C, famlies_dtype_t dtype, const famlies_options_t* opt,
              Plan* out);

void fill_info(const Plan& p, famlies_plan_info_t* info);

// The direct bf16 kernel (csrc/k_box.cu) accumulates the whole contracted
// range in tensor memory: at most this many k.
constexpr int64_t kBoxMaxK = 16384;
// Whether plan p (kernel TC_BF16 or TC_BF16_DIRECT) fits the direct bf16
// kernel.  Host only: no device work.
bool box_applicable(const Plan& p);

}  // namespace famlies
