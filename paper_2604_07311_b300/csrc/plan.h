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
  // Symmetric packed operand (famlies_contract_sym): n > 0 when the row
  // (side 0) or column (side 1) operand is stored as the lower triangle of
  // a symmetric n x n matrix; its classes are then one mode each (rows and
  // k of extent n) and its tables hold the offsets of the dense layout.
  int64_t sym_n = 0;
  int sym_side = -1;
};

// Validates and plans; returns FAMLIES_OK or a FAMLIES_ERR_* code.  Never
// touches the device.  `alpha` decides scale_only (alpha == 0 => A and B
// are not read and need not alias-check).
int make_plan(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
              const famlies_tensor_t* C, famlies_dtype_t dtype, const famlies_options_t* opt,
              Plan* out);

void fill_info(const Plan& p, famlies_plan_info_t* info);

}  // namespace famlies
