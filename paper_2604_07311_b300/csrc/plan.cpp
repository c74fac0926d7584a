// Planner: descriptor validation, label classification, index fusion and
// the choice of which operand supplies the kernel's rows.
//
// Classification follows Einstein summation over labels (the contraction of
// Sec. 2.3 of the paper): C-and-A-only labels form class M, C-and-B-only
// class N, A-and-B-only class K, labels in all three the batch class.
// Index fusion merges adjacent modes of a class whose strides chain
// (stride_outer == stride_inner * extent_inner) in EVERY operand holding the
// class, so a dense column-major 4-index contraction becomes a plain GEMM
// without moving any data (the tensor-to-matrix mapping without explicit
// conversion, Sec. 1 "Challenges" and Sec. 2.3 block-scatter item).
#include "plan.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace famlies {

namespace {

int elem_size_in(famlies_dtype_t dt) {
  switch (dt) {
    case FAMLIES_F64:
    case FAMLIES_F64_EMU: return 8;
    case FAMLIES_F32: return 4;
    case FAMLIES_BF16: return 2;
  }
  return 0;
}

int elem_size_out(famlies_dtype_t dt) {
  switch (dt) {
    case FAMLIES_F64:
    case FAMLIES_F64_EMU: return 8;
    case FAMLIES_F32:
    case FAMLIES_BF16: return 4;
  }
  return 0;
}

int check_tensor(const famlies_tensor_t* t) {
  if (!t) return FAMLIES_ERR_INVALID_ARG;
  if (t->ndim < 0 || t->ndim > kMaxModes) return FAMLIES_ERR_INVALID_ARG;
  if (t->ndim > 0 && (!t->extents || !t->strides || !t->labels)) return FAMLIES_ERR_INVALID_ARG;
  for (int i = 0; i < t->ndim; ++i) {
    if (t->extents[i] < 0 || t->strides[i] < 0) return FAMLIES_ERR_INVALID_ARG;
    for (int j = i + 1; j < t->ndim; ++j)
      if (t->labels[i] == t->labels[j]) return FAMLIES_ERR_LABEL;
  }
  if (t->size_bytes < 0) return FAMLIES_ERR_INVALID_ARG;
  return FAMLIES_OK;
}

int find(const famlies_tensor_t* t, int32_t lab) {
  for (int i = 0; i < t->ndim; ++i)
    if (t->labels[i] == lab) return i;
  return -1;
}

bool is_empty(const famlies_tensor_t* t) {
  for (int i = 0; i < t->ndim; ++i)
    if (t->extents[i] == 0) return true;
  return false;
}

// Number of reachable elements (max offset + 1), 0 for an empty tensor.
// Returns -1 on overflow.
int64_t span_of(const famlies_tensor_t* t) {
  if (is_empty(t)) return 0;
  __int128 off = 0;
  for (int i = 0; i < t->ndim; ++i) off += (__int128)(t->extents[i] - 1) * t->strides[i];
  if (off > (__int128)INT64_MAX / 16) return -1;
  return (int64_t)off + 1;
}

// C's modes of extent > 1, sorted by stride, must each start past the span
// of the smaller ones; then no two index tuples share an address.
bool c_layout_ok(const famlies_tensor_t* c) {
  int idx[kMaxModes];
  int n = 0;
  for (int i = 0; i < c->ndim; ++i)
    if (c->extents[i] > 1) idx[n++] = i;
  std::sort(idx, idx + n, [&](int x, int y) { return c->strides[x] < c->strides[y]; });
  int64_t reach = 0;  // max offset reachable with the modes so far
  for (int j = 0; j < n; ++j) {
    int64_t s = c->strides[idx[j]];
    if (s <= reach) return false;
    reach += (c->extents[idx[j]] - 1) * s;
  }
  return true;
}

bool ranges_overlap(const void* p, int64_t pbytes, const void* q, int64_t qbytes) {
  if (pbytes <= 0 || qbytes <= 0) return false;
  uintptr_t a0 = (uintptr_t)p, a1 = a0 + (uintptr_t)pbytes;
  uintptr_t b0 = (uintptr_t)q, b1 = b0 + (uintptr_t)qbytes;
  return a0 < b1 && b0 < a1;
}

// Sorts a class by the stride of the operand selected by `key` (0: sa,
// 1: sb, 2: sc; ties broken by the others), then merges chained modes.
void fuse(ClassModes& cm, int key, bool has_a, bool has_b, bool has_c) {
  auto st = [&](const Mode& m, int w) { return w == 0 ? m.sa : (w == 1 ? m.sb : m.sc); };
  std::stable_sort(cm.m, cm.m + cm.n, [&](const Mode& x, const Mode& y) {
    for (int w : {key, 0, 1, 2})
      if (st(x, w) != st(y, w)) return st(x, w) < st(y, w);
    return false;
  });
  int out = 0;
  for (int i = 0; i < cm.n; ++i) {
    if (out > 0) {
      Mode& p = cm.m[out - 1];
      const Mode& q = cm.m[i];
      bool ok = (!has_a || q.sa == p.sa * p.ext) && (!has_b || q.sb == p.sb * p.ext) &&
                (!has_c || q.sc == p.sc * p.ext);
      if (ok) {
        p.ext *= q.ext;
        continue;
      }
    }
    cm.m[out++] = cm.m[i];
  }
  cm.n = out;
}

}  // namespace

int make_plan(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
              const famlies_tensor_t* C, famlies_dtype_t dtype, const famlies_options_t* opt,
              Plan* out) {
  if (!out) return FAMLIES_ERR_INVALID_ARG;
  if (dtype != FAMLIES_F64 && dtype != FAMLIES_F64_EMU && dtype != FAMLIES_F32 &&
      dtype != FAMLIES_BF16)
    return FAMLIES_ERR_INVALID_ARG;
  int rc;
  if ((rc = check_tensor(A)) || (rc = check_tensor(B)) || (rc = check_tensor(C))) return rc;

  Plan p;
  p.dtype = dtype;
  p.es_a = p.es_b = elem_size_in(dtype);
  p.es_c = elem_size_out(dtype);

  // ---- classification
  ClassModes M, N, K, Lb;
  for (int i = 0; i < C->ndim; ++i) {
    int ia = find(A, C->labels[i]), ib = find(B, C->labels[i]);
    if (ia < 0 && ib < 0) return FAMLIES_ERR_LABEL;
    if (ia >= 0 && A->extents[ia] != C->extents[i]) return FAMLIES_ERR_EXTENT_MISMATCH;
    if (ib >= 0 && B->extents[ib] != C->extents[i]) return FAMLIES_ERR_EXTENT_MISMATCH;
    Mode md{C->extents[i], ia >= 0 ? A->strides[ia] : 0, ib >= 0 ? B->strides[ib] : 0,
            C->strides[i]};
    ClassModes& cls = (ia >= 0 && ib >= 0) ? Lb : (ia >= 0 ? M : N);
    cls.m[cls.n++] = md;
  }
  for (int i = 0; i < A->ndim; ++i) {
    if (find(C, A->labels[i]) >= 0) continue;
    int ib = find(B, A->labels[i]);
    if (ib < 0) return FAMLIES_ERR_LABEL;
    if (B->extents[ib] != A->extents[i]) return FAMLIES_ERR_EXTENT_MISMATCH;
    K.m[K.n++] = Mode{A->extents[i], A->strides[i], B->strides[ib], 0};
  }
  for (int i = 0; i < B->ndim; ++i)
    if (find(C, B->labels[i]) < 0 && find(A, B->labels[i]) < 0) return FAMLIES_ERR_LABEL;

  // ---- spans, bounds, layout and aliasing
  int64_t sa = span_of(A), sb = span_of(B), sc = span_of(C);
  if (sa < 0 || sb < 0 || sc < 0) return FAMLIES_ERR_UNSUPPORTED;
  if (A->size_bytes > 0 && sa * p.es_a > A->size_bytes) return FAMLIES_ERR_OUT_OF_BOUNDS;
  if (B->size_bytes > 0 && sb * p.es_b > B->size_bytes) return FAMLIES_ERR_OUT_OF_BOUNDS;
  if (C->size_bytes > 0 && sc * p.es_c > C->size_bytes) return FAMLIES_ERR_OUT_OF_BOUNDS;
  p.c_empty = is_empty(C);
  if (!p.c_empty && !C->data) return FAMLIES_ERR_INVALID_ARG;
  if (!c_layout_ok(C)) return FAMLIES_ERR_UNSUPPORTED;
  bool k_empty = false;
  for (int i = 0; i < K.n; ++i) k_empty |= (K.m[i].ext == 0);
  p.scale_only = !p.c_empty && (alpha == 0.0 || k_empty);
  bool reads_ab = !p.c_empty && !p.scale_only;
  if (reads_ab) {
    if (!A->data || !B->data) return FAMLIES_ERR_INVALID_ARG;
    if (ranges_overlap(C->data, sc * p.es_c, A->data, sa * p.es_a) ||
        ranges_overlap(C->data, sc * p.es_c, B->data, sb * p.es_b))
      return FAMLIES_ERR_ALIAS;
  }

  // ---- drop extent-1 modes (they change no offset), then fuse
  auto drop1 = [](ClassModes& cm) {
    int o = 0;
    for (int i = 0; i < cm.n; ++i)
      if (cm.m[i].ext != 1) cm.m[o++] = cm.m[i];
    cm.n = o;
  };
  drop1(M); drop1(N); drop1(K); drop1(Lb);

  // Role choice: the kernels put class M on the rows (tensor-memory lanes,
  // one output row per epilogue thread), so C's unit-stride mode should be
  // an M mode for coalesced stores.  Swap A and B when it is an N mode.
  auto min_stride_mode = [&](const ClassModes& cm, int64_t& best) {
    for (int i = 0; i < cm.n; ++i) best = std::min(best, cm.m[i].sc);
  };
  int64_t bm = INT64_MAX, bn = INT64_MAX;
  min_stride_mode(M, bm);
  min_stride_mode(N, bn);
  p.swapped = bn < bm;
  const famlies_tensor_t* rowop = p.swapped ? B : A;
  const famlies_tensor_t* colop = p.swapped ? A : B;
  if (p.swapped) {
    std::swap(M, N);
    for (ClassModes* cm : {&M, &N, &K, &Lb})
      for (int i = 0; i < cm->n; ++i) std::swap(cm->m[i].sa, cm->m[i].sb);
    std::swap(sa, sb);
  }
  p.a = rowop->data;
  p.b = colop->data;
  p.c = C->data;
  p.span_a = sa;
  p.span_b = sb;
  p.span_c = sc;

  fuse(M, 2, true, false, true);
  fuse(N, 2, false, true, true);
  fuse(K, 0, true, true, false);
  fuse(Lb, 2, true, true, true);
  p.M = M; p.N = N; p.K = K; p.L = Lb;
  p.m = M.total();
  p.n = N.total();
  p.k = K.total();
  p.l = Lb.total();
  const int64_t lim = (int64_t)1 << 31;
  if (p.m >= lim || p.n >= lim || p.k >= lim || p.l >= lim) return FAMLIES_ERR_UNSUPPORTED;

  // ---- contiguity of each operand along one class (first fused mode)
  auto unit = [](const ClassModes& cm, int w) {
    if (cm.n == 0) return false;
    const Mode& m = cm.m[0];
    return (w == 0 ? m.sa : (w == 1 ? m.sb : m.sc)) == 1;
  };
  p.a_contig = unit(p.M, 0) ? 1 : (unit(p.K, 0) ? 2 : 0);
  // For the column operand, check its own smallest K stride.
  ClassModes Kb = p.K;
  std::stable_sort(Kb.m, Kb.m + Kb.n, [](const Mode& x, const Mode& y) { return x.sb < y.sb; });
  p.b_contig = unit(p.N, 1) ? 1 : (unit(Kb, 1) ? 2 : 0);
  p.c_contig = unit(p.M, 2) ? 1 : (unit(p.N, 2) ? 2 : 0);

  // ---- kernel choice
  const int force = opt ? opt->kernel : 0;
  if (force < 0 || force > 5) return FAMLIES_ERR_INVALID_ARG;
  if (force >= 4 && dtype != FAMLIES_BF16 && !p.c_empty && !p.scale_only) return FAMLIES_ERR_UNSUPPORTED;
  if (p.c_empty) p.kernel = FAMLIES_KERNEL_NONE;
  else if (p.scale_only) p.kernel = FAMLIES_KERNEL_SCALE;
  else switch (dtype) {
    case FAMLIES_F64:
      if (force >= 2) return FAMLIES_ERR_UNSUPPORTED;
      p.kernel = FAMLIES_KERNEL_SIMT_F64;
      break;
    case FAMLIES_F32:
      p.kernel = force == 1 ? FAMLIES_KERNEL_SIMT_F32
                            : (force == 3 ? FAMLIES_KERNEL_TC_TF32X3_GATHER : FAMLIES_KERNEL_TC_TF32X3);
      break;
    case FAMLIES_BF16:
      if (force == 1) return FAMLIES_ERR_UNSUPPORTED;
      p.kernel = force == 3 ? FAMLIES_KERNEL_TC_BF16_GATHER : FAMLIES_KERNEL_TC_BF16;
      break;
    case FAMLIES_F64_EMU:
      if (force == 1 || force == 3) return FAMLIES_ERR_UNSUPPORTED;
      p.kernel = FAMLIES_KERNEL_TC_EMU;
      break;
  }
  // Options left at 0 take FAMLIES_FORCE_TILE / FAMLIES_SLICES from the
  // environment when set, else the built-in choices.
  auto env_int = [](const char* name) {
    const char* e = std::getenv(name);
    return e ? std::atoi(e) : 0;
  };
  p.tile_n = opt && opt->tile_n ? opt->tile_n : env_int("FAMLIES_FORCE_TILE");
  if (opt && (opt->ctas_per_mma < 0 || opt->ctas_per_mma > 2)) return FAMLIES_ERR_INVALID_ARG;
  p.cta_pair = opt && opt->ctas_per_mma == 2 ? 1 : 0;
  if (p.tile_n != 0 && p.tile_n != 64 && p.tile_n != 128 && p.tile_n != 192 && p.tile_n != 256)
    return FAMLIES_ERR_INVALID_ARG;
  // bf16: the direct kernel (tiles staged from the caller's strides) when
  // the call fits it, unless another kernel was asked for
  if (p.kernel == FAMLIES_KERNEL_TC_BF16 && (force == 0 || force >= 4)) {
    p.kernel = FAMLIES_KERNEL_TC_BF16_DIRECT;
    if (!box_applicable(p)) {
      if (force >= 4) return FAMLIES_ERR_UNSUPPORTED;
      p.kernel = FAMLIES_KERNEL_TC_BF16;
    }
  }
  p.force_gather = force == 5 ? 3 : 0;
  int s = opt && opt->slices ? opt->slices : env_int("FAMLIES_SLICES");
  if (s == 0) s = 6;
  if (s < 2 || s > 7) return FAMLIES_ERR_INVALID_ARG;
  p.slices = s;
  *out = p;
  return FAMLIES_OK;
}

void fill_info(const Plan& p, famlies_plan_info_t* info) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->m = p.m;
  info->n = p.n;
  info->k = p.k;
  info->batch = p.l;
  info->m_modes = p.M.n;
  info->n_modes = p.N.n;
  info->k_modes = p.K.n;
  info->batch_modes = p.L.n;
  info->swapped = p.swapped;
  info->kernel = p.kernel;
  info->ctas_per_mma = 1;
  info->slices = p.dtype == FAMLIES_F64_EMU ? p.slices : 0;
  info->a_contig = p.a_contig;
  info->b_contig = p.b_contig;
  info->c_contig = p.c_contig;
}

}  // namespace famlies
