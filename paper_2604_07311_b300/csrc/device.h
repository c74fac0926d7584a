// Device-side argument blocks shared by the kernels and the host launchers.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "plan.h"

namespace famlies {

// Offset tables ("block-scatter" vectors): element (m, n, k, l) of the
// contraction reads A at a + am[m] + ak[k] + al[l], B at b + bn[n] + bk[k]
// + bl[l] and writes C at c + cm[m] + cn[n] + cl[l] (offsets in elements).
struct Tables {
  const int64_t* am;
  const int64_t* cm;
  const int64_t* bn;
  const int64_t* cn;
  const int64_t* ak;
  const int64_t* bk;
  const int64_t* al;
  const int64_t* bl;
  const int64_t* cl;
};

struct GemmArgs {
  const void* a;
  const void* b;
  void* c;
  Tables t;
  int64_t m, n, k, l;
  double alpha, beta;
  int a_contig, b_contig;  // 1: unit stride along rows/cols, 2: along k
  int64_t wait_limit;      // iteration cap of every bounded wait
  int* status;             // device status word (first error recorded wins)
  int stall_test;          // testing: product kernels first wait on a barrier nothing completes
  int64_t sym_n;           // > 0: operand sym_side is a packed symmetric matrix (see Plan)
  int sym_side;
  Band band;               // tridiagonal factor (see Plan) of operand band_op - 1 (0: none)
  int band_op;
  int tri;                 // 0: all of C; 1: only row >= col; 2: only row <= col
  Krp krp;                 // Khatri-Rao operand (see Plan) is operand krp_op - 1 (0: none)
  int krp_op;
  void* part;              // CUDA-core split K: partial results [split][l][n][m] (null: none)
  int emit_mode;           // fp64 split in a network: consumer exponents recorded (see Plan)
  int32_t* emit_e;
  int32_t* emit_flag;
  int32_t* emit_list;
  cudaEvent_t ev_begin, ev_end;  // host only: recorded around the product kernel
};

inline void mark_begin(const GemmArgs& g, cudaStream_t s) {
  if (g.ev_begin) cudaEventRecord(g.ev_begin, s);
}
inline void mark_end(const GemmArgs& g, cudaStream_t s) {
  if (g.ev_end) cudaEventRecord(g.ev_end, s);
}

// One offset table: out[i] = sum_d digit_d(i) * st[d] for the mixed-radix
// digits of i over ext[0..n).
struct TableJob {
  int n;
  int64_t ext[kMaxModes];
  int64_t st[kMaxModes];
  int64_t total;
  int64_t* out;
};
void plan_table_jobs(const Plan& p, int64_t* ws, TableJob jobs[9], Tables* t);
cudaError_t launch_tables_grouped(const TableJob* jobs, int64_t njobs, int64_t max_total,
                                  cudaStream_t s);

// Grouped execution of many plans of one packed kernel (csrc/grouped.cu).
int run_grouped(const std::vector<const Plan*>& ps, const std::vector<double>& alpha,
                const std::vector<double>& beta, cudaStream_t s, bool use_graph, int* status,
                int64_t wait_limit);

// Address of the device status word of the current device, and a host-side
// read-and-clear of it (both defined next to the word itself).
int* device_status_ptr();
int read_clear_status(int* value);

// ---- launchers (each returns a cudaError_t from the launch)
cudaError_t launch_tables(const Plan& p, int64_t* ws, Tables* t, cudaStream_t s);
cudaError_t launch_scale(const Plan& p, const Tables& t, double beta, cudaStream_t s);
// ws: workspace of simt_workspace_bytes(p) bytes, or null (no K split).
cudaError_t launch_simt(const Plan& p, const GemmArgs& g, void* ws, cudaStream_t s);
// Bytes of the partial tiles a CUDA-core launch splits K into (0: no split).
int64_t simt_workspace_bytes(const Plan& p);
cudaError_t launch_tc(const Plan& p, const GemmArgs& g, int tile_n, void* ws, cudaStream_t s);
// Direct bf16 kernel (csrc/k_box.cu; box_applicable in plan.h), no offset
// tables: its workspace (a re-padded copy of each operand whose strides no
// tensor map can address; 0 bytes when both can be read as they stand, or
// when Plan::force_gather stages them by gather warps), and its launch (the
// re-pad copies, then the product; *launches counts them).
int64_t box_workspace_bytes(const Plan& p);
cudaError_t launch_box(const Plan& p, const GemmArgs& g, void* ws, cudaStream_t s, int* launches);
int64_t tc_workspace_bytes(const Plan& p);
// Packed paths (bf16, tf32 split, fp64 split): workspace size and launch.
int64_t packed_workspace_bytes(const Plan& p);
cudaError_t launch_packed(const Plan& p, const GemmArgs& g, void* ws, cudaStream_t s);
// Kernel launches launch_packed makes for plan p.
int packed_launches(const Plan& p);
// CTAs per tensor-core MMA of the packed product (2: CTA pairs).
int packed_ctas_per_mma(const Plan& p);

// Whether C's element (row r, column c) of the kernel's indices is updated
// under triangle mode tri (see Plan::tri).
__host__ __device__ __forceinline__ bool tri_keep(int tri, int64_t r, int64_t c) {
  return tri == 0 || (tri == 1 ? r >= c : r <= c);
}

// Element p of a banded operand row (see Band): x is the source, base the
// row's offset, its k offsets koff[q] (koff null: q * ks).  One fixed order
// of operations, so that every kernel computing it gets the same value.
template <class T>
__device__ __forceinline__ T band_at(const T* __restrict__ x, int64_t base, const int64_t* koff,
                                     int64_t ks, int64_t p, int64_t k, const Band& b) {
  const T* s = (const T*)b.sub;
  const T* d = (const T*)b.diag;
  const T* u = (const T*)b.sup;
  auto at = [&](int64_t q) { return x[base + (koff ? koff[q] : q * ks)]; };
  auto fm = [](T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return fmaf(a, b, c);
    else return fma(a, b, c);
  };
  T v = d ? d[p] * at(p) : T(0);
  if (p > 0) v = fm(s[p - 1], at(p - 1), v);
  if (p + 1 < k) v = fm(u ? u[p] : -s[p], at(p + 1), v);
  return v;
}

// Element (r, k) of a Khatri-Rao operand (see Krp) whose k offset is off.
template <class T>
__device__ __forceinline__ T krp_at(const Krp& q, int64_t r, int64_t off) {
  T v = T(1);
  for (int f = 0; f < q.nf; ++f) {
    const int64_t i = (off / q.st[f]) % q.ext[f];
    const T u = ((const T*)q.u[f])[i * q.rs[f] + r * q.cs[f]];
    v = f == 0 ? u : v * u;
  }
  return v;
}

// x as the nearest binary64 value (ties to even), formed with integer
// instructions only (B300's fp64 pipe is narrow and the fp64-split epilogues
// convert one integer sum per output): the leading set bit of |x| at
// position p gives the biased exponent p + 1023, the 52 bits below it the
// fraction, and the 11 bits after those decide the rounding (above half:
// up; exactly half: up when the kept fraction is odd); a carry out of the
// fraction raises the exponent.  Exact for |x| < 2^53.
__device__ __forceinline__ double i64_to_f64_rn(int64_t x) {
  if (x == 0) return 0.0;
  const unsigned long long sign = x < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long u = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
  const int lz = __clzll((long long)u);
  const unsigned long long m = u << lz;          // leading 1 at bit 63
  unsigned long long mant = m >> 11;             // 53 bits, leading 1 at bit 52
  const unsigned long long rem = m & 0x7FFull;   // the bits rounded away
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
  unsigned long long e = (unsigned long long)(63 - lz + 1023);
  if (mant >> 53) {  // rounding carried into bit 53
    mant >>= 1;
    ++e;
  }
  return __longlong_as_double((long long)(sign | (e << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// How the end of an fp64-split tile applies alpha and beta, classified once
// per thread: alpha = +-2^p (p in the normal range) goes into the int64
// sum's sign and the scaling exponent in integer arithmetic (one rounding in
// all), any other alpha takes one fp64 multiply; beta = 0 leaves C unread,
// beta = 1 costs one fp64 add, any other beta one fma.  The fp64 pipe is
// narrow on this GPU (one warp instruction occupies it for ~16 cycles): a
// finish that compared and multiplied in fp64 per output was bound by it.
struct FinishScale {
  bool a_neg;  // alpha = -2^p
  bool a_gen;  // alpha is not a power of two: multiply
  int a_p;     // alpha = +-2^p
  int b_kind;  // 0: beta = 0, 1: beta = 1, 2: other
};
__device__ __forceinline__ FinishScale finish_scale(double alpha, double beta) {
  FinishScale f;
  const unsigned long long u = (unsigned long long)__double_as_longlong(alpha);
  const int E = (int)((u >> 52) & 0x7FF);
  const bool pow2 = (u & 0xFFFFFFFFFFFFFull) == 0 && E >= 1 && E <= 2046;
  f.a_gen = !pow2;
  f.a_neg = pow2 && (u >> 63) != 0;
  f.a_p = pow2 ? E - 1023 : 0;
  f.b_kind = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
  return f;
}

// A network's fused epilogue: folds output value v into the row exponent
// bound and non-finite flag that the consuming step's split would compute
// for its row ci (exponent max(E, 1) - 1022 over the row's biased exponents
// E; E = 2047 flags the row and lists it once).  `e` is the largest exponent
// already folded by this thread (or warp) for ci, so that callers can reduce
// before the atomic; returns nothing.
__device__ __forceinline__ int f64_row_exp(double v, bool* bad) {
  const int E = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  *bad = E == 0x7FF;
  return (E > 1 ? E : 1) - 1022;
}
__device__ __forceinline__ void emit_mark(int32_t* flag, int32_t* list, int64_t ci) {
  if (atomicExch(&flag[ci], 1) == 0) {
    const int pos = atomicAdd(&list[0], 1);
    list[1 + pos] = (int32_t)ci;
  }
}

// Number of int64 entries the offset tables of a plan need.
inline int64_t table_entries(const Plan& p) {
  return 2 * p.m + 2 * p.n + 2 * p.k + 3 * p.l;
}

inline int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace famlies
