// Packing kernels: strided operand -> K-major slices for the TMA product.
//
// The pack is the one place an operand is re-laid out, and it fuses the
// tensor-to-matrix mapping (offset tables, Sec. 2.3 block-scatter item) with
// the precision split into slices.  Each 64 x 64 tile is read coalesced along
// the operand's unit-stride index into shared memory and written as 16-byte
// K-major chunks, so both the reads and the writes are full-width.  All of
// it is bound by HBM bandwidth.
#include <cstdint>

#include <cuda_bf16.h>

#include "packed.h"

namespace famlies {

namespace {

constexpr int PR = 64;      // rows per pack tile
constexpr int PK = 64;      // k per pack tile
constexpr int KCH = 1024;   // k per block in the exponent pass

__device__ __forceinline__ void mark_row(const PackOp& o, int64_t idx) {
  if (atomicExch(&o.flag[idx], 1) == 0) {
    const int pos = atomicAdd(&o.list[0], 1);
    o.list[1 + pos] = (int32_t)idx;
  }
}

// Exponent bound of one fp64 value: |x| < 2^(max(E,1) - 1022) for its biased
// exponent field E; E == 2047 marks Inf/NaN.
__device__ __forceinline__ void exp_update(double v, int& mx, int& bad) {
  const int E = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  if (E == 0x7FF) bad = 1;
  else mx = max(mx, max(E, 1) - 1022);
}

// Processes tiles b0, b0 + bstep, ... of one operand.
__device__ __forceinline__ void rowexp_body(const PackArgs& pa, const PackOp& o, int64_t b0,
                                            int64_t bstep) {
  const double* __restrict__ X = (const double*)o.x;
  const int64_t tiles_r = (o.rows + PR - 1) / PR, tiles_k = (pa.k + KCH - 1) / KCH;
  __shared__ int smx[4][PR], sbad[4][PR];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int64_t b = b0; b < tiles_r * tiles_k * pa.l; b += bstep) {
    const int64_t tr = b % tiles_r, rest = b / tiles_r;
    const int64_t tk = rest % tiles_k, il = rest / tiles_k;
    const int64_t lo = o.loff[il];
    const int64_t k0 = tk * KCH, k1 = min(pa.k, k0 + KCH);
    if (o.contig == 2) {
      // unit stride along k: a warp sweeps one row at a time
      for (int j = 0; j < PR / 8; ++j) {
        const int64_t gr = tr * PR + warp + 8 * j;
        if (gr >= o.rows) break;
        const int64_t base = lo + o.roff[gr];
        int mx = -1100, bad = 0;
        for (int64_t k = k0 + lane; k < k1; k += 32) exp_update(__ldg(X + base + o.koff[k]), mx, bad);
        mx = __reduce_max_sync(0xffffffffu, mx);
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (lane == 0) {
          atomicMax(&o.e[il * o.rows + gr], mx);
          if (bad) mark_row(o, il * o.rows + gr);
        }
      }
    } else {
      // neighbouring threads take neighbouring rows; 4 k-lanes per row
      const int r = tid % PR, kl = tid / PR;
      const int64_t gr = tr * PR + r;
      int mx = -1100, bad = 0;
      if (gr < o.rows) {
        const int64_t base = lo + o.roff[gr];
        for (int64_t k = k0 + kl; k < k1; k += 4) exp_update(__ldg(X + base + o.koff[k]), mx, bad);
      }
      smx[kl][r] = mx;
      sbad[kl][r] = bad;
      __syncthreads();
      if (tid < PR && gr < o.rows) {
        int m = max(max(smx[0][tid], smx[1][tid]), max(smx[2][tid], smx[3][tid]));
        int bd = sbad[0][tid] | sbad[1][tid] | sbad[2][tid] | sbad[3][tid];
        atomicMax(&o.e[il * o.rows + gr], m);
        if (bd) mark_row(o, il * o.rows + gr);
      }
      __syncthreads();
    }
  }
}

template <int PMODE>
struct PackT;
template <> struct PackT<PACK_BF16> { using T = uint16_t; };
template <> struct PackT<PACK_TF32> { using T = float; };
template <> struct PackT<PACK_F64> { using T = double; };

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int PMODE>
__device__ __forceinline__ void pack_body(const PackArgs& pa, const PackOp& o, int64_t b0,
                                          int64_t bstep) {
  using T = typename PackT<PMODE>::T;
  __shared__ T tile[PR][PK + 1];
  const T* __restrict__ X = (const T*)o.x;
  const int64_t tiles_r = (o.rows + PR - 1) / PR, tiles_k = (pa.k + PK - 1) / PK;
  const size_t slice_stride = (size_t)pa.l * o.rows * pa.kp;  // elements per slice
  const int tid = threadIdx.x;
  for (int64_t b = b0; b < tiles_r * tiles_k * pa.l; b += bstep) {
    const int64_t tr = b % tiles_r, rest = b / tiles_r;
    const int64_t tk = rest % tiles_k, il = rest / tiles_k;
    const int64_t lo = o.loff[il];
    for (int e = tid; e < PR * PK; e += 256) {
      int r, kk;
      if (o.contig == 2) { kk = e % PK; r = e / PK; } else { r = e % PR; kk = e / PR; }
      const int64_t gr = tr * PR + r, gk = tk * PK + kk;
      T v = T(0);
      if (gr < o.rows && gk < pa.k) v = __ldg(X + lo + o.roff[gr] + o.koff[gk]);
      tile[r][kk] = v;
    }
    __syncthreads();
    for (int it = tid; it < PR * 8; it += 256) {
      const int r = it >> 3, c = it & 7;
      const int64_t gr = tr * PR + r, gk0 = tk * PK + c * 8;
      if (gr >= o.rows || gk0 >= pa.k) continue;
      const size_t rowbase = ((size_t)il * o.rows + gr) * pa.kp + gk0;
      if constexpr (PMODE == PACK_BF16) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          w[j] = (uint32_t)tile[r][c * 8 + 2 * j] | ((uint32_t)tile[r][c * 8 + 2 * j + 1] << 16);
        *(uint4*)((uint16_t*)o.out + rowbase) = make_uint4(w[0], w[1], w[2], w[3]);
      } else if constexpr (PMODE == PACK_TF32) {
        uint32_t hi[8], lo32[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float x = tile[r][c * 8 + j];
          hi[j] = tf32_bits(x);
          lo32[j] = tf32_bits(x - __uint_as_float(hi[j]));
        }
        uint4* ph = (uint4*)((float*)o.out + rowbase);
        uint4* pl = (uint4*)((float*)o.out + slice_stride + rowbase);
        ph[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        ph[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
        pl[0] = make_uint4(lo32[0], lo32[1], lo32[2], lo32[3]);
        pl[1] = make_uint4(lo32[4], lo32[5], lo32[6], lo32[7]);
      } else {
        // Integer arithmetic only (the fp64 pipe is narrow): with
        // t = x * 2^-e_r in (-1, 1), F = round(t * 2^(b S)) is taken from
        // x's significand and exponent bits, then split into balanced base
        // 2^b digits from the bottom: d_S..d_2 in [-2^(b-1), 2^(b-1)), the
        // remaining top digit |d_1| <= 2^b.  F = sum_i d_i 2^(b (S - i)), so
        // |t - sum_i d_i 2^(-b i)| <= 2^(-b S - 1).
        const int64_t ri = il * o.rows + gr;
        const int ex = o.e[ri];
        const bool bad = o.flag[ri] != 0;
        const int b = pa.bits, S = pa.slices, bs = b * S;
        const int64_t half = (int64_t)1 << (b - 1), mask = ((int64_t)1 << b) - 1;
        int64_t F[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint64_t bitsx = (uint64_t)__double_as_longlong(tile[r][c * 8 + j]);
          const int E = (int)((bitsx >> 52) & 0x7FF);
          const uint64_t mant = (bitsx & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
          const int sh = max(E, 1) - 1075 - ex + bs;  // F = mant * 2^sh
          int64_t f = 0;
          if (!bad && mant != 0) {
            if (sh >= 0) f = (int64_t)(mant << sh);
            else if (sh > -63) f = (int64_t)((mant + (1ull << (-sh - 1))) >> (-sh));
          }
          F[j] = (bitsx >> 63) ? -f : f;
        }
        // Peeling the digits from the bottom (d = ((F + h) & mask) - h,
        // F = (F - d) >> b) is the same as adding the bias
        // h * (1 + 2^b + ... + 2^(b(S-2))) once and reading the lower S-1
        // digits as b-bit fields minus h; the top digit is what remains
        // above them (arithmetic shift).  No digit then waits on another.
        int64_t bias = 0;
        for (int s = 0; s < S - 1; ++s) bias += half << (b * s);
#pragma unroll
        for (int j = 0; j < 8; ++j) F[j] += bias;
        // slice 0 (most significant) first; each slice's digits are read
        // straight from the biased values, so only those stay in registers
        for (int s = 0; s < S; ++s) {
          const int sh2 = b * (S - 1 - s);
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const int32_t d0 = s == 0 ? (int32_t)(F[j] >> sh2)
                                      : (int32_t)((F[j] >> sh2) & mask) - (int32_t)half;
            const int32_t d1 = s == 0 ? (int32_t)(F[j + 1] >> sh2)
                                      : (int32_t)((F[j + 1] >> sh2) & mask) - (int32_t)half;
            // small integers are exact in fp32 and bf16: 1.5 * 2^23 + d holds
            // d in its low significand bits, and the subtraction is exact
            const float f0 = __int_as_float(0x4B400000 + d0) - 12582912.0f;
            const float f1 = __int_as_float(0x4B400000 + d1) - 12582912.0f;
            w[j / 2] = (__float_as_uint(f0) >> 16) | (__float_as_uint(f1) & 0xFFFF0000u);
          }
          *(uint4*)((uint16_t*)o.out + (size_t)s * slice_stride + rowbase) =
              make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void fixup_body(const GemmArgs& g, const int32_t* __restrict__ list_a,
                                           const int32_t* __restrict__ list_b,
                                           const int32_t* __restrict__ flag_a) {
  const int64_t na = list_a[0], nb = list_b[0];
  if (na == 0 && nb == 0) return;
  const double* __restrict__ A = (const double*)g.a;
  const double* __restrict__ B = (const double*)g.b;
  double* __restrict__ C = (double*)g.c;
  const int64_t total = na * g.n + nb * g.m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t m, n, il;
    if (idx < na * g.n) {
      const int64_t e = list_a[1 + idx / g.n];
      il = e / g.m;
      m = e % g.m;
      n = idx % g.n;
    } else {
      const int64_t j = idx - na * g.n;
      const int64_t e = list_b[1 + j / g.m];
      il = e / g.n;
      n = e % g.n;
      m = j % g.m;
      if (flag_a[il * g.m + m]) continue;  // done by the row pass
    }
    const int64_t ab = g.t.al[il] + g.t.am[m], bb = g.t.bl[il] + g.t.bn[n];
    double acc = 0.0;
    for (int64_t k = 0; k < g.k; ++k) acc = fma(A[ab + g.t.ak[k]], B[bb + g.t.bk[k]], acc);
    double* p = C + g.t.cl[il] + g.t.cm[m] + g.t.cn[n];
    double v = g.alpha * acc;
    if (g.beta != 0.0) v = fma(g.beta, *p, v);
    *p = v;
  }
}

int grid_for(int64_t blocks) {
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

// One problem per launch: blockIdx.z picks the operand.
__global__ void __launch_bounds__(256) k_rowexp(PackArgs pa) {
  rowexp_body(pa, pa.op[blockIdx.z], blockIdx.x, gridDim.x);
}

template <int PMODE>
__global__ void __launch_bounds__(256) k_pack(PackArgs pa) {
  pack_body<PMODE>(pa, pa.op[blockIdx.z], blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_fixup(GemmArgs g, const int32_t* list_a,
                                               const int32_t* list_b, const int32_t* flag_a) {
  fixup_body(g, list_a, list_b, flag_a);
}

// Many problems per launch.  The tiles of every (problem, operand) segment
// are numbered consecutively (off[s] = first tile of segment s = 2p + op,
// off[nseg] = total); the blocks stride over that flat range, so large and
// small problems share the grid evenly.
__device__ __forceinline__ int segment_of(const int64_t* off, int nseg, int64_t g) {
  int lo = 0, hi = nseg;  // largest s with off[s] <= g
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int64_t kOneTile = (int64_t)1 << 62;  // a step that ends a body's loop after one tile

__global__ void __launch_bounds__(256) k_rowexp_grouped(const PackArgs* __restrict__ pas,
                                                        const int64_t* __restrict__ off, int nseg) {
  const int64_t total = off[nseg];
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int s = segment_of(off, nseg, g);
    const PackArgs& pa = pas[s >> 1];
    rowexp_body(pa, pa.op[s & 1], g - off[s], kOneTile);
  }
}

template <int PMODE>
__global__ void __launch_bounds__(256) k_pack_grouped(const PackArgs* __restrict__ pas,
                                                      const int64_t* __restrict__ off, int nseg) {
  const int64_t total = off[nseg];
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int s = segment_of(off, nseg, g);
    const PackArgs& pa = pas[s >> 1];
    pack_body<PMODE>(pa, pa.op[s & 1], g - off[s], kOneTile);
  }
}

__global__ void __launch_bounds__(256) k_fixup_grouped(const GemmArgs* __restrict__ gs,
                                                       const PackArgs* __restrict__ pas, int n) {
  for (int p = blockIdx.y; p < n; p += gridDim.y)
    fixup_body(gs[p], pas[p].op[0].list, pas[p].op[1].list, pas[p].op[0].flag);
}

}  // namespace

static void prefer_shared_carveout();

int64_t rowexp_tiles(int64_t rows, int64_t k, int64_t l) {
  return ((rows + PR - 1) / PR) * ((k + KCH - 1) / KCH) * l;
}
int64_t pack_tiles(int64_t rows, int64_t k, int64_t l) {
  return ((rows + PR - 1) / PR) * ((k + PK - 1) / PK) * l;
}

cudaError_t launch_rowexp_grouped(const PackArgs* pas, const int64_t* off, int n, int64_t total,
                                  cudaStream_t s) {
  if (n <= 0 || total <= 0) return cudaSuccess;
  k_rowexp_grouped<<<grid_for(total), 256, 0, s>>>(pas, off, 2 * n);
  return cudaGetLastError();
}

cudaError_t launch_pack_grouped(int pmode, const PackArgs* pas, const int64_t* off, int n,
                                int64_t total, cudaStream_t s) {
  if (n <= 0 || total <= 0) return cudaSuccess;
  prefer_shared_carveout();
  const int grid = grid_for(total);
  if (pmode == PACK_BF16) k_pack_grouped<PACK_BF16><<<grid, 256, 0, s>>>(pas, off, 2 * n);
  else if (pmode == PACK_TF32) k_pack_grouped<PACK_TF32><<<grid, 256, 0, s>>>(pas, off, 2 * n);
  else k_pack_grouped<PACK_F64><<<grid, 256, 0, s>>>(pas, off, 2 * n);
  return cudaGetLastError();
}

cudaError_t launch_fixup_grouped(const GemmArgs* gs, const PackArgs* pas, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid(4, (unsigned)(n > 32768 ? 32768 : n));
  k_fixup_grouped<<<grid, 256, 0, s>>>(gs, pas, n);
  return cudaGetLastError();
}

cudaError_t launch_rowexp(const PackArgs& pa, cudaStream_t s) {
  int64_t blocks = 0;
  for (int i = 0; i < 2; ++i) {
    const int64_t b = ((pa.op[i].rows + PR - 1) / PR) * ((pa.k + KCH - 1) / KCH) * pa.l;
    blocks = b > blocks ? b : blocks;
  }
  k_rowexp<<<dim3(grid_for(blocks), 1, 2), 256, 0, s>>>(pa);
  return cudaGetLastError();
}

// The pack kernels stage 64 x 64 tiles in shared memory (33 KB for fp64):
// ask for the largest shared-memory carveout so that several blocks fit
// per SM and keep enough loads in flight.
static void prefer_shared_carveout() {
  static bool done = false;
  if (done) return;
  const int c = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(k_pack<PACK_BF16>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_pack<PACK_TF32>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_pack<PACK_F64>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_pack_grouped<PACK_BF16>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_pack_grouped<PACK_TF32>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaFuncSetAttribute(k_pack_grouped<PACK_F64>, cudaFuncAttributePreferredSharedMemoryCarveout, c);
  cudaGetLastError();
  done = true;
}

cudaError_t launch_pack(int pmode, const PackArgs& pa, cudaStream_t s) {
  prefer_shared_carveout();
  int64_t blocks = 0;
  for (int i = 0; i < 2; ++i) {
    const int64_t b = ((pa.op[i].rows + PR - 1) / PR) * ((pa.k + PK - 1) / PK) * pa.l;
    blocks = b > blocks ? b : blocks;
  }
  const dim3 grid(grid_for(blocks), 1, 2);
  if (pmode == PACK_BF16) k_pack<PACK_BF16><<<grid, 256, 0, s>>>(pa);
  else if (pmode == PACK_TF32) k_pack<PACK_TF32><<<grid, 256, 0, s>>>(pa);
  else k_pack<PACK_F64><<<grid, 256, 0, s>>>(pa);
  return cudaGetLastError();
}

cudaError_t launch_fixup(const GemmArgs& g, const PackArgs& pa, cudaStream_t s) {
  k_fixup<<<num_sms() * 2, 256, 0, s>>>(g, pa.op[0].list, pa.op[1].list, pa.op[0].flag);
  return cudaGetLastError();
}

}  // namespace famlies
