// Packing kernels: strided operand -> K-major slices for the TMA product.
//
// The pack is the one place an operand is re-laid out, and it fuses the
// tensor-to-matrix mapping (offset tables, Sec. 2.3 block-scatter item) with
// the precision split into slices.  Each 64 x 64 tile is read coalesced along
// the operand's unit-stride index into shared memory and written as 16-byte
// K-major chunks, so both the reads and the writes are full-width.  All of
// it is bound by HBM bandwidth.
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "packed.h"

namespace famlies {

namespace {

constexpr int PR = 64;      // rows per pack tile
constexpr int PK = 64;      // k per pack tile
constexpr int KCH = 1024;   // k per block in the exponent pass

__host__ __device__ inline int64_t n_pack_tiles(int64_t rows, int64_t k, int64_t l) {
  return ((rows + PR - 1) / PR) * ((k + PK - 1) / PK) * l;
}

__device__ __forceinline__ void mark_row(const PackOp& o, int64_t idx) {
  if (atomicExch(&o.flag[idx], 1) == 0) {
    const int pos = atomicAdd(&o.list[0], 1);
    o.list[1 + pos] = (int32_t)idx;
  }
}

// Element (p, q) of a symmetric n x n matrix stored as its lower triangle,
// column by column: column q holds rows q..n-1 and starts at q n - q (q-1)/2.
__host__ __device__ __forceinline__ int64_t sym_at(int64_t p, int64_t q, int64_t n) {
  if (p < q) {
    const int64_t t = p;
    p = q;
    q = t;
  }
  return q * n - q * (q - 1) / 2 + (p - q);
}

// Offsets of row r and contracted index k of an operand: affine when the
// class fused to one mode, otherwise read from the offset tables.
__device__ __forceinline__ int64_t row_off(const PackOp& o, int64_t r) {
  return (o.affine & 1) ? r * o.rs : o.roff[r];
}
__device__ __forceinline__ int64_t k_off(const PackOp& o, int64_t k) {
  return (o.affine & 2) ? k * o.ks : o.koff[k];
}

// Exponent bound of one fp64 value: |x| < 2^(max(E,1) - 1022) for its biased
// exponent field E; E == 2047 marks Inf/NaN.
__device__ __forceinline__ void exp_update(double v, int& mx, int& bad) {
  const int E = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
  if (E == 0x7FF) bad = 1;
  else mx = max(mx, max(E, 1) - 1022);
}

// Exponent bound and non-finite flag over X[base + k_off(k)] for k = k0,
// k0 + step, ... < k1, with U independent loads in flight per thread (the
// offsets may come from a table: one more dependent load each).
template <int U>
__device__ __forceinline__ void scan_row(const PackOp& o, const double* __restrict__ X, int64_t base,
                                         int64_t k0, int64_t k1, int step, int& mx, int& bad) {
  if (o.affine & 2) {  // affine offsets: the plain loop measures faster
    for (int64_t k = k0; k < k1; k += step) exp_update(__ldg(X + base + k * o.ks), mx, bad);
    return;
  }
  for (int64_t k = k0; k < k1; k += (int64_t)U * step) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      // past the end: the last element again (it changes neither result),
      // so that no load is predicated
      const int64_t kk = min(k + (int64_t)u * step, k1 - 1);
      v[u] = __ldg(X + base + k_off(o, kk));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) exp_update(v[u], mx, bad);
  }
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
        const int64_t base = lo + row_off(o, gr);
        int mx = -1100, bad = 0;
        scan_row<4>(o, X, base, k0 + lane, k1, 32, mx, bad);
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
        const int64_t base = lo + row_off(o, gr);
        scan_row<4>(o, X, base, k0 + kl, k1, 4, mx, bad);
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

// fp64 split of 8 consecutive values of one row into S slices of
// kSplitBits = 8-bit digits, in integer arithmetic only (the fp64 pipe is
// narrow).  With t = x * 2^-e_r in (-1, 1), F = round(t * 2^(8 S)) is taken
// from x's significand and exponent bits, then split into balanced base-256
// digits: d_S..d_2 in [-128, 128), the remaining top digit |d_1| <= 256
// (all exact in bf16's 8-bit significand), and F = sum_i d_i 2^(8 (S - i)),
// so |t - sum_i d_i 2^(-8 i)| <= 2^(-8 S - 1).  S is a template argument so
// that every digit is a fixed byte of F.
template <int S>
__device__ __forceinline__ void split8(const double* v, int ex, bool bad, uint16_t* out,
                                       size_t slice_stride) {
  static_assert(kSplitBits == 8, "digits are read as bytes");
  static_assert(S >= 2 && S <= kMaxSplitSlices, "F must fit in 63 bits");
  constexpr int bs = 8 * S, top = 8 * (S - 1);
  if (bad) {  // recomputed natively afterwards: zero slices
#pragma unroll
    for (int s = 0; s < S; ++s) *(uint4*)(out + (size_t)s * slice_stride) = make_uint4(0, 0, 0, 0);
    return;
  }
  // Peeling the digits from the bottom (d = ((F + 128) & 255) - 128,
  // F = (F - d) >> 8) is the same as adding the bias 0x80 in each of the
  // lower S-1 bytes once and reading those bytes minus 128; the top digit
  // is what remains above them (arithmetic shift).  No digit then waits on
  // another.
  constexpr int64_t bias = [] {
    int64_t t = 0;
    for (int s = 0; s < S - 1; ++s) t |= (int64_t)0x80 << (8 * s);
    return t;
  }();
  uint32_t lo[8], hi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t u = (uint64_t)__double_as_longlong(v[j]);
    const int E = (int)(((uint32_t)(u >> 32) >> 20) & 0x7FF);
    const uint64_t mant = (u & 0xFFFFFFFFFFFFFull) | ((uint64_t)(E != 0) << 52);
    // F = mant * 2^-n; |x| < 2^ex bounds n below by 53 - bs
    const int n = ex + (1075 - bs) - max(E, 1);
    uint64_t f;
    if constexpr (bs > 53) {
      f = n <= 0 ? mant << (-n) : (n <= 54 ? (mant + (1ull << (n - 1))) >> n : 0);
    } else {
      f = n <= 54 ? (mant + (1ull << (n - 1))) >> n : 0;
    }
    const uint64_t F = (uint64_t)(((int64_t)u < 0 ? -(int64_t)f : (int64_t)f) + bias);
    lo[j] = (uint32_t)F;
    hi[j] = (uint32_t)(F >> 32);
  }
  // slice 0 (most significant) first.  Small integers are exact in fp32
  // and bf16: the float with bits 0x4B400000 + d is 1.5 * 2^23 + d, so
  // subtracting 1.5 * 2^23 gives d exactly.  A lower digit's byte is
  // permuted straight into those bits and 128 more is subtracted.
#pragma unroll
  for (int s = 0; s < S; ++s) {
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (s == 0) {
        const int32_t d = (int32_t)(((int64_t)hi[j] << 32 | lo[j]) >> top);
        f[j] = __int_as_float(0x4B400000 + d) - 12582912.0f;
      } else {
        const int byte = S - 1 - s;  // digit s sits in byte `byte` of F
        const uint32_t word = byte < 4 ? lo[j] : hi[j];
        const uint32_t w = __byte_perm(word, 0x4B400000u, 0x7650 | (byte & 3));
        f[j] = __uint_as_float(w) - (12582912.0f + 128.0f);
      }
    }
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      w[j] = __byte_perm(__float_as_uint(f[2 * j]), __float_as_uint(f[2 * j + 1]), 0x7632);
    *(uint4*)(out + (size_t)s * slice_stride) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// One tile of one operand to pack: tile b of pa.op[...] = *o.
struct PackTile {
  const PackArgs* pa;
  const PackOp* o;
  int64_t b;
};

// Asynchronous global -> shared copy of one element, zero-filled when
// `valid` is false (no bytes are then read), so that the next tile's loads
// are in flight while the current tile is split and stored.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int TLD = PK + 1;  // shared tile row length (padded against bank conflicts)

// Stages a PR x PK tile of the operand in shared memory (buf[r][kk]),
// reading along the operand's unit-stride index: with unit stride along k
// the threads of a warp take consecutive k of one row, otherwise
// consecutive rows at one k.  Entries past the operand's edge are zero.
// Entries a thread moves per tile (PR = PK = 64 with 256 threads: 16), in
// the order load_tile visits them; entry i of thread t is row
// t / PK + 4 i, column t % PK (unit stride along k) or row t % PR, column
// t / PR + 4 i (otherwise).
constexpr int PER_THREAD = PR * PK / 256;

__device__ __forceinline__ int stage_slot(int contig, int i) {
  return contig == 2 ? (threadIdx.x / PK + i * (256 / PK)) * TLD + threadIdx.x % PK
                     : (threadIdx.x % PR) * TLD + threadIdx.x / PR + i * (256 / PR);
}

// 4- and 8-byte values go straight to shared memory by asynchronous copies;
// 2-byte values (no asynchronous copy that small) are loaded into registers
// (`regs`) and stored by store_regs once the current tile is converted.
template <int PMODE>
__device__ __forceinline__ void load_tile(const PackTile& t, typename PackT<PMODE>::T* buf,
                                          typename PackT<PMODE>::T (&regs)[PER_THREAD]) {
  using T = typename PackT<PMODE>::T;
  constexpr int NT = 256;
  const PackArgs& pa = *t.pa;
  const PackOp& o = *t.o;
  const T* __restrict__ X = (const T*)o.x;
  const int64_t tiles_r = (o.rows + PR - 1) / PR, tiles_k = (pa.k + PK - 1) / PK;
  const int64_t tr = t.b % tiles_r, rest = t.b / tiles_r;
  const int64_t tk = rest % tiles_k, il = rest / tiles_k;
  const int64_t r0 = tr * PR, k0 = tk * PK;
  const int rmax = (int)min((int64_t)PR, o.rows - r0), kmax = (int)min((int64_t)PK, pa.k - k0);
  const T* const base = X + o.loff[il];
  int slot = 0;  // entries are visited in order: the i-th put is entry i
  auto put = [&](T* dst, const T* src, bool ok) {
    if constexpr (sizeof(T) >= 4) cp_async_elem<sizeof(T)>(dst, ok ? src : X, ok);
    else regs[slot] = ok ? __ldg(src) : T(0);
    ++slot;
  };
  if (o.contig == 2) {
    const int kk = threadIdx.x % PK;
    const bool kok = kk < kmax;
    const T* src = base + (kok ? k_off(o, k0 + kk) : 0);
    T* dst = buf + kk;
    if (o.affine & 1) {
      const int64_t step = (NT / PK) * o.rs;
      src += (r0 + threadIdx.x / PK) * o.rs;
#pragma unroll
      for (int i = 0; i < PR / (NT / PK); ++i, src += step) {
        const int r = threadIdx.x / PK + i * (NT / PK);
        put(dst + r * TLD, src, kok && r < rmax);
      }
    } else {
      // the table reads first, all in flight together, then the copies
      constexpr int NI = PR / (NT / PK);
      int64_t off[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int r = threadIdx.x / PK + i * (NT / PK);
        off[i] = kok && r < rmax ? o.roff[r0 + r] : -1;
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int r = threadIdx.x / PK + i * (NT / PK);
        put(dst + r * TLD, src + (off[i] >= 0 ? off[i] : 0), off[i] >= 0);
      }
    }
  } else {
    const int r = threadIdx.x % PR;
    const bool rok = r < rmax;
    const T* src = base + (rok ? row_off(o, r0 + r) : 0);
    T* dst = buf + r * TLD;
    if (o.affine & 2) {
      const int64_t step = (NT / PR) * o.ks;
      src += (k0 + threadIdx.x / PR) * o.ks;
#pragma unroll
      for (int i = 0; i < PK / (NT / PR); ++i, src += step) {
        const int kk = threadIdx.x / PR + i * (NT / PR);
        put(dst + kk, src, rok && kk < kmax);
      }
    } else {
      constexpr int NI = PK / (NT / PR);
      int64_t off[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int kk = threadIdx.x / PR + i * (NT / PR);
        off[i] = rok && kk < kmax ? o.koff[k0 + kk] : -1;
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int kk = threadIdx.x / PR + i * (NT / PR);
        put(dst + kk, src + (off[i] >= 0 ? off[i] : 0), off[i] >= 0);
      }
    }
  }
}

template <int PMODE>
__device__ __forceinline__ void store_regs(const PackTile& t, typename PackT<PMODE>::T* buf,
                                           const typename PackT<PMODE>::T (&regs)[PER_THREAD]) {
#pragma unroll
  for (int i = 0; i < PER_THREAD; ++i) buf[stage_slot(t.o->contig, i)] = regs[i];
}

// Converts a staged tile and writes it as 16-byte K-major chunks of every
// slice.  TR: the staged tile holds the transpose (buf[kk][r]), as the
// symmetric pack uses one staged block for both of its mirror images.
template <int PMODE, bool TR = false>
__device__ __forceinline__ void emit_tile(const PackTile& t, const typename PackT<PMODE>::T* buf) {
  const PackArgs& pa = *t.pa;
  const PackOp& o = *t.o;
  const int64_t tiles_r = (o.rows + PR - 1) / PR, tiles_k = (pa.k + PK - 1) / PK;
  const int64_t tr = t.b % tiles_r, rest = t.b / tiles_r;
  const int64_t tk = rest % tiles_k, il = rest / tiles_k;
  const size_t slice_stride = (size_t)pa.l * o.rows * pa.kp;  // elements per slice
  for (int it = threadIdx.x; it < PR * 8; it += 256) {
    const int r = it >> 3, c = it & 7;
    const int64_t gr = tr * PR + r, gk0 = tk * PK + c * 8;
    if (gr >= o.rows || gk0 >= pa.k) continue;
    const size_t rowbase = ((size_t)il * o.rows + gr) * pa.kp + gk0;
    typename PackT<PMODE>::T vt[8];
    if constexpr (TR) {
#pragma unroll
      for (int j = 0; j < 8; ++j) vt[j] = buf[(c * 8 + j) * TLD + r];
    }
    const auto* v = TR ? vt : buf + r * TLD + c * 8;
    if constexpr (PMODE == PACK_BF16) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = (uint32_t)v[2 * j] | ((uint32_t)v[2 * j + 1] << 16);
      *(uint4*)((uint16_t*)o.out + rowbase) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (PMODE == PACK_TF32) {
      uint32_t hi[8], lo32[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float x = v[j];
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
      const int64_t ri = il * o.rows + gr;
      uint16_t* out = (uint16_t*)o.out + rowbase;
      const int ex = o.e[ri];
      const bool bad = o.flag[ri] != 0;
      switch (pa.slices) {
        case 2: split8<2>(v, ex, bad, out, slice_stride); break;
        case 3: split8<3>(v, ex, bad, out, slice_stride); break;
        case 4: split8<4>(v, ex, bad, out, slice_stride); break;
        case 5: split8<5>(v, ex, bad, out, slice_stride); break;
        case 6: split8<6>(v, ex, bad, out, slice_stride); break;
        default: split8<7>(v, ex, bad, out, slice_stride); break;
      }
    }
  }
}

// ---------------------------------------------------------------- symmetric
// The operand is the lower triangle of a symmetric n x n matrix stored
// column by column (famlies_contract_sym).  Both kernels walk its PR x PK
// blocks (P, Q) with P >= Q, numbered row by row of the block triangle, and
// read each stored element once, along the stored columns.

// Block (P, Q) of lower-triangle block number t: t = P (P + 1) / 2 + Q.
__device__ __forceinline__ void tri_block(int64_t t, int64_t& P, int64_t& Q) {
  int64_t p = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((p + 1) * (p + 2) / 2 <= t) ++p;
  while (p * (p + 1) / 2 > t) --p;
  P = p;
  Q = t - p * (p + 1) / 2;
}

// Row exponent bounds: a stored element (p, q) bounds row p and, being also
// element (q, p), row q.
__device__ __forceinline__ void rowexp_sym_body(const PackOp& o, int32_t* __restrict__ scr) {
  const double* __restrict__ X = (const double*)o.x;
  const int64_t n = o.sym_n, nb = (n + PR - 1) / PR, nblk = nb * (nb + 1) / 2;
  __shared__ int rmx[4][PR], rbad[4][PR];
  __shared__ int cmx[2][4][PK / 4], cbad[2][4][PK / 4];
  const int tid = threadIdx.x, r = tid % PR, qi = tid / PR, lane = tid & 31, wh = (tid >> 5) & 1;
  for (int64_t t = blockIdx.x; t < nblk; t += gridDim.x) {
    int64_t P, Q;
    tri_block(t, P, Q);
    const int64_t p = P * PR + r;
    int mxr = -1100, badr = 0;
#pragma unroll
    for (int i = 0; i < PK / 4; ++i) {
      const int64_t q = Q * PK + qi + 4 * i;
      int mxc = -1100, badc = 0;
      if (p < n && q < n && p >= q) {  // consecutive p of one stored column
        exp_update(__ldg(X + sym_at(p, q, n)), mxc, badc);
        mxr = max(mxr, mxc);
        badr |= badc;
      }
      mxc = __reduce_max_sync(0xffffffffu, mxc);
      badc = __reduce_or_sync(0xffffffffu, badc);
      if (lane == 0) {
        cmx[wh][qi][i] = mxc;
        cbad[wh][qi][i] = badc;
      }
    }
    rmx[qi][r] = mxr;
    rbad[qi][r] = badr;
    __syncthreads();
    // the tile's maxima go to its scratch entry (k_rowexp_sym_reduce takes
    // each row's maximum over its tiles): rows P * PR + r at [0, PR), the
    // mirror images, rows Q * PK + j, at [PR, PR + PK)
    if (tid < PR) {
      const int64_t pp = P * PR + tid;
      const int m = max(max(rmx[0][tid], rmx[1][tid]), max(rmx[2][tid], rmx[3][tid]));
      const int b = rbad[0][tid] | rbad[1][tid] | rbad[2][tid] | rbad[3][tid];
      scr[t * (PR + PK) + tid] = m;
      if (pp < n && b) mark_row(o, pp);
    } else if (tid < PR + PK) {
      const int j = tid - PR, jq = j % 4, ji = j / 4;
      const int64_t qq = Q * PK + jq + 4 * ji;
      const int m = max(cmx[0][jq][ji], cmx[1][jq][ji]);
      const int b = cbad[0][jq][ji] | cbad[1][jq][ji];
      scr[t * (PR + PK) + PR + jq + 4 * ji] = m;
      if (qq < n && b) mark_row(o, qq);
    }
    __syncthreads();
  }
}

// Stages block (P, Q): buf[r][kk] = element (P PR + r, Q PK + kk), read along
// the stored columns (diagonal blocks also read their mirrored half).
__device__ __forceinline__ void load_sym_block(const PackOp& o, int64_t P, int64_t Q, double* buf) {
  const double* __restrict__ X = (const double*)o.x;
  const int64_t n = o.sym_n;
  const int r = threadIdx.x % PR;
  const int64_t p = P * PR + r;
#pragma unroll
  for (int i = 0; i < PER_THREAD; ++i) {
    const int kk = threadIdx.x / PR + i * (256 / PR);
    const int64_t q = Q * PK + kk;
    const bool ok = p < n && q < n;
    cp_async_elem<8>(buf + r * TLD + kk, ok ? X + sym_at(p, q, n) : X, ok);
  }
}

// Slices of the symmetric operand: block (P, Q) gives rows P x k Q and, off
// the diagonal, its transpose, rows Q x k P; double-buffered like
// pack_pipeline.
__device__ __forceinline__ void pack_sym_body(const PackArgs& pa, const PackOp& o) {
  extern __shared__ __align__(16) unsigned char pack_smem[];
  double* const buf0 = (double*)pack_smem;
  auto buf = [&](int j) { return buf0 + (j & 1) * (PR * TLD); };
  const int64_t n = o.sym_n, nb = (n + PR - 1) / PR, nblk = nb * (nb + 1) / 2;
  if ((int64_t)blockIdx.x >= nblk) return;
  int64_t P, Q;
  tri_block(blockIdx.x, P, Q);
  load_sym_block(o, P, Q, buf(0));
  cp_async_commit();
  int i = 0;
  for (int64_t t = blockIdx.x; t < nblk; t += gridDim.x, ++i) {
    int64_t Pn = P, Qn = Q;
    if (t + gridDim.x < nblk) {
      tri_block(t + gridDim.x, Pn, Qn);
      load_sym_block(o, Pn, Qn, buf(i + 1));
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    // tile numbers as emit_tile decodes them: row block + nb * k block
    emit_tile<PACK_F64>(PackTile{&pa, &o, P + nb * Q}, buf(i));
    if (P != Q) emit_tile<PACK_F64, true>(PackTile{&pa, &o, Q + nb * P}, buf(i));
    __syncthreads();
    P = Pn;
    Q = Qn;
  }
}

// Dynamic shared memory of the pack kernels: two staged tiles.
template <int PMODE>
constexpr int pack_smem_bytes() {
  return 2 * PR * TLD * (int)sizeof(typename PackT<PMODE>::T);
}

// Packs tiles g0, g0 + gstep, ... < total (loc maps a flat index to its
// tile) with two shared-memory buffers: the loads of the next tile are
// issued before the current one is converted.
template <int PMODE, class Locate>
__device__ __forceinline__ void pack_pipeline(int64_t g0, int64_t gstep, int64_t total, Locate loc) {
  using T = typename PackT<PMODE>::T;
  extern __shared__ __align__(16) unsigned char pack_smem[];
  T* const buf0 = (T*)pack_smem;
  auto buf = [&](int j) { return buf0 + (j & 1) * (PR * TLD); };
  if (g0 >= total) return;
  T regs[PER_THREAD];
  PackTile cur = loc(g0);
  load_tile<PMODE>(cur, buf(0), regs);
  if constexpr (sizeof(T) < 4) store_regs<PMODE>(cur, buf(0), regs);
  cp_async_commit();
  int i = 0;
  for (int64_t g = g0; g < total; g += gstep, ++i) {
    PackTile nxt = cur;
    const bool more = g + gstep < total;
    if (more) {
      nxt = loc(g + gstep);
      load_tile<PMODE>(nxt, buf(i + 1), regs);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of the current tile have landed
    __syncthreads();     // ... and everyone else's; the tile before is emitted
    emit_tile<PMODE>(cur, buf(i));
    if constexpr (sizeof(T) < 4) {
      // the register-held loads of the next tile return while this one is
      // converted; buf(i + 1) was last read by the emit before the barrier
      if (more) store_regs<PMODE>(nxt, buf(i + 1), regs);
    } else {
      __syncthreads();   // the buffer is free for the tile after next
    }
    cur = nxt;
  }
}

// ---------------------------------------------------------- generated operands
// Values of a generated operand's 64 x 64 tile (row tile tr, k tile tk)
// into buf[r * TLD + kk], zero past its edges; thread t computes row t % PR.
// Band: sub/diag/sup against the affine source (the same arithmetic as
// band_at everywhere).  Khatri-Rao: the factor digits of the tile's k
// offsets are decoded once per tile into dig (shared, [factor][kk]), then
// each value is the product of its factors' entries, in factor order.
template <class T>
__device__ __forceinline__ void gen_tile(const PackArgs& pa, const PackOp& o, int64_t tr, int64_t tk, T* buf,
                                         int32_t* dig) {
  const int r = threadIdx.x % PR;
  const int64_t row = tr * PR + r;
  if (o.gen == 1) {
    const T* __restrict__ X = (const T*)o.x;
#pragma unroll 4
    for (int i = 0; i < PER_THREAD; ++i) {
      const int kk = threadIdx.x / PR + i * (256 / PR);
      const int64_t p = tk * PK + kk;
      buf[r * TLD + kk] =
          (row < o.rows && p < pa.k) ? band_at<T>(X, row * o.rs, nullptr, o.ks, p, pa.k, o.band) : T(0);
    }
    return;
  }
  // Khatri-Rao: lanes run along k, so that a warp reads consecutive rows of
  // the first factor (its fastest digit) and one row of the others
  const Krp& q = o.krp;
  for (int i = threadIdx.x; i < q.nf * PK; i += 256) {
    const int f = i / PK, kk = i % PK;
    const int64_t k = tk * PK + kk;
    const int64_t off = k < pa.k ? ((o.affine & 2) ? k * o.ks : o.koff[k]) : 0;
    dig[i] = (int32_t)((off / q.st[f]) % q.ext[f]);
  }
  __syncthreads();
  const int kk = threadIdx.x % PK;
  const int64_t k = tk * PK + kk;
#pragma unroll 4
  for (int i = 0; i < PER_THREAD; ++i) {
    const int rr = threadIdx.x / PK + i * (256 / PK);
    const int64_t rw = tr * PR + rr;
    T v = T(0);
    if (rw < o.rows && k < pa.k)
      for (int f = 0; f < q.nf; ++f) {
        const T u = ((const T*)q.u[f])[(int64_t)dig[f * PK + kk] * q.rs[f] + rw * q.cs[f]];
        v = f == 0 ? u : v * u;
      }
    buf[rr * TLD + kk] = v;
  }
}

// Row exponents and non-finite flags of a generated operand (fp64 split):
// per tile, thread (r, g) scans row r's k = 16 g .. 16 g + 15 of the staged
// values.
__device__ __forceinline__ void rowexp_gen_body(const PackArgs& pa, const PackOp& o) {
  __shared__ double buf[PR * TLD];
  __shared__ int32_t dig[kMaxModes * PK];
  __shared__ int smx[4][PR], sbad[4][PR];
  const int64_t tiles_r = (o.rows + PR - 1) / PR, tiles_k = (pa.k + PK - 1) / PK;
  const int64_t items = tiles_r * tiles_k;
  const int r = threadIdx.x % PR, g = threadIdx.x / PR;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t tr = it % tiles_r, tk = it / tiles_r;
    gen_tile<double>(pa, o, tr, tk, buf, dig);
    __syncthreads();
    int mx = -1100, bad = 0;
    const int64_t krem = pa.k - tk * PK;
    const int kmax = krem < PK ? (int)krem : PK;
#pragma unroll 4
    for (int j = 0; j < PK / 4; ++j)
      if (g * (PK / 4) + j < kmax) exp_update(buf[r * TLD + g * (PK / 4) + j], mx, bad);
    smx[g][r] = mx;
    sbad[g][r] = bad;
    __syncthreads();
    if (threadIdx.x < PR) {
      const int t = threadIdx.x;
      const int64_t rr = tr * PR + t;
      const int m = max(max(smx[0][t], smx[1][t]), max(smx[2][t], smx[3][t]));
      const int bd = sbad[0][t] | sbad[1][t] | sbad[2][t] | sbad[3][t];
      if (rr < o.rows && m > -1100) atomicMax(&o.e[rr], m);
      if (rr < o.rows && bd) mark_row(o, rr);
    }
    __syncthreads();
  }
}

// Slices of a generated operand: each tile's values are staged in shared
// memory and emitted like any staged tile.
template <int PMODE>
__device__ __forceinline__ void pack_gen_body(const PackArgs& pa, const PackOp& o) {
  using T = typename PackT<PMODE>::T;
  extern __shared__ __align__(16) unsigned char pack_smem[];
  __shared__ int32_t dig[kMaxModes * PK];
  T* const buf = (T*)pack_smem;
  const int64_t tiles_r = (o.rows + PR - 1) / PR, tiles_k = (pa.k + PK - 1) / PK;
  const int64_t items = tiles_r * tiles_k;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    gen_tile<T>(pa, o, it % tiles_r, it / tiles_r, buf, dig);
    __syncthreads();
    // tile number as emit_tile decodes it: row tile + tiles_r * k tile
    emit_tile<PMODE>(PackTile{&pa, &o, it}, buf);
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
    if (!tri_keep(g.tri, m, n)) continue;  // outside the updated triangle
    const int64_t ab = g.t.al[il] + g.t.am[m], bb = g.t.bl[il] + g.t.bn[n];
    double acc = 0.0;
    if (g.krp_op) {
      for (int64_t k = 0; k < g.k; ++k) {
        const double va = g.krp_op == 1 ? krp_at<double>(g.krp, m, g.t.ak[k]) : A[ab + g.t.ak[k]];
        const double vb = g.krp_op == 2 ? krp_at<double>(g.krp, n, g.t.bk[k]) : B[bb + g.t.bk[k]];
        acc = fma(va, vb, acc);
      }
    } else if (g.band_op) {
      for (int64_t k = 0; k < g.k; ++k) {
        const double va = g.band_op == 1 ? band_at<double>(A, ab, g.t.ak, 0, k, g.k, g.band) : A[ab + g.t.ak[k]];
        const double vb = g.band_op == 2 ? band_at<double>(B, bb, g.t.bk, 0, k, g.k, g.band) : B[bb + g.t.bk[k]];
        acc = fma(va, vb, acc);
      }
    } else if (g.sym_n > 0) {
      // the tables hold offsets p + n q of the dense symmetric matrix
      const int64_t sn = g.sym_n;
      for (int64_t k = 0; k < g.k; ++k) {
        int64_t oa = ab + g.t.ak[k], ob = bb + g.t.bk[k];
        if (g.sym_side == 0) oa = sym_at(oa % sn, oa / sn, sn);
        else ob = sym_at(ob % sn, ob / sn, sn);
        acc = fma(A[oa], B[ob], acc);
      }
    } else {
      for (int64_t k = 0; k < g.k; ++k) acc = fma(A[ab + g.t.ak[k]], B[bb + g.t.bk[k]], acc);
    }
    double* p = C + g.t.cl[il] + g.t.cm[m] + g.t.cn[n];
    double v = g.alpha * acc;
    if (g.beta != 0.0) v = fma(g.beta, *p, v);
    *p = v;
    if (g.emit_mode) {  // a network's fused epilogue: the consumer's exponents
      bool bad = false;
      const int ve = f64_row_exp(v, &bad);
      const int64_t ci = g.emit_mode == 1 ? m : n;
      atomicMax(&g.emit_e[ci], ve);
      if (bad) emit_mark(g.emit_flag, g.emit_list, ci);
    }
  }
}

// ------------------------------------------------------------ one-pass split
// An fp64-split operand whose k is one unit-stride mode (each row a run of k
// consecutive values, k <= kRowPackMaxK): its row exponents, flags and slices
// in one read.  tpr threads hold a row in registers, 8 consecutive values
// per group, RP_G groups each (value 8 (g tpr + t) + j in v[g][j]), reduce
// its exponent bound and flag, then split it from the registers.  The next
// row's loads go out group by group as the current row's slices are
// written, so they are in flight while it is split.  512 / tpr rows per
// block at a time; one block per SM.
constexpr int RP_THREADS = 512;
constexpr int RP_G = 4;

template <int S>
__global__ void __launch_bounds__(RP_THREADS, 1) k_rowpack(const __grid_constant__ PackArgs pa, int side,
                                                           int tpr) {
  const PackOp& o = pa.op[side];
  const double* __restrict__ X = (const double*)o.x;
  const int64_t K = pa.k, total = pa.l * o.rows;
  const int rpb = RP_THREADS / tpr;
  const int slot = threadIdx.x / tpr, t = threadIdx.x % tpr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t slice_stride = (size_t)pa.l * o.rows * pa.kp;  // elements per slice
  __shared__ int smx[2][RP_THREADS / 32], sbad[2][RP_THREADS / 32];
  double v[RP_G][8];
  auto row_src = [&](int64_t ri) {
    const int64_t il = pa.l == 1 ? 0 : ri / o.rows;
    return X + o.loff[il] + row_off(o, ri - il * o.rows);
  };
  // group g of this thread's share of the row at p (zeros past k or for no row)
  auto load = [&](const double* p, int g, bool ok) {
    const int64_t k0 = 8 * ((int64_t)g * tpr + t);
    if (ok && k0 + 8 <= K) {
      if (((uintptr_t)p & 15) == 0) {
        const double2* q = (const double2*)(p + k0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double2 d = __ldg(q + j);
          v[g][2 * j] = d.x;
          v[g][2 * j + 1] = d.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[g][j] = __ldg(p + k0 + j);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[g][j] = ok && k0 + j < K ? __ldg(p + k0 + j) : 0.0;
    }
  };
  const int64_t step = (int64_t)gridDim.x * rpb;
  int64_t base = (int64_t)blockIdx.x * rpb;  // the block's first row in this pass of the grid
  {
    const bool ok = base + slot < total;
    const double* p = ok ? row_src(base + slot) : X;
#pragma unroll
    for (int g = 0; g < RP_G; ++g) load(p, g, ok);
  }
  for (int par = 0; base < total; base += step, par ^= 1) {
    const int64_t ri = base + slot, rn = ri + step;
    const bool ok = ri < total, okn = rn < total;
    // values past k were loaded as zeros: their bound, -1021, is the least
    // any value gives, so they change neither result
    int mx = -1100, bad = 0;
#pragma unroll
    for (int g = 0; g < RP_G; ++g)
#pragma unroll
      for (int j = 0; j < 8; ++j) exp_update(v[g][j], mx, bad);
    mx = __reduce_max_sync(0xffffffffu, mx);
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (tpr > 32) {  // across the row's warps (parity-double-buffered: one barrier per round)
      if (lane == 0) {
        smx[par][warp] = mx;
        sbad[par][warp] = bad;
      }
      __syncthreads();
      const int w0 = slot * (tpr >> 5);
      for (int w = w0; w < w0 + (tpr >> 5); ++w) {
        mx = max(mx, smx[par][w]);
        bad |= sbad[par][w];
      }
    }
    if (ok && t == 0) {
      o.e[ri] = mx;
      if (bad) mark_row(o, ri);
    }
    const double* pn = okn ? row_src(rn) : X;
    uint16_t* out = (uint16_t*)o.out + (size_t)(ok ? ri : 0) * pa.kp;
#pragma unroll
    for (int g = 0; g < RP_G; ++g) {
      const int64_t k0 = 8 * ((int64_t)g * tpr + t);
      if (ok && k0 < K) split8<S>(v[g], mx, bad != 0, out + k0, slice_stride);
      load(pn, g, okn);
    }
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
__global__ void __launch_bounds__(256, 3) k_pack(const __grid_constant__ PackArgs pa) {
  const PackOp* o = &pa.op[blockIdx.z];
  pack_pipeline<PMODE>(blockIdx.x, gridDim.x, n_pack_tiles(o->rows, pa.k, pa.l),
                       [&](int64_t g) { return PackTile{&pa, o, g}; });
}

__global__ void __launch_bounds__(256) k_rowexp_sym(const __grid_constant__ PackArgs pa, int side,
                                                   int32_t* scr) {
  rowexp_sym_body(pa.op[side], scr);
}

// Row p's exponent bound: the maximum over the tiles of the triangle that
// hold row p, as a row (tiles (P, Q), Q <= P) or as a mirror image (tiles
// (Q, P), Q >= P), P = p / PR.  Block P takes rows P * PR + r, its four
// thread groups every fourth tile, combined in shared memory; one writer
// per row.
__global__ void __launch_bounds__(256) k_rowexp_sym_reduce(const __grid_constant__ PackArgs pa, int side,
                                                          const int32_t* __restrict__ scr) {
  const PackOp& o = pa.op[side];
  const int64_t n = o.sym_n, nb = (n + PR - 1) / PR, P = blockIdx.x;
  const int r = threadIdx.x % PR, g = threadIdx.x / PR;
  __shared__ int part[4][PR];
  int m = -1100;
  for (int64_t Q = g; Q <= P; Q += 4) m = max(m, scr[(P * (P + 1) / 2 + Q) * (PR + PK) + r]);
  for (int64_t Q = P + g; Q < nb; Q += 4) m = max(m, scr[(Q * (Q + 1) / 2 + P) * (PR + PK) + PR + r]);
  part[g][r] = m;
  __syncthreads();
  if (threadIdx.x < PR) {
    const int64_t p = P * PR + r;
    const int mm = max(max(part[0][r], part[1][r]), max(part[2][r], part[3][r]));
    if (p < n && mm > -1100) o.e[p] = mm;
  }
}

__global__ void __launch_bounds__(256) k_rowexp_gen(const __grid_constant__ PackArgs pa, int side) {
  rowexp_gen_body(pa, pa.op[side]);
}

template <int PMODE>
__global__ void __launch_bounds__(256) k_pack_gen(const __grid_constant__ PackArgs pa, int side) {
  pack_gen_body<PMODE>(pa, pa.op[side]);
}

__global__ void __launch_bounds__(256, 3) k_pack_sym(const __grid_constant__ PackArgs pa, int side) {
  pack_sym_body(pa, pa.op[side]);
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
__global__ void __launch_bounds__(256, 3) k_pack_grouped(const PackArgs* __restrict__ pas,
                                                      const int64_t* __restrict__ off, int nseg) {
  pack_pipeline<PMODE>(blockIdx.x, gridDim.x, off[nseg], [&](int64_t g) {
    const int s = segment_of(off, nseg, g);
    const PackArgs* pa = pas + (s >> 1);
    return PackTile{pa, &pa->op[s & 1], g - off[s]};
  });
}

__global__ void __launch_bounds__(256) k_fixup_grouped(const GemmArgs* __restrict__ gs,
                                                       const PackArgs* __restrict__ pas, int n) {
  for (int p = blockIdx.y; p < n; p += gridDim.y)
    fixup_body(gs[p], pas[p].op[0].list, pas[p].op[1].list, pas[p].op[0].flag);
}

}  // namespace

static cudaError_t configure_pack_kernels();

void set_affine(PackOp& o, const ClassModes& R, const ClassModes& K, int which) {
  auto st = [&](const Mode& m) { return which == 0 ? m.sa : m.sb; };
  o.affine = 0;
  o.rs = o.ks = 0;
  if (R.n <= 1) { o.affine |= 1; o.rs = R.n ? st(R.m[0]) : 0; }
  if (K.n <= 1) { o.affine |= 2; o.ks = K.n ? st(K.m[0]) : 0; }
}

int64_t rowexp_tiles(int64_t rows, int64_t k, int64_t l) {
  return ((rows + PR - 1) / PR) * ((k + KCH - 1) / KCH) * l;
}
int64_t pack_tiles(int64_t rows, int64_t k, int64_t l) { return n_pack_tiles(rows, k, l); }

cudaError_t launch_rowexp_grouped(const PackArgs* pas, const int64_t* off, int n, int64_t total,
                                  cudaStream_t s) {
  if (n <= 0 || total <= 0) return cudaSuccess;
  k_rowexp_grouped<<<grid_for(total), 256, 0, s>>>(pas, off, 2 * n);
  return cudaGetLastError();
}

cudaError_t launch_pack_grouped(int pmode, const PackArgs* pas, const int64_t* off, int n,
                                int64_t total, cudaStream_t s) {
  if (n <= 0 || total <= 0) return cudaSuccess;
  if (cudaError_t e = configure_pack_kernels(); e != cudaSuccess) return e;
  const int grid = grid_for(total);
  if (pmode == PACK_BF16)
    k_pack_grouped<PACK_BF16><<<grid, 256, pack_smem_bytes<PACK_BF16>(), s>>>(pas, off, 2 * n);
  else if (pmode == PACK_TF32)
    k_pack_grouped<PACK_TF32><<<grid, 256, pack_smem_bytes<PACK_TF32>(), s>>>(pas, off, 2 * n);
  else
    k_pack_grouped<PACK_F64><<<grid, 256, pack_smem_bytes<PACK_F64>(), s>>>(pas, off, 2 * n);
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

// The pack kernels stage two 64 x 64 tiles in dynamic shared memory (65 KB
// for fp64): allow that size and ask for the largest shared-memory carveout
// so that several blocks fit per SM.  Once per device.
template <class Kernel>
static void configure(Kernel kernel, int smem) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

static cudaError_t configure_pack_kernels() {
  constexpr int kMaxDev = 64;
  static bool done[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < kMaxDev && done[dev]) return cudaSuccess;
  configure(k_pack<PACK_BF16>, pack_smem_bytes<PACK_BF16>());
  configure(k_pack<PACK_TF32>, pack_smem_bytes<PACK_TF32>());
  configure(k_pack<PACK_F64>, pack_smem_bytes<PACK_F64>());
  configure(k_pack_grouped<PACK_BF16>, pack_smem_bytes<PACK_BF16>());
  configure(k_pack_grouped<PACK_TF32>, pack_smem_bytes<PACK_TF32>());
  configure(k_pack_grouped<PACK_F64>, pack_smem_bytes<PACK_F64>());
  configure(k_pack_sym, pack_smem_bytes<PACK_F64>());
  e = cudaGetLastError();
  if (e == cudaSuccess && dev < kMaxDev) done[dev] = true;
  return e;
}

cudaError_t launch_rowpack(const PackArgs& pa, int side, cudaStream_t s) {
  const PackOp& o = pa.op[side];
  if (pa.k < kRowPackMinK || pa.k > kRowPackMaxK || !(o.affine & 2) || o.ks != 1) return cudaErrorInvalidValue;
  static_assert(kRowPackMaxK <= (int64_t)RP_THREADS * RP_G * 8, "a row must fit the block's registers");
  int tpr = 32;  // threads per row: the fewest that hold k in RP_G groups of 8
  while ((int64_t)tpr * RP_G * 8 < pa.k) tpr *= 2;
  const int64_t rows = pa.l * o.rows;
  if (rows <= 0) return cudaSuccess;
  const int64_t per = RP_THREADS / tpr;
  const int grid = (int)std::min<int64_t>((rows + per - 1) / per, num_sms());
  switch (pa.slices) {
    case 2: k_rowpack<2><<<grid, RP_THREADS, 0, s>>>(pa, side, tpr); break;
    case 3: k_rowpack<3><<<grid, RP_THREADS, 0, s>>>(pa, side, tpr); break;
    case 4: k_rowpack<4><<<grid, RP_THREADS, 0, s>>>(pa, side, tpr); break;
    case 5: k_rowpack<5><<<grid, RP_THREADS, 0, s>>>(pa, side, tpr); break;
    case 6: k_rowpack<6><<<grid, RP_THREADS, 0, s>>>(pa, side, tpr); break;
    default: k_rowpack<7><<<grid, RP_THREADS, 0, s>>>(pa, side, tpr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_pack(int pmode, const PackArgs& pa, cudaStream_t s) {
  if (cudaError_t e = configure_pack_kernels(); e != cudaSuccess) return e;
  int64_t blocks = 0;
  for (int i = 0; i < 2; ++i) {
    const int64_t b = ((pa.op[i].rows + PR - 1) / PR) * ((pa.k + PK - 1) / PK) * pa.l;
    blocks = b > blocks ? b : blocks;
  }
  const dim3 grid(grid_for(blocks), 1, 2);
  if (pmode == PACK_BF16)
    k_pack<PACK_BF16><<<grid, 256, pack_smem_bytes<PACK_BF16>(), s>>>(pa);
  else if (pmode == PACK_TF32)
    k_pack<PACK_TF32><<<grid, 256, pack_smem_bytes<PACK_TF32>(), s>>>(pa);
  else
    k_pack<PACK_F64><<<grid, 256, pack_smem_bytes<PACK_F64>(), s>>>(pa);
  return cudaGetLastError();
}

static int64_t sym_blocks(const PackOp& o) {
  const int64_t nb = (o.sym_n + PR - 1) / PR;
  return nb * (nb + 1) / 2;
}

int64_t sym_scratch_bytes(int64_t n) {
  const int64_t nb = (n + PR - 1) / PR;
  return nb * (nb + 1) / 2 * (PR + PK) * (int64_t)sizeof(int32_t);
}

cudaError_t launch_rowexp_sym(const PackArgs& pa, int side, int32_t* scr, cudaStream_t s) {
  const int64_t nblk = sym_blocks(pa.op[side]);
  if (nblk <= 0) return cudaSuccess;
  k_rowexp_sym<<<grid_for(nblk), 256, 0, s>>>(pa, side, scr);
  const int64_t nb = (pa.op[side].sym_n + PR - 1) / PR;
  k_rowexp_sym_reduce<<<(unsigned)nb, 256, 0, s>>>(pa, side, scr);
  return cudaGetLastError();
}

cudaError_t launch_pack_sym(const PackArgs& pa, int side, cudaStream_t s) {
  if (cudaError_t e = configure_pack_kernels(); e != cudaSuccess) return e;
  const int64_t nblk = sym_blocks(pa.op[side]);
  if (nblk <= 0) return cudaSuccess;
  k_pack_sym<<<grid_for(nblk), 256, pack_smem_bytes<PACK_F64>(), s>>>(pa, side);
  return cudaGetLastError();
}

cudaError_t launch_rowexp_gen(const PackArgs& pa, int side, cudaStream_t s) {
  const PackOp& o = pa.op[side];
  const int64_t items = ((o.rows + PR - 1) / PR) * ((pa.k + PK - 1) / PK);
  if (items <= 0) return cudaSuccess;
  k_rowexp_gen<<<grid_for(items), 256, 0, s>>>(pa, side);
  return cudaGetLastError();
}

cudaError_t launch_pack_gen(int pmode, const PackArgs& pa, int side, cudaStream_t s) {
  const PackOp& o = pa.op[side];
  const int64_t items = ((o.rows + PR - 1) / PR) * ((pa.k + PK - 1) / PK);
  if (items <= 0) return cudaSuccess;
  if (pmode == PACK_TF32)
    k_pack_gen<PACK_TF32><<<grid_for(items), 256, PR * TLD * sizeof(float), s>>>(pa, side);
  else
    k_pack_gen<PACK_F64><<<grid_for(items), 256, PR * TLD * sizeof(double), s>>>(pa, side);
  return cudaGetLastError();
}

cudaError_t launch_fixup(const GemmArgs& g, const PackArgs& pa, cudaStream_t s) {
  k_fixup<<<num_sms() * 2, 256, 0, s>>>(g, pa.op[0].list, pa.op[1].list, pa.op[0].flag);
  return cudaGetLastError();
}

}  // namespace famlies
