// Tensor-core contraction with operand tiles gathered straight from the
// strided tensors (bf16 inputs, and fp32 inputs through a three-term tf32
// split).  No operand is transposed or packed in global memory.
//
// The paper fuses the tensor-to-matrix re-organisation into the packing step
// of the level-3 product (Sec. 1 "Challenges", tensor item; Sec. 2.3 block-
// scatter item; Fig. 2's packed A~/B~).  Here the "packing" is the staging of
// each operand tile into shared memory: producer warps read the tile through
// the offset tables (coalesced along whichever index is unit-stride in that
// operand) and write it in the 128-byte-swizzled K-major layout that
// tcgen05.mma reads directly.  One thread issues the MMAs into a
// double-buffered fp32 accumulator in tensor memory; four epilogue warps
// drain it (one output row per thread), apply alpha/beta and scatter to C's
// strided layout while the next tile accumulates.  The grid is persistent:
// one CTA per SM walks the tile list.
//
// Warp roles: 0-3 epilogue, 4 MMA issue (+ tensor-memory allocation),
// 5-12 producers.  Every wait is bounded; on expiry the CTA records
// FAMLIES_ERR_DEVICE_TIMEOUT, stops all roles, and frees its tensor memory.
#include <cstdint>

#include <cuda_bf16.h>

#include "device.h"
#include "ptx.cuh"

namespace famlies {

namespace {

constexpr int64_t kIrregular = INT64_MIN;

template <bool TF32, int BN>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int ROWB = 128;           // bytes of one swizzled smem row
  static constexpr int EPC = TF32 ? 4 : 8;   // elements per 16-byte chunk
  static constexpr int KB = 8 * EPC;         // k per stage (8 chunks per row)
  static constexpr int NT = TF32 ? 2 : 1;    // hi (+ lo) copies of each tile
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int STAGE_BYTES = NT * (A_BYTES + B_BYTES);
  static constexpr int STAGES = (196 * 1024) / STAGE_BYTES > 8 ? 8 : (196 * 1024) / STAGE_BYTES;
  static constexpr int EPI_WARPS = 4;
  static constexpr int PROD_WARPS = 8;
  static constexpr int PT = 32 * PROD_WARPS;
  static constexpr int THREADS = 32 * (EPI_WARPS + 1 + PROD_WARPS);
  static constexpr int MMA_K = TF32 ? 8 : 16;  // k of one MMA (32 bytes)
  static constexpr int KSTEPS = KB / MMA_K;
  static constexpr uint32_t TMEM_COLS = 2 * BN;
  static constexpr uint32_t IDESC = ptx::idesc_make(BM, BN, TF32 ? 2u : 1u);
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
};

struct TcArgs {
  GemmArgs g;
  const int64_t* aks;  // per 16-byte k-chunk: constant stride of the row operand, or irregular
  const int64_t* bks;
};

// Loads EPC consecutive-k values of one operand row (zero beyond K).
template <bool TF32>
__device__ __forceinline__ void gather_chunk(const void* X, int64_t base, const int64_t* koff,
                                             const int64_t* kstr, int64_t K, int64_t kc,
                                             uint32_t (&out)[TF32 ? 8 : 4]) {
  constexpr int EPC = TF32 ? 4 : 8;
  const int64_t st = kstr[kc / EPC];
  if (TF32) {
    const float* p = (const float*)X;
    float v[4];
    if (st != kIrregular) {
      const float* q = p + base + koff[kc];
      if (st == 1 && (((uintptr_t)q) & 15) == 0) {
        float4 f = __ldg((const float4*)q);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = __ldg(q + e * st);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (kc + e < K) ? __ldg(p + base + koff[kc + e]) : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t hi = ptx::tf32_round(v[e]);
      float lo = v[e] - __uint_as_float(hi);
      out[e] = hi;
      out[4 + e] = ptx::tf32_round(lo);
    }
  } else {
    const unsigned short* p = (const unsigned short*)X;
    unsigned short v[8];
    if (st != kIrregular) {
      const unsigned short* q = p + base + koff[kc];
      if (st == 1 && (((uintptr_t)q) & 15) == 0) {
        uint4 u = __ldg((const uint4*)q);
        out[0] = u.x; out[1] = u.y; out[2] = u.z; out[3] = u.w;
        return;
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = __ldg(q + e * st);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (kc + e < K) ? __ldg(p + base + koff[kc + e]) : (unsigned short)0;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = (uint32_t)v[2 * e] | ((uint32_t)v[2 * e + 1] << 16);
  }
}

// Stages one operand tile (R rows x KB k) of stage memory `s_hi` (and the
// tf32 low part at `s_lo`).  Thread pt of PT producer threads.
template <bool TF32, int R, int PT>
__device__ __forceinline__ void fill_tile(uint32_t s_hi, uint32_t s_lo, const void* X, int64_t xl,
                                          const int64_t* roff, int64_t rows, int64_t r0,
                                          const int64_t* koff, const int64_t* kstr, int64_t K,
                                          int64_t k0, int contig, int pt) {
  constexpr int EPC = TF32 ? 4 : 8;
  constexpr int NI = R * 8 / PT;  // items (row, chunk) per thread
  static_assert(NI >= 1 && (R * 8) % PT == 0, "tile/thread split");
#pragma unroll
  for (int j = 0; j < NI; ++j) {
    int r, c;
    if (contig == 2) {  // unit stride along k: neighbouring threads take neighbouring chunks
      c = pt & 7;
      r = (pt >> 3) + j * (PT / 8);
    } else {            // otherwise neighbouring threads take neighbouring rows
      const int i = pt + j * PT;
      r = i % R;
      c = i / R;
    }
    const int64_t gr = r0 + r, kc = k0 + (int64_t)c * EPC;
    uint32_t w[TF32 ? 8 : 4];
    if (gr < rows && kc < K) {
      gather_chunk<TF32>(X, xl + roff[gr], koff, kstr, K, kc, w);
    } else {
#pragma unroll
      for (int e = 0; e < (TF32 ? 8 : 4); ++e) w[e] = 0u;
    }
    const uint32_t off = (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
    ptx::st_shared_v4(s_hi + off, w[0], w[1], w[2], w[3]);
    if constexpr (TF32) ptx::st_shared_v4(s_lo + off, w[4], w[5], w[6], w[7]);
  }
}

__device__ __forceinline__ void record_timeout(volatile int* abort, int* status) {
  *abort = 1;
  atomicCAS(status, 0, FAMLIES_ERR_DEVICE_TIMEOUT);
}

template <bool TF32, int BN>
__global__ void __launch_bounds__(TcCfg<TF32, BN>::THREADS, 1) k_tc(const TcArgs args) {
  using Cfg = TcCfg<TF32, BN>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const GemmArgs& g = args.g;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t tiles_m = (g.m + Cfg::BM - 1) / Cfg::BM, tiles_n = (g.n + BN - 1) / BN;
  const int64_t ntiles = tiles_m * tiles_n * g.l;
  const int64_t nkb = (g.k + Cfg::KB - 1) / Cfg::KB;
  const int64_t lim = g.wait_limit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      ptx::mbar_init(&full[s], Cfg::PT);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&tfull[b], 1);
      ptx::mbar_init(&tempty[b], Cfg::EPI_WARPS);
    }
    ptx::mbar_init(done, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == Cfg::EPI_WARPS) {
    ptx::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == Cfg::EPI_WARPS) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, acc = 0, accph = 0;
      // testing: `done` completes only after this thread's last commit
      bool ok = !g.stall_test || ptx::mbar_wait(done, 0, lim, abort);
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        if (!ptx::mbar_wait(&tempty[acc], accph ^ 1, lim, abort)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t dt = tmem_base + acc * BN;
        for (int64_t kb = 0; kb < nkb; ++kb) {
          if (!ptx::mbar_wait(&full[stage], phase, lim, abort)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t a_hi = ptx::smem_u32(smem + stage * Cfg::STAGE_BYTES);
          const uint32_t b_hi = a_hi + Cfg::A_BYTES;
          const uint64_t da = ptx::sdesc_kmajor_sw128(a_hi), db = ptx::sdesc_kmajor_sw128(b_hi);
#pragma unroll
          for (int kk = 0; kk < Cfg::KSTEPS; ++kk) {
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            if (TF32) {
              const uint32_t a_lo = b_hi + Cfg::B_BYTES, b_lo = a_lo + Cfg::A_BYTES;
              const uint64_t dal = ptx::sdesc_kmajor_sw128(a_lo), dbl = ptx::sdesc_kmajor_sw128(b_lo);
              ptx::mma_tf32(dt, dal + 2 * kk, db + 2 * kk, Cfg::IDESC, first);
              ptx::mma_tf32(dt, da + 2 * kk, dbl + 2 * kk, Cfg::IDESC, 1u);
              ptx::mma_tf32(dt, da + 2 * kk, db + 2 * kk, Cfg::IDESC, 1u);
            } else {
              ptx::mma_f16(dt, da + 2 * kk, db + 2 * kk, Cfg::IDESC, first);
            }
          }
          ptx::mma_commit(&empty[stage]);
          if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        ptx::mma_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) accph ^= 1;
      }
      if (!ok) record_timeout(abort, g.status);
      // All issued MMAs must finish before tensor memory is released.
      ptx::mma_commit(done);
      for (int64_t i = 0; i < ((int64_t)1 << 24); ++i)
        if (ptx::mbar_try_wait(done, 0)) break;
    }
    __syncwarp();
  } else if (warp > Cfg::EPI_WARPS) {
    // ------------------------------------------------------------ producers
    const int pt = threadIdx.x - 32 * (Cfg::EPI_WARPS + 1);
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int64_t tm = t % tiles_m, rest = t / tiles_m;
      const int64_t tn = rest % tiles_n, il = rest / tiles_n;
      const int64_t al = g.t.al[il], bl = g.t.bl[il];
      for (int64_t kb = 0; kb < nkb; ++kb) {
        if (!ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort)) { ok = false; break; }
        const uint32_t a_hi = ptx::smem_u32(smem + stage * Cfg::STAGE_BYTES);
        const uint32_t b_hi = a_hi + Cfg::A_BYTES;
        const uint32_t a_lo = b_hi + Cfg::B_BYTES, b_lo = a_lo + Cfg::A_BYTES;
        const int64_t k0 = kb * Cfg::KB;
        fill_tile<TF32, Cfg::BM, Cfg::PT>(a_hi, a_lo, g.a, al, g.t.am, g.m, tm * Cfg::BM, g.t.ak,
                                          args.aks, g.k, k0, g.a_contig, pt);
        fill_tile<TF32, BN, Cfg::PT>(b_hi, b_lo, g.b, bl, g.t.bn, g.n, tn * BN, g.t.bk, args.bks,
                                     g.k, k0, g.b_contig, pt);
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(&full[stage]);
        if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1; }
      }
    }
    if (!ok && !*abort) record_timeout(abort, g.status);
  } else {
    // ------------------------------------------------------------ epilogue
    float* C = (float*)g.c;
    const float alpha = (float)g.alpha, beta = (float)g.beta;
    uint32_t acc = 0, accph = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t tm = t % tiles_m, rest = t / tiles_m;
      const int64_t tn = rest % tiles_n, il = rest / tiles_n;
      if (!ptx::mbar_wait(&tfull[acc], accph, lim, abort)) {
        if (!*abort) record_timeout(abort, g.status);
        break;
      }
      ptx::tc_fence_after();
      const int64_t row = tm * Cfg::BM + warp * 32 + lane;
      const bool rv = row < g.m;
      const int64_t crow = rv ? g.t.cl[il] + g.t.cm[row] : 0;
      const int64_t n0 = tn * BN;
#pragma unroll 1
      for (int q = 0; q < BN / 32; ++q) {
        uint32_t r[32];
        ptx::tmem_ld32(tmem_base + ((uint32_t)(warp * 32) << 16) + acc * BN + q * 32, r);
        ptx::tmem_ld_wait();
        if (rv) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int64_t col = n0 + q * 32 + i;
            if (col < g.n) {
              float* p = C + crow + g.t.cn[col];
              float v = alpha * __uint_as_float(r[i]);
              if (beta != 0.f) v = fmaf(beta, *p, v);
              *p = v;
            }
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) accph ^= 1;
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == Cfg::EPI_WARPS) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

// Per 16-byte k-chunk of EPC elements: the constant stride between
// neighbouring offsets inside the chunk, or kIrregular when they are not
// evenly spaced or the chunk runs past K.
__global__ void k_kstride(const int64_t* __restrict__ off, int64_t K, int epc, int64_t* __restrict__ out) {
  const int64_t nq = (K + epc - 1) / epc;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = q * epc;
    int64_t st = kIrregular;
    if (k + epc <= K) {
      st = off[k + 1] - off[k];
      for (int e = 2; e < epc; ++e)
        if (off[k + e] - off[k + e - 1] != st) { st = kIrregular; break; }
    }
    out[q] = st;
  }
}

template <bool TF32, int BN>
cudaError_t launch_one(const TcArgs& a, cudaStream_t s) {
  using Cfg = TcCfg<TF32, BN>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc<TF32, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t tiles = ((a.g.m + Cfg::BM - 1) / Cfg::BM) * ((a.g.n + BN - 1) / BN) * a.g.l;
  const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
  mark_begin(a.g, s);
  k_tc<TF32, BN><<<grid, Cfg::THREADS, Cfg::SMEM_BYTES, s>>>(a);
  mark_end(a.g, s);
  return cudaGetLastError();
}

}  // namespace

int64_t tc_workspace_bytes(const Plan& p) {
  return 2 * ((p.k + 3) / 4 + 1) * (int64_t)sizeof(int64_t);
}

cudaError_t launch_tc(const Plan& p, const GemmArgs& g, int tile_n, void* ws, cudaStream_t s) {
  const bool tf32 = p.kernel == FAMLIES_KERNEL_TC_TF32X3_GATHER;
  const int epc = tf32 ? 4 : 8;
  const int64_t nq = (p.k + epc - 1) / epc;
  int64_t* aks = (int64_t*)ws;
  int64_t* bks = aks + nq + 1;
  const int blocks = (int)((nq + 255) / 256 < 1024 ? (nq + 255) / 256 : 1024);
  k_kstride<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g.t.ak, p.k, epc, aks);
  k_kstride<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g.t.bk, p.k, epc, bks);
  TcArgs a;
  a.g = g;
  a.aks = aks;
  a.bks = bks;
  int bn = tile_n;
  if (bn != 64 && bn != 128 && bn != 256) bn = p.n > 128 ? 256 : (p.n > 64 ? 128 : 64);
  if (tf32) return bn == 64 ? launch_one<true, 64>(a, s) : launch_one<true, 128>(a, s);
  if (bn == 64) return launch_one<false, 64>(a, s);
  if (bn == 128) return launch_one<false, 128>(a, s);
  return launch_one<false, 256>(a, s);
}

}  // namespace famlies
