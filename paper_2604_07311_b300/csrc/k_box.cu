// bf16 tensor-core contraction whose operand tiles are staged straight from
// the caller's strided tensors: no pack, no offset tables, no transposed copy.
//
// The paper asks for tensor contractions that reach level-3 performance
// without converting the tensors to matrices (Sec. 1 "Challenges", tensor
// item; Sec. 2.3, the block-scatter mapping of TBLIS) and for transposition
// expressed as a change of strides (Sec. 2.1, "Variations on
// functionality").  Here every output tile is a box over the label modes:
// the row class (at most two modes m0, m1 after index fusion) contributes
// bm0 x bm1 = 128 rows, the column class bn0 x bn1 = BN columns and the
// contracted class bk0 x bk1 = 64 k per pipeline stage.  Each operand tile
// lands in shared memory in the layout the tensor cores read:
//   MN-major  the operand is unit-stride along its first row mode: each
//             shared-memory row holds a run of `run` consecutive rows of the
//             operand for one k (one k per row, the tile a stack of such
//             runs); the MMA reads it with the transpose bit set.
//   K-major   the operand is unit-stride along the first contracted mode:
//             each shared-memory row holds a run of bk0 consecutive k for one
//             row index (bk1 such sub-tiles per stage).
// A run is 32, 64 or 128 bytes and the tile uses the swizzle of that span.
// When the operand's strides are multiples of 16 bytes a 5-D TMA map over
// the caller's tensor fills the tile (one copy per run column or k
// sub-tile); otherwise gather warps load aligned 16-byte chunks, shift them
// to the run's 2-byte alignment and store them swizzled (e.g. a first-mode
// stride padded to 103 elements, 206 bytes).
//
// Warp roles: 0-7 drain the fp32 accumulator (two warps per 32-lane
// quadrant, each half the columns), 8 issues TMA copies, 9 allocates tensor
// memory and one of its threads issues tcgen05.mma into a double-buffered
// accumulator, 10.. (when an operand is gathered) gather warps.  The grid is
// persistent (one CTA per SM walks the tile list, column tiles fastest).
// The whole k range accumulates in tensor memory (fp32, at most 16384 k so
// that rounding stays below 1e-5 relative), drained once per tile:
// C = alpha * acc + beta * C at C's own strides.  Every wait is bounded; on
// expiry the CTA records FAMLIES_ERR_DEVICE_TIMEOUT, the roles stop, copies
// and MMAs in flight are waited for (bounded) and tensor memory is freed.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include <cuda.h>

#include "device.h"
#include "pair_gemm.h"
#include "ptx.cuh"

namespace famlies {

namespace {

constexpr int BM = 128;
constexpr int KB = 64;  // k per stage
constexpr int EPI_WARPS = 8;
constexpr int NGATHER = 6;  // gather warps when an operand is gathered (16 warps in all: 4 per SM sub-partition)
constexpr int GU = 8;       // gather rounds whose loads are in flight together

// One operand as the kernel stages it.  Modes: 0 = first row mode, 1 =
// second row mode, 2 = first contracted mode, 3 = second contracted mode,
// 4 = batch; absent modes have extent 1.
struct BoxOp {
  const void* x;
  int64_t e[5];  // extents
  int64_t s[5];  // strides in elements
  int mn;        // 1: MN-major tile (unit stride along mode 0), 0: K-major (along mode 2)
  int tma;       // 1: filled by TMA, 0: by the gather warps
  int run;       // elements per shared-memory row (32/64/128 bytes)
  int b0, b1;    // row box (b0 * b1 = the operand's tile rows)
  int lrun, lb0, lapr;  // log2 of run, b0 and b0 / run (all powers of two)
  // TMA: single = 1 when one copy fills the whole tile (the map's dimensions
  // are the roles below), else one copy per run column (MN-major only)
  int single;
  int8_t role[5];
};

// What each tensor-map dimension's coordinate is (see encode_op).
enum : int8_t { ROLE_ZERO = 0, ROLE_R0, ROLE_K0, ROLE_K1, ROLE_RHI, ROLE_R1, ROLE_L };

struct BoxArgs {
  BoxOp op[2];            // 0: row operand (tile rows 128), 1: column operand (BN)
  int bk0, bk1;           // contracted box (bk0 * bk1 = KB)
  int lbk0;               // log2(bk0)
  int64_t t0[2], t1[2];   // tiles along the row modes of each operand
  int64_t nk0, nk1;       // k blocks along the two contracted modes
  int64_t l;              // batch extent
  float* c;
  int64_t cs[5];          // C strides: m0, m1, n0, n1, batch
  // split K of the last, partly empty round: items [0, full) are whole
  // tiles; the `tail` tiles after them run as `splits` items each over parts
  // of the k blocks, writing fp32 partial tiles part[split][tail tile][BN][BM]
  // that k_box_reduce sums in split order (splits == 1: no split)
  int64_t full, tail;
  int splits;
  float* part;
  float alpha, beta;
  int* status;
  int64_t wait_limit;
  int stall_test;
};

template <int BN, int NG>
struct BoxCfg {
  static constexpr int A_BYTES = BM * KB * 2;
  static constexpr int B_BYTES = BN * KB * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (200 * 1024) / STAGE_BYTES > 8 ? 8 : (200 * 1024) / STAGE_BYTES;
  static constexpr int THREADS = 32 * (EPI_WARPS + 2 + NG);
  // two accumulator buffers of BN columns, allocated as a power of two
  static constexpr uint32_t TMEM_COLS = 2 * BN <= 128 ? 128 : (2 * BN <= 256 ? 256 : 512);
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static_assert(STAGES >= 2 && SMEM_BYTES <= 227 * 1024, "shared memory budget");
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "tile bases stay 1024-aligned");
};

__device__ __forceinline__ void record_timeout(volatile int* abort, int* status) {
  *abort = 1;
  atomicCAS(status, 0, FAMLIES_ERR_DEVICE_TIMEOUT);
}

struct TileIx {
  int64_t tm0, tm1, tn0, tn1, il;
};

// Tile t of the launch: column tiles fastest, then row tiles, then batch.
__device__ __forceinline__ TileIx tile_ix(const BoxArgs& a, int64_t t) {
  const int64_t tn_all = a.t0[1] * a.t1[1], tm_all = a.t0[0] * a.t1[0];
  const int64_t tn = t % tn_all, rest = t / tn_all;
  const int64_t tm = rest % tm_all;
  TileIx x;
  x.il = rest / tm_all;
  x.tm0 = tm % a.t0[0];
  x.tm1 = tm / a.t0[0];
  x.tn0 = tn % a.t0[1];
  x.tn1 = tn / a.t0[1];
  return x;
}

// Work item t: a tile and the k blocks [kb_lo, kb_hi) it covers; split >= 0
// for a split item (ti: its index among the tail tiles).
struct Item {
  TileIx T;
  int64_t kb_lo, kb_hi, ti;
  int split;
};

__device__ __forceinline__ Item item_at(const BoxArgs& a, int64_t t, int64_t nkb) {
  Item it;
  int64_t tile = t;
  it.split = -1;
  it.ti = 0;
  it.kb_lo = 0;
  it.kb_hi = nkb;
  if (a.splits > 1 && t >= a.full) {
    const int64_t u = t - a.full;
    it.ti = u % a.tail;
    it.split = (int)(u / a.tail);
    tile = a.full + it.ti;
    it.kb_lo = nkb * it.split / a.splits;
    it.kb_hi = nkb * (it.split + 1) / a.splits;
  }
  it.T = tile_ix(a, tile);
  return it;
}

__device__ __forceinline__ uint4 ldg_nc_v4(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// A gather warp's share of one operand tile of one stage.  A "run" is one
// shared-memory row: `run` consecutive elements of the operand (2-byte
// aligned in global memory).  L = run/8 + 1 lanes serve a run: lane j < run/8
// loads the 16-byte-aligned chunk j covering the run and writes output chunk
// j, built from its chunk and lane j+1's (a shuffle) shifted by the run's
// misalignment; lane run/8 loads the chunk after the last one when the run
// is misaligned.  A chunk is loaded only when it holds an element of the
// run inside the tensor (so no load leaves the 16-byte block of a valid
// element); elements outside the tensor are stored as zeros.
//   tbase  element offset of the tile's origin (row modes and batch)
//   kbase  element offset of the stage's first k (both contracted modes)
//   lim0/lim1  row-mode indices left inside the tensor from the tile origin
//   klim0/klim1  contracted indices left from the stage's first k
struct GatherCtx {
  int64_t tbase, kbase;
  int lim0, lim1, klim0, klim1;
};

template <int ROWS, int NG>
__device__ __forceinline__ void gather_tile(const BoxOp& X, uint32_t tile, const GatherCtx& cx, int bk0m1, int lbk0,
                                            int bk1, int lane, int gw) {
  const int R = X.run, nq = R >> 3, L = nq + 1, rpw = 32 / L;
  const int g = lane / L, j = lane - g * L;
  const int RB = 2 * R;
  const int runs = X.mn ? (ROWS >> X.lrun) * KB : ROWS * bk1;
  const int per_round = rpw * NG;
  const int rounds = (runs + per_round - 1) / per_round;
  const char* base = (const char*)X.x + 2 * (cx.tbase + cx.kbase);
  const int aprm1 = (1 << X.lapr) - 1, b0m1 = X.b0 - 1;
  for (int r = 0; r < rounds; r += GU) {
    uint4 w[GU];
    uint32_t soff[GU];
    int meta[GU];  // -1: no run in this slot; else (elements inside the tensor) << 4 | misalignment
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int q = ((r + u) * NG + gw) * rpw + g;
      w[u] = make_uint4(0u, 0u, 0u, 0u);
      meta[u] = -1;
      soff[u] = 0;
      if (!((r + u) < rounds && g < rpw && q < runs)) continue;
      meta[u] = 0;
      int rr0, rr1, kk0, kk1, lim;
      if (X.mn) {  // run (a, kr): a = run column (a0 along mode 0, a1 along mode 1), kr = k row
        const int a = q >> 6, kr = q & 63;
        rr0 = (a & aprm1) << X.lrun;
        rr1 = a >> X.lapr;
        kk0 = kr & bk0m1;
        kk1 = kr >> lbk0;
        soff[u] = (uint32_t)((a * KB + kr) * RB);
        lim = cx.lim0 - rr0;
      } else {     // run (js, lr): js = k sub-tile, lr = tile row
        const int js = q / ROWS, lr = q - js * ROWS;
        rr0 = lr & b0m1;
        rr1 = lr >> X.lb0;
        kk0 = 0;
        kk1 = js;
        soff[u] = (uint32_t)((js * ROWS + lr) * RB);
        lim = cx.klim0;
      }
      if (!(rr0 < cx.lim0 && rr1 < cx.lim1 && kk0 < cx.klim0 && kk1 < cx.klim1)) continue;
      const int nv = lim < R ? lim : R;
      const char* p = base + 2 * ((int64_t)rr0 * X.s[0] + (int64_t)rr1 * X.s[1] + (int64_t)kk0 * X.s[2] +
                                  (int64_t)kk1 * X.s[3]);
      const int off = (int)((uintptr_t)p & 15);
      meta[u] = (nv << 4) | off;
      const char* c = p - off + 16 * j;
      if ((j < nq || off != 0) && c < p + 2 * nv) w[u] = ldg_nc_v4(c);
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      uint32_t win[8];
      win[0] = w[u].x; win[1] = w[u].y; win[2] = w[u].z; win[3] = w[u].w;
      win[4] = __shfl_down_sync(0xffffffffu, w[u].x, 1);
      win[5] = __shfl_down_sync(0xffffffffu, w[u].y, 1);
      win[6] = __shfl_down_sync(0xffffffffu, w[u].z, 1);
      win[7] = __shfl_down_sync(0xffffffffu, w[u].w, 1);
      if (meta[u] < 0 || j >= nq) continue;
      // bytes [off, off + 16) of the 32-byte window: word shift, then byte shift
      const int off = meta[u] & 15, nv = meta[u] >> 4;
      uint32_t t6[6], v5[5], o[4];
#pragma unroll
      for (int i = 0; i < 6; ++i) t6[i] = (off & 8) ? win[i + 2] : win[i];
#pragma unroll
      for (int i = 0; i < 5; ++i) v5[i] = (off & 4) ? t6[i + 1] : t6[i];
      const uint32_t sh = (uint32_t)(off & 3) * 8u;
#pragma unroll
      for (int i = 0; i < 4; ++i) o[i] = __funnelshift_r(v5[i], v5[i + 1], sh);
      const int first = 8 * j;
      if (first + 8 > nv) {  // elements past the tensor's edge (or the whole chunk) are zero
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = first + 2 * i;
          if (e >= nv) o[i] = 0u;
          else if (e + 1 >= nv) o[i] &= 0xFFFFu;
        }
      }
      const uint32_t so = soff[u] + 16u * (uint32_t)j;
      ptx::st_shared_v4(tile + ptx::swizzle_off(so, RB), o[0], o[1], o[2], o[3]);
    }
  }
}

// The TMA copies of one operand tile: one copy of the whole tile when the
// map holds every dimension, else (MN-major) one per run column (a1 along
// the second row mode, a0 along the first).  The copy coordinates of a tile
// are fixed but for the contracted ones: tile_coords() forms them once per
// tile (contracted coordinates 0), tma_tile() adds the stage's k0s and k1s
// with independent selects (the single issuing thread's latency paces the
// whole pipeline).
struct TmaCoords {
  int32_t c[5];
};

__device__ __forceinline__ TmaCoords tile_coords(const BoxOp& X, int32_t r0, int32_t r1, int32_t il) {
  TmaCoords t;
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    const int8_t r = X.role[d];
    t.c[d] = r == ROLE_R0 ? r0 : r == ROLE_RHI ? (r0 >> X.lrun) : r == ROLE_R1 ? r1 : r == ROLE_L ? il : 0;
  }
  return t;
}

template <int ROWS>
__device__ __forceinline__ void tma_tile(const BoxOp& X, const CUtensorMap* map, uint8_t* tile, uint64_t* bar,
                                         const TmaCoords& t, int32_t k0s, int32_t k1s) {
  int32_t c[5];
#pragma unroll
  for (int d = 0; d < 5; ++d)
    c[d] = t.c[d] + (X.role[d] == ROLE_K0 ? k0s : 0) + (X.role[d] == ROLE_K1 ? k1s : 0);
  if (X.single) {
    ptx::tma_load_5d(tile, map, bar, c[0], c[1], c[2], c[3], c[4]);
    return;
  }
  // fallback map {r0, k0, k1, r1, batch}, box {run, bk0, bk1, 1, 1}
  const int R = X.run, RB = 2 * R;
  const int apr = 1 << X.lapr;
  uint8_t* dst = tile;
  for (int a1 = 0; a1 < X.b1; ++a1)
    for (int a0 = 0; a0 < apr; ++a0, dst += KB * RB)
      ptx::tma_load_5d(dst, map, bar, c[0] + a0 * R, c[1], c[2], c[3] + a1, c[4]);
}

// Descriptor of k-step s (16 k) of an operand tile at `tile` (ROWS rows).
template <int ROWS>
__device__ __forceinline__ uint64_t op_desc(const BoxOp& X, uint32_t tile, int s, int bk0) {
  const uint32_t RB = 2u * (uint32_t)X.run;
  if (X.mn)  // k rows of RB bytes; 8-row groups RB*8 apart; runs along M (N) KB*RB apart
    return ptx::sdesc(tile + (uint32_t)s * 16u * RB, (uint32_t)KB * RB, 8u * RB, (int)RB);
  // rows of RB bytes (bk0 k); k-step s lies in sub-tile 16s / bk0 at byte 2 (16s mod bk0)
  const int js = (16 * s) / bk0, kin = (16 * s) % bk0;
  return ptx::sdesc(tile + (uint32_t)(js * ROWS) * RB + 2u * (uint32_t)kin, 16u, 8u * RB, (int)RB);
}

template <int BN, int NG>
__global__ void __launch_bounds__(BoxCfg<BN, NG>::THREADS, 1)
    k_box(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
          const __grid_constant__ BoxArgs args) {
  using Cfg = BoxCfg<BN, NG>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const BoxArgs& A = args;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t nkb = A.nk0 * A.nk1;
  const int64_t nitems = A.splits > 1 ? A.full + A.tail * A.splits : A.t0[0] * A.t1[0] * A.t0[1] * A.t1[1] * A.l;
  const int64_t lim = A.wait_limit;
  const bool tma0 = A.op[0].tma, tma1 = A.op[1].tma;
  const bool any_tma = tma0 || tma1;
  const bool any_gather = NG > 0 && (!tma0 || !tma1);

  if (threadIdx.x == 0) {
    // full[s]: the TMA thread's arrival (with the copies' bytes) plus every
    // gather thread's; empty[s]: the MMA's commit
    const uint32_t arrivals = (any_tma ? 1u : 0u) + (any_gather ? 32u * NG : 0u);
    for (int s = 0; s < Cfg::STAGES; ++s) {
      ptx::mbar_init(&full[s], arrivals);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&tfull[b], 1);
      ptx::mbar_init(&tempty[b], EPI_WARPS);
    }
    ptx::mbar_init(done, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == EPI_WARPS + 1) {
    ptx::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == EPI_WARPS) {
    // ------------------------------------------------------------ TMA copies
    if (lane == 0 && any_tma) {
      if (tma0) ptx::prefetch_tmap(&map_a);
      if (tma1) ptx::prefetch_tmap(&map_b);
      const uint32_t bytes = (tma0 ? (uint32_t)Cfg::A_BYTES : 0u) + (tma1 ? (uint32_t)Cfg::B_BYTES : 0u);
      int stage = 0;
      uint32_t phase = 0, pending = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        const Item I = item_at(A, t, nkb);
        const TileIx& T = I.T;
        const TmaCoords ta = tile_coords(A.op[0], (int32_t)(T.tm0 * A.op[0].b0), (int32_t)(T.tm1 * A.op[0].b1),
                                         (int32_t)T.il);
        const TmaCoords tb = tile_coords(A.op[1], (int32_t)(T.tn0 * A.op[1].b0), (int32_t)(T.tn1 * A.op[1].b1),
                                         (int32_t)T.il);
        int32_t kb0 = (int32_t)(I.kb_lo % A.nk0), k0s = kb0 * A.bk0, k1s = (int32_t)(I.kb_lo / A.nk0) * A.bk1;
        for (int64_t kb = I.kb_lo; kb < I.kb_hi; ++kb) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort)) { ok = false; break; }
          uint8_t* st = smem + stage * Cfg::STAGE_BYTES;
          ptx::mbar_arrive_expect_tx(&full[stage], bytes);
          if (tma0) tma_tile<BM>(A.op[0], &map_a, st, &full[stage], ta, k0s, k1s);
          if (tma1) tma_tile<BN>(A.op[1], &map_b, st + Cfg::A_BYTES, &full[stage], tb, k0s, k1s);
          pending = (pending & ~(0x101u << stage)) | (1u << stage) | (phase << (stage + 8));
          if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1; }
          if (++kb0 == A.nk0) { kb0 = 0; k0s = 0; k1s += A.bk1; } else { k0s += A.bk0; }
        }
      }
      if (!ok && !*abort) record_timeout(abort, A.status);
      // copies still in flight land before the CTA leaves (bounded)
      for (int s = 0; s < Cfg::STAGES; ++s) {
        if (!(pending & (1u << s))) continue;
        const uint32_t ph = (pending >> (s + 8)) & 1u;
        for (int64_t i = 0; i < ((int64_t)1 << 22); ++i)
          if (ptx::mbar_try_wait(&full[s], ph)) break;
      }
    }
    __syncwarp();
  } else if (warp == EPI_WARPS + 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = ptx::idesc_make_mn(BM, BN, 1u, (uint32_t)A.op[0].mn, (uint32_t)A.op[1].mn);
      // descriptors of stage 0's k-steps; stage s adds its byte offset / 16
      // to the start-address field (addresses stay below 256 KB: no carry)
      uint64_t da[KB / 16], db[KB / 16];
      const uint32_t t0 = ptx::smem_u32(smem);
#pragma unroll
      for (int s = 0; s < KB / 16; ++s) {
        da[s] = op_desc<BM>(A.op[0], t0, s, A.bk0);
        db[s] = op_desc<BN>(A.op[1], t0 + Cfg::A_BYTES, s, A.bk0);
      }
      int stage = 0;
      uint32_t phase = 0, acc = 0, accph = 0;
      // testing: `done` completes only after this thread's last commit
      bool ok = !A.stall_test || ptx::mbar_wait(done, 0, lim, abort);
      for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
        int64_t kb_lo = 0, kb_hi = nkb;
        if (A.splits > 1 && t >= A.full) {
          const int sp = (int)((t - A.full) / A.tail);
          kb_lo = nkb * sp / A.splits;
          kb_hi = nkb * (sp + 1) / A.splits;
        }
        if (!ptx::mbar_wait(&tempty[acc], accph ^ 1, lim, abort)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t dt = tmem_base + acc * BN;
        for (int64_t kb = kb_lo; kb < kb_hi; ++kb) {
          if (!ptx::mbar_wait(&full[stage], phase, lim, abort)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint64_t so = (uint64_t)((uint32_t)(stage * Cfg::STAGE_BYTES) >> 4);
#pragma unroll
          for (int s = 0; s < KB / 16; ++s)
            ptx::mma_f16(dt, da[s] + so, db[s] + so, idesc, (kb != kb_lo || s) ? 1u : 0u);
          ptx::mma_commit(&empty[stage]);
          if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        ptx::mma_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) accph ^= 1;
      }
      if (!ok && !*abort) record_timeout(abort, A.status);
      // every issued MMA finishes before tensor memory is released
      ptx::mma_commit(done);
      for (int64_t i = 0; i < ((int64_t)1 << 24); ++i)
        if (ptx::mbar_try_wait(done, 0)) break;
    }
    __syncwarp();
  } else if (warp >= EPI_WARPS + 2) {
    // ------------------------------------------------------------ gather warps
    if constexpr (NG > 0) {
      const int gw = warp - (EPI_WARPS + 2);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < nitems && ok && any_gather; t += gridDim.x) {
        const Item I = item_at(A, t, nkb);
        const TileIx& T = I.T;
        GatherCtx cx[2];
        const int64_t tr0[2] = {T.tm0, T.tn0}, tr1[2] = {T.tm1, T.tn1};
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          const BoxOp& X = A.op[w];
          const int64_t o0 = tr0[w] * X.b0, o1 = tr1[w] * X.b1;
          cx[w].tbase = o0 * X.s[0] + o1 * X.s[1] + T.il * X.s[4];
          cx[w].lim0 = (int)min(X.e[0] - o0, (int64_t)1 << 30);
          cx[w].lim1 = (int)min(X.e[1] - o1, (int64_t)1 << 30);
        }
        int64_t kb0 = I.kb_lo % A.nk0, k0s = kb0 * A.bk0, k1s = (I.kb_lo / A.nk0) * A.bk1;
        for (int64_t kb = I.kb_lo; kb < I.kb_hi; ++kb) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort)) { ok = false; break; }
          const uint32_t st = ptx::smem_u32(smem + stage * Cfg::STAGE_BYTES);
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const BoxOp& X = A.op[w];
            cx[w].kbase = k0s * X.s[2] + k1s * X.s[3];
            cx[w].klim0 = (int)min(X.e[2] - k0s, (int64_t)1 << 30);
            cx[w].klim1 = (int)min(X.e[3] - k1s, (int64_t)1 << 30);
          }
          if (!tma0) gather_tile<BM, NG>(A.op[0], st, cx[0], A.bk0 - 1, A.lbk0, A.bk1, lane, gw);
          if (!tma1) gather_tile<BN, NG>(A.op[1], st + Cfg::A_BYTES, cx[1], A.bk0 - 1, A.lbk0, A.bk1, lane, gw);
          ptx::fence_proxy_async_smem();  // generic-proxy stores -> tensor-core reads
          ptx::mbar_arrive(&full[stage]);
          if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1; }
          if (++kb0 == A.nk0) { kb0 = 0; k0s = 0; k1s += A.bk1; } else { k0s += A.bk0; }
        }
      }
      if (!ok && !*abort) record_timeout(abort, A.status);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int CPT = BN / 2;  // columns per thread
    const int qd = warp & 3, hf = warp >> 2;
    const uint32_t lane_addr = (uint32_t)(qd * 32) << 16;
    const BoxOp& P = A.op[0];
    const BoxOp& Q = A.op[1];
    uint32_t acc = 0, accph = 0;
    for (int64_t t = blockIdx.x; t < nitems; t += gridDim.x) {
      const Item I = item_at(A, t, nkb);
      const TileIx& T = I.T;
      if (!ptx::mbar_wait(&tfull[acc], accph, lim, abort)) {
        if (!*abort) record_timeout(abort, A.status);
        break;
      }
      ptx::tc_fence_after();
      const int lr = qd * 32 + lane;
      if (I.split >= 0) {
        // a split item: its fp32 partial tile, column by column (rows
        // contiguous), summed with alpha and beta by k_box_reduce
        float* pt = A.part + ((size_t)I.split * (size_t)A.tail + (size_t)I.ti) * BM * BN + lr;
#pragma unroll 1
        for (int q = 0; q < CPT / 32; ++q) {
          uint32_t r[32];
          ptx::tmem_ld32(tmem_base + lane_addr + acc * BN + hf * CPT + q * 32, r);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 32; ++i) pt[(size_t)(hf * CPT + q * 32 + i) * BM] = __uint_as_float(r[i]);
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
        acc ^= 1;
        if (acc == 0) accph ^= 1;
        continue;
      }
      const int64_t r0 = T.tm0 * P.b0 + lr % P.b0, r1 = T.tm1 * P.b1 + lr / P.b0;
      const bool rv = r0 < P.e[0] && r1 < P.e[1];
      const int64_t crow = r0 * A.cs[0] + r1 * A.cs[1] + T.il * A.cs[4];
#pragma unroll 1
      for (int q = 0; q < CPT / 32; ++q) {
        uint32_t r[32];
        ptx::tmem_ld32(tmem_base + lane_addr + acc * BN + hf * CPT + q * 32, r);
        ptx::tmem_ld_wait();
        if (!rv) continue;
        // groups of 8 columns share the second column mode's index (the
        // first mode's box is at least 16 wide): consecutive first-mode
        // indices, one stride apart in C
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          const int lc = hf * CPT + q * 32 + g8 * 8;
          const int64_t c0 = T.tn0 * Q.b0 + lc % Q.b0, c1 = T.tn1 * Q.b1 + lc / Q.b0;
          const int nv = c1 < Q.e[1] ? (int)(Q.e[0] - c0 < 8 ? Q.e[0] - c0 : 8) : 0;
          float* cp = A.c + crow + c0 * A.cs[2] + c1 * A.cs[3];
          const int64_t cs = A.cs[2];
          float old[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) old[i] = (i < nv && A.beta != 0.f) ? cp[i * cs] : 0.f;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            float v = A.alpha * __uint_as_float(r[g8 * 8 + i]);
            if (A.beta != 0.f) v = fmaf(A.beta, old[i], v);
            if (i < nv) cp[i * cs] = v;
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
  if (warp == EPI_WARPS + 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

// ----------------------------------------------------------------- host side
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// The operand's 5-D tensor map over the caller's tensor (dimensions of
// extent 1 pad it to rank 5).  The box's shared-memory order (first
// dimension fastest) is the tile layout the MMA descriptors describe:
//   K-major   {k0, r0, r1, k1, batch}, box {bk0, b0, b1, bk1, 1}: sub-tile
//             kk1, row rr0 + b0 rr1, bk0 k each; one copy per stage.
//   MN-major  {r0 within a run, k0, k1, run index, r1, batch}, box {run, bk0,
//             bk1, b0/run, b1, 1}: run column a0 + (b0/run) a1, k row kk0 +
//             bk0 kk1; one copy per stage when the first row mode's extent is
//             a multiple of the run (or the box holds one run) and at most
//             five dimensions remain after dropping those of extent 1 and
//             box 1.  Otherwise {r0, k0, k1, r1, batch} with box {run, bk0,
//             bk1, 1, 1}, one copy per run column.
// False when a stride or the base is not 16-byte aligned or the driver
// rejects the map (the gather warps then stage the operand).
bool encode_op(CUtensorMap* map, BoxOp& X, int bk0, int bk1) {
  EncodeFn enc = encode_fn();
  if (!enc || ((uintptr_t)X.x & 15) != 0) return false;
  struct Dim {
    int64_t ext, stride;  // stride in elements (dimension 0: 1)
    int box;
    int8_t role;
  };
  Dim d[6];
  int nd = 0;
  const int apr = X.mn ? X.b0 / X.run : 1;
  X.single = 1;
  if (!X.mn) {
    d[nd++] = {X.e[2], 1, bk0, ROLE_K0};
    d[nd++] = {X.e[0], X.s[0], X.b0, ROLE_R0};
    d[nd++] = {X.e[1], X.s[1], X.b1, ROLE_R1};
    d[nd++] = {X.e[3], X.s[3], bk1, ROLE_K1};
    d[nd++] = {X.e[4], X.s[4], 1, ROLE_L};
  } else {
    const bool split = apr > 1;
    if (split && X.e[0] % X.run != 0) X.single = 0;
    if (X.single) {
      d[nd++] = {split ? X.run : X.e[0], 1, X.run, split ? ROLE_ZERO : ROLE_R0};
      d[nd++] = {X.e[2], X.s[2], bk0, ROLE_K0};
      if (X.e[3] > 1 || bk1 > 1) d[nd++] = {X.e[3], X.s[3], bk1, ROLE_K1};
      if (split) d[nd++] = {X.e[0] / X.run, X.run, apr, ROLE_RHI};
      if (X.e[1] > 1 || X.b1 > 1) d[nd++] = {X.e[1], X.s[1], X.b1, ROLE_R1};
      if (X.e[4] > 1) d[nd++] = {X.e[4], X.s[4], 1, ROLE_L};
      if (nd > 5) X.single = 0;
    }
    if (!X.single) {
      nd = 0;
      d[nd++] = {X.e[0], 1, X.run, ROLE_R0};
      d[nd++] = {X.e[2], X.s[2], bk0, ROLE_K0};
      d[nd++] = {X.e[3], X.s[3], bk1, ROLE_K1};
      d[nd++] = {X.e[1], X.s[1], 1, ROLE_R1};
      d[nd++] = {X.e[4], X.s[4], 1, ROLE_L};
    }
  }
  while (nd < 5) d[nd++] = {1, 1, 1, ROLE_ZERO};
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int i = 0; i < 5; ++i) {
    dims[i] = (cuuint64_t)d[i].ext;
    box[i] = (cuuint32_t)d[i].box;
    X.role[i] = d[i].role;
    if (d[i].box > 256 || d[i].ext < 1) return false;
    if (i == 0) continue;
    // a dimension of extent 1 is never stepped: any legal stride will do
    const int64_t bytes = d[i].ext > 1 ? d[i].stride * 2 : 16;
    if (bytes <= 0 || bytes % 16 != 0 || bytes >= ((int64_t)1 << 40)) return false;
    strides[i - 1] = (cuuint64_t)bytes;
  }
  const CUtensorMapSwizzle sw = X.run == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                            : (X.run == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(X.x), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The two modes of a class as an ordered pair for one operand: first the
// mode with unit stride in that operand when `unit_first`, else the one
// with the smaller stride in C (the epilogue's coalescing order).
struct Pair {
  Mode m[2];
  int n;
};

// An absent mode (extent 1: only index 0 is ever formed) takes stride 1 in
// both operands, so that an empty class can serve as a unit-stride mode.
constexpr Mode kAbsent{1, 1, 1, 0};

Pair order_class(const ClassModes& cm, int which, bool want_unit) {
  Pair p;
  p.n = cm.n;
  const Mode absent = kAbsent;
  p.m[0] = cm.n > 0 ? cm.m[0] : absent;
  p.m[1] = cm.n > 1 ? cm.m[1] : absent;
  auto st = [&](const Mode& m) { return which == 0 ? m.sa : (which == 1 ? m.sb : m.sc); };
  bool swap;
  if (want_unit && cm.n == 2 && st(p.m[1]) == 1 && st(p.m[0]) != 1) swap = true;
  else if (want_unit && cm.n == 2 && st(p.m[0]) == 1) swap = false;
  else swap = cm.n == 2 && p.m[1].sc < p.m[0].sc;
  if (swap) std::swap(p.m[0], p.m[1]);
  return p;
}

// Box (b0, b1), b0 * b1 = rows, b0 a power of two (a run of the shared-
// memory layout is a power-of-two number of elements and divides b0),
// minimising the padded volume; ties go to the longer first box (longer
// contiguous runs, wider swizzle).
void pick_box(int64_t e0, int64_t e1, int rows, int min_b0, int* b0, int* b1) {
  int64_t best = -1;
  for (int c0 = 256; c0 >= min_b0; c0 /= 2) {
    if (c0 > rows || rows % c0) continue;
    const int c1 = rows / c0;
    const int64_t vol = ((e0 + c0 - 1) / c0) * c0 * ((e1 + c1 - 1) / c1) * c1;
    if (best < 0 || vol < best) {
      best = vol;
      *b0 = c0;
      *b1 = c1;
    }
  }
}

struct BoxPlan {
  BoxArgs a;
  int bn;
  int64_t tiles;
};

// Splits of the tail (the last, partly empty round of the persistent grid):
// s items per tail tile take ceil(tail s / SMs) / s rounds instead of one;
// s minimises that (each step up must save 2 %), up to 4 when whole rounds
// precede the tail, else up to max(16, SMs / tiles), and each split keeps at
// least 4 k blocks (256 k).  Returns s; *rounds gets the launch's rounds.
int tail_splits(int64_t tiles, int64_t sms, int64_t nkb, double* rounds_out) {
  const int64_t full = (tiles / sms) * sms, tail = tiles - full;
  auto rounds = [&](int64_t sp) { return (double)((tail * sp + sms - 1) / sms) * (1.0 / (double)sp + 0.01); };
  int64_t best = 1;
  if (tail > 0) {
    const int64_t most = full == 0 ? std::max<int64_t>(16, (sms + tail - 1) / tail) : 4;
    const int64_t cap = std::min<int64_t>(most, nkb / 4);
    for (int64_t sp = 2; sp <= cap; ++sp)
      if (rounds(sp) < 0.98 * rounds(best)) best = sp;
  }
  if (rounds_out) *rounds_out = (double)(full / sms) + (tail > 0 ? rounds(best) : 0.0);
  return (int)best;
}

double split_rounds(int64_t tiles, int64_t sms, int64_t nkb) {
  double r = 0.0;
  tail_splits(tiles, sms, nkb, &r);
  return r;
}

// Structural plan (no device work, no tensor maps): false when the call
// does not fit the kernel (the packed path then serves it).
bool plan_box(const Plan& p, int tile_n, BoxPlan* out) {
  if (p.kernel != FAMLIES_KERNEL_TC_BF16_DIRECT && p.kernel != FAMLIES_KERNEL_TC_BF16) return false;
  if (p.M.n > 2 || p.N.n > 2 || p.K.n > 2 || p.L.n > 1) return false;
  if (p.k > kBoxMaxK || p.tri || p.sym_n || p.band_side >= 0 || p.krp_side >= 0) return false;
  BoxArgs& a = out->a;
  std::memset(&a, 0, sizeof(a));
  const ClassModes* R[2] = {&p.M, &p.N};
  // majorness per operand: MN-major when a row mode is unit-stride, else
  // K-major when a contracted mode is
  int unit_k[2] = {-1, -1};
  bool mn[2];
  for (int w = 0; w < 2; ++w) {
    mn[w] = R[w]->n == 0;  // an empty row class: its absent mode is unit-stride
    for (int i = 0; i < R[w]->n; ++i)
      if ((w == 0 ? R[w]->m[i].sa : R[w]->m[i].sb) == 1) mn[w] = true;
    if (!mn[w]) {
      if (p.K.n == 0) unit_k[w] = 0;
      for (int i = 0; i < p.K.n; ++i)
        if ((w == 0 ? p.K.m[i].sa : p.K.m[i].sb) == 1) unit_k[w] = i;
    }
    if (!mn[w] && unit_k[w] < 0) return false;  // no unit stride: the pack serves it
  }
  if (unit_k[0] >= 0 && unit_k[1] >= 0 && unit_k[0] != unit_k[1]) return false;
  const int uk = unit_k[0] >= 0 ? unit_k[0] : unit_k[1];
  // contracted modes: the K-major operand's unit mode first
  Mode km[2] = {p.K.n > 0 ? p.K.m[0] : kAbsent, p.K.n > 1 ? p.K.m[1] : kAbsent};
  if (uk == 1) std::swap(km[0], km[1]);
  // contracted box: a K-major operand's run is bk0 (16/32/64 k)
  int bk0 = 64, bk1 = 1;
  pick_box(km[0].ext, km[1].ext, KB, 16, &bk0, &bk1);
  a.bk0 = bk0;
  a.bk1 = bk1;
  a.nk0 = (km[0].ext + bk0 - 1) / bk0;
  a.nk1 = (km[1].ext + bk1 - 1) / bk1;
  // row boxes
  Pair pr[2];
  for (int w = 0; w < 2; ++w) pr[w] = order_class(*R[w], w, mn[w]);
  // tile width: fewest padded rounds of the persistent grid, weighted by a
  // tile's relative cost per column (narrow tiles feed the MMA less per
  // byte staged)
  const int64_t sms = num_sms();
  int rb0 = 128, rb1 = 1;
  pick_box(pr[0].m[0].ext, pr[0].m[1].ext, BM, 16, &rb0, &rb1);
  const int64_t t0a = (pr[0].m[0].ext + rb0 - 1) / rb0, t1a = (pr[0].m[1].ext + rb1 - 1) / rb1;
  const int cands[4] = {256, 192, 128, 64};
  const double eff[4] = {1.0, 1.04, 1.12, 1.5};
  double best = -1;
  int bn = 256, cb0 = 256, cb1 = 1;
  for (int c = 0; c < 4; ++c) {
    if (tile_n && cands[c] != tile_n) continue;
    int b0 = cands[c], b1 = 1;
    pick_box(pr[1].m[0].ext, pr[1].m[1].ext, cands[c], 16, &b0, &b1);
    const int64_t tiles = t0a * t1a * ((pr[1].m[0].ext + b0 - 1) / b0) * ((pr[1].m[1].ext + b1 - 1) / b1) *
                          (p.l > 0 ? p.l : 1);
    const double cost = split_rounds(tiles, sms, a.nk0 * a.nk1) * cands[c] * eff[c];
    if (best < 0 || cost < best - 1e-9) {
      best = cost;
      bn = cands[c];
      cb0 = b0;
      cb1 = b1;
    }
  }
  if (best < 0) return false;
  out->bn = bn;
  const int rows[2] = {BM, bn};
  const int b0s[2] = {rb0, cb0}, b1s[2] = {rb1, cb1};
  const void* xs[2] = {p.a, p.b};
  for (int w = 0; w < 2; ++w) {
    BoxOp& X = a.op[w];
    X.x = xs[w];
    auto st = [&](const Mode& m) { return w == 0 ? m.sa : m.sb; };
    X.e[0] = pr[w].m[0].ext; X.s[0] = st(pr[w].m[0]);
    X.e[1] = pr[w].m[1].ext; X.s[1] = st(pr[w].m[1]);
    X.e[2] = km[0].ext; X.s[2] = st(km[0]);
    X.e[3] = km[1].ext; X.s[3] = st(km[1]);
    X.e[4] = p.L.n ? p.L.m[0].ext : 1;
    X.s[4] = p.L.n ? st(p.L.m[0]) : 0;
    X.mn = mn[w] ? 1 : 0;
    X.b0 = b0s[w];
    X.b1 = b1s[w];
    X.run = mn[w] ? std::min(X.b0, 64) : bk0;
    if (mn[w] && X.s[0] != 1) return false;
    if (!mn[w] && X.s[2] != 1) return false;
    X.tma = 0;
    a.t0[w] = (X.e[0] + X.b0 - 1) / X.b0;
    a.t1[w] = (X.e[1] + X.b1 - 1) / X.b1;
  }
  // the shared-memory layouts the descriptors describe: runs of 16, 32 or
  // 64 elements that tile each box exactly
  for (int w = 0; w < 2; ++w) {
    const BoxOp& X = a.op[w];
    if (X.run != 16 && X.run != 32 && X.run != 64) return false;
    if (X.b0 * X.b1 != rows[w] || (X.b0 & (X.b0 - 1)) != 0) return false;
    if (X.mn ? (X.b0 % X.run != 0) : (X.run != bk0)) return false;
  }
  if (bk0 * bk1 != KB || (bk0 & (bk0 - 1)) != 0) return false;
  auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return l; };
  a.lbk0 = lg(bk0);
  for (int w = 0; w < 2; ++w) {
    BoxOp& X = a.op[w];
    X.lrun = lg(X.run);
    X.lb0 = lg(X.b0);
    X.lapr = X.mn ? lg(X.b0 / X.run) : 0;
  }
  a.l = p.L.n ? p.L.m[0].ext : 1;
  a.cs[0] = pr[0].m[0].sc;
  a.cs[1] = pr[0].m[1].sc;
  a.cs[2] = pr[1].m[0].sc;
  a.cs[3] = pr[1].m[1].sc;
  a.cs[4] = p.L.n ? p.L.m[0].sc : 0;
  out->tiles = a.t0[0] * a.t1[0] * a.t0[1] * a.t1[1] * a.l;
  return out->tiles > 0;
}

// Split K: C = alpha * (sum of the splits' partial tiles, in split order) +
// beta * C for the tail tiles.  Grid (column chunks, tail tiles); thread t
// owns row t % 128 and columns chunk * 16 + t / 128 + 2 j.
__global__ void __launch_bounds__(256) k_box_reduce(const BoxArgs a, int bn) {
  constexpr int COLS = 16, PER = COLS / 2;
  const BoxOp& P = a.op[0];
  const BoxOp& Q = a.op[1];
  const int lr = threadIdx.x % BM, lq = threadIdx.x / BM;
  const size_t per_tile = (size_t)BM * bn, per_split = (size_t)a.tail * per_tile;
  const int64_t ti = blockIdx.y;
  const int c0 = blockIdx.x * COLS;
  const TileIx T = tile_ix(a, a.full + ti);
  const int64_t r0 = T.tm0 * P.b0 + lr % P.b0, r1 = T.tm1 * P.b1 + lr / P.b0;
  if (!(r0 < P.e[0] && r1 < P.e[1])) return;
  const int64_t crow = r0 * a.cs[0] + r1 * a.cs[1] + T.il * a.cs[4];
  float sum[PER], old[PER];
  int64_t off[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int lc = c0 + lq + 2 * j;
    const int64_t n0 = T.tn0 * Q.b0 + lc % Q.b0, n1 = T.tn1 * Q.b1 + lc / Q.b0;
    off[j] = (n0 < Q.e[0] && n1 < Q.e[1]) ? crow + n0 * a.cs[2] + n1 * a.cs[3] : -1;
    sum[j] = 0.f;
  }
  const float* pt = a.part + (size_t)ti * per_tile + (size_t)(c0 + lq) * BM + lr;
  for (int sp = 0; sp < a.splits; ++sp) {
    float v[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) v[j] = pt[(size_t)sp * per_split + (size_t)(2 * j) * BM];
#pragma unroll
    for (int j = 0; j < PER; ++j) sum[j] += v[j];
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) old[j] = (off[j] >= 0 && a.beta != 0.f) ? a.c[off[j]] : 0.f;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    float v = a.alpha * sum[j];
    if (a.beta != 0.f) v = fmaf(a.beta, old[j], v);
    if (off[j] >= 0) a.c[off[j]] = v;
  }
}

void plan_splits(BoxPlan& bp, int64_t nkb) {
  BoxArgs& a = bp.a;
  const int64_t sms = num_sms();
  a.full = (bp.tiles / sms) * sms;
  a.tail = bp.tiles - a.full;
  a.splits = tail_splits(bp.tiles, sms, nkb, nullptr);
}

template <int BN, int NG>
cudaError_t launch_cfg(const CUtensorMap& ma, const CUtensorMap& mb, const BoxArgs& a, int grid, cudaStream_t s) {
  using Cfg = BoxCfg<BN, NG>;
  constexpr int kMaxDev = 64;
  static bool attr[kMaxDev] = {};
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return e;
  if (dev >= kMaxDev || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_box<BN, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDev) attr[dev] = true;
  }
  k_box<BN, NG><<<grid, Cfg::THREADS, Cfg::SMEM_BYTES, s>>>(ma, mb, a);
  return cudaGetLastError();
}

template <int NG>
cudaError_t launch_ng(int bn, const CUtensorMap& ma, const CUtensorMap& mb, const BoxArgs& a, int grid,
                      cudaStream_t s) {
  switch (bn) {
    case 64: return launch_cfg<64, NG>(ma, mb, a, grid, s);
    case 128: return launch_cfg<128, NG>(ma, mb, a, grid, s);
    case 192: return launch_cfg<192, NG>(ma, mb, a, grid, s);
    default: return launch_cfg<256, NG>(ma, mb, a, grid, s);
  }
}


// Re-pad copy of an operand whose strides (or base) no tensor map can
// address (e.g. a first-mode stride padded to an odd number of elements):
// the same elements in the same mode order, the unit-stride mode u first
// with stride 1 and each other mode's stride the span before it rounded up
// to 8 elements (16 bytes).  Not a transpose: only the padding changes, so
// that the product's copies can read the operand as a tensor map.
struct RepadArgs {
  int64_t e[5];   // extents
  int64_t ss[5];  // source strides (elements)
  int64_t ds[5];  // destination strides
  int u;          // the unit-stride mode
  int64_t rows;   // product of the other extents
};

// One thread per 16-byte destination chunk (8 consecutive elements along u of
// one row: a fixed index of every mode but u), so every thread's loads are
// independent of every other's; index arithmetic in 32 bits (the host
// checks that the chunk count fits).  Destination rows start on 16-byte
// boundaries, so a full chunk is one aligned 16-byte store.
__global__ void __launch_bounds__(256) k_repad(const uint16_t* __restrict__ src, uint16_t* __restrict__ dst,
                                               const RepadArgs r) {
  uint32_t m4[4], e4[4];
  int nm = 0;
  for (int m = 0; m < 5; ++m)
    if (m != r.u) {
      m4[nm] = (uint32_t)m;
      e4[nm++] = (uint32_t)r.e[m];
    }
  const uint32_t eu = (uint32_t)r.e[r.u], cpr = (eu + 7) / 8;
  const int64_t ssu = r.ss[r.u];
  const uint32_t items = (uint32_t)(r.rows * cpr);
  for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
    uint32_t rest = it / cpr;
    const uint32_t x0 = (it - rest * cpr) * 8;
    int64_t so = 0, dof = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t q = rest / e4[j], i = rest - q * e4[j];
      rest = q;
      so += (int64_t)i * r.ss[m4[j]];
      dof += (int64_t)i * r.ds[m4[j]];
    }
    const uint32_t n = eu - x0 < 8 ? eu - x0 : 8;
    uint32_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = e < (int)n ? src[so + (int64_t)(x0 + e) * ssu] : 0u;
    if (n == 8) {
      *(uint4*)(dst + dof + x0) = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16),
                                             v[6] | (v[7] << 16));
    } else {
      for (uint32_t e = 0; e < n; ++e) dst[dof + x0 + e] = (uint16_t)v[e];
    }
  }
}

// Fills r and the re-padded operand's view; returns the copy's bytes.
int64_t repad_layout(const BoxOp& X, RepadArgs* r, BoxOp* out) {
  std::memset(r, 0, sizeof(*r));
  r->u = X.mn ? 0 : 2;
  int order[4], n = 0;
  for (int m = 0; m < 5; ++m)
    if (m != r->u) order[n++] = m;
  std::stable_sort(order, order + 4, [&](int x, int y) { return X.s[x] < X.s[y]; });
  *out = X;
  r->rows = 1;
  for (int m = 0; m < 5; ++m) {
    r->e[m] = X.e[m];
    r->ss[m] = X.s[m];
    if (m != r->u) r->rows *= X.e[m];
  }
  r->ds[r->u] = 1;
  int64_t span = X.e[r->u];
  for (int i = 0; i < 4; ++i) {
    const int m = order[i];
    r->ds[m] = (span + 7) / 8 * 8;
    span = r->ds[m] * X.e[m];
  }
  int64_t last = 0;
  for (int m = 0; m < 5; ++m) {
    out->s[m] = r->ds[m];
    last += (X.e[m] - 1) * r->ds[m];
  }
  return (last + 1) * 2;
}

// Host side of one direct call: plan, tensor maps, and which operands need
// the re-pad copy first (their workspace offsets).
struct BoxLaunch {
  BoxPlan bp;
  CUtensorMap maps[2];
  bool repad[2];
  RepadArgs rp[2];
  int64_t off[2];
  int64_t ws;
};

bool prepare_box(const Plan& p, int force_gather, BoxLaunch* L) {
  if (!plan_box(p, p.tile_n, &L->bp)) return false;
  BoxArgs& a = L->bp.a;
  std::memset(L->maps, 0, sizeof(L->maps));
  plan_splits(L->bp, a.nk0 * a.nk1);
  L->ws = a.splits > 1 ? ((int64_t)a.splits * a.tail * BM * L->bp.bn * 4 + 255) / 256 * 256 : 0;
  for (int w = 0; w < 2; ++w) {
    L->repad[w] = false;
    L->off[w] = 0;
    BoxOp& X = a.op[w];
    X.tma = 0;
    if (force_gather & (1 << w)) continue;  // the gather warps stage it
    if (encode_op(&L->maps[w], X, a.bk0, a.bk1)) {
      X.tma = 1;
      continue;
    }
    BoxOp padded;
    const int64_t bytes = repad_layout(X, &L->rp[w], &padded);
    if (L->rp[w].rows * ((X.e[L->rp[w].u] + 7) / 8) >= ((int64_t)1 << 32)) continue;  // gathered instead
    L->repad[w] = true;
    L->off[w] = L->ws;
    L->ws += (bytes + 255) / 256 * 256;
    X = padded;  // strides now; the base is set at launch
  }
  return true;
}

}  // namespace

bool box_applicable(const Plan& p) {
  BoxPlan bp;
  return plan_box(p, p.tile_n, &bp);
}

int64_t box_workspace_bytes(const Plan& p) {
  BoxLaunch L;
  return prepare_box(p, p.force_gather, &L) ? L.ws : -1;
}

cudaError_t launch_box(const Plan& p, const GemmArgs& g, void* ws, cudaStream_t s, int* launches) {
  BoxLaunch L;
  if (!prepare_box(p, p.force_gather, &L)) return cudaErrorNotSupported;
  BoxArgs& a = L.bp.a;
  int n = 0;
  for (int w = 0; w < 2; ++w) {
    if (!L.repad[w]) continue;
    if (!ws) return cudaErrorInvalidValue;
    uint16_t* dst = (uint16_t*)((char*)ws + L.off[w]);
    const int64_t chunks = L.rp[w].rows * ((L.rp[w].e[L.rp[w].u] + 7) / 8);
    const int64_t blocks = std::min<int64_t>((chunks + 255) / 256, (int64_t)num_sms() * 16);
    k_repad<<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>((const uint16_t*)a.op[w].x, dst, L.rp[w]);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
    ++n;
    a.op[w].x = dst;
    a.op[w].tma = encode_op(&L.maps[w], a.op[w], a.bk0, a.bk1) ? 1 : 0;  // else gathered from the copy
  }
  a.c = (float*)g.c;
  a.alpha = (float)g.alpha;
  a.beta = (float)g.beta;
  a.status = g.status;
  a.wait_limit = g.wait_limit;
  a.stall_test = g.stall_test;
  a.part = a.splits > 1 ? (float*)ws : nullptr;  // the partial tiles lead the workspace
  if (a.splits > 1 && !ws) return cudaErrorInvalidValue;
  const int64_t items = a.splits > 1 ? a.full + a.tail * a.splits : L.bp.tiles;
  const int grid = (int)std::min<int64_t>(items, num_sms());
  const bool gather = !a.op[0].tma || !a.op[1].tma;
  mark_begin(g, s);
  cudaError_t e = gather ? launch_ng<NGATHER>(L.bp.bn, L.maps[0], L.maps[1], a, grid, s)
                         : launch_ng<0>(L.bp.bn, L.maps[0], L.maps[1], a, grid, s);
  mark_end(g, s);
  ++n;
  if (e == cudaSuccess && a.splits > 1) {
    // grid.y over the tail tiles (fewer than the SMs, so within its limit)
    k_box_reduce<<<dim3((unsigned)(L.bp.bn / 16), (unsigned)a.tail), 256, 0, s>>>(a, L.bp.bn);
    e = cudaGetLastError();
    ++n;
  }
  if (launches) *launches = n;
  return e;
}

}  // namespace famlies
