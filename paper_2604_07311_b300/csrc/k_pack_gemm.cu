// Packed tensor-core contraction: one re-layout pass per operand, then a
// TMA-fed tcgen05 product over pairs of packed "slices".
//
// Pack.  Each operand is read once through its offset tables (coalesced
// along its unit-stride index, transposed through shared memory) and written
// K-major, one 16-byte chunk per thread, as S slices P[s][l][r][k]:
//   plain bf16   S = 1, the bf16 values themselves;
//   tf32 split   S = 2, hi = tf32(x) and lo = tf32(x - hi) (fp32 words);
//   fp64 split   S = s, integer digits of x scaled by its row's power of two:
//                x = 2^e_r * sum_i d_i 2^(-b i) + remainder, |d_1| <= 2^b,
//                |d_i| <= 2^(b-1) for i > 1 (round-to-nearest digits), every
//                digit exact in bf16.  e_r bounds the row's largest
//                magnitude (a first, read-only pass).  Rows holding Inf/NaN
//                are flagged and recomputed natively afterwards.
// This is the BLIS packing step of Fig. 2 with the tensor re-organisation
// and the precision split fused into it (Sec. 1 "Challenges"; mixed
// precision, Sec. 1.5; packing hoisted with data re-organisation, Girder 2).
//
// Product.  A persistent, warp-specialised kernel: one thread issues TMA
// loads of slice tiles into a shared-memory ring, one thread issues
// tcgen05.mma into a double-buffered fp32 accumulator in tensor memory, and
// eight epilogue warps drain it.  The work of one output tile is a list of
// "units"; a unit accumulates a set of slice pairs over a k range.
//   bf16 / tf32: one unit (all pairs, all of K); epilogue C = alpha*acc +
//                beta*C in fp32.
//   fp64 split:  the pairs with i + j = d (a "diagonal", weight 2^(-b d))
//                for d = s+1 down to 2; a unit covers a k range short enough
//                that the fp32 accumulator stays an exact integer (< 2^24),
//                the epilogue adds it into int32 running sums and, at each
//                diagonal's end, adds them (scaled by the diagonal's weight)
//                into an int64 tile sum with reductions performed at L2; the
//                tile's end converts the sum once to fp64 and writes
//                C = alpha * 2^(e_m+e_n) * sum + beta * C.
// The fp32 accumulation is exact because every partial sum is an integer
// below 2^24, and so is the int64 recombination down to the finest weight K
// allows; only the final scaling and the alpha/beta update use fp64
// arithmetic (B300's fp64 pipe is narrow).
//
// Grouped launches (many independent problems, e.g. the blocks of a
// block-sparse contraction) run the same kernel over a device tile list:
// each entry names its problem, whose descriptor (TMA maps in global memory,
// C's offset tables, scalars) the roles read per tile.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "device.h"
#include "packed.h"
#include "pair_gemm.h"
#include "ptx.cuh"

namespace famlies {

namespace {

constexpr int BM = kPairBM;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 32 * (EPI_WARPS + 2);  // + TMA producer, MMA issuer

struct PairArgs {
  Prob single;           // the problem of a single-problem launch
  const Prob* probs;     // grouped: problem descriptors (device)
  const TileEntry* tiles;  // grouped: tile list (device)
  int64_t ntiles;        // grouped: tile count
  Sched sc;
  double* G;             // fp64 split: per-CTA fp64 tile sums
  int splits;            // single problem: K splits of each tail tile
  int tailed;            // single problem: tail items write tile slots finished by k_split_finish /
                         // k_split_reduce (K splits, or the deferred finish of short-K tiles)
  int64_t full;          // splits > 1: the leading tiles that run whole (the rest is the tail)
  int64_t* xtail;        // fp64 split, splits > 1: int64 sums of the tail tiles [tail][BN][BM];
                         // grouped with defer: the sums of every tile of the list [tile][BN][BM]
  int defer;             // grouped, fp64 split: tiles leave their sums in xtail for k_group_finish
  int stall_test;        // testing: the MMA issuer first waits on a barrier nothing completes
  float* part;           // fp32 output, splits > 1: partial tail tiles [split][tail][BN][BM]
  int* status;
  int64_t wait_limit;
};

// CG: CTAs per MMA.  With 2 (a cluster pair, cta_group::2) a tile is
// 2 BM x BN: each CTA stages its BM rows of A and BN / 2 of B's columns and
// holds its BM rows of the accumulator; the MMA reads both CTAs' halves.
template <int KIND, int BN, int MODE = PAIR_MODE_F32OUT, int CG = 1>
struct PCfg {
  static constexpr int KB = pair_stage_k(KIND);            // k per stage
  static constexpr int ROWB = pair_row_bytes(KIND);        // bytes of one tile row in a stage
  static constexpr int MMA_K = KIND == PAIR_KIND_BF16 ? 16 : 8;
  static constexpr int KSTEPS = KB / MMA_K;
  static constexpr int TM = BM * CG;                       // rows of an output tile
  static constexpr int B_ROWS = BN / CG;                   // this CTA's columns of B per stage
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = B_ROWS * ROWB;
  // Ring stages (as many as ~200 KB holds, at most 8).  The row operand's
  // tiles fill one region and the column operand's another, stage s of each
  // guarded by one barrier pair.  (Separate producers and rings of different
  // depth per operand measured slower on both the fp64 split and bf16.)
  // (A pair's 32 KB stages take the whole 227 KB: seven of them.)
  static constexpr int RING = CG == 2 ? 227 * 1024 - 1536 : 200 * 1024;
  static constexpr int STAGES = RING / (A_BYTES + B_BYTES) > 8 ? 8 : RING / (A_BYTES + B_BYTES);
  static constexpr int B_OFF = STAGES * A_BYTES;
  static constexpr int BAR_OFF = B_OFF + STAGES * B_BYTES;
  // Accumulator buffers in tensor memory: two of 256 columns, or four of
  // 128 (64) columns, so that short units of narrower tiles are drained
  // while the next ones accumulate.
  static constexpr int NACC = BN == 256 ? 2 : 4;
  static constexpr uint32_t TMEM_COLS = NACC * BN;
  static constexpr uint32_t IDESC = ptx::idesc_make(TM, BN, KIND == PAIR_KIND_BF16 ? 1u : 2u);
  static constexpr int SMEM_BYTES = BAR_OFF + 1024 + 512;
  static_assert(STAGES >= 2 && SMEM_BYTES <= 227 * 1024, "shared memory budget");
};

__device__ __forceinline__ void record_timeout(volatile int* abort, int* status) {
  *abort = 1;
  atomicCAS(status, 0, FAMLIES_ERR_DEVICE_TIMEOUT);
}

// One work item: an output tile (tm, tn, il) of problem P and, with split K,
// the part of its k blocks [kb_lo, kb_hi) this item covers.
struct TileRef {
  const Prob* P;
  int64_t tm, tn, il;
  int64_t tile;  // single problems: the tile's number
  int split;
  int kb_lo, kb_hi;
};

// Output tiles of a single problem: the whole grid of bn-wide tiles, or
// those of its triangle list; and the coordinates of tile number `tile`
// (column tiles fastest, then row tiles, then the batch).
// rm: rows of a tile (BM, or 2 BM for a CTA pair).
__host__ __device__ __forceinline__ int64_t prob_tiles(const Prob& P, int bn, int rm = BM) {
  return P.tri_list ? P.tri_tiles : ((P.m + rm - 1) / rm) * ((P.n + bn - 1) / bn) * P.l;
}
__device__ __forceinline__ void tile_coords(const Prob& P, int bn, int64_t tile, int64_t& tm, int64_t& tn,
                                            int64_t& il, int rm = BM) {
  if (P.tri_list) {
    const int2 e = P.tri_list[tile];
    tm = e.x;
    tn = e.y;
    il = 0;
    return;
  }
  const int64_t tiles_m = (P.m + rm - 1) / rm, tiles_n = (P.n + bn - 1) / bn;
  tn = tile % tiles_n;
  const int64_t rest = tile / tiles_n;
  tm = rest % tiles_m;
  il = rest / tiles_m;
}

template <int BN, bool GROUPED, bool SPLITK, int RM = BM>
__device__ __forceinline__ int64_t tile_count(const PairArgs& a) {
  if (GROUPED) return a.ntiles;
  const int64_t ntile = prob_tiles(a.single, BN, RM);
  return SPLITK ? a.full + (ntile - a.full) * a.splits : ntile;
}

// Item t of the launch.  Single problems walk column tiles fastest, so the
// CTAs running at the same time share A tiles through L2.  With split K the
// first `full` items are whole tiles (whole rounds of the persistent grid);
// each tail tile then runs as `splits` items over parts of its k range,
// splits the slowest index (concurrent CTAs read the same k range).  A split
// covers whole units of the fp32-output schedule, or any k blocks for the
// fp64 split (each diagonal forms its units inside the range).
template <int BN, bool GROUPED, int KB, bool SPLITK, int RM = BM>
__device__ __forceinline__ TileRef tile_at(const PairArgs& a, int64_t t) {
  if (GROUPED) {
    const TileEntry e = a.tiles[t];
    const Prob* P = a.probs + e.p;
    return TileRef{P, e.tm, e.tn, e.il, 0, -1, 0, (int)((P->k + KB - 1) / KB)};
  }
  const Prob& P = a.single;
  const int nkb = (int)((P.k + KB - 1) / KB);
  int64_t tile = t;
  int split = -1, lo = 0, hi = nkb;
  if (SPLITK && t >= a.full) {
    const int64_t tail = prob_tiles(P, BN, RM) - a.full, u = t - a.full;
    tile = a.full + u % tail;
    split = (int)(u / tail);
    const int kcb = a.sc.ndiag > 1 ? 1 : a.sc.kcb[0];
    const int64_t units = (nkb + kcb - 1) / kcb;
    lo = (int)(units * split / a.splits) * kcb;
    hi = (int)(units * (split + 1) / a.splits) * kcb;
    hi = hi < nkb ? hi : nkb;
  }
  int64_t tm, tn, il;
  tile_coords(P, BN, tile, tm, tn, il, RM);
  return TileRef{&a.single, tm, tn, il, tile, split, lo, hi};
}

// The end of an fp64-split tile: C = alpha * 2^(e_m + e_n - xunit) * X + beta
// * C for this thread's row and CPT columns (X: the int64 tile sums), in
// groups of columns whose table entries, X and C are loaded together.  X is
// read from L2 (the reductions that built it ran there).  AK, BK: alpha and
// beta classified as FinishScale does (AK 0: alpha = +-2^p, applied in
// integer arithmetic; BK: beta 0, 1 or other), fixed at compile time so that
// no fp64 instruction of an untaken choice runs.
template <int CPT, bool FINE, int AK, int BK>
__device__ __forceinline__ void finish_cols(const Prob& P, const int64_t* Xt, const Sched& sc, int64_t il,
                                         int64_t row, int64_t crow, int64_t col0, int lc0, int bnp) {
  // the fine sums follow the coarse ones in the tile's slot (tiles 2 CPT wide)
  const int64_t* Lt = Xt + (size_t)BM * (2 * CPT);
  const int xunit = sc.xunit, xlo = sc.xlo;
  double* C = (double*)P.c;
  const double alpha = P.alpha, beta = P.beta;
  const FinishScale fs = finish_scale(P.alpha, P.beta);
  const int er = P.ea[il * P.m + row] - xunit + fs.a_p;
  const int32_t* ebl = P.eb + il * P.n;
  const int32_t* fbl = P.fb + il * P.n;
  const double lsc = ldexp(1.0, xunit - xlo);
  constexpr int FG = 8;
#pragma unroll 1
  for (int j0 = 0; j0 < CPT; j0 += FG) {
    bool use[FG];
    int ecol[FG];
    int64_t coff[FG];
    int64_t g[FG], gl[FG];
    double cold[FG];
#pragma unroll
    for (int j = 0; j < FG; ++j) {
      const int64_t col = col0 + j0 + j;
      use[j] = lc0 + j0 + j < bnp && col < P.n && tri_keep(P.tri, row, col);
      ecol[j] = use[j] ? ebl[col] : 0;
      coff[j] = use[j] ? P.cn[col] : 0;
      use[j] = use[j] && !fbl[col];
      g[j] = __ldcg(Xt + (size_t)(j0 + j) * BM);
      gl[j] = FINE ? __ldcg(Lt + (size_t)(j0 + j) * BM) : 0;
    }
#pragma unroll
    for (int j = 0; j < FG; ++j) cold[j] = (use[j] && BK) ? C[crow + coff[j]] : 0.0;
#pragma unroll
    for (int j = 0; j < FG; ++j) {
      const int e = er + ecol[j];
      // the two sums in units of 2^-xunit (lsc: an exact power of two),
      // alpha's sign applied to them; converted with integer instructions
      const int64_t g0 = fs.a_neg ? -g[j] : g[j], g1 = fs.a_neg ? -gl[j] : gl[j];
      const double x = FINE ? fma(i64_to_f64_rn(g1), lsc, i64_to_f64_rn(g0)) : i64_to_f64_rn(g0);
      // x * 2^e by adding e to x's exponent field (integer arithmetic: the
      // fp64 pipe is narrow) when the result stays a normal number
      const long long xb = __double_as_longlong(x);
      const int ex = (int)((xb >> 52) & 0x7FF);
      const double scaled = (ex != 0 && ex + e >= 1 && ex + e <= 2046)
                                ? __longlong_as_double(xb + ((long long)e << 52))
                                : ldexp(x, e);
      // (compile-time choices: no fp64 instruction for a branch not taken)
      double v = scaled;
      if constexpr (AK == 1) v = alpha * scaled;
      if constexpr (BK == 1) v = v + cold[j];
      if constexpr (BK == 2) v = fma(beta, cold[j], v);
      if (use[j]) C[crow + coff[j]] = v;
      if (P.emit_mode) {  // a network's fused epilogue: the consumer's exponents
        bool bad = false;
        const int ve = use[j] ? f64_row_exp(v, &bad) : -2000;
        const unsigned act = __activemask();  // the lanes finishing this tile
        const int64_t ci = P.emit_mode == 1 ? row : col0 + j0 + j;
        if (P.emit_mode == 1) {
          if (ve > -2000) atomicMax(&P.emit_e[ci], ve);
          if (use[j] && bad) emit_mark(P.emit_flag, P.emit_list, ci);
        } else {
          const int wm = __reduce_max_sync(act, ve);
          const unsigned wb = __reduce_or_sync(act, (use[j] && bad) ? 1u : 0u);
          if ((threadIdx.x & 31) == (unsigned)(__ffs(act) - 1) && ci < P.n) {
            if (wm > -2000) atomicMax(&P.emit_e[ci], wm);
            if (wb) emit_mark(P.emit_flag, P.emit_list, ci);
          }
        }
      }
    }
  }
}

// finish_cols for the problem's alpha and beta (the same for every tile of
// a single problem; per problem in a grouped launch): the choice is made once
// per call, outside the loops over columns.  Not inlined: one call site in
// the product kernel keeps its registers out of the drain loop's budget.
template <int CPT, bool FINE>
__device__ __noinline__ void finish_tile(const Prob& P, const int64_t* Xt, const Sched& sc, int64_t il,
                                         int64_t row, int64_t crow, int64_t col0, int lc0, int bnp) {
  const FinishScale fs = finish_scale(P.alpha, P.beta);
  if (!fs.a_gen) {
    if (fs.b_kind == 0) finish_cols<CPT, FINE, 0, 0>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
    else if (fs.b_kind == 1) finish_cols<CPT, FINE, 0, 1>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
    else finish_cols<CPT, FINE, 0, 2>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
  } else {
    if (fs.b_kind == 0) finish_cols<CPT, FINE, 1, 0>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
    else if (fs.b_kind == 1) finish_cols<CPT, FINE, 1, 1>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
    else finish_cols<CPT, FINE, 1, 2>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
  }
}

// Items of a CTA: its own for CG = 1, its cluster's for a pair (both CTAs
// of a cluster walk the same items; CTAs of a cluster have consecutive
// numbers).
template <int CG>
__device__ __forceinline__ int64_t first_item() { return CG == 2 ? blockIdx.x >> 1 : blockIdx.x; }
template <int CG>
__device__ __forceinline__ int64_t item_step() { return CG == 2 ? gridDim.x >> 1 : gridDim.x; }

// The TMA producer: walks the CTA's unit sequence (tiles, diagonals, units,
// pairs, k blocks, exactly as the MMA issuer consumes it) and fills stage s
// of both operand regions per k block.  On a timeout it sets the abort flag;
// before returning it waits (bounded) for its copies still in flight.
// A CTA pair: each CTA loads its own rows of A and columns of B, and both
// count their bytes on the even CTA's stage barrier (the one the MMA issuer
// waits on); the stage is free again once the issuer's commit reaches this
// CTA's own empty barrier.
// A diagonal's k blocks [kb_lo, kb_hi) run in units of kcb blocks (the last
// one ragged).  Odd diagonals take the units from the top down, so that each
// diagonal starts on the k range its predecessor read last, while those
// operand tiles may still be in L2 (the integer sums do not depend on the
// order).  The producer and the issuer walk the same sequence; the drain
// only counts units.
__device__ __forceinline__ int unit_count(const TileRef& T, int kcb) {
  return (T.kb_hi - T.kb_lo + kcb - 1) / kcb;
}
__device__ __forceinline__ void unit_range(const TileRef& T, int kcb, int di, int uu, int nun, int& kb0,
                                           int& kb1) {
  const int u = (di & 1) ? nun - 1 - uu : uu;
  kb0 = T.kb_lo + u * kcb;
  kb1 = kb0 + kcb < T.kb_hi ? kb0 + kcb : T.kb_hi;
}

template <class Cfg, int BN, bool GROUPED, bool SPLITK, int CG>
__device__ __forceinline__ void produce(const PairArgs& args, const CUtensorMap* map_a,
                                        const CUtensorMap* map_b, uint8_t* ring_a, uint8_t* ring_b,
                                        uint64_t* full, uint64_t* empty, int64_t ntiles,
                                        int64_t lim, volatile int* abort) {
  constexpr int S = Cfg::STAGES;
  const uint32_t rank = CG == 2 ? ptx::cluster_rank() : 0;
  const uint32_t full0 = CG == 2 ? ptx::mapa(full, 0) : 0;  // the even CTA's barriers
  const Sched& sc = args.sc;
  if (!GROUPED) {
    ptx::prefetch_tmap(map_a);
    ptx::prefetch_tmap(map_b);
  }
  int stage = 0;
  uint32_t phase = 0;
  uint32_t pending = 0;  // bit s: stage s holds a copy issued in phase bit (s+8)
  bool ok = true;
  // the row operand's tiles are read by the CTAs of one row of tiles at
  // about the same time, the column operand's by every row of tiles: keep
  // the latter in L2.  A grouped list interleaves the tiles of many problems
  // longest first, so neither holds there and its loads take no hint
  // (evict-first made the 2000-block batch ~8 % slower).
  const uint64_t pol_a = ptx::policy_evict_first(), pol_b = ptx::policy_evict_last();
  for (int64_t t = first_item<CG>(); t < ntiles && ok; t += item_step<CG>()) {
    const TileRef T = tile_at<BN, GROUPED, Cfg::KB, SPLITK, Cfg::TM>(args, t);
    const CUtensorMap* ma = GROUPED ? T.P->map_a : map_a;
    const CUtensorMap* mb = GROUPED ? T.P->map_b : map_b;
    const int l = (int)T.P->l;
    const int bnp = GROUPED ? T.P->bn : BN;  // this tile's width
    const uint32_t bytes = (uint32_t)(CG * Cfg::A_BYTES + bnp * Cfg::ROWB);  // both CTAs' for a pair
    const int row_a = (int)(T.tm * Cfg::TM + rank * BM), row_b = (int)(T.tn * bnp + rank * Cfg::B_ROWS);
    for (int di = 0; di < sc.ndiag && ok; ++di) {
      const int kcb = sc.kcb[di];
      const int nun = unit_count(T, kcb);
      for (int uu = 0; uu < nun && ok; ++uu) {
        int kb0, kb1;
        unit_range(T, kcb, di, uu, nun, kb0, kb1);
        for (int p = 0; p < sc.npairs[di] && ok; ++p) {
          // slices are stored [slice][batch][rows][k]
          const int za = sc.pa[di][p] * l + (int)T.il;
          const int zb = sc.pb[di][p] * l + (int)T.il;
          for (int kb = kb0; kb < kb1; ++kb) {
            if constexpr (CG == 2) {
              if (!ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort)) { ok = false; break; }
              if (rank == 0) ptx::mbar_arrive_expect_tx(&full[stage], bytes);
              const uint32_t fb = full0 + 8u * (uint32_t)stage;
              ptx::tma_load_3d_pair(ring_a + stage * Cfg::A_BYTES, ma, fb, kb * Cfg::KB, row_a, za);
              ptx::tma_load_3d_pair(ring_b + stage * Cfg::B_BYTES, mb, fb, kb * Cfg::KB, row_b, zb);
            } else {
              if (!ptx::mbar_wait(&empty[stage], phase ^ 1, lim, abort)) { ok = false; break; }
              ptx::mbar_arrive_expect_tx(&full[stage], bytes);
              if constexpr (GROUPED) {
                ptx::tma_load_3d(ring_a + stage * Cfg::A_BYTES, ma, &full[stage], kb * Cfg::KB, row_a, za);
                ptx::tma_load_3d(ring_b + stage * Cfg::B_BYTES, mb, &full[stage], kb * Cfg::KB, row_b, zb);
              } else {
                ptx::tma_load_3d_hint(ring_a + stage * Cfg::A_BYTES, ma, &full[stage], kb * Cfg::KB, row_a, za,
                                      pol_a);
                ptx::tma_load_3d_hint(ring_b + stage * Cfg::B_BYTES, mb, &full[stage], kb * Cfg::KB, row_b, zb,
                                      pol_b);
              }
            }
            pending = (pending & ~(0x101u << stage)) | (1u << stage) | (phase << (stage + 8));
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
        }
      }
    }
  }
  if (!ok && !*abort) record_timeout(abort, args.status);
  // Copies still in flight must land before the CTA leaves: wait (bounded)
  // for the phase each stage was last filled in.  (The odd CTA of a pair
  // cannot wait on the even CTA's barriers: the pair's closing cluster
  // barrier follows the issuer's wait for its last MMA, which read every
  // stage both CTAs filled.)
  if (CG == 2 && rank != 0) return;
  for (int s = 0; s < S; ++s) {
    if (!(pending & (1u << s))) continue;
    const uint32_t ph = (pending >> (s + 8)) & 1u;
    for (int64_t i = 0; i < ((int64_t)1 << 22); ++i)
      if (ptx::mbar_try_wait(&full[s], ph)) break;
  }
}

template <int KIND, int MODE, int BN, bool GROUPED, bool SPLITK, int CG = 1>
__global__ void __launch_bounds__(THREADS, 1)
    k_pair_gemm(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                const __grid_constant__ PairArgs args) {
  static_assert(CG == 1 || (CG == 2 && KIND == PAIR_KIND_BF16 && !GROUPED), "CTA pairs: bf16 single problems");
  using Cfg = PCfg<KIND, BN, MODE, CG>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + Cfg::BAR_OFF);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* tfull = empty + Cfg::STAGES;
  uint64_t* tempty = tfull + Cfg::NACC;
  uint64_t* done = tempty + Cfg::NACC;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const Sched& sc = args.sc;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t ntiles = tile_count<BN, GROUPED, SPLITK, Cfg::TM>(args);
  const int64_t lim = args.wait_limit;
  const uint32_t rank = CG == 2 ? ptx::cluster_rank() : 0;  // 0: the CTA that issues the MMAs

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < Cfg::NACC; ++b) {
      ptx::mbar_init(&tfull[b], 1);
      ptx::mbar_init(&tempty[b], EPI_WARPS * CG);  // a pair: both CTAs' epilogue warps
    }
    ptx::mbar_init(done, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == EPI_WARPS + 1) {
    if constexpr (CG == 2) {
      ptx::tmem_alloc_pair(tmem_slot, Cfg::TMEM_COLS);
      ptx::tmem_relinquish_pair();
    } else {
      ptx::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
      ptx::tmem_relinquish();
    }
  }
  ptx::tc_fence_before();
  // a pair: the other CTA's barriers are initialised before anything reaches them
  if constexpr (CG == 2) {
    __syncwarp();
    ptx::cluster_sync();
  } else {
    __syncthreads();
  }
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == EPI_WARPS) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0)
      produce<Cfg, BN, GROUPED, SPLITK, CG>(args, &map_a, &map_b, smem, smem + Cfg::B_OFF, full, empty,
                                            ntiles, lim, abort);
    __syncwarp();
  } else if (warp == EPI_WARPS + 1) {
    // ------------------------------------------------------------ MMA issue
    // (a pair: the even CTA's thread issues for both; each commit is sent
    // to the barrier of each CTA, one commit per CTA)
    if (lane == 0 && rank == 0) {
      int stage = 0;
      uint32_t phase = 0, acc = 0, accph = 0;
      const uint32_t empty0 = CG == 2 ? ptx::mapa(empty, 0) : 0, empty1 = CG == 2 ? ptx::mapa(empty, 1) : 0;
      const uint32_t tfull0 = CG == 2 ? ptx::mapa(tfull, 0) : 0, tfull1 = CG == 2 ? ptx::mapa(tfull, 1) : 0;
      auto wait = [&](uint64_t* bar, uint32_t par) { return ptx::mbar_wait(bar, par, lim, abort); };
      // testing: `done` completes only after this thread's last commit
      bool ok = !args.stall_test || ptx::mbar_wait(done, 0, lim, abort);
      for (int64_t t = first_item<CG>(); t < ntiles && ok; t += item_step<CG>()) {
        const TileRef T = tile_at<BN, GROUPED, Cfg::KB, SPLITK, Cfg::TM>(args, t);
        // the MMA's N is this tile's width (the instruction descriptor's N field)
        const uint32_t idesc =
            GROUPED ? ptx::idesc_make(BM, T.P->bn, KIND == PAIR_KIND_BF16 ? 1u : 2u) : Cfg::IDESC;
        for (int di = 0; di < sc.ndiag && ok; ++di) {
          const int kcb = sc.kcb[di];
          const int nun = unit_count(T, kcb);
          for (int uu = 0; uu < nun && ok; ++uu) {
            int kb0, kb1;
            unit_range(T, kcb, di, uu, nun, kb0, kb1);
            if (!wait(&tempty[acc], accph ^ 1)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t dt = tmem_base + acc * BN;
            uint32_t accumulate = 0;
            for (int p = 0; p < sc.npairs[di] && ok; ++p) {
              for (int kb = kb0; kb < kb1; ++kb) {
                if (!wait(&full[stage], phase)) { ok = false; break; }
                ptx::tc_fence_after();
                const uint64_t da = ptx::sdesc_kmajor<Cfg::ROWB>(ptx::smem_u32(smem + stage * Cfg::A_BYTES));
                const uint64_t db =
                    ptx::sdesc_kmajor<Cfg::ROWB>(ptx::smem_u32(smem + Cfg::B_OFF + stage * Cfg::B_BYTES));
#pragma unroll
                for (int kk = 0; kk < Cfg::KSTEPS; ++kk) {
                  if (CG == 2)
                    ptx::mma_f16_pair(dt, da + 2 * kk, db + 2 * kk, idesc, accumulate);
                  else if (KIND == PAIR_KIND_BF16)
                    ptx::mma_f16(dt, da + 2 * kk, db + 2 * kk, idesc, accumulate);
                  else
                    ptx::mma_tf32(dt, da + 2 * kk, db + 2 * kk, idesc, accumulate);
                  accumulate = 1;
                }
                if constexpr (CG == 2) {
                  ptx::mma_commit_pair(empty0 + 8u * (uint32_t)stage);
                  ptx::mma_commit_pair(empty1 + 8u * (uint32_t)stage);
                } else {
                  ptx::mma_commit(&empty[stage]);
                }
                if (++stage == Cfg::STAGES) { stage = 0; phase ^= 1; }
              }
            }
            if (!ok) break;
            if constexpr (CG == 2) {
              ptx::mma_commit_pair(tfull0 + 8u * acc);
              ptx::mma_commit_pair(tfull1 + 8u * acc);
            } else {
              ptx::mma_commit(&tfull[acc]);
            }
            if (++acc == Cfg::NACC) { acc = 0; accph ^= 1; }
          }
        }
      }
      if (!ok && !*abort) record_timeout(abort, args.status);
      if constexpr (CG == 2) ptx::mma_commit_pair(ptx::mapa(done, 0));
      else ptx::mma_commit(done);
      for (int64_t i = 0; i < ((int64_t)1 << 24); ++i)
        if (ptx::mbar_try_wait(done, 0)) break;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    constexpr int CPT = BN / 2;  // columns per thread
    const int qd = warp & 3, hf = warp >> 2;
    const uint32_t lane_addr = (uint32_t)(qd * 32) << 16;
    uint32_t acc = 0, accph = 0;
    bool ok = true;
    // a pair: the accumulator buffer is released to the even CTA's issuer
    const uint32_t tempty0 = CG == 2 ? ptx::mapa(tempty, 0) : 0;
    auto wait_full = [&](uint32_t b, uint32_t par) { return ptx::mbar_wait(&tfull[b], par, lim, abort); };
    auto release = [&](uint32_t b) {
      if (CG == 2 && rank != 0) ptx::mbar_arrive_cluster(tempty0 + 8u * b);
      else ptx::mbar_arrive(&tempty[b]);
    };
    for (int64_t t = first_item<CG>(); t < ntiles && ok; t += item_step<CG>()) {
      const TileRef T = tile_at<BN, GROUPED, Cfg::KB, SPLITK, Cfg::TM>(args, t);
      const Prob& P = *T.P;
      const int nkb = T.kb_hi - T.kb_lo;  // k blocks of this item
      const int64_t il = T.il;
      const int64_t row = T.tm * Cfg::TM + rank * BM + qd * 32 + lane;
      const int bnp = GROUPED ? P.bn : BN;  // this tile's width
      const int lc0 = hf * CPT;             // first tile-local column of this thread
      const int64_t col0 = T.tn * bnp + lc0;
      const bool rv = row < P.m;
      const int64_t crow = rv ? P.cl[il] + P.cm[row] : 0;
      if (MODE == PAIR_MODE_F32OUT) {
        // Each unit's tensor-memory sum is added into fp32 registers with
        // round-to-nearest, which bounds how much rounding any one
        // accumulator sees over a long k.
        float S[CPT];
        const int kcb = sc.kcb[0];
        const int nunits = (nkb + kcb - 1) / kcb;
        for (int u = 0; u < nunits; ++u) {
          if (!wait_full(acc, accph)) { ok = false; break; }
          ptx::tc_fence_after();
#pragma unroll
          for (int q = 0; q < CPT / 32; ++q) {
            if (lc0 + q * 32 >= bnp) continue;  // beyond this tile's width (warp-uniform)
            uint32_t r[32];
            ptx::tmem_ld32(tmem_base + lane_addr + acc * BN + hf * CPT + q * 32, r);
            ptx::tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 32; ++i)
              S[q * 32 + i] = (u == 0) ? __uint_as_float(r[i]) : S[q * 32 + i] + __uint_as_float(r[i]);
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) release(acc);
          if (++acc == Cfg::NACC) { acc = 0; accph ^= 1; }
        }
        if (!ok) break;
        if (SPLITK && T.split >= 0) {
          // a split of a tail tile: its partial tile, reduced (with alpha,
          // beta) by k_split_reduce
          const int64_t tail = prob_tiles(P, BN) - args.full;
          float* Pt = args.part + ((size_t)T.split * (size_t)tail + (size_t)(T.tile - args.full)) * BM * BN +
                      (size_t)lc0 * BM + qd * 32 + lane;
#pragma unroll
          for (int j = 0; j < CPT; ++j) Pt[(size_t)j * BM] = S[j];
        } else if (rv) {
          float* C = (float*)P.c;
          const float alpha = (float)P.alpha, beta = (float)P.beta;
#pragma unroll
          for (int j = 0; j < CPT; ++j) {
            const int64_t col = col0 + j;
            if (lc0 + j < bnp && col < P.n && tri_keep(P.tri, row, col)) {
              float* p = C + crow + P.cn[col];
              float v = alpha * S[j];
              if (beta != 0.f) v = fmaf(beta, *p, v);
              *p = v;
            }
          }
        }
      } else {
        // fp64 split: int32 running sums per diagonal, two int64 tile sums:
        // Xt in units of 2^-xunit (the diagonals whose weight is at least
        // that) and Lt in units of 2^-xlo (the finer ones), so that every
        // flush is an exact shift however long K is and however many
        // splits share a tile.
        int32_t S[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) S[j] = 0;
        // tile sums: a slot per CTA for a whole tile; for a split of a tail
        // tile the tile's slot, shared by its splits through the reductions
        // and finished by k_split_finish.  A slot holds the coarse sums, then
        // the fine ones (BM x BN each); the fine diagonals are di < nlow (the
        // walk runs from the least significant diagonal up).
        const bool part_item = SPLITK && T.split >= 0;
        constexpr bool FINE = MODE == PAIR_MODE_EMU_FINE;
        constexpr size_t slot = (size_t)BM * BN * (FINE ? 2 : 1);
        // a pair's tail tiles (every tile split, no batch): each CTA's half
        // has the slot of its BM-row tile, numbered as k_split_finish numbers them
        const int64_t xi = CG == 2 ? (2 * T.tm + rank) * ((P.n + BN - 1) / BN) + T.tn : T.tile - args.full;
        // a deferred grouped tile (one CTA owns it, so its first flush
        // stores) keeps its sums in its own slot for k_group_finish
        const bool deferred = GROUPED && args.defer;
        int64_t* Xt = (part_item  ? args.xtail + (size_t)xi * slot
                       : deferred ? args.xtail + (size_t)t * slot
                                  : (int64_t*)args.G + (size_t)blockIdx.x * slot) +
                      (size_t)(hf * CPT) * BM + qd * 32 + lane;
        bool first_flush = true;
        for (int di = 0; di < sc.ndiag && ok; ++di) {
          const int kcb = sc.kcb[di];
          const int nunits = (nkb + kcb - 1) / kcb;
          if (FINE && di == sc.nlow) first_flush = true;  // the first diagonal of the coarse sums
          for (int u = 0; u < nunits; ++u) {
            if (!wait_full(acc, accph)) { ok = false; break; }
            ptx::tc_fence_after();
            const bool last_unit = (u == nunits - 1);
            const bool flush = last_unit || ((u + 1) % sc.flush_every[di]) == 0;
#pragma unroll
            for (int q = 0; q < CPT / 32; ++q) {
              if (lc0 + q * 32 >= bnp) continue;  // beyond this tile's width (warp-uniform)
              uint32_t r[32];
              ptx::tmem_ld32(tmem_base + lane_addr + acc * BN + hf * CPT + q * 32, r);
              ptx::tmem_ld_wait();
#pragma unroll
              for (int i = 0; i < 32; ++i) S[q * 32 + i] += __float2int_rn(__uint_as_float(r[i]));
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) release(acc);
            if (++acc == Cfg::NACC) { acc = 0; accph ^= 1; }
            if (!flush) continue;
            // sum += S * 2^xshift in int64 (exact, order-free): the first
            // flush into a tile's sum stores, later ones are fire-and-forget
            // reductions performed at L2, so no flush waits on memory.
            {
              const int xs = sc.xshift[di];
              int64_t* D = (FINE && di < sc.nlow) ? Xt + (size_t)BM * BN : Xt;
              const bool first = first_flush && !part_item;
#pragma unroll
              for (int j = 0; j < CPT; ++j) {
                int64_t v = (int64_t)S[j];
                v = xs >= 0 ? (int64_t)((uint64_t)v << xs) : ((v + ((int64_t)1 << (-xs - 1))) >> (-xs));
                if (first) D[(size_t)j * BM] = v;
                else atomicAdd((unsigned long long*)(D + (size_t)j * BM), (unsigned long long)v);
                S[j] = 0;
              }
              first_flush = false;
            }
            if (part_item || deferred || !(last_unit && di == sc.ndiag - 1) || !rv || P.fa[il * P.m + row])
              continue;
            finish_tile<CPT, FINE>(P, Xt, sc, il, row, crow, col0, lc0, bnp);
          }
        }
      }
    }
    if (!ok && !*abort) record_timeout(abort, args.status);
  }

  ptx::tc_fence_before();
  // a pair: neither CTA leaves (nor frees its tensor memory) while the
  // issuer's MMAs may still read its shared memory or write its tensor memory
  if constexpr (CG == 2) {
    __syncwarp();
    ptx::cluster_sync();
  } else {
    __syncthreads();
  }
  if (warp == EPI_WARPS + 1) {
    ptx::tc_fence_after();
    if constexpr (CG == 2) ptx::tmem_dealloc_pair(tmem_base, Cfg::TMEM_COLS);
    else ptx::tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

// Split-K finishing kernels.  Work item: a tile (numbered as tile_at numbers
// them) and a chunk of SPLIT_COLS of its columns; thread t owns row t % BM
// and every other column of the chunk from t / BM, so that the partial
// reads and the C accesses run along rows; each thread issues the loads of
// all its columns before the stores.
constexpr int SPLIT_COLS = 16;
constexpr int SPLIT_PER_THREAD = SPLIT_COLS / (256 / BM);

// fp32 output: C = alpha * (sum of the splits' partial tiles, in split order)
// + beta * C.
__global__ void __launch_bounds__(256, 4) k_split_reduce(const float* __restrict__ part, int splits,
                                                     int64_t full, int bn, Prob P) {
  const int chunks = bn / SPLIT_COLS;
  const int64_t tail = prob_tiles(P, bn) - full, items = tail * chunks;
  const size_t per = (size_t)BM * bn, total = (size_t)tail * per;
  float* C = (float*)P.c;
  const float alpha = (float)P.alpha, beta = (float)P.beta;
  const int lr = threadIdx.x % BM, lq = threadIdx.x / BM;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t ti = it / chunks, tile = full + ti;  // ti: index among the tail tiles
    const int c0 = (int)(it % chunks) * SPLIT_COLS;
    int64_t tm, tn, il;
    tile_coords(P, bn, tile, tm, tn, il);
    const int64_t row = tm * BM + lr;
    if (row >= P.m) continue;
    const int64_t crow = P.cl[il] + P.cm[row];
    float sum[SPLIT_PER_THREAD], old[SPLIT_PER_THREAD];
    int64_t off[SPLIT_PER_THREAD];
#pragma unroll
    for (int j = 0; j < SPLIT_PER_THREAD; ++j) {
      const int lc = c0 + lq + j * (256 / BM);
      const int64_t col = tn * bn + lc;
      off[j] = col < P.n && tri_keep(P.tri, row, col) ? crow + P.cn[col] : -1;
      const size_t at = (size_t)ti * per + (size_t)lc * BM + lr;
      float acc = 0.f;
      for (int sp = 0; sp < splits; ++sp) acc += part[(size_t)sp * total + at];
      sum[j] = acc;
    }
#pragma unroll
    for (int j = 0; j < SPLIT_PER_THREAD; ++j) old[j] = (off[j] >= 0 && beta != 0.f) ? C[off[j]] : 0.f;
#pragma unroll
    for (int j = 0; j < SPLIT_PER_THREAD; ++j) {
      float v = alpha * sum[j];
      if (beta != 0.f) v = fmaf(beta, old[j], v);
      if (off[j] >= 0) C[off[j]] = v;
    }
  }
}

// fp64 split: the splits of a tile added their int64 sums into one slot;
// C = alpha * 2^(e_m + e_n - xunit) * sum + beta * C (rows and columns
// holding Inf/NaN are left to the native fix-up).  Item: a tail tile and
// FIN_COLS of its columns.  The item's column tables (C offset, exponent;
// offset -1 for a column left to the fix-up or past the edge) are staged in
// shared memory once, beside each thread's row tables; thread t then owns
// row t % BM and the item's columns t / BM + 2 j, a group at a time, with
// the sums and the C entries of a group loaded together.  An item thus waits on
// the tables once and then on one level of loads per group (a 16-column
// item that fetched its own tables waited on three levels and kept the
// kernel at ~2.8 TB/s).  AK, BK: alpha and beta classified on the host (see
// FinishScale).
constexpr int FIN_COLS = 64;

template <bool FINE, int AK, int BK>
__global__ void __launch_bounds__(256, 3) k_split_finish(const int64_t* __restrict__ X, int64_t full,
                                                     int bn, int xunit, int xlo, Prob P) {
  // columns per group: 8, or 4 with the second (fine) sums, whose loads
  // and converts would not fit the register budget at 8
  constexpr int FIN_G = FINE ? 4 : 8;
  __shared__ int64_t s_cn[FIN_COLS];
  __shared__ int32_t s_ec[FIN_COLS];
  const int chunks = (bn + FIN_COLS - 1) / FIN_COLS;
  const int64_t items = (prob_tiles(P, bn) - full) * chunks;
  const size_t per = (size_t)BM * bn, slot = per * (FINE ? 2 : 1);
  const double lsc = ldexp(1.0, xunit - xlo);
  const FinishScale fs = finish_scale(P.alpha, P.beta);
  double* C = (double*)P.c;
  const int lr = threadIdx.x % BM, lq = threadIdx.x / BM;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t ti = it / chunks, tile = full + ti;  // ti: index among the tail tiles
    const int c0 = (int)(it % chunks) * FIN_COLS;
    int64_t tm, tn, il;
    tile_coords(P, bn, tile, tm, tn, il);
    const int64_t row = tm * BM + lr;
    const bool rv = row < P.m;
    __syncthreads();  // the previous item's reads of the column tables are done
    if (threadIdx.x < FIN_COLS) {
      const int lc = c0 + (int)threadIdx.x;
      const int64_t col = tn * bn + lc;
      const bool ok = lc < bn && col < P.n;
      const int32_t fb = ok ? P.fb[il * P.n + col] : 1;
      const int64_t cn = ok ? P.cn[col] : 0;
      const int32_t ec = ok ? P.eb[il * P.n + col] : 0;
      s_cn[threadIdx.x] = (ok && !fb) ? cn : -1;
      s_ec[threadIdx.x] = ec;
    }
    const bool rskip = !rv || P.fa[il * P.m + (rv ? row : 0)];
    const int64_t crow = P.cl[il] + (rv ? P.cm[row] : 0);
    const int er = (rv ? P.ea[il * P.m + row] : 0) - xunit + fs.a_p;
    __syncthreads();
    const int64_t* Xt = X + (size_t)ti * slot + lr;
    int rmx = -2000;
    bool rbad = false;
#pragma unroll 1
    for (int g0 = 0; g0 < FIN_COLS / 2; g0 += FIN_G) {
      int64_t x[FIN_G], xl[FIN_G], off[FIN_G];
      int32_t ec[FIN_G];
      double old[FIN_G];
#pragma unroll
      for (int j = 0; j < FIN_G; ++j) {
        const int cc = lq + 2 * (g0 + j);  // column within the item
        const int lc = c0 + cc;            // column within the tile
        const int64_t cn = s_cn[cc];
        off[j] = (!rskip && cn >= 0 && tri_keep(P.tri, row, tn * bn + lc)) ? crow + cn : -1;
        ec[j] = s_ec[cc];
        x[j] = lc < bn ? Xt[(size_t)lc * BM] : 0;
        xl[j] = (FINE && lc < bn) ? Xt[per + (size_t)lc * BM] : 0;
      }
#pragma unroll
      for (int j = 0; j < FIN_G; ++j) old[j] = (off[j] >= 0 && BK) ? C[off[j]] : 0.0;
#pragma unroll
      for (int j = 0; j < FIN_G; ++j) {
        // alpha's sign on the sums, their conversion and scaling in integer
        // instructions (see FinishScale)
        const int64_t x0 = fs.a_neg ? -x[j] : x[j], x1 = fs.a_neg ? -xl[j] : xl[j];
        const double xd = FINE ? fma(i64_to_f64_rn(x1), lsc, i64_to_f64_rn(x0)) : i64_to_f64_rn(x0);
        const int e = er + ec[j];
        const long long xb = __double_as_longlong(xd);
        const int ex = (int)((xb >> 52) & 0x7FF);
        const double scaled = (ex != 0 && ex + e >= 1 && ex + e <= 2046)
                                  ? __longlong_as_double(xb + ((long long)e << 52))
                                  : ldexp(xd, e);
        // (compile-time choices: no fp64 instruction for a branch not taken)
        double v = scaled;
        if constexpr (AK == 1) v = P.alpha * scaled;
        if constexpr (BK == 1) v = v + old[j];
        if constexpr (BK == 2) v = fma(P.beta, old[j], v);
        if (off[j] >= 0) C[off[j]] = v;
        if (P.emit_mode) {  // a network's fused epilogue: the consumer's exponents
          bool bad = false;
          const int ve = off[j] >= 0 ? f64_row_exp(v, &bad) : -2000;
          if (P.emit_mode == 1) {
            rmx = max(rmx, ve);
            rbad = rbad || (off[j] >= 0 && bad);
          } else {  // consumer row = this column: reduce over the warp's 32 rows
            const int wm = __reduce_max_sync(0xffffffffu, ve);
            const unsigned wb = __reduce_or_sync(0xffffffffu, (off[j] >= 0 && bad) ? 1u : 0u);
            const int64_t col = tn * bn + c0 + lq + 2 * (g0 + j);
            if ((threadIdx.x & 31) == 0 && col < P.n) {
              if (wm > -2000) atomicMax(&P.emit_e[col], wm);
              if (wb) emit_mark(P.emit_flag, P.emit_list, col);
            }
          }
        }
      }
    }
    if (P.emit_mode == 1 && rv) {
      if (rmx > -2000) atomicMax(&P.emit_e[row], rmx);
      if (rbad) emit_mark(P.emit_flag, P.emit_list, row);
    }
  }
}

// k_split_finish for the problem's alpha and beta (classified as FinishScale
// does on the device): power-of-two alpha and beta 0 or 1 take no fp64
// multiply.
template <bool FINE>
cudaError_t launch_split_finish_a(bool agen, int bk, int grid, const int64_t* X, int64_t full, int bn, int xunit,
                                  int xlo, const Prob& P, cudaStream_t s) {
  if (!agen) {
    if (bk == 0) k_split_finish<FINE, 0, 0><<<grid, 256, 0, s>>>(X, full, bn, xunit, xlo, P);
    else if (bk == 1) k_split_finish<FINE, 0, 1><<<grid, 256, 0, s>>>(X, full, bn, xunit, xlo, P);
    else k_split_finish<FINE, 0, 2><<<grid, 256, 0, s>>>(X, full, bn, xunit, xlo, P);
  } else {
    if (bk == 0) k_split_finish<FINE, 1, 0><<<grid, 256, 0, s>>>(X, full, bn, xunit, xlo, P);
    else if (bk == 1) k_split_finish<FINE, 1, 1><<<grid, 256, 0, s>>>(X, full, bn, xunit, xlo, P);
    else k_split_finish<FINE, 1, 2><<<grid, 256, 0, s>>>(X, full, bn, xunit, xlo, P);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_finish(bool fine, int grid, const int64_t* X, int64_t full, int bn, int xunit, int xlo,
                                const Prob& P, cudaStream_t s) {
  uint64_t u;
  std::memcpy(&u, &P.alpha, sizeof(u));
  const int E = (int)((u >> 52) & 0x7FF);
  const bool agen = !((u & 0xFFFFFFFFFFFFFull) == 0 && E >= 1 && E <= 2046);
  const int bk = P.beta == 0.0 ? 0 : (P.beta == 1.0 ? 1 : 2);
  return fine ? launch_split_finish_a<true>(agen, bk, grid, X, full, bn, xunit, xlo, P, s)
              : launch_split_finish_a<false>(agen, bk, grid, X, full, bn, xunit, xlo, P, s);
}

// Grouped, fp64 split, deferred: every tile of the list left its int64 sums
// in its slot (xtail [tile][bn][BM], bn the launch's widest tile); this
// finishes them all after the product, like k_split_finish, per item a tile
// and FIN_COLS of its columns, with the tile's own problem (tables, width,
// alpha and beta, classified per item at run time; the branches are uniform
// across an item) and no fp64 instruction for alpha = +-2^p or beta 0.
template <bool FINE>
__global__ void __launch_bounds__(256, 3) k_group_finish(const int64_t* __restrict__ X, const Prob* __restrict__ probs,
                                                     const TileEntry* __restrict__ tiles, int64_t ntiles, int bn,
                                                     int xunit, int xlo) {
  constexpr int FIN_G = FINE ? 4 : 8;
  __shared__ int64_t s_cn[FIN_COLS];
  __shared__ int32_t s_ec[FIN_COLS];
  const int chunks = (bn + FIN_COLS - 1) / FIN_COLS;
  const int64_t items = ntiles * chunks;
  const size_t per = (size_t)BM * bn, slot = per * (FINE ? 2 : 1);
  const double lsc = ldexp(1.0, xunit - xlo);
  const int lr = threadIdx.x % BM, lq = threadIdx.x / BM;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t ti = it / chunks;
    const int c0 = (int)(it % chunks) * FIN_COLS;
    const TileEntry te = tiles[ti];
    const Prob& P = probs[te.p];
    const int bnp = P.bn;  // this tile's width
    if (c0 >= bnp) continue;  // the whole block skips the item together
    const int64_t tm = te.tm, tn = te.tn, il = te.il;
    const FinishScale fs = finish_scale(P.alpha, P.beta);
    double* C = (double*)P.c;
    const int64_t row = tm * BM + lr;
    const bool rv = row < P.m;
    __syncthreads();  // the previous item's reads of the column tables are done
    if (threadIdx.x < FIN_COLS) {
      const int lc = c0 + (int)threadIdx.x;
      const int64_t col = tn * bnp + lc;
      const bool ok = lc < bnp && col < P.n;
      const int32_t fb = ok ? P.fb[il * P.n + col] : 1;
      const int64_t cn = ok ? P.cn[col] : 0;
      const int32_t ec = ok ? P.eb[il * P.n + col] : 0;
      s_cn[threadIdx.x] = (ok && !fb) ? cn : -1;
      s_ec[threadIdx.x] = ec;
    }
    const bool rskip = !rv || P.fa[il * P.m + (rv ? row : 0)];
    const int64_t crow = P.cl[il] + (rv ? P.cm[row] : 0);
    const int er = (rv ? P.ea[il * P.m + row] : 0) - xunit + fs.a_p;
    __syncthreads();
    const int64_t* Xt = X + (size_t)ti * slot + lr;
#pragma unroll 1
    for (int g0 = 0; g0 < FIN_COLS / 2; g0 += FIN_G) {
      int64_t x[FIN_G], xl[FIN_G], off[FIN_G];
      int32_t ec[FIN_G];
      double old[FIN_G];
#pragma unroll
      for (int j = 0; j < FIN_G; ++j) {
        const int cc = lq + 2 * (g0 + j);  // column within the item
        const int lc = c0 + cc;            // column within the tile
        const int64_t cn = s_cn[cc];
        off[j] = (!rskip && cn >= 0) ? crow + cn : -1;
        ec[j] = s_ec[cc];
        x[j] = off[j] >= 0 ? Xt[(size_t)lc * BM] : 0;
        xl[j] = (FINE && off[j] >= 0) ? Xt[per + (size_t)lc * BM] : 0;
      }
#pragma unroll
      for (int j = 0; j < FIN_G; ++j) old[j] = (off[j] >= 0 && fs.b_kind != 0) ? C[off[j]] : 0.0;
#pragma unroll
      for (int j = 0; j < FIN_G; ++j) {
        if (off[j] < 0) continue;
        const int64_t x0 = fs.a_neg ? -x[j] : x[j], x1 = fs.a_neg ? -xl[j] : xl[j];
        const double xd = FINE ? fma(i64_to_f64_rn(x1), lsc, i64_to_f64_rn(x0)) : i64_to_f64_rn(x0);
        const int e = er + ec[j];
        const long long xb = __double_as_longlong(xd);
        const int ex = (int)((xb >> 52) & 0x7FF);
        const double scaled = (ex != 0 && ex + e >= 1 && ex + e <= 2046)
                                  ? __longlong_as_double(xb + ((long long)e << 52))
                                  : ldexp(xd, e);
        double v = fs.a_gen ? P.alpha * scaled : scaled;
        if (fs.b_kind == 1) v = v + old[j];
        else if (fs.b_kind == 2) v = fma(P.beta, old[j], v);
        C[off[j]] = v;
      }
    }
  }
}


// The tiles of a triangle of C (tri 1: row >= col, 2: row <= col): row tile
// tm meets it in the column tiles [lo, hi).
__host__ __device__ __forceinline__ void tri_run(int tri, int64_t tm, int bn, int64_t tiles_n, int64_t& lo,
                                                 int64_t& hi) {
  if (tri == 1) {
    lo = 0;
    hi = (tm * BM + BM - 1) / bn + 1;
    hi = hi < tiles_n ? hi : tiles_n;
  } else {
    lo = tm * BM / bn;
    lo = lo < tiles_n ? lo : tiles_n;
    hi = tiles_n;
  }
}

// Writes the triangle's tile list, row tile by row tile (column tiles
// fastest, so the CTAs running together share row tiles through L2):
// thread tm writes its row tile's run after the earlier runs.
__global__ void __launch_bounds__(256) k_tri_tiles(int tri, int64_t tiles_m, int64_t tiles_n, int bn,
                                                  int2* __restrict__ out) {
  for (int64_t tm = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tm < tiles_m;
       tm += (int64_t)gridDim.x * blockDim.x) {
    int64_t off = 0, lo, hi;
    for (int64_t t = 0; t < tm; ++t) {
      tri_run(tri, t, bn, tiles_n, lo, hi);
      off += hi - lo;
    }
    tri_run(tri, tm, bn, tiles_n, lo, hi);
    for (int64_t tn = lo; tn < hi; ++tn) out[off++] = make_int2((int)tm, (int)tn);
  }
}

int64_t tri_tile_count(const Plan& p, int bn) {
  const int64_t tiles_m = (p.m + BM - 1) / BM, tiles_n = (p.n + bn - 1) / bn;
  int64_t n = 0, lo, hi;
  for (int64_t tm = 0; tm < tiles_m; ++tm) {
    tri_run(p.tri, tm, bn, tiles_n, lo, hi);
    n += hi - lo;
  }
  return n;
}

// Output tiles the product of plan p runs (host side of prob_tiles).
int64_t plan_tiles(const Plan& p, int bn) {
  return p.tri ? tri_tile_count(p, bn) : ((p.m + BM - 1) / BM) * ((p.n + bn - 1) / bn) * p.l;
}

// ----------------------------------------------------------------- launch
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// K splits of a single problem.  A persistent launch over T tiles on the
// SMs runs whole rounds of tiles and then a last, partly empty one (the
// tail: T mod SMs tiles; all of them when T < SMs).  The tail tiles may each
// run as s items over parts of their k range: the tail then takes
// ceil(tail * s / SMs) / s rounds instead of one (plus a little per item for
// its pipeline start and flushes).  s minimises that, each step up taken
// when it saves more than 2 %: when all tiles fit in one round up to
// max(16, SMs / tiles) (a few tall tiles with a long K fill the SMs), else
// up to 4 (more splits of long tiles only multiply the partial-sum
// traffic), and no more than the k range allows (whole units of the
// fp32-output schedule, at least 512 k for the fp64 split).  Partial tiles
// meet in k_split_reduce (fp32 output) or in an int64 slot per tile finished
// by k_split_finish (fp64 split).
struct SplitPlan {
  int splits;    // 1: no split
  int64_t full;  // leading tiles that run whole
  int64_t tail;  // tiles that run split
};

// Most workspace the deferred finish of short-K fp64-split tiles may take.
constexpr int64_t kDeferredFinishBytes = (int64_t)2 << 30;

SplitPlan split_plan(const Plan& p, int bn) {
  const int64_t tiles = plan_tiles(p, bn);
  const int64_t sms = num_sms();
  const bool emu = p.kernel == FAMLIES_KERNEL_TC_EMU;
  const int kind = p.kernel == FAMLIES_KERNEL_TC_TF32X3 ? PAIR_KIND_TF32 : PAIR_KIND_BF16;
  const int kb = pair_stage_k(kind);
  const int64_t nkb = (p.k + kb - 1) / kb;
  const int64_t unit = emu ? 512 / kb : f32out_unit_stages(kind);
  const int64_t pieces = emu ? nkb / unit : (nkb + unit - 1) / unit;
  const int64_t full = (tiles / sms) * sms, tail = tiles - full;
  // fp64 split with short K: every tile's sums go to its slot and a separate
  // kernel finishes them (a tile's finish otherwise stalls the product's
  // epilogue for about half its time).  The slots take 8 bytes per output
  // element (16 with the fine sums); above kDeferredFinishBytes of them the
  // tiles finish inside the product instead.
  if (emu && p.k <= 512) {
    const Sched sc = make_pair_sched(p.kernel, p.slices, kSplitBits, p.k, 1);
    const int64_t slot_bytes = (int64_t)BM * bn * 8 * (sc.nlow ? 2 : 1);
    if (tiles * slot_bytes <= kDeferredFinishBytes) return SplitPlan{1, 0, tiles};
  }
  // all tiles in one round: enough splits to fill the SMs (at least 16)
  const int64_t most = full == 0 ? std::max<int64_t>(16, (sms + tail - 1) / tail) : 4;
  const int64_t cap = pieces < most ? pieces : most;
  SplitPlan none{1, tiles, 0};
  if (cap <= 1 || tail == 0) return none;
  auto rounds = [&](int64_t sp) {
    return (double)((tail * sp + sms - 1) / sms) * (1.0 / (double)sp + 0.01);
  };
  int64_t best = 1;
  for (int64_t sp = 2; sp <= cap; ++sp)
    if (rounds(sp) < 0.98 * rounds(best)) best = sp;
  // fp64 split with whole rounds too: splitting every tile instead (so every
  // tile is finished outside the product kernel, whose epilogue then never
  // stalls on a tile's end) measures faster when it needs no more rounds
  if (emu && full > 0 && cap >= 2) {
    const double whole = (double)(full / sms) + (best > 1 ? rounds(best) : 1.0);
    for (int64_t sp = 2; sp <= 4 && sp <= cap; ++sp) {
      const double all = (double)((tiles * sp + sms - 1) / sms) / (double)sp;
      if (all <= whole + 1e-9) return SplitPlan{(int)sp, 0, tiles};
    }
  }
  if (best == 1) return none;
  return SplitPlan{(int)best, full, tail};
}


int grid_of(const Plan& p, int bn) {
  const SplitPlan sp = split_plan(p, bn);
  const int64_t items = sp.full + sp.tail * sp.splits;
  return (int)(items < num_sms() ? items : num_sms());
}

// ------------------------------------------------------------- CTA pairs
// The fp64 split's product on CTA pairs (cta_group::2, 256 x 256 tiles):
// per SM, each MMA reads 128 rows of A and 128 columns of B from shared
// memory instead of 128 rows and all 256 columns, so the operand traffic
// through shared memory (TMA writes plus MMA reads) drops by a third for
// the same tensor work.

template <int MODE, bool SPLITK>
cudaError_t pair2_attr() {
  using Cfg = PCfg<PAIR_KIND_BF16, 256, MODE, 2>;
  constexpr int kMaxDev = 64;
  static bool attr[kMaxDev] = {};
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return e;
  if (dev < kMaxDev && attr[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_pair_gemm<PAIR_KIND_BF16, MODE, 256, false, SPLITK, 2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
  if (e == cudaSuccess && dev < kMaxDev) attr[dev] = true;
  return e;
}

cudaLaunchConfig_t pair2_config(int grid, int smem, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Clusters of two CTAs of the pair kernel that fit on the device at once (0
// when the query fails: pairs are then not used).  Once per device.
int pair_clusters() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static int known[kMaxDev] = {};  // clusters + 1; 0: not asked yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (known[dev]) return known[dev] - 1;
  int n = 0;
  using Cfg = PCfg<PAIR_KIND_BF16, 256, PAIR_MODE_EMU, 2>;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = pair2_config(2 * (num_sms() / 2), Cfg::SMEM_BYTES, nullptr, at);
  if (pair2_attr<PAIR_MODE_EMU, false>() != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, k_pair_gemm<PAIR_KIND_BF16, PAIR_MODE_EMU, 256, false, false, 2>,
                                     &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  known[dev] = n + 1;
  return n;
}

// The product's schedule: CTAs per MMA, the split of its tiles (in tiles of
// cg * BM rows), its grid, and the int64 slots of the tail tiles' sums
// (BM x bn each).
struct ProductPlan {
  int cg;
  SplitPlan sp;
  int grid;
  int64_t xslots;
};

// Pairs (when the options ask for them) run the fp64 split's single
// problems with 256-wide tiles, no batch, no triangle and K past the
// deferred-finish range, when there is at least one whole round of pair
// tiles.  Either no tile is split (each finishes in the product) or every
// tile is split in s and k_split_finish finishes them, whichever takes
// fewer rounds.  (On the ladder product the pairs halve each SM's operand
// traffic through shared memory but measured a few per cent slower than one
// SM per MMA: that kernel waits on operand latency, not on bandwidth, so
// one SM per MMA stays the default.)
ProductPlan product_plan(const Plan& p, int bn) {
  const SplitPlan sp1 = split_plan(p, bn);
  ProductPlan r{1, sp1, grid_of(p, bn), sp1.tail};
  if (!p.cta_pair || p.kernel != FAMLIES_KERNEL_TC_EMU || bn != 256 || p.tri || p.l != 1 || p.k <= 512) return r;
  const int nc = pair_clusters();
  const int64_t tm2 = (p.m + 2 * BM - 1) / (2 * BM), pt = tm2 * ((p.n + bn - 1) / bn);
  if (nc < 1 || pt < nc) return r;
  int best = 1;
  double cost = 1e30;
  for (int s = 1; s <= 4; ++s) {  // rounds of the persistent grid, a little more per split
    const double c = (double)((pt * s + nc - 1) / nc) / (double)s + 0.01 * (s - 1);
    if (c < cost - 1e-9) {
      cost = c;
      best = s;
    }
  }
  r.cg = 2;
  r.sp = best == 1 ? SplitPlan{1, pt, 0} : SplitPlan{best, 0, pt};
  r.grid = 2 * (int)std::min<int64_t>(r.sp.full + r.sp.tail * r.sp.splits, nc);
  r.xslots = best == 1 ? 0 : 2 * pt;  // both halves of every pair tile
  return r;
}

struct Layout {
  size_t a, b, ea, eb, fa, fb, la, lb, G, xtail, part, tri, sym, total;
};

Layout layout_of(const Plan& p) {
  const bool emu = p.kernel == FAMLIES_KERNEL_TC_EMU;
  const bool tf32 = p.kernel == FAMLIES_KERNEL_TC_TF32X3;
  const int S = emu ? p.slices : (tf32 ? 2 : 1);
  const int es = tf32 ? 4 : 2;
  const size_t kp = (size_t)((p.k + 7) / 8 * 8);
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  Layout L{};
  size_t off = 0;
  L.a = off; off += up((size_t)S * p.l * p.m * kp * es);
  L.b = off; off += up((size_t)S * p.l * p.n * kp * es);
  if (emu) {
    const int bn = pair_bn_for(p.n, p.tile_n);
    L.ea = off; off += up((size_t)p.l * p.m * 4);
    L.eb = off; off += up((size_t)p.l * p.n * 4);
    L.fa = off; off += up((size_t)p.l * p.m * 4);
    L.fb = off; off += up((size_t)p.l * p.n * 4);
    L.la = off; off += up((size_t)(p.l * p.m + 1) * 4);
    L.lb = off; off += up((size_t)(p.l * p.n + 1) * 4);
    // per-CTA tile sums for the tiles that run whole; split K (and the
    // deferred finish) adds one slot per tail tile; one int64 sum per
    // element, two when the fine diagonals keep their own
    const ProductPlan pp = product_plan(p, bn);
    const size_t sums = make_pair_sched(p.kernel, p.slices, kSplitBits, p.k, pp.sp.splits).nlow ? 2 : 1;
    L.G = off; off += pp.sp.full > 0 ? up(sums * pp.grid * BM * bn * 8) : 0;
    L.xtail = off; off += up(sums * pp.xslots * BM * bn * 8);
  } else {
    const int bn = pair_bn_for(p.n, p.tile_n);
    const SplitPlan sp = split_plan(p, bn);
    if (sp.tail > 0) {
      L.part = off; off += up((size_t)sp.splits * sp.tail * BM * bn * 4);
    }
  }
  if (p.sym_n > 0) {  // per-tile maxima of the symmetric operand's exponent pass
    L.sym = off;
    off += up((size_t)sym_scratch_bytes(p.sym_n));
  }
  if (p.tri) {
    L.tri = off;
    off += up((size_t)tri_tile_count(p, pair_bn_for(p.n, p.tile_n)) * sizeof(int2));
  }
  L.total = off;
  return L;
}

template <int KIND, int MODE, int BN, bool GROUPED, bool SPLITK>
cudaError_t launch_pair_k(const CUtensorMap& ma, const CUtensorMap& mb, const PairArgs& a, int grid,
                          cudaStream_t s) {
  using Cfg = PCfg<KIND, BN, MODE>;
  constexpr int kMaxDev = 64;
  static bool attr[kMaxDev] = {};  // per device: function attributes are per context
  int dev = 0;
  if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return e;
  if (dev >= kMaxDev || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_pair_gemm<KIND, MODE, BN, GROUPED, SPLITK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev < kMaxDev) attr[dev] = true;
  }
  k_pair_gemm<KIND, MODE, BN, GROUPED, SPLITK><<<grid, THREADS, Cfg::SMEM_BYTES, s>>>(ma, mb, a);
  return cudaGetLastError();
}

template <int KIND, int MODE, int BN, bool GROUPED>
cudaError_t launch_pair(const CUtensorMap& ma, const CUtensorMap& mb, const PairArgs& a, int grid,
                        cudaStream_t s) {
  // split K only for single problems (a separate instantiation, so that the
  // common kernel carries none of its bookkeeping)
  if constexpr (!GROUPED) {
    if (a.tailed) return launch_pair_k<KIND, MODE, BN, GROUPED, true>(ma, mb, a, grid, s);
  }
  return launch_pair_k<KIND, MODE, BN, GROUPED, false>(ma, mb, a, grid, s);
}

template <int KIND, int MODE, bool GROUPED>
cudaError_t launch_pair_bn(int bn, const CUtensorMap& ma, const CUtensorMap& mb,
                           const PairArgs& a, int grid, cudaStream_t s) {
  if (bn == 64) return launch_pair<KIND, MODE, 64, GROUPED>(ma, mb, a, grid, s);
  if (bn == 128) return launch_pair<KIND, MODE, 128, GROUPED>(ma, mb, a, grid, s);
  return launch_pair<KIND, MODE, 256, GROUPED>(ma, mb, a, grid, s);
}

// The pair kernel (fp64 split, 256-wide tiles) as clusters of two.
template <int MODE, bool SPLITK>
cudaError_t launch_pair2_k(const CUtensorMap& ma, const CUtensorMap& mb, const PairArgs& a, int grid,
                           cudaStream_t s) {
  using Cfg = PCfg<PAIR_KIND_BF16, 256, MODE, 2>;
  if (cudaError_t e = pair2_attr<MODE, SPLITK>(); e != cudaSuccess) return e;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = pair2_config(grid, Cfg::SMEM_BYTES, s, at);
  return cudaLaunchKernelEx(&cfg, k_pair_gemm<PAIR_KIND_BF16, MODE, 256, false, SPLITK, 2>, ma, mb, a);
}

cudaError_t launch_pair2(int mode, const CUtensorMap& ma, const CUtensorMap& mb, const PairArgs& a, int grid,
                         cudaStream_t s) {
  if (mode == PAIR_MODE_EMU_FINE)
    return a.tailed ? launch_pair2_k<PAIR_MODE_EMU_FINE, true>(ma, mb, a, grid, s)
                    : launch_pair2_k<PAIR_MODE_EMU_FINE, false>(ma, mb, a, grid, s);
  return a.tailed ? launch_pair2_k<PAIR_MODE_EMU, true>(ma, mb, a, grid, s)
                  : launch_pair2_k<PAIR_MODE_EMU, false>(ma, mb, a, grid, s);
}

template <bool GROUPED>
cudaError_t launch_pair_any(int kind, int mode, int bn, const CUtensorMap& ma,
                            const CUtensorMap& mb, const PairArgs& a, int grid, cudaStream_t s) {
  if (mode == PAIR_MODE_EMU) return launch_pair_bn<PAIR_KIND_BF16, PAIR_MODE_EMU, GROUPED>(bn, ma, mb, a, grid, s);
  if (mode == PAIR_MODE_EMU_FINE)
    return launch_pair_bn<PAIR_KIND_BF16, PAIR_MODE_EMU_FINE, GROUPED>(bn, ma, mb, a, grid, s);
  if (kind == PAIR_KIND_TF32)
    return launch_pair_bn<PAIR_KIND_TF32, PAIR_MODE_F32OUT, GROUPED>(bn, ma, mb, a, grid, s);
  return launch_pair_bn<PAIR_KIND_BF16, PAIR_MODE_F32OUT, GROUPED>(bn, ma, mb, a, grid, s);
}

}  // namespace

bool make_slice_map(CUtensorMap* map, void* base, bool f32, int64_t k, int64_t kp, int64_t rows,
                    int64_t z, int box_k, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  const int es = f32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)z};
  cuuint64_t strides[2] = {(cuuint64_t)(kp * es), (cuuint64_t)(kp * es * rows)};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  // the swizzle spans one stage row (see pair_row_bytes)
  const int rowb = box_k * es;
  return enc(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
             base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A bf16 operand that TMA can read as it stands: its contracted modes fused
// to one unit-stride mode, at most one row mode and one batch mode, every
// stride a multiple of 16 bytes and the base 16-byte aligned.  which: 0 for
// the row operand (strides sa), 1 for the column operand (sb).
struct DirectView {
  const void* base;
  int64_t row_stride, batch_stride;  // elements
};

static bool direct_view(const ClassModes& R, const ClassModes& K, const ClassModes& Lb, int which,
                        const void* base, DirectView* v) {
  auto st = [&](const Mode& m) { return which == 0 ? m.sa : m.sb; };
  if (K.n != 1 || st(K.m[0]) != 1 || R.n > 1 || Lb.n > 1) return false;
  if (((uintptr_t)base & 15) != 0) return false;
  v->base = base;
  v->row_stride = R.n ? st(R.m[0]) : 8;
  v->batch_stride = Lb.n ? st(Lb.m[0]) : 8;
  return v->row_stride % 8 == 0 && v->batch_stride % 8 == 0 && v->row_stride > 0 &&
         v->batch_stride > 0;
}

static bool make_view_map(CUtensorMap* map, const DirectView& v, int64_t k, int64_t rows, int64_t l,
                          int box_k, int box_rows) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)l};
  cuuint64_t strides[2] = {(cuuint64_t)(v.row_stride * 2), (cuuint64_t)(v.batch_stride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(v.base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             box_k * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int pair_bn_for(int64_t n, int request) {
  if (request == 64 || request == 128 || request == 256) return request;
  return n > 128 ? 256 : (n > 64 ? 128 : 64);
}

// Unit schedule.  fp64 split with s slices of b bits: diagonal q = i + j
// (0-based slice indices, i + j <= s - 1) has weight 2^(-b (q + 2)); a unit
// covers kcb 64-wide k blocks so that its exact integer sum stays <= 2^24.
Sched make_pair_sched(int kernel, int slices, int bits, int64_t k, int64_t parts) {
  const int stage_k = pair_stage_k(PAIR_KIND_BF16);  // the fp64 split's slices are bf16
  Sched sc;
  std::memset(&sc, 0, sizeof(sc));
  if (kernel != FAMLIES_KERNEL_TC_EMU) {
    const bool tf32 = kernel == FAMLIES_KERNEL_TC_TF32X3;
    sc.ndiag = 1;
    sc.slices = tf32 ? 2 : 1;
    sc.kcb[0] = f32out_unit_stages(tf32 ? PAIR_KIND_TF32 : PAIR_KIND_BF16);
    sc.flush_every[0] = 1;
    if (tf32) {  // lo*hi + hi*lo + hi*hi, hi = slice 0, lo = slice 1
      sc.npairs[0] = 3;
      sc.pa[0][0] = 1; sc.pb[0][0] = 0;
      sc.pa[0][1] = 0; sc.pb[0][1] = 1;
      sc.pa[0][2] = 0; sc.pb[0][2] = 0;
    } else {
      sc.npairs[0] = 1;
    }
    return sc;
  }
  const int s = slices;
  sc.ndiag = s;
  sc.slices = s;
  auto maxd = [&](int i) { return (int64_t)1 << (i == 0 ? bits : bits - 1); };
  for (int di = 0; di < s; ++di) {
    const int q = s - 1 - di;  // least significant diagonal first
    int64_t bound = 0;
    for (int i = 0; i <= q; ++i) {
      sc.pa[di][i] = (int8_t)i;
      sc.pb[di][i] = (int8_t)(q - i);
      bound += maxd(i) * maxd(q - i);
    }
    sc.npairs[di] = q + 1;
    sc.shift[di] = bits * (q + 2);
    int64_t kcb = (((int64_t)1 << 24) / bound) / stage_k;
    sc.kcb[di] = (int)(kcb < 1 ? 1 : kcb);
    int64_t fe = (((int64_t)1 << 31) - 1) / (bound * sc.kcb[di] * stage_k);
    sc.flush_every[di] = (int)(fe < 1 ? 1 : fe);
  }
  // |tile sum| <= sum over diagonals of k * bound * 2^-shift (in units of 1);
  // in units of 2^-xunit it must stay below 2^62.  No finer than the least
  // significant diagonal's weight (that is already exact).
  double T = 0.0;
  for (int di = 0; di < s; ++di) {
    const int q = s - 1 - di;
    int64_t bound = 0;
    for (int i = 0; i <= q; ++i) bound += maxd(i) * maxd(q - i);
    T += std::ldexp((double)(k < 1 ? 1 : k) * (double)bound, -sc.shift[di]);
  }
  int xunit = (int)std::floor(62.0 - std::log2(T)) - 1;
  if (xunit > sc.shift[0]) xunit = sc.shift[0];  // di = 0 is the least significant diagonal
  sc.xunit = xunit;
  // Diagonals finer than 2^-xunit are rounded to it at each flush (at most
  // half a unit) if they go into the coarse sum.  The digits themselves
  // carry each scaled element to 2^-(bits*slices), so over k terms the
  // split's own error grows like sqrt(k) 2^-(bits*slices) and the flushes'
  // like sqrt(nflush) 2^-xunit (random walks).  When the latter would pass
  // a quarter of the former, i.e. nflush 4^(bits*slices - xunit) > k / 16
  // (long K, many splits sharing a tile), the fine diagonals get a second,
  // exact sum in units of 2^-xlo (their own finest weight, unless K makes
  // even their sum too large).
  const int64_t kk = k < 1 ? 1 : k, np = parts < 1 ? 1 : parts;
  const int64_t kpart = (kk + np - 1) / np, nkb_part = (kpart + stage_k - 1) / stage_k;
  double TL = 0.0, nflush = 0.0;
  int nfine = 0;
  for (int di = 0; di < s; ++di) {
    if (sc.shift[di] <= xunit) continue;
    ++nfine;
    const int q = s - 1 - di;
    int64_t bound = 0;
    for (int i = 0; i <= q; ++i) bound += maxd(i) * maxd(q - i);
    TL += std::ldexp((double)kk * (double)bound, -sc.shift[di]);
    const int64_t units = (nkb_part + sc.kcb[di] - 1) / sc.kcb[di];
    nflush += (double)np * (double)((units + sc.flush_every[di] - 1) / sc.flush_every[di]);
  }
  const bool fine = nfine > 0 && nflush * std::ldexp(1.0, 2 * (bits * s - xunit)) > (double)kk / 16.0;
  sc.xlo = sc.shift[0];
  if (fine && TL > 0.0) {
    const int cap = (int)std::floor(62.0 - std::log2(TL)) - 1;
    if (sc.xlo > cap) sc.xlo = cap;
  }
  sc.nlow = fine ? nfine : 0;  // shifts fall as di rises, so the fine diagonals are di < nlow
  for (int di = 0; di < s; ++di)
    sc.xshift[di] = (di < sc.nlow ? sc.xlo : xunit) - sc.shift[di];
  return sc;
}

cudaError_t launch_group_finish(bool fine, const int64_t* X, const Prob* probs, const TileEntry* tiles,
                                int64_t ntiles, int bn, int xunit, int xlo, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const int64_t items = ntiles * ((bn + FIN_COLS - 1) / FIN_COLS);
  const int grid = (int)std::min<int64_t>(items, (int64_t)num_sms() * 24);
  if (fine) k_group_finish<true><<<grid, 256, 0, s>>>(X, probs, tiles, ntiles, bn, xunit, xlo);
  else k_group_finish<false><<<grid, 256, 0, s>>>(X, probs, tiles, ntiles, bn, xunit, xlo);
  return cudaGetLastError();
}

cudaError_t launch_pair_grouped(int kind, int mode, int bn, const Prob* probs,
                                const TileEntry* tiles, int64_t ntiles, const Sched& sc,
                                double* G, int64_t* slots, int grid, int* status, int64_t wait_limit,
                                cudaStream_t s) {
  PairArgs a;
  std::memset(&a, 0, sizeof(a));
  a.probs = probs;
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.sc = sc;
  a.G = G;
  a.xtail = slots;
  a.defer = slots != nullptr;
  a.status = status;
  a.wait_limit = wait_limit;
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  if (mode == PAIR_MODE_EMU && sc.nlow) mode = PAIR_MODE_EMU_FINE;
  return launch_pair_any<true>(kind, mode, bn, unused, unused, a, grid, s);
}

int64_t packed_workspace_bytes(const Plan& p) { return (int64_t)layout_of(p).total; }

int packed_ctas_per_mma(const Plan& p) { return product_plan(p, pair_bn_for(p.n, p.tile_n)).cg; }

// fp64 split: the operands (bit 0: A, bit 1: B) split in one pass by
// k_rowpack (k one unit-stride mode of a length it holds in registers;
// neither symmetric nor generated).
static int rowpack_sides(const Plan& p) {
  if (p.kernel != FAMLIES_KERNEL_TC_EMU || p.k < kRowPackMinK || p.k > kRowPackMaxK || p.K.n != 1) return 0;
  int mask = 0;
  for (int side = 0; side < 2; ++side) {
    const bool own = (p.sym_n > 0 && p.sym_side == side) || p.band_side == side || p.krp_side == side;
    if (!own && (side == 0 ? p.K.m[0].sa : p.K.m[0].sb) == 1) mask |= 1 << side;
  }
  return mask;
}

int packed_launches(const Plan& p) {
  const int tri = p.tri ? 1 : 0;  // the triangle's tile list
  if (p.kernel == FAMLIES_KERNEL_TC_EMU) {
    // exponents + pack of the generic operands (one launch each for both),
    // one launch per one-pass operand, product (+ split finish) + fix-up
    const int rp = rowpack_sides(p);
    const int own = p.sym_n > 0 ? p.sym_side : (p.band_side >= 0 ? p.band_side : p.krp_side);
    int generic = 0, one_pass = 0;
    for (int side = 0; side < 2; ++side) {
      if (rp >> side & 1) ++one_pass;
      else if (side != own) ++generic;
    }
    return (generic ? 2 : 0) + one_pass + 2 + (product_plan(p, pair_bn_for(p.n, p.tile_n)).sp.tail > 0 ? 1 : 0) +
           tri + (p.band_side >= 0 || p.krp_side >= 0 ? 2 : 0) +  // (+ a generated operand's own)
           (p.sym_n > 0 ? 3 : 0);  // (+ a symmetric operand's exponents, their reduction, pack)
  }
  DirectView v;
  const bool tf32 = p.kernel == FAMLIES_KERNEL_TC_TF32X3;
  const bool da = !tf32 && direct_view(p.M, p.K, p.L, 0, p.a, &v);
  const bool db = !tf32 && direct_view(p.N, p.K, p.L, 1, p.b, &v);
  return ((da && db) ? 0 : 1) + 1 + (split_plan(p, pair_bn_for(p.n, p.tile_n)).tail > 0 ? 1 : 0) + tri +
         (p.band_side >= 0 || p.krp_side >= 0 ? 1 : 0);
}

cudaError_t launch_packed(const Plan& p, const GemmArgs& g, void* ws, cudaStream_t s) {
  const bool emu = p.kernel == FAMLIES_KERNEL_TC_EMU;
  const bool tf32 = p.kernel == FAMLIES_KERNEL_TC_TF32X3;
  const int bits = kSplitBits;
  const Layout L = layout_of(p);
  char* w = (char*)ws;
  const int64_t kp = (p.k + 7) / 8 * 8;
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.k = p.k;
  pa.kp = kp;
  pa.l = p.l;
  pa.slices = emu ? p.slices : (tf32 ? 2 : 1);
  pa.op[0] = PackOp{g.a, g.t.am, g.t.ak, g.t.al, p.m, p.a_contig, w + L.a, nullptr, nullptr, nullptr};
  pa.op[1] = PackOp{g.b, g.t.bn, g.t.bk, g.t.bl, p.n, p.b_contig, w + L.b, nullptr, nullptr, nullptr};
  set_affine(pa.op[0], p.M, p.K, 0);
  set_affine(pa.op[1], p.N, p.K, 1);
  const bool sym = p.sym_n > 0;
  if (sym) pa.op[p.sym_side].sym_n = p.sym_n;
  // a generated operand: banded (its source affine) or Khatri-Rao, no batch
  const int gside = p.band_side >= 0 ? p.band_side : p.krp_side;
  const bool gen = gside >= 0;
  if (gen) {
    PackOp& o = pa.op[gside];
    if (p.l != 1 || (p.band_side >= 0 && o.affine != 3)) return cudaErrorNotSupported;
    o.gen = p.band_side >= 0 ? 1 : 2;
    o.band = p.band;
    o.krp = p.krp;
  }
  const int own = sym ? p.sym_side : gside;  // packed by its own kernels (-1: none)
  const int rp = rowpack_sides(p);           // split in one pass
  cudaError_t e;
  if (emu) {
    pa.op[0].e = (int32_t*)(w + L.ea);
    pa.op[1].e = (int32_t*)(w + L.eb);
    pa.op[0].flag = (int32_t*)(w + L.fa);
    pa.op[1].flag = (int32_t*)(w + L.fb);
    pa.op[0].list = (int32_t*)(w + L.la);
    pa.op[1].list = (int32_t*)(w + L.lb);
    // an operand whose exponents, flags and list the step that produced it
    // recorded (a network's fused epilogue): no exponent pass over it (a
    // one-pass split stores the same values again)
    for (int side = 0; side < 2; ++side) {
      if (!p.pre_e[side]) continue;
      pa.op[side].e = p.pre_e[side];
      pa.op[side].flag = p.pre_flag[side];
      pa.op[side].list = p.pre_list[side];
    }
    // exponents start at a large negative value, flags and list counts at 0
    if ((e = cudaMemsetAsync(w + L.ea, 0x80, L.fa - L.ea, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w + L.fa, 0, L.G - L.fa, s)) != cudaSuccess) return e;
    // the generic kernels skip a symmetric or generated operand and one
    // split in one pass
    PackArgs pg = pa;
    if (own >= 0) pg.op[own].rows = 0;
    for (int side = 0; side < 2; ++side)
      if (p.pre_e[side] || (rp >> side & 1)) pg.op[side].rows = 0;
    nvtxRangePushA("exponents");
    e = pg.op[0].rows || pg.op[1].rows ? launch_rowexp(pg, s) : cudaSuccess;
    nvtxRangePop();
    if (e != cudaSuccess) return e;
    if (sym && (e = launch_rowexp_sym(pa, p.sym_side, (int32_t*)(w + L.sym), s)) != cudaSuccess) return e;
    if (gen && (e = launch_rowexp_gen(pa, gside, s)) != cudaSuccess) return e;
  }
  const int bn = pair_bn_for(p.n, p.tile_n);
  const int S = pa.slices;
  const int kind = tf32 ? PAIR_KIND_TF32 : PAIR_KIND_BF16;
  const int kbk = pair_stage_k(kind);
  CUtensorMap ma, mb;
  // bf16 operands already laid out like a slice (k unit-stride, aligned
  // rows and batches) are read by TMA straight from the caller's tensor;
  // only the others are packed.
  DirectView va, vb;
  const bool da = !emu && !tf32 && !gen && direct_view(p.M, p.K, p.L, 0, p.a, &va);
  const bool db = !emu && !tf32 && !gen && direct_view(p.N, p.K, p.L, 1, p.b, &vb);
  if (da) pa.op[0].rows = 0;  // nothing to pack
  if (db) pa.op[1].rows = 0;
  if (!da || !db) {
    struct Range {  // closes on every exit of the block
      Range() { nvtxRangePushA("pack"); }
      ~Range() { nvtxRangePop(); }
    } range;
    PackArgs pg = pa;
    if (own >= 0) pg.op[own].rows = 0;
    for (int side = 0; side < 2; ++side) {
      if (!(rp >> side & 1)) continue;
      if ((e = launch_rowpack(pa, side, s)) != cudaSuccess) return e;
      pg.op[side].rows = 0;
    }
    if ((pg.op[0].rows || pg.op[1].rows) &&
        (e = launch_pack(emu ? PACK_F64 : (tf32 ? PACK_TF32 : PACK_BF16), pg, s)) != cudaSuccess)
      return e;
    if (sym && (e = launch_pack_sym(pa, p.sym_side, s)) != cudaSuccess) return e;
    if (gen && (e = launch_pack_gen(emu ? PACK_F64 : PACK_TF32, pa, gside, s)) != cudaSuccess)
      return e;
  }
  const bool ok_a = da ? make_view_map(&ma, va, p.k, p.m, p.l, kbk, BM)
                       : make_slice_map(&ma, w + L.a, tf32, p.k, kp, p.m, (int64_t)S * p.l, kbk, BM);
  // the product's schedule (a CTA pair stages half of B's tile columns per CTA)
  const ProductPlan pp = emu ? product_plan(p, bn) : ProductPlan{1, split_plan(p, bn), grid_of(p, bn), 0};
  const bool ok_b = db ? make_view_map(&mb, vb, p.k, p.n, p.l, kbk, bn)
                       : make_slice_map(&mb, w + L.b, tf32, p.k, kp, p.n, (int64_t)S * p.l, kbk, bn / pp.cg);
  if (!ok_a || !ok_b) return cudaErrorInvalidValue;
  PairArgs a;
  std::memset(&a, 0, sizeof(a));
  a.single = Prob{nullptr, nullptr, g.c, g.t.cm, g.t.cn, g.t.cl, pa.op[0].e, pa.op[1].e,
                  pa.op[0].flag, pa.op[1].flag, p.m, p.n, p.k, p.l, g.alpha, g.beta, bn};
  a.single.emit_mode = emu ? g.emit_mode : 0;
  a.single.emit_e = g.emit_e;
  a.single.emit_flag = g.emit_flag;
  a.single.emit_list = g.emit_list;
  if (p.tri) {
    if (p.l != 1) return cudaErrorNotSupported;
    const int64_t tiles_m = (p.m + BM - 1) / BM, tiles_n = (p.n + bn - 1) / bn;
    int2* list = (int2*)(w + L.tri);
    k_tri_tiles<<<(int)std::min<int64_t>((tiles_m + 255) / 256, 1024), 256, 0, s>>>(p.tri, tiles_m, tiles_n,
                                                                                   bn, list);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    a.single.tri = p.tri;
    a.single.tri_list = list;
    a.single.tri_tiles = tri_tile_count(p, bn);
  }
  const SplitPlan spl = pp.sp;
  a.sc = make_pair_sched(p.kernel, p.slices, bits, p.k, spl.splits);
  a.G = emu ? (double*)(w + L.G) : nullptr;
  a.splits = spl.splits;
  a.tailed = spl.tail > 0 ? 1 : 0;
  a.full = spl.full;
  a.xtail = emu && a.tailed ? (int64_t*)(w + L.xtail) : nullptr;
  a.part = !emu && a.tailed ? (float*)(w + L.part) : nullptr;
  a.status = g.status;
  a.wait_limit = g.wait_limit;
  a.stall_test = g.stall_test;
  const int grid = pp.grid;
  const int split_grid = (int)std::min<int64_t>(spl.tail * (bn / SPLIT_COLS), (int64_t)num_sms() * 16);
  if (emu && a.tailed &&
      (e = cudaMemsetAsync(a.xtail, 0, (size_t)(a.sc.nlow ? 2 : 1) * pp.xslots * BM * bn * 8, s)) != cudaSuccess)
    return e;
  mark_begin(g, s);
  nvtxRangePushA("product");
  const int mode = emu ? (a.sc.nlow ? PAIR_MODE_EMU_FINE : PAIR_MODE_EMU) : PAIR_MODE_F32OUT;
  e = pp.cg == 2 ? launch_pair2(mode, ma, mb, a, grid, s) : launch_pair_any<false>(kind, mode, bn, ma, mb, a, grid, s);
  nvtxRangePop();
  mark_end(g, s);  // the events bracket the product kernel alone
  if (e == cudaSuccess && a.tailed) {
    if (emu) {
      // finished per BM-row tile (a pair's split tiles: every tile, full = 0)
      const int64_t ftiles = pp.cg == 2 ? ((p.m + BM - 1) / BM) * ((p.n + bn - 1) / bn) : spl.tail;
      const int fg = (int)std::min<int64_t>(ftiles * ((bn + FIN_COLS - 1) / FIN_COLS), (int64_t)num_sms() * 24);
      e = launch_split_finish(a.sc.nlow != 0, fg, a.xtail, a.full, bn, a.sc.xunit, a.sc.xlo, a.single, s);
    }
    else
      k_split_reduce<<<split_grid, 256, 0, s>>>(a.part, a.splits, a.full, bn, a.single);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  if (emu) {
    nvtxRangePushA("fixup");
    e = launch_fixup(g, pa, s);
    nvtxRangePop();
  }
  return e;
}

}  // namespace famlies
