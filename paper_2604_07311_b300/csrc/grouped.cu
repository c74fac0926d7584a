// Grouped execution of many independent contractions (the blocks of a
// block-sparse contraction: the "tensor-of-tensors" tiling of Sec. 2.3, run
// as a task list in the spirit of the algorithms-by-blocks runtimes of
// Sec. 2.4 with no dependencies between tasks).
//
// One call = one launch per stage, whatever the number of problems:
//   offset tables -> [fp64 split: row exponents] -> pack -> product -> [fix-up]
// Every problem's descriptors (offset-table jobs, pack arguments, TMA maps,
// epilogue descriptor) travel to the device in one copy; the product kernel
// walks a device tile list sorted longest-first, so the persistent CTAs
// balance the uneven blocks.  With use_graph the launches are captured once
// into a CUDA graph per problem set and replayed.  The tile width of the
// product is picked by timing the candidates on the first call for a given
// shape class (the autotuner) and remembered for the process, or across
// processes in the file FAMLIES_TUNE_CACHE names.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <unistd.h>

#include <cuda.h>
#include <cuda_runtime.h>

#include "device.h"
#include "packed.h"
#include "pair_gemm.h"
#include "plan.h"

namespace famlies {

namespace {

auto up256 = [](size_t x) { return (x + 255) / 256 * 256; };

// Most workspace the deferred finish of a grouped set's tiles may take.
constexpr size_t kGroupDeferBytes = (size_t)2 << 30;

// FAMLIES_GROUP_DEFER=0: grouped tiles finish inside the product (as they
// do anyway when their slots would pass kGroupDeferBytes).
bool group_defer_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("FAMLIES_GROUP_DEFER");
    v = (e && e[0] == '0') ? 0 : 1;
  }
  return v == 1;
}

struct ProbLayout {
  size_t tab, a, b;    // in the per-problem region
  size_t ea, eb;       // in the exponent region
  size_t fa, fb, la, lb;  // in the flag region
};

struct GroupSetup {
  int n = 0;
  int kernel = 0, kind = 0, mode = 0, slices = 1;
  size_t ws_main = 0, ws_exp = 0, ws_flag = 0, ws_g = 0, ws_defer = 0, ws_total = 0;
  bool fine = false;  // fp64 split: the schedule keeps the fine diagonals' second sums
  std::vector<ProbLayout> lay;
  int64_t ntiles = 0, max_table = 1, rowexp_total = 0, pack_total = 0, kmax = 1;
  size_t blob_probs = 0, blob_gargs = 0, blob_pargs = 0, blob_jobs = 0, blob_tiles = 0,
         blob_maps = 0, blob_offr = 0, blob_offp = 0, blob_bytes = 0;
  size_t c_bytes = 0;  // sum of C spans (autotuning scratch)
};

GroupSetup layout_group(const std::vector<const Plan*>& ps, int bn_max) {
  GroupSetup G;
  G.n = (int)ps.size();
  G.kernel = ps[0]->kernel;
  const bool emu = G.kernel == FAMLIES_KERNEL_TC_EMU;
  const bool tf32 = G.kernel == FAMLIES_KERNEL_TC_TF32X3;
  G.kind = tf32 ? PAIR_KIND_TF32 : PAIR_KIND_BF16;
  G.mode = emu ? PAIR_MODE_EMU : PAIR_MODE_F32OUT;
  G.slices = emu ? ps[0]->slices : (tf32 ? 2 : 1);
  const int es = tf32 ? 4 : 2;
  G.lay.resize(G.n);
  for (int i = 0; i < G.n; ++i) {
    const Plan& p = *ps[i];
    ProbLayout& L = G.lay[i];
    const size_t kp = (size_t)((p.k + 7) / 8 * 8);
    L.tab = G.ws_main; G.ws_main += up256((size_t)table_entries(p) * 8);
    L.a = G.ws_main; G.ws_main += up256((size_t)G.slices * p.l * p.m * kp * es);
    L.b = G.ws_main; G.ws_main += up256((size_t)G.slices * p.l * p.n * kp * es);
    if (emu) {
      L.ea = G.ws_exp; G.ws_exp += up256((size_t)p.l * p.m * 4);
      L.eb = G.ws_exp; G.ws_exp += up256((size_t)p.l * p.n * 4);
      L.fa = G.ws_flag; G.ws_flag += up256((size_t)p.l * p.m * 4);
      L.fb = G.ws_flag; G.ws_flag += up256((size_t)p.l * p.n * 4);
      L.la = G.ws_flag; G.ws_flag += up256((size_t)(p.l * p.m + 1) * 4);
      L.lb = G.ws_flag; G.ws_flag += up256((size_t)(p.l * p.n + 1) * 4);
    }
    int64_t tmax = std::max(std::max(p.m, p.n), std::max(p.k, p.l));
    G.max_table = std::max(G.max_table, tmax);
    G.kmax = std::max(G.kmax, p.k);
    G.rowexp_total += rowexp_tiles(p.m, p.k, p.l) + rowexp_tiles(p.n, p.k, p.l);
    G.pack_total += pack_tiles(p.m, p.k, p.l) + pack_tiles(p.n, p.k, p.l);
    G.c_bytes += up256((size_t)p.span_c * p.es_c);
  }
  if (emu) G.ws_g = up256((size_t)2 * num_sms() * kPairBM * bn_max * 8);  // two sums per element
  if (emu) {
    // Deferred finish: a slot of int64 sums per tile (bn_max columns, two
    // sums with the fine diagonals), sized for the widest tile list any
    // candidate width gives; above kGroupDeferBytes the tiles finish inside
    // the product instead.
    G.fine = make_pair_sched(G.kernel, G.slices, kSplitBits, G.kmax).nlow != 0;
    size_t most = 0;
    for (int bw = 64; bw <= bn_max; bw *= 2) {
      size_t tiles = 0;
      for (const Plan* p : ps) {
        const int w = std::min(pair_bn_for(p->n, 0), bw);
        tiles += (size_t)p->l * (size_t)((p->m + kPairBM - 1) / kPairBM) * (size_t)((p->n + w - 1) / w);
      }
      most = std::max(most, tiles * kPairBM * bw);
    }
    const size_t bytes = up256(most * 8 * (G.fine ? 2 : 1));
    if (bytes <= kGroupDeferBytes && group_defer_enabled()) G.ws_defer = bytes;
  }
  G.ws_total = G.ws_main + G.ws_exp + G.ws_flag + G.ws_g + G.ws_defer;
  return G;
}

// Tile width of one problem in a launch whose widest tile is cap: the
// narrowest of 64/128/256 that covers the problem's columns, at most cap.
int width_for(const Plan& p, int cap) { return std::min(pair_bn_for(p.n, 0), cap); }

// Fills the host image of the descriptor blob whose device copy starts at
// d_blob, for workspace d_ws and product tile width bn.  Returns false if a
// TMA map cannot be encoded.
bool build_blob(const std::vector<const Plan*>& ps, const double* alpha, const double* beta,
                GroupSetup& G, int bn, char* d_ws, char* d_blob, int* status, int64_t wait_limit,
                std::vector<char>& blob) {
  const int n = G.n;
  std::vector<TileEntry> tiles;
  std::vector<int64_t> cost;
  for (int i = 0; i < n; ++i) {
    const Plan& p = *ps[i];
    const int bw = width_for(p, bn);
    const int64_t tm_n = (p.m + kPairBM - 1) / kPairBM, tn_n = (p.n + bw - 1) / bw;
    const int64_t c = (p.k + 63) / 64 * (bw / 64);  // work of one tile
    for (int64_t il = 0; il < p.l; ++il)
      for (int64_t tm = 0; tm < tm_n; ++tm)
        for (int64_t tn = 0; tn < tn_n; ++tn) {
          tiles.push_back(TileEntry{i, (int32_t)tm, (int32_t)tn, (int32_t)il});
          cost.push_back(c);
        }
  }
  // longest first: the persistent CTAs then take the remaining tiles
  // greedily, which bounds the imbalance by the shortest tile
  std::vector<size_t> order(tiles.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  G.ntiles = (int64_t)tiles.size();

  size_t off = 0;
  G.blob_probs = off; off += up256(sizeof(Prob) * n);
  G.blob_gargs = off; off += up256(sizeof(GemmArgs) * n);
  G.blob_pargs = off; off += up256(sizeof(PackArgs) * n);
  G.blob_jobs = off; off += up256(sizeof(TableJob) * 9 * n);
  G.blob_tiles = off; off += up256(sizeof(TileEntry) * tiles.size());
  G.blob_maps = off; off += up256(sizeof(CUtensorMap) * 2 * n);
  G.blob_offr = off; off += up256(sizeof(int64_t) * (2 * n + 1));
  G.blob_offp = off; off += up256(sizeof(int64_t) * (2 * n + 1));
  G.blob_bytes = off;
  blob.assign(off, 0);

  Prob* probs = (Prob*)(blob.data() + G.blob_probs);
  GemmArgs* gargs = (GemmArgs*)(blob.data() + G.blob_gargs);
  PackArgs* pargs = (PackArgs*)(blob.data() + G.blob_pargs);
  TableJob* jobs = (TableJob*)(blob.data() + G.blob_jobs);
  TileEntry* tl = (TileEntry*)(blob.data() + G.blob_tiles);
  CUtensorMap* maps = (CUtensorMap*)(blob.data() + G.blob_maps);
  const CUtensorMap* d_maps = (const CUtensorMap*)(d_blob + G.blob_maps);
  char* d_exp = d_ws + G.ws_main;
  char* d_flag = d_exp + G.ws_exp;
  const bool emu = G.mode == PAIR_MODE_EMU;
  const bool tf32 = G.kind == PAIR_KIND_TF32;
  for (int i = 0; i < n; ++i) {
    const Plan& p = *ps[i];
    const ProbLayout& L = G.lay[i];
    Tables t;
    plan_table_jobs(p, (int64_t*)(d_ws + L.tab), jobs + 9 * i, &t);
    GemmArgs& g = gargs[i];
    std::memset(&g, 0, sizeof(g));
    g.a = p.a; g.b = p.b; g.c = p.c; g.t = t;
    g.m = p.m; g.n = p.n; g.k = p.k; g.l = p.l;
    g.alpha = alpha[i]; g.beta = beta[i];
    g.a_contig = p.a_contig; g.b_contig = p.b_contig;
    g.wait_limit = wait_limit; g.status = status;
    PackArgs& pa = pargs[i];
    std::memset(&pa, 0, sizeof(pa));
    const int64_t kp = (p.k + 7) / 8 * 8;
    pa.k = p.k; pa.kp = kp; pa.l = p.l; pa.slices = G.slices;
    pa.op[0] = PackOp{p.a, t.am, t.ak, t.al, p.m, p.a_contig, d_ws + L.a, nullptr, nullptr, nullptr};
    pa.op[1] = PackOp{p.b, t.bn, t.bk, t.bl, p.n, p.b_contig, d_ws + L.b, nullptr, nullptr, nullptr};
    set_affine(pa.op[0], p.M, p.K, 0);
    set_affine(pa.op[1], p.N, p.K, 1);
    if (emu) {
      pa.op[0].e = (int32_t*)(d_exp + L.ea);
      pa.op[1].e = (int32_t*)(d_exp + L.eb);
      pa.op[0].flag = (int32_t*)(d_flag + L.fa);
      pa.op[1].flag = (int32_t*)(d_flag + L.fb);
      pa.op[0].list = (int32_t*)(d_flag + L.la);
      pa.op[1].list = (int32_t*)(d_flag + L.lb);
    }
    const int kbk = pair_stage_k(G.kind);
    if (!make_slice_map(&maps[2 * i], d_ws + L.a, tf32, p.k, kp, p.m, (int64_t)G.slices * p.l, kbk,
                        kPairBM) ||
        !make_slice_map(&maps[2 * i + 1], d_ws + L.b, tf32, p.k, kp, p.n,
                        (int64_t)G.slices * p.l, kbk, width_for(p, bn)))
      return false;
    probs[i] = Prob{d_maps + 2 * i, d_maps + 2 * i + 1, p.c, t.cm, t.cn, t.cl, pa.op[0].e,
                    pa.op[1].e, pa.op[0].flag, pa.op[1].flag, p.m, p.n, p.k, p.l,
                    alpha[i], beta[i], width_for(p, bn)};
  }
  for (size_t i = 0; i < order.size(); ++i) tl[i] = tiles[order[i]];
  // flat tile numbering of the exponent and pack passes, per (problem, operand)
  int64_t* offr = (int64_t*)(blob.data() + G.blob_offr);
  int64_t* offp = (int64_t*)(blob.data() + G.blob_offp);
  offr[0] = offp[0] = 0;
  for (int i = 0; i < n; ++i) {
    const Plan& p = *ps[i];
    offr[2 * i + 1] = offr[2 * i] + rowexp_tiles(p.m, p.k, p.l);
    offr[2 * i + 2] = offr[2 * i + 1] + rowexp_tiles(p.n, p.k, p.l);
    offp[2 * i + 1] = offp[2 * i] + pack_tiles(p.m, p.k, p.l);
    offp[2 * i + 2] = offp[2 * i + 1] + pack_tiles(p.n, p.k, p.l);
  }
  return true;
}

struct DevPtrs {
  const Prob* probs;
  const GemmArgs* gargs;
  const PackArgs* pargs;
  const TableJob* jobs;
  const TileEntry* tiles;
  const int64_t* offr;
  const int64_t* offp;
};

DevPtrs dev_ptrs(const GroupSetup& G, char* d_blob) {
  return DevPtrs{(const Prob*)(d_blob + G.blob_probs), (const GemmArgs*)(d_blob + G.blob_gargs),
                 (const PackArgs*)(d_blob + G.blob_pargs), (const TableJob*)(d_blob + G.blob_jobs),
                 (const TileEntry*)(d_blob + G.blob_tiles), (const int64_t*)(d_blob + G.blob_offr),
                 (const int64_t*)(d_blob + G.blob_offp)};
}

cudaError_t enqueue_prepare(const GroupSetup& G, char* d_ws, const DevPtrs& d, cudaStream_t s) {
  cudaError_t e;
  char* d_exp = d_ws + G.ws_main;
  char* d_flag = d_exp + G.ws_exp;
  const bool emu = G.mode == PAIR_MODE_EMU;
  if (emu) {
    if ((e = cudaMemsetAsync(d_exp, 0x80, G.ws_exp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_flag, 0, G.ws_flag, s)) != cudaSuccess) return e;
  }
  if ((e = launch_tables_grouped(d.jobs, 9 * (int64_t)G.n, G.max_table, s)) != cudaSuccess) return e;
  if (emu && (e = launch_rowexp_grouped(d.pargs, d.offr, G.n, G.rowexp_total, s)) != cudaSuccess)
    return e;
  const int pmode = emu ? PACK_F64 : (G.kind == PAIR_KIND_TF32 ? PACK_TF32 : PACK_BF16);
  return launch_pack_grouped(pmode, d.pargs, d.offp, G.n, G.pack_total, s);
}

cudaError_t enqueue_product(const GroupSetup& G, int bn, const Prob* probs, const TileEntry* tiles,
                            char* d_ws, int* status, int64_t wait_limit, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(G.ntiles, num_sms());
  const Sched sc = make_pair_sched(G.kernel, G.slices, kSplitBits, G.kmax);
  double* Gsum = G.mode == PAIR_MODE_EMU ? (double*)(d_ws + G.ws_main + G.ws_exp + G.ws_flag) : nullptr;
  int64_t* slots = G.ws_defer ? (int64_t*)(d_ws + G.ws_main + G.ws_exp + G.ws_flag + G.ws_g) : nullptr;
  return launch_pair_grouped(G.kind, G.mode, bn, probs, tiles, G.ntiles, sc, Gsum, slots, grid, status,
                             wait_limit, s);
}

// After the product: the deferred finish of every tile (when the product
// left its sums in slots), then the native recomputation of the rows and
// columns that hold Inf/NaN.
cudaError_t enqueue_finish(const GroupSetup& G, const DevPtrs& d, char* d_ws, int bn, cudaStream_t s) {
  if (G.mode != PAIR_MODE_EMU) return cudaSuccess;
  if (G.ws_defer) {
    const Sched sc = make_pair_sched(G.kernel, G.slices, kSplitBits, G.kmax);
    const cudaError_t e =
        launch_group_finish(sc.nlow != 0, (const int64_t*)(d_ws + G.ws_main + G.ws_exp + G.ws_flag + G.ws_g),
                            d.probs, d.tiles, G.ntiles, bn, sc.xunit, sc.xlo, s);
    if (e != cudaSuccess) return e;
  }
  return launch_fixup_grouped(d.gargs, d.pargs, G.n, s);
}

// ------------------------------------------------------------ autotuner
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

// FAMLIES_LOG=1: one line per grouped call on stderr (problems, chunks, the
// product's tile width and where it came from).
bool grouped_log() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("FAMLIES_LOG");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v == 1;
}

// Tuned widths kept across processes: FAMLIES_TUNE_CACHE names a JSON file,
// one object mapping each shape-class key to its width ({"sm148 k2 ...": 128,
// ...}).  It is read on the first lookup (entries whose width is not 64, 128
// or 256 are ignored) and rewritten, through a temporary file and a rename,
// whenever this process tunes a new class (each process through a
// temporary file of its own); two processes tuning at once keep the last
// writer's set.  The keys hold the SM count, so a file moved
// to another kind of GPU is not taken for it.
const char* tune_cache_path() {
  const char* e = std::getenv("FAMLIES_TUNE_CACHE");
  return (e && e[0]) ? e : nullptr;
}

void load_tune_cache_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = std::fopen(path, "rb");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  size_t i = 0;
  while ((i = text.find('"', i)) != std::string::npos) {
    const size_t j = text.find('"', i + 1);
    if (j == std::string::npos) break;
    const size_t c = text.find(':', j);
    if (c == std::string::npos) break;
    char* end = nullptr;
    const long w = std::strtol(text.c_str() + c + 1, &end, 10);
    if (w == 64 || w == 128 || w == 256) g_tune.emplace(text.substr(i + 1, j - i - 1), (int)w);
    i = end && end > text.c_str() + c + 1 ? (size_t)(end - text.c_str()) : c + 1;
  }
}

void save_tune_cache_locked() {
  const char* path = tune_cache_path();
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return;
  std::fputs("{\n", f);
  size_t n = 0;
  for (const auto& kv : g_tune)
    std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++n < g_tune.size() ? "," : "");
  std::fputs("}\n", f);
  const bool ok = std::fclose(f) == 0;
  if (ok) std::rename(tmp.c_str(), path);
  else std::remove(tmp.c_str());
}

std::string tune_key(const std::vector<const Plan*>& ps) {
  std::vector<int64_t> m, n, k;
  for (const Plan* p : ps) { m.push_back(p->m); n.push_back(p->n); k.push_back(p->k); }
  auto med = [](std::vector<int64_t>& v) {
    std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
    return v[v.size() / 2];
  };
  auto lg = [](int64_t x) { int b = 0; while ((int64_t)1 << (b + 1) <= x) ++b; return b; };
  char buf[160];
  std::snprintf(buf, sizeof(buf), "sm%d k%d s%d m%d n%d k%d c%d", num_sms(), ps[0]->kernel, ps[0]->slices,
                lg(med(m)), lg(med(n)), lg(med(k)), lg((int64_t)ps.size()));
  return buf;
}

// Without tuning: the cap that lets every problem use its own best width.
int heuristic_bn(const std::vector<const Plan*>& ps) {
  int cap = 64;
  for (const Plan* p : ps) cap = std::max(cap, pair_bn_for(p->n, 0));
  return cap;
}

bool autotune_enabled() {
  const char* e = std::getenv("FAMLIES_AUTOTUNE");
  return !(e && e[0] == '0');
}

// Times each candidate width on the packed problems with C redirected to
// scratch, so the caller's C is untouched; returns the fastest.
int tune_bn(const std::vector<const Plan*>& ps, const double* alpha, const double* beta,
            GroupSetup& G, char* d_ws, int* status, int64_t wait_limit, cudaStream_t s) {
  const int cands[3] = {64, 128, 256};
  int best = heuristic_bn(ps);
  float best_ms = 1e30f;
  char* scratch = nullptr;
  if (cudaMallocAsync((void**)&scratch, G.c_bytes + 256, s) != cudaSuccess) {
    cudaGetLastError();
    return best;
  }
  cudaMemsetAsync(scratch, 0, G.c_bytes + 256, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int bn : cands) {
    // a width beyond twice the widest problem only adds empty columns
    int64_t maxn = 0;
    for (const Plan* p : ps) maxn = std::max(maxn, p->n);
    if (bn > 64 && bn / 2 >= maxn) continue;
    std::vector<char> blob;
    char* d_blob = nullptr;
    GroupSetup Gb = G;
    // first pass sizes the descriptors, the second writes device addresses
    if (!build_blob(ps, alpha, beta, Gb, bn, d_ws, nullptr, status, wait_limit, blob)) continue;
    if (cudaMallocAsync((void**)&d_blob, Gb.blob_bytes, s) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    build_blob(ps, alpha, beta, Gb, bn, d_ws, d_blob, status, wait_limit, blob);
    Prob* probs = (Prob*)(blob.data() + Gb.blob_probs);
    size_t coff = 0;
    for (int i = 0; i < Gb.n; ++i) {  // redirect C to scratch (same offsets)
      probs[i].c = scratch + coff;
      coff += up256((size_t)ps[i]->span_c * ps[i]->es_c);
    }
    cudaMemcpyAsync(d_blob, blob.data(), Gb.blob_bytes, cudaMemcpyHostToDevice, s);
    const DevPtrs d = dev_ptrs(Gb, d_blob);
    cudaEventRecord(e0, s);
    cudaError_t err = enqueue_product(Gb, bn, d.probs, d.tiles, d_ws, status, wait_limit, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = bn;
    }
    cudaGetLastError();
    cudaFreeAsync(d_blob, s);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(scratch, s);
  return best;
}

int pick_bn(const std::vector<const Plan*>& ps, const double* alpha, const double* beta,
            GroupSetup& G, char* d_ws, int* status, int64_t wait_limit, cudaStream_t s,
            bool can_tune) {
  const std::string key = tune_key(ps);
  auto log = [&](int bn, const char* how) {
    if (grouped_log())
      std::fprintf(stderr, "famlies: grouped %zu problems [%s]: tile width %d (%s)\n", ps.size(), key.c_str(), bn,
                   how);
    return bn;
  };
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_cache_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return log(it->second, "tuned");
  }
  if (!can_tune || !autotune_enabled()) return log(heuristic_bn(ps), "heuristic");
  const int bn = tune_bn(ps, alpha, beta, G, d_ws, status, wait_limit, s);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = bn;
  save_tune_cache_locked();
  return log(bn, "timed now");
}

// ------------------------------------------------------------ graph cache
struct GraphEntry {
  uint64_t key;
  char* ws;                  // persistent workspace of the captured set
  std::vector<char*> blobs;  // persistent descriptor blocks, one per chunk
  cudaGraphExec_t exec;
};
std::mutex g_graph_mu;
std::list<GraphEntry> g_graphs;  // most recent first
constexpr size_t kGraphCap = 4;

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

uint64_t set_key(const std::vector<const Plan*>& ps, const double* alpha, const double* beta,
                 int dev) {
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &dev, sizeof(dev));
  for (size_t i = 0; i < ps.size(); ++i) {
    const Plan& p = *ps[i];
    h = fnv(h, &p.kernel, sizeof(p.kernel));
    h = fnv(h, &p.slices, sizeof(p.slices));
    h = fnv(h, &p.a, sizeof(p.a));
    h = fnv(h, &p.b, sizeof(p.b));
    h = fnv(h, &p.c, sizeof(p.c));
    for (const ClassModes* cm : {&p.M, &p.N, &p.K, &p.L}) {
      h = fnv(h, &cm->n, sizeof(cm->n));
      h = fnv(h, cm->m, sizeof(Mode) * cm->n);
    }
    h = fnv(h, &alpha[i], sizeof(double));
    h = fnv(h, &beta[i], sizeof(double));
  }
  return h;
}

// Problems in call order, cut into chunks whose workspace stays within
// the budget (a problem larger than the budget forms its own chunk).
// Small chunks keep the packed slices within TLB reach and close in time to
// their use; every chunk still runs as one launch per stage.
std::vector<std::pair<size_t, size_t>> make_chunks(const std::vector<const Plan*>& ps) {
  const char* env = std::getenv("FAMLIES_BATCH_WORKSPACE_MB");
  size_t budget = env ? (size_t)std::atoll(env) << 20 : (size_t)4096 << 20;
  if (budget < ((size_t)16 << 20)) budget = (size_t)16 << 20;
  // each problem's own workspace, laid out once: all of it, and without the
  // per-CTA sums, which the problems of a chunk share
  std::vector<size_t> whole(ps.size()), shared(ps.size());
  for (size_t i = 0; i < ps.size(); ++i) {
    const GroupSetup one = layout_group({ps[i]}, 256);
    whole[i] = one.ws_total;
    shared[i] = one.ws_total - one.ws_g;
  }
  std::vector<std::pair<size_t, size_t>> out;
  size_t i0 = 0;
  while (i0 < ps.size()) {
    size_t i1 = i0 + 1, used = whole[i0];
    while (i1 < ps.size() && used + shared[i1] <= budget) used += shared[i1++];
    out.emplace_back(i0, i1);
    i0 = i1;
  }
  return out;
}

struct ChunkRun {
  std::vector<const Plan*> ps;
  const double* alpha;
  const double* beta;
  GroupSetup G;
  int bn = 256;
  std::vector<char> blob;
  char* d_blob = nullptr;
  size_t blob_cap = 0;
};

// Descriptor capacity: the narrowest width gives the longest tile list.
size_t blob_capacity(ChunkRun& c, char* ws, int* status, int64_t wait_limit) {
  GroupSetup G64 = c.G;
  std::vector<char> tmp;
  build_blob(c.ps, c.alpha, c.beta, G64, 64, ws, nullptr, status, wait_limit, tmp);
  return G64.blob_bytes;
}

}  // namespace

int run_grouped(const std::vector<const Plan*>& all, const std::vector<double>& alpha,
                const std::vector<double>& beta, cudaStream_t s, bool use_graph, int* status,
                int64_t wait_limit) {
  if (all.empty()) return FAMLIES_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  // a set captured before replays its graph: no chunking or layout needed
  uint64_t key = 0;
  if (use_graph) {
    key = set_key(all, alpha.data(), beta.data(), dev);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
      if (it->key != key) continue;
      g_graphs.splice(g_graphs.begin(), g_graphs, it);
      return cudaGraphLaunch(g_graphs.front().exec, s) == cudaSuccess ? FAMLIES_OK : FAMLIES_ERR_CUDA;
    }
  }
  const auto ranges = make_chunks(all);
  std::vector<ChunkRun> chunks(ranges.size());
  size_t ws_max = 0;
  for (size_t c = 0; c < ranges.size(); ++c) {
    ChunkRun& r = chunks[c];
    r.ps.assign(all.begin() + ranges[c].first, all.begin() + ranges[c].second);
    r.alpha = alpha.data() + ranges[c].first;
    r.beta = beta.data() + ranges[c].first;
    r.G = layout_group(r.ps, 256);
    ws_max = std::max(ws_max, r.G.ws_total);
  }
  // workspace (one, reused by the chunks in turn) and descriptor blocks
  char* ws = nullptr;
  cudaError_t e = use_graph ? cudaMalloc((void**)&ws, ws_max + 256)
                            : cudaMallocAsync((void**)&ws, ws_max + 256, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_ALLOC;
  }
  auto release = [&]() {
    for (ChunkRun& r : chunks) {
      if (!r.d_blob) continue;
      if (use_graph) cudaFree(r.d_blob); else cudaFreeAsync(r.d_blob, s);
      r.d_blob = nullptr;
    }
    if (use_graph) cudaFree(ws); else cudaFreeAsync(ws, s);
  };
  for (ChunkRun& r : chunks) {
    r.blob_cap = blob_capacity(r, ws, status, wait_limit);
    e = use_graph ? cudaMalloc((void**)&r.d_blob, r.blob_cap)
                  : cudaMallocAsync((void**)&r.d_blob, r.blob_cap, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      r.d_blob = nullptr;
      if (use_graph) cudaStreamSynchronize(s);
      release();
      return FAMLIES_ERR_ALLOC;
    }
  }
  // Eager part on the caller's stream.  Without a graph: every stage of
  // every chunk.  With a graph: only what the tuner needs (the packed slices
  // of a chunk whose shape class has no tuned width yet); the graph below
  // then computes the result exactly once.
  int rc = FAMLIES_OK;
  for (ChunkRun& r : chunks) {
    const std::string tk = tune_key(r.ps);
    bool tuned;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      load_tune_cache_locked();
      auto it = g_tune.find(tk);
      tuned = it != g_tune.end();
      r.bn = tuned ? it->second : heuristic_bn(r.ps);
    }
    if (tuned && grouped_log())
      std::fprintf(stderr, "famlies: grouped %zu problems [%s]: tile width %d (tuned)\n", r.ps.size(), tk.c_str(),
                   r.bn);
    const bool need_prepare = !use_graph || !tuned;
    if (!need_prepare) continue;
    if (!build_blob(r.ps, r.alpha, r.beta, r.G, r.bn, ws, r.d_blob, status, wait_limit, r.blob)) {
      rc = FAMLIES_ERR_CUDA;
      break;
    }
    cudaMemcpyAsync(r.d_blob, r.blob.data(), r.G.blob_bytes, cudaMemcpyHostToDevice, s);
    DevPtrs d = dev_ptrs(r.G, r.d_blob);
    if (enqueue_prepare(r.G, ws, d, s) != cudaSuccess) { rc = FAMLIES_ERR_CUDA; break; }
    if (!tuned) {
      const int bn = pick_bn(r.ps, r.alpha, r.beta, r.G, ws, status, wait_limit, s, true);
      if (bn != r.bn) {
        r.bn = bn;
        build_blob(r.ps, r.alpha, r.beta, r.G, r.bn, ws, r.d_blob, status, wait_limit, r.blob);
        cudaMemcpyAsync(r.d_blob, r.blob.data(), r.G.blob_bytes, cudaMemcpyHostToDevice, s);
        d = dev_ptrs(r.G, r.d_blob);
      }
    }
    if (!use_graph) {
      if (enqueue_product(r.G, r.bn, d.probs, d.tiles, ws, status, wait_limit, s) != cudaSuccess ||
          enqueue_finish(r.G, d, ws, r.bn, s) != cudaSuccess) {
        rc = FAMLIES_ERR_CUDA;
        break;
      }
    }
  }
  if (rc != FAMLIES_OK || !use_graph) {
    cudaGetLastError();
    release();
    return rc;
  }

  // Graph: final descriptors of every chunk, then one capture of all stages
  // of all chunks in order (they share the workspace), instantiate, replay.
  cudaStreamSynchronize(s);
  for (ChunkRun& r : chunks) {
    build_blob(r.ps, r.alpha, r.beta, r.G, r.bn, ws, r.d_blob, status, wait_limit, r.blob);
    cudaMemcpy(r.d_blob, r.blob.data(), r.G.blob_bytes, cudaMemcpyHostToDevice);
  }
  cudaStream_t cs;
  cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t ek = cudaSuccess;
    for (ChunkRun& r : chunks) {
      const DevPtrs d = dev_ptrs(r.G, r.d_blob);
      if (ek == cudaSuccess) ek = enqueue_prepare(r.G, ws, d, cs);
      if (ek == cudaSuccess) ek = enqueue_product(r.G, r.bn, d.probs, d.tiles, ws, status, wait_limit, cs);
      if (ek == cudaSuccess) ek = enqueue_finish(r.G, d, ws, r.bn, cs);
    }
    e = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess && ek != cudaSuccess) e = ek;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release();
    return FAMLIES_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_graph_mu);
  if (g_graphs.size() >= kGraphCap) {
    cudaDeviceSynchronize();  // an evicted graph may still run on some stream
    GraphEntry& old = g_graphs.back();
    cudaGraphExecDestroy(old.exec);
    for (char* b : old.blobs) cudaFree(b);
    cudaFree(old.ws);
    g_graphs.pop_back();
  }
  GraphEntry ge;
  ge.key = key;
  ge.ws = ws;
  ge.exec = exec;
  for (ChunkRun& r : chunks) ge.blobs.push_back(r.d_blob);
  g_graphs.push_front(ge);
  return cudaGraphLaunch(exec, s) == cudaSuccess ? FAMLIES_OK : FAMLIES_ERR_CUDA;
}

}  // namespace famlies
