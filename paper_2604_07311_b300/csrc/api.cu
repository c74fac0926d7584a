// C ABI entry points: validate and plan on the host, take stream-ordered
// workspace, build the offset tables on the device, launch the kernel the
// plan names, release the workspace.  Nothing here computes on the host.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <list>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "device.h"
#include "plan.h"

using namespace famlies;

namespace {

// Checks (once per device) that the current device is an sm_103 part, the
// only target these kernels are built for.
int check_device() {
  static std::mutex mu;
  static int cached[64];
  static bool init = false;
  std::lock_guard<std::mutex> lk(mu);
  if (!init) {
    for (int& c : cached) c = 1;  // 1 = unknown
    init = true;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_NO_DEVICE;
  }
  if (dev < 0 || dev >= 64) return FAMLIES_ERR_NO_DEVICE;
  if (cached[dev] == 1) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaGetLastError();
    cached[dev] = (major == 10 && minor == 3) ? FAMLIES_OK : FAMLIES_ERR_NO_DEVICE;
    if (cached[dev] == FAMLIES_OK) {
      // Keep freed stream-ordered workspace mapped in the device's default
      // pool between calls instead of returning it at every synchronisation
      // (re-mapping gigabytes of slices each call costs milliseconds).
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      cudaGetLastError();
    }
  }
  return cached[dev];
}

int64_t env_wait_limit() {
  static int64_t v = -1;
  if (v < 0) {
    const char* e = std::getenv("FAMLIES_WAIT_LIMIT");
    v = e ? std::atoll(e) : 0;
    if (v <= 0) v = (int64_t)1 << 26;  // ~ seconds of polling, far above any real wait
  }
  return v;
}

// FAMLIES_LOG=1: one line per planned call on stderr (kernel, sizes, role swap).
bool env_log() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("FAMLIES_LOG");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v == 1;
}

// A profiler range around one library call (host side: enqueue order).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

const char* kernel_name(int k) {
  static const char* names[] = {"none", "scale", "simt_f64", "simt_f32", "tc_bf16", "tc_tf32x3",
                                "tc_emu", "tc_bf16_gather", "tc_tf32x3_gather", "tc_bf16_direct"};
  return (k >= 0 && k <= 9) ? names[k] : "?";
}

struct Workspace {
  void* ptr = nullptr;
  cudaStream_t s = nullptr;
  bool owned = true;  // false: the workspace belongs to a plan-cache entry
  ~Workspace() {
    if (ptr && owned) cudaFreeAsync(ptr, s);
  }
};

// Plan cache.  Repeated calls with the same shapes, strides, dtype, knobs
// and stream (a training loop, an iterative solver) keep their workspace
// and the offset tables in it: such a call skips the allocation, the free
// and the table kernel.  The key holds the fused label classes (extents and
// strides of every operand), which fix the tables and the workspace layout,
// plus the device and the stream, so that calls sharing an entry are ordered
// by their stream.  Not used while the stream is being captured into a graph
// (a captured call allocates its own workspace), nor for entries above
// 256 MB; at most 16 entries, the least recently used one not held by a call
// in progress freed when a new one is needed.  Each call that used an entry
// records an event on its stream after its last kernel; eviction waits for
// that event before it frees the workspace (in stream order: it came from
// the stream-ordered allocator, whose memory a plain free may unmap under
// kernels still queued).  FAMLIES_PLAN_CACHE=0 turns it off.
class PlanCache {
 public:
  struct Entry {
    std::vector<int64_t> key;
    void* ws = nullptr;
    int64_t bytes = 0;
    uint64_t used = 0;
    bool tables = false;         // the tables have been built in ws
    cudaEvent_t done = nullptr;  // after the last kernel of the last call that used ws
    int holders = 0;             // calls between get() and release()
  };

  static bool enabled() {
    static int v = -1;
    if (v < 0) {
      const char* e = std::getenv("FAMLIES_PLAN_CACHE");
      v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
  }

  // The entry for key (created with `bytes` of workspace allocated on s when
  // missing), or null when the cache cannot serve the call.
  // A returned entry is held until release(entry, stream), which the caller
  // makes once the call's kernels are enqueued.
  Entry* get(const std::vector<int64_t>& key, int64_t bytes, cudaStream_t s) {
    if (bytes > kMaxBytes) return nullptr;
    std::lock_guard<std::mutex> lk(mu_);
    ++clock_;
    for (Entry& e : entries_)
      if (e.key == key && e.bytes >= bytes) {
        e.used = clock_;
        ++e.holders;
        return &e;
      }
    if (entries_.size() >= kMaxEntries) {
      auto lru = entries_.end();
      for (auto it = entries_.begin(); it != entries_.end(); ++it)
        if (it->holders == 0 && (lru == entries_.end() || it->used < lru->used)) lru = it;
      if (lru == entries_.end()) return nullptr;  // every entry is in use: no caching
      // the last call that used it may still be queued on its stream
      if (lru->done) {
        cudaEventSynchronize(lru->done);
        cudaEventDestroy(lru->done);
      } else {
        cudaDeviceSynchronize();
      }
      cudaFreeAsync(lru->ws, s);
      cudaGetLastError();
      entries_.erase(lru);
    }
    Entry e;
    e.key = key;
    e.bytes = bytes;
    e.used = clock_;
    e.holders = 1;
    if (cudaMallocAsync(&e.ws, bytes > 0 ? bytes : 256, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    entries_.push_back(std::move(e));
    return &entries_.back();
  }

  // The call holding e has enqueued its kernels on s.
  void release(Entry* e, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(mu_);
    if (!e->done && cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      e->done = nullptr;
    }
    if (e->done && cudaEventRecord(e->done, s) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(e->done);
      e->done = nullptr;  // eviction then waits for the whole device
    }
    --e->holders;
  }

 private:
  static constexpr int64_t kMaxBytes = (int64_t)256 << 20;
  static constexpr size_t kMaxEntries = 16;
  std::mutex mu_;
  std::list<Entry> entries_;  // stable addresses: entries are held across a call
  uint64_t clock_ = 0;
};

PlanCache& plan_cache() {
  static PlanCache* c = new PlanCache();  // never destroyed: entries live until exit
  return *c;
}

// Releases a held plan-cache entry when the call's scope ends (after its
// kernels are enqueued, on every return path).
struct CacheHold {
  PlanCache::Entry* e = nullptr;
  cudaStream_t s = nullptr;
  ~CacheHold() {
    if (e) plan_cache().release(e, s);
  }
};


// The cache key of plan p on stream s, or an empty key when p is not cached
// (operands that carry device pointers in the plan: symmetric, banded,
// Khatri-Rao; triangle updates).
std::vector<int64_t> cache_key(const Plan& p, cudaStream_t s) {
  std::vector<int64_t> k;
  if (p.sym_n || p.band_side >= 0 || p.krp_side >= 0 || p.tri || p.emit_mode || p.pre_e[0] || p.pre_e[1])
    return k;
  int dev = 0;
  cudaGetDevice(&dev);
  k = {dev, (int64_t)(intptr_t)s, (int64_t)p.dtype, p.kernel, p.slices, p.tile_n, p.force_gather,
       p.cta_pair, (int64_t)p.swapped, p.m, p.n, p.k, p.l};
  for (const ClassModes* cm : {&p.M, &p.N, &p.K, &p.L}) {
    k.push_back(cm->n);
    for (int i = 0; i < cm->n; ++i) {
      k.push_back(cm->m[i].ext);
      k.push_back(cm->m[i].sa);
      k.push_back(cm->m[i].sb);
      k.push_back(cm->m[i].sc);
    }
  }
  return k;
}

bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown: do not cache
  }
  return st != cudaStreamCaptureStatusNone;
}

int run_plan(const Plan& p, double alpha, double beta, cudaStream_t s,
             const famlies_options_t* opt, famlies_plan_info_t* info) {
  fill_info(p, info);
  if (env_log())
    std::fprintf(stderr,
                 "famlies: %s m=%lld n=%lld k=%lld batch=%lld modes=%d/%d/%d/%d swapped=%d slices=%d%s%s%s\n",
                 kernel_name(p.kernel), (long long)p.m, (long long)p.n, (long long)p.k, (long long)p.l, p.M.n,
                 p.N.n, p.K.n, p.L.n, (int)p.swapped, p.slices, p.sym_n ? " symmetric" : "",
                 p.band_side >= 0 ? " banded" : "", p.krp_side >= 0 ? " khatri-rao" : "");
  if (p.kernel == FAMLIES_KERNEL_NONE) return FAMLIES_OK;
  Range range(kernel_name(p.kernel));
  int rc = check_device();
  if (rc) return rc;
  if (p.kernel == FAMLIES_KERNEL_TC_BF16_DIRECT) {
    // no offset tables: tiles come straight from the operands (workspace
    // only for an operand that must be re-padded for its tensor map)
    const int64_t wsb = box_workspace_bytes(p);
    if (wsb < 0) return FAMLIES_ERR_UNSUPPORTED;
    Workspace ws;
    ws.s = s;
    PlanCache::Entry* ce = nullptr;
    if (wsb > 0 && PlanCache::enabled() && !stream_capturing(s)) {
      const std::vector<int64_t> key = cache_key(p, s);
      if (!key.empty()) ce = plan_cache().get(key, wsb, s);
    }
    CacheHold hold{ce, s};
    if (ce) {
      ws.ptr = ce->ws;
      ws.owned = false;
    } else if (wsb > 0 && cudaMallocAsync(&ws.ptr, wsb, s) != cudaSuccess) {
      cudaGetLastError();
      ws.ptr = nullptr;
      return FAMLIES_ERR_ALLOC;
    }
    GemmArgs g = {};
    g.a = p.a;
    g.b = p.b;
    g.c = p.c;
    g.m = p.m;
    g.n = p.n;
    g.k = p.k;
    g.l = p.l;
    g.alpha = alpha;
    g.beta = beta;
    g.wait_limit = (opt && opt->wait_limit > 0) ? opt->wait_limit : env_wait_limit();
    g.status = device_status_ptr();
    if (!g.status) return FAMLIES_ERR_CUDA;
    g.stall_test = opt ? opt->stall_test : 0;
    g.ev_begin = opt ? (cudaEvent_t)opt->events[0] : nullptr;
    g.ev_end = opt ? (cudaEvent_t)opt->events[1] : nullptr;
    int nl = 0;
    cudaError_t err = launch_box(p, g, ws.ptr, s, &nl);
    if (info) info->launches = nl;
    if (err != cudaSuccess) {
      cudaGetLastError();
      return err == cudaErrorNotSupported ? FAMLIES_ERR_UNSUPPORTED : FAMLIES_ERR_CUDA;
    }
    return FAMLIES_OK;
  }
  int64_t tab_bytes = table_entries(p) * (int64_t)sizeof(int64_t);
  int64_t extra = 0;
  if (p.kernel == FAMLIES_KERNEL_TC_EMU || p.kernel == FAMLIES_KERNEL_TC_BF16 ||
      p.kernel == FAMLIES_KERNEL_TC_TF32X3)
    extra = packed_workspace_bytes(p);
  else if (p.kernel == FAMLIES_KERNEL_TC_BF16_GATHER || p.kernel == FAMLIES_KERNEL_TC_TF32X3_GATHER)
    extra = tc_workspace_bytes(p);
  else if (p.kernel == FAMLIES_KERNEL_SIMT_F64 || p.kernel == FAMLIES_KERNEL_SIMT_F32)
    extra = simt_workspace_bytes(p);
  extra = (extra + 255) / 256 * 256;
  tab_bytes = (tab_bytes + 255) / 256 * 256;
  Workspace ws;
  ws.s = s;
  PlanCache::Entry* ce = nullptr;
  if (PlanCache::enabled() && !stream_capturing(s)) {
    const std::vector<int64_t> key = cache_key(p, s);
    if (!key.empty()) ce = plan_cache().get(key, tab_bytes + extra, s);
  }
  CacheHold hold{ce, s};
  if (ce) {
    ws.ptr = ce->ws;
    ws.owned = false;
  } else if (cudaMallocAsync(&ws.ptr, tab_bytes + extra, s) != cudaSuccess) {
    cudaGetLastError();
    ws.ptr = nullptr;
    return FAMLIES_ERR_ALLOC;
  }
  Tables t;
  int launches = 0;
  int64_t* tab = (int64_t*)((char*)ws.ptr + extra);
  bool reused = false;
  if (ce && ce->tables) {  // the cached workspace already holds this plan's tables
    TableJob jobs[9];
    plan_table_jobs(p, tab, jobs, &t);
    reused = true;
  } else {
    if (launch_tables(p, tab, &t, s) != cudaSuccess) return FAMLIES_ERR_CUDA;
    ++launches;
    if (ce) ce->tables = true;
  }
  cudaError_t err = cudaSuccess;
  if (p.kernel == FAMLIES_KERNEL_SCALE) {
    err = launch_scale(p, t, beta, s);
    ++launches;
  } else {
    GemmArgs g = {};
    g.a = p.a;
    g.b = p.b;
    g.c = p.c;
    g.t = t;
    g.m = p.m;
    g.n = p.n;
    g.k = p.k;
    g.l = p.l;
    g.alpha = alpha;
    g.beta = beta;
    g.a_contig = p.a_contig;
    g.b_contig = p.b_contig;
    g.wait_limit = (opt && opt->wait_limit > 0) ? opt->wait_limit : env_wait_limit();
    g.status = device_status_ptr();
    if (!g.status) return FAMLIES_ERR_CUDA;
    g.stall_test = opt ? opt->stall_test : 0;
    g.sym_n = p.sym_n;
    g.sym_side = p.sym_side;
    g.band = p.band;
    g.band_op = p.band_side + 1;
    g.tri = p.tri;
    g.krp = p.krp;
    g.krp_op = p.krp_side + 1;
    g.emit_mode = p.emit_mode;
    g.emit_e = p.emit_e;
    g.emit_flag = p.emit_flag;
    g.emit_list = p.emit_list;
    g.ev_begin = opt ? (cudaEvent_t)opt->events[0] : nullptr;
    g.ev_end = opt ? (cudaEvent_t)opt->events[1] : nullptr;
    switch (p.kernel) {
      case FAMLIES_KERNEL_SIMT_F64:
      case FAMLIES_KERNEL_SIMT_F32:
        err = launch_simt(p, g, extra ? ws.ptr : nullptr, s);
        launches += extra ? 2 : 1;  // (+ the split reduction)
        break;
      case FAMLIES_KERNEL_TC_BF16_GATHER:
      case FAMLIES_KERNEL_TC_TF32X3_GATHER:
        err = launch_tc(p, g, p.tile_n, ws.ptr, s);
        launches += 3;  // two k-stride tables + the product
        break;
      case FAMLIES_KERNEL_TC_BF16:
      case FAMLIES_KERNEL_TC_TF32X3:
      case FAMLIES_KERNEL_TC_EMU:
        err = launch_packed(p, g, ws.ptr, s);
        launches += packed_launches(p);
        break;
      default:
        return FAMLIES_ERR_UNSUPPORTED;
    }
  }
  if (info) {
    info->launches = launches;
    info->cached = reused ? 1 : 0;
    info->ctas_per_mma = p.kernel == FAMLIES_KERNEL_TC_EMU ? packed_ctas_per_mma(p) : 1;
  }
  if (err != cudaSuccess) {
    cudaGetLastError();
    return err == cudaErrorNotSupported ? FAMLIES_ERR_UNSUPPORTED : FAMLIES_ERR_CUDA;
  }
  return FAMLIES_OK;
}

}  // namespace

extern "C" {

int famlies_version(void) { return 100; }

const char* famlies_error_string(int code) {
  switch (code) {
    case FAMLIES_OK: return "success";
    case FAMLIES_ERR_INVALID_ARG: return "invalid argument (null pointer, ndim, negative extent or stride, dtype)";
    case FAMLIES_ERR_LABEL: return "bad label set (label in one tensor only, or repeated within a tensor)";
    case FAMLIES_ERR_EXTENT_MISMATCH: return "extent mismatch for a shared label";
    case FAMLIES_ERR_ALIAS: return "C overlaps A or B";
    case FAMLIES_ERR_OUT_OF_BOUNDS: return "reachable element beyond size_bytes";
    case FAMLIES_ERR_UNSUPPORTED: return "unsupported layout or size";
    case FAMLIES_ERR_ALLOC: return "workspace allocation failed";
    case FAMLIES_ERR_CUDA: return "CUDA runtime error";
    case FAMLIES_ERR_DEVICE_TIMEOUT: return "a kernel's bounded wait expired";
    case FAMLIES_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    case FAMLIES_ERR_SCRATCH: return "call needs more than the no-allocation entry point's fixed 1 MiB scratch";
  }
  return "unknown error code";
}

int famlies_plan(const famlies_tensor_t* A, const famlies_tensor_t* B, const famlies_tensor_t* C,
                 famlies_dtype_t dtype, const famlies_options_t* opt, famlies_plan_info_t* info) {
  Plan p;
  int rc = make_plan(1.0, A, B, C, dtype, opt, &p);
  if (rc) return rc;
  fill_info(p, info);
  return FAMLIES_OK;
}

int famlies_contract_ex(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
                        double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                        void* stream, const famlies_options_t* opt, famlies_plan_info_t* info) {
  Plan p;
  int rc = make_plan(alpha, A, B, C, dtype, opt, &p);
  if (rc) return rc;
  return run_plan(p, alpha, beta, (cudaStream_t)stream, opt, info);
}

int famlies_contract_sym(double alpha, const famlies_symtensor_t* A, const famlies_tensor_t* B,
                         double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                         void* stream, const famlies_options_t* opt, famlies_plan_info_t* info) {
  if (!A || !B || !C || A->ndim < 2 || A->ndim > FAMLIES_MAX_NDIM || A->ndim % 2 ||
      !A->extents || !A->labels)
    return FAMLIES_ERR_INVALID_ARG;
  if (dtype != FAMLIES_F64_EMU) return FAMLIES_ERR_UNSUPPORTED;
  const int h = A->ndim / 2;
  int64_t n = 1;
  for (int i = 0; i < h; ++i) {
    if (A->extents[i] < 0 || A->extents[i] != A->extents[i + h]) return FAMLIES_ERR_INVALID_ARG;
    n *= A->extents[i];
  }
  if (n > ((int64_t)1 << 30)) return FAMLIES_ERR_UNSUPPORTED;  // packed bytes must fit int64
  const int64_t packed = n * (n + 1) / 2;
  if (A->size_bytes > 0 && packed * 8 > A->size_bytes) return FAMLIES_ERR_OUT_OF_BOUNDS;
  // Plan A as its dense expansion (first mode fastest): the halves' fused
  // indices p and q then have strides 1 and n.  A stand-in address keeps the
  // planner's aliasing check (which would see n^2 elements) off the packed
  // data; the packed range is checked here instead.
  int64_t st[FAMLIES_MAX_NDIM];
  int64_t acc = 1;
  for (int i = 0; i < A->ndim; ++i) {
    st[i] = acc;
    acc *= A->extents[i];
  }
  famlies_tensor_t dense = {A->ndim, A->extents, st, A->labels, (void*)(uintptr_t)256, 0};
  famlies_options_t o = {};
  if (opt) o = *opt;
  o.kernel = 2;  // the packed tensor-core path
  Plan p;
  int rc = make_plan(alpha, &dense, B, C, dtype, &o, &p);
  if (rc) return rc;
  if (p.kernel == FAMLIES_KERNEL_NONE || p.kernel == FAMLIES_KERNEL_SCALE)
    return run_plan(p, alpha, beta, (cudaStream_t)stream, &o, info);  // A is not read
  if (p.kernel != FAMLIES_KERNEL_TC_EMU) return FAMLIES_ERR_UNSUPPORTED;
  if (!A->data) return FAMLIES_ERR_INVALID_ARG;
  if (n == 1) {  // a 1 x 1 triangle is its own dense matrix
    dense.data = const_cast<void*>(A->data);
    dense.size_bytes = A->size_bytes;
    return famlies_contract_ex(alpha, &dense, B, beta, C, dtype, stream, &o, info);
  }
  {
    const int64_t sc = p.span_c * p.es_c;
    const char* c0 = (const char*)C->data;
    const char* a0 = (const char*)A->data;
    if (c0 < a0 + packed * 8 && a0 < c0 + sc) return FAMLIES_ERR_ALIAS;
  }
  // A's side and classes: one mode each (after fusion) for its rows and k,
  // of extent n, with strides 1 and n in the dense expansion.
  const int side = p.swapped ? 1 : 0;
  const ClassModes& R = side == 0 ? p.M : p.N;
  if (R.n != 1 || p.K.n != 1 || p.L.n != 0 || R.m[0].ext != n || p.K.m[0].ext != n)
    return FAMLIES_ERR_UNSUPPORTED;
  const int64_t sr = side == 0 ? R.m[0].sa : R.m[0].sb;
  const int64_t sk = side == 0 ? p.K.m[0].sa : p.K.m[0].sb;
  if (!((sr == 1 && sk == n) || (sr == n && sk == 1))) return FAMLIES_ERR_UNSUPPORTED;
  if (side == 0) p.a = A->data;
  else p.b = A->data;
  p.sym_n = n;
  p.sym_side = side;
  return run_plan(p, alpha, beta, (cudaStream_t)stream, &o, info);
}

int famlies_gemmt_tridiag(int64_t n, int64_t k, double alpha, const void* A, int64_t rs_a,
                          int64_t cs_a, const void* t_sub, const void* t_diag, const void* t_sup,
                          double beta, void* C, int64_t rs_c, int64_t cs_c, famlies_dtype_t dtype,
                          void* stream, const famlies_options_t* opt, famlies_plan_info_t* info) {
  if (n < 0 || k < 0 || rs_a < 0 || cs_a < 0 || rs_c < 0 || cs_c < 0) return FAMLIES_ERR_INVALID_ARG;
  if (dtype != FAMLIES_F64 && dtype != FAMLIES_F64_EMU && dtype != FAMLIES_F32)
    return FAMLIES_ERR_UNSUPPORTED;
  if (k > 1 && !t_sub) return FAMLIES_ERR_INVALID_ARG;
  // The operation as a contraction C[i,j] = A[i,p] B[p,j] whose column
  // operand B is A^T with the band applied along p: both operands read A.
  const int64_t ea[2] = {n, k}, sa[2] = {rs_a, cs_a};
  const int64_t eb[2] = {k, n}, sb[2] = {cs_a, rs_a};
  const int64_t ec[2] = {n, n}, scs[2] = {rs_c, cs_c};
  const int32_t la[2] = {1, 3}, lb[2] = {3, 2}, lc[2] = {1, 2};
  famlies_tensor_t ta = {2, ea, sa, la, const_cast<void*>(A), 0};
  famlies_tensor_t tb = {2, eb, sb, lb, const_cast<void*>(A), 0};
  famlies_tensor_t tc = {2, ec, scs, lc, C, 0};
  famlies_options_t o = {};
  if (opt) o = *opt;
  o.kernel = dtype == FAMLIES_F64 ? 1 : 2;  // CUDA cores / packed tensor cores
  Plan p;
  int rc = make_plan(alpha, &ta, &tb, &tc, dtype, &o, &p);
  if (rc) return rc;
  // kernel indices: rows are C's i unless the planner put C's unit stride
  // (then j) on the rows
  p.tri = p.swapped ? 2 : 1;
  if (p.kernel != FAMLIES_KERNEL_NONE && p.kernel != FAMLIES_KERNEL_SCALE) {
    if (p.kernel != FAMLIES_KERNEL_SIMT_F64 && p.kernel != FAMLIES_KERNEL_TC_EMU &&
        p.kernel != FAMLIES_KERNEL_TC_TF32X3)
      return FAMLIES_ERR_UNSUPPORTED;
    p.band_side = p.swapped ? 0 : 1;
    p.band.sub = t_sub;
    p.band.diag = t_diag;
    p.band.sup = t_sup;
  }
  return run_plan(p, alpha, beta, (cudaStream_t)stream, &o, info);
}

int famlies_mttkrp(double alpha, const famlies_tensor_t* X, int32_t mode, const famlies_matrix_t* U,
                   double beta, const famlies_matrix_t* M, famlies_dtype_t dtype, void* stream,
                   const famlies_options_t* opt, famlies_plan_info_t* info) {
  if (!X || !U || !M || X->ndim < 2 || X->ndim > FAMLIES_MAX_NDIM || mode < 0 || mode >= X->ndim ||
      !X->extents || !X->strides)
    return FAMLIES_ERR_INVALID_ARG;
  if (dtype != FAMLIES_F64 && dtype != FAMLIES_F64_EMU && dtype != FAMLIES_F32)
    return FAMLIES_ERR_UNSUPPORTED;
  const int N = X->ndim;
  const int64_t R = M->cols;
  const int es = dtype == FAMLIES_F32 ? 4 : 8;
  if (R < 0 || M->rows != X->extents[mode] || M->rs < 0 || M->cs < 0) return FAMLIES_ERR_EXTENT_MISMATCH;
  auto span = [](const famlies_matrix_t& a) {
    return (a.rows == 0 || a.cols == 0) ? (int64_t)0 : (a.rows - 1) * a.rs + (a.cols - 1) * a.cs + 1;
  };
  auto overlap = [&](const famlies_matrix_t& a) {
    const char* a0 = (const char*)a.data;
    const char* m0 = (const char*)M->data;
    return span(a) > 0 && span(*M) > 0 && a0 < m0 + span(*M) * es && m0 < a0 + span(a) * es;
  };
  // The contraction M[i, r] = X[.., i, ..] KR[(i_m), r] whose column operand,
  // the Khatri-Rao product KR, has a dense layout (the other modes in order,
  // first fastest, then r) that the kernels decode instead of reading.
  int32_t lx[FAMLIES_MAX_NDIM], lb[FAMLIES_MAX_NDIM];
  int64_t eb[FAMLIES_MAX_NDIM], sb[FAMLIES_MAX_NDIM];
  const int32_t RL = 99;  // r's label (X's modes are 1..N)
  Krp q;
  int64_t acc = 1;
  for (int m = 0; m < N; ++m) {
    lx[m] = m + 1;
    if (m == mode) continue;
    const famlies_matrix_t& u = U[m];
    if (u.rows != X->extents[m] || u.cols != R || u.rs < 0 || u.cs < 0) return FAMLIES_ERR_EXTENT_MISMATCH;
    if (overlap(u)) return FAMLIES_ERR_ALIAS;
    eb[q.nf] = X->extents[m];
    sb[q.nf] = acc;
    lb[q.nf] = m + 1;
    q.u[q.nf] = u.data;
    q.rs[q.nf] = u.rs;
    q.cs[q.nf] = u.cs;
    q.ext[q.nf] = X->extents[m] > 0 ? X->extents[m] : 1;
    q.st[q.nf] = acc;
    ++q.nf;
    const int64_t e = X->extents[m] > 0 ? X->extents[m] : 1;
    if (acc > ((int64_t)1 << 62) / e) return FAMLIES_ERR_UNSUPPORTED;  // the Khatri-Rao layout's offsets
    acc *= e;
  }
  if (R > 0 && acc > ((int64_t)1 << 62) / R) return FAMLIES_ERR_UNSUPPORTED;
  eb[q.nf] = R;
  sb[q.nf] = acc;
  lb[q.nf] = RL;
  famlies_tensor_t tx = {N, X->extents, X->strides, lx, X->data, X->size_bytes};
  // a stand-in address: the Khatri-Rao operand is generated, never read
  famlies_tensor_t tb = {q.nf + 1, eb, sb, lb, (void*)(uintptr_t)256, 0};
  const int64_t ec[2] = {M->rows, R}, scs[2] = {M->rs, M->cs};
  const int32_t lc[2] = {mode + 1, RL};
  famlies_tensor_t tm = {2, ec, scs, lc, const_cast<void*>(M->data), 0};
  famlies_options_t o = {};
  if (opt) o = *opt;
  o.kernel = dtype == FAMLIES_F64 ? 1 : 2;  // CUDA cores / packed tensor cores
  Plan p;
  int rc = make_plan(alpha, &tx, &tb, &tm, dtype, &o, &p);
  if (rc) return rc;
  if (p.kernel != FAMLIES_KERNEL_NONE && p.kernel != FAMLIES_KERNEL_SCALE) {
    if (p.kernel != FAMLIES_KERNEL_SIMT_F64 && p.kernel != FAMLIES_KERNEL_TC_EMU &&
        p.kernel != FAMLIES_KERNEL_TC_TF32X3)
      return FAMLIES_ERR_UNSUPPORTED;
    for (int f = 0; f < q.nf; ++f)
      if (!q.u[f]) return FAMLIES_ERR_INVALID_ARG;
    p.krp = q;
    p.krp_side = p.swapped ? 0 : 1;
  }
  return run_plan(p, alpha, beta, (cudaStream_t)stream, &o, info);
}

int famlies_network(const famlies_tensor_t* tensors, int32_t ntensors,
                    const famlies_step_t* steps, int32_t nsteps, famlies_dtype_t dtype,
                    void* stream, const famlies_options_t* opt) {
  if (!tensors || ntensors <= 0 || nsteps < 0 || (nsteps > 0 && !steps))
    return FAMLIES_ERR_INVALID_ARG;
  // Which tensors are intermediates, and is each one written (with beta = 0)
  // before it is read?
  std::vector<char> inter(ntensors), written(ntensors, 0);
  bool any_inter = false;
  for (int i = 0; i < ntensors; ++i) inter[i] = tensors[i].data == nullptr;
  for (int i = 0; i < nsteps; ++i) {
    const famlies_step_t& st = steps[i];
    if (st.a < 0 || st.a >= ntensors || st.b < 0 || st.b >= ntensors || st.c < 0 ||
        st.c >= ntensors || st.c == st.a || st.c == st.b)
      return FAMLIES_ERR_INVALID_ARG;
    if ((inter[st.a] && !written[st.a]) || (inter[st.b] && !written[st.b]))
      return FAMLIES_ERR_INVALID_ARG;
    if (inter[st.c] && !written[st.c] && st.beta != 0.0) return FAMLIES_ERR_INVALID_ARG;
    written[st.c] = 1;
    any_inter = any_inter || inter[st.a] || inter[st.b] || inter[st.c];
  }
  if (any_inter && dtype == FAMLIES_BF16) return FAMLIES_ERR_UNSUPPORTED;
  const int64_t es = (dtype == FAMLIES_F32) ? 4 : 8;

  // Descriptors with the intermediates' dense strides; device memory for them.
  std::vector<famlies_tensor_t> t(tensors, tensors + ntensors);
  std::vector<std::vector<int64_t>> dense(ntensors);
  std::vector<int64_t> bytes(ntensors, 0);
  for (int i = 0; i < ntensors; ++i) {
    if (!inter[i]) continue;
    if (t[i].ndim < 0 || t[i].ndim > FAMLIES_MAX_NDIM || (t[i].ndim > 0 && !t[i].extents))
      return FAMLIES_ERR_INVALID_ARG;
    dense[i].resize(t[i].ndim > 0 ? t[i].ndim : 1);
    int64_t n = 1;
    for (int d = 0; d < t[i].ndim; ++d) {
      if (t[i].extents[d] < 0) return FAMLIES_ERR_INVALID_ARG;
      dense[i][d] = n;
      n *= t[i].extents[d];
    }
    t[i].strides = dense[i].data();
    bytes[i] = n * es;
    t[i].size_bytes = bytes[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<void*> owned;
  auto release = [&] {
    for (void* q : owned) cudaFreeAsync(q, s);
    owned.clear();
  };
  if (any_inter) {
    int rc = check_device();
    if (rc) return rc;
    for (int i = 0; i < ntensors; ++i) {
      if (!inter[i] || !written[i]) continue;
      void* q = nullptr;
      // a zero-size intermediate still gets a distinct address (alias checks)
      if (cudaMallocAsync(&q, bytes[i] > 0 ? bytes[i] : 256, s) != cudaSuccess) {
        cudaGetLastError();
        release();
        return FAMLIES_ERR_ALLOC;
      }
      owned.push_back(q);
      t[i].data = q;
    }
  }
  // Plan every step first, so that a planning error launches nothing.
  std::vector<Plan> plans(nsteps);
  for (int i = 0; i < nsteps; ++i) {
    const famlies_step_t& st = steps[i];
    int rc = make_plan(st.alpha, &t[st.a], &t[st.b], &t[st.c], dtype, opt, &plans[i]);
    if (rc) {
      release();
      return rc;
    }
  }
  // Fused epilogues (fp64 split).  The split of a consuming step needs each
  // of its rows' exponent bound and Inf/NaN flag, a maximum over the whole
  // row, which a scan of the intermediate would compute.  When the
  // intermediate is written once (beta = 0) by an fp64-split step and its
  // first reader is an fp64-split step whose row class for it is exactly
  // the producer's row or column class (same modes in the same order, so the
  // two fused row indices agree; no batch labels), the producer's finish
  // records those exponents and flags as it writes each value, and the
  // consumer skips its exponent pass over the intermediate.  (Its digit
  // slices cannot be written by the producer: a row's exponent is only known
  // once every tile of that row is done.)
  if (dtype == FAMLIES_F64_EMU && any_inter) {
    for (int x = 0; x < ntensors; ++x) {
      if (!inter[x] || !written[x]) continue;
      int prod = -1, writes = 0, cons = -1;
      for (int i = 0; i < nsteps; ++i)
        if (steps[i].c == x) {
          ++writes;
          if (prod < 0) prod = i;
        }
      if (writes != 1) continue;
      for (int i = prod + 1; i < nsteps && cons < 0; ++i)
        if (steps[i].a == x || steps[i].b == x) cons = i;
      if (cons < 0 || steps[cons].a == steps[cons].b) continue;
      Plan& P = plans[prod];
      Plan& Q = plans[cons];
      auto plain = [](const Plan& q) {
        return q.kernel == FAMLIES_KERNEL_TC_EMU && q.l == 1 && !q.sym_n && q.band_side < 0 && q.krp_side < 0 &&
               !q.tri;
      };
      if (!plain(P) || !plain(Q)) continue;
      const int side = Q.a == t[x].data ? 0 : (Q.b == t[x].data ? 1 : -1);
      if (side < 0) continue;
      const ClassModes& R = side == 0 ? Q.M : Q.N;
      auto same = [&](const ClassModes& pc) {
        if (pc.n != R.n) return false;
        for (int d = 0; d < pc.n; ++d)
          if (pc.m[d].ext != R.m[d].ext || pc.m[d].sc != (side == 0 ? R.m[d].sa : R.m[d].sb)) return false;
        return true;
      };
      const int mode = same(P.M) ? 1 : (same(P.N) ? 2 : 0);
      if (!mode) continue;
      const int64_t rows = R.total();
      void* q = nullptr;
      const size_t eb = ((size_t)rows * 4 + 255) / 256 * 256;
      if (cudaMallocAsync(&q, 2 * eb + (size_t)(rows + 1) * 4, s) != cudaSuccess) {
        cudaGetLastError();
        continue;  // unfused: the consumer scans the intermediate itself
      }
      owned.push_back(q);
      int32_t* e = (int32_t*)q;
      int32_t* flag = (int32_t*)((char*)q + eb);
      int32_t* list = (int32_t*)((char*)q + 2 * eb);
      // exponents start at a large negative value, flags and the list count at 0
      if (cudaMemsetAsync(e, 0x80, (size_t)rows * 4, s) != cudaSuccess ||
          cudaMemsetAsync(flag, 0, eb + (size_t)(rows + 1) * 4, s) != cudaSuccess) {
        cudaGetLastError();
        release();
        return FAMLIES_ERR_CUDA;
      }
      P.emit_mode = mode;
      P.emit_e = e;
      P.emit_flag = flag;
      P.emit_list = list;
      Q.pre_e[side] = e;
      Q.pre_flag[side] = flag;
      Q.pre_list[side] = list;
    }
  }
  for (int i = 0; i < nsteps; ++i) {
    int rc = run_plan(plans[i], steps[i].alpha, steps[i].beta, s, opt, nullptr);
    if (rc) {
      release();
      return rc;
    }
  }
  release();
  return FAMLIES_OK;
}

int famlies_contract(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
                     double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                     void* stream) {
  return famlies_contract_ex(alpha, A, B, beta, C, dtype, stream, nullptr, nullptr);
}

namespace {

// The copy stream of a device (for host calls whose copies overlap compute).
cudaStream_t copy_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}

int find_label(const famlies_tensor_t* t, int32_t label) {
  for (int i = 0; i < t->ndim; ++i)
    if (t->labels[i] == label) return i;
  return -1;
}

// Host-buffer contraction whose larger input X sits in pinned memory and is
// large: X is copied in chunks along its outermost mode on a copy stream,
// and each chunk's contraction runs on the call's stream as soon as its
// bytes have landed, so the transfers and the kernels overlap.  A chunk of
// a contracted label adds into C (beta for the first chunk, then 1); a
// chunk of a free or batch label writes its own part of C.  Returns 1 when
// the path does not apply (the caller then copies whole operands).
int contract_host_chunked(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B, double beta,
                          const famlies_tensor_t* C, famlies_dtype_t dtype, cudaStream_t s,
                          const famlies_options_t* opt, const Plan& p) {
  constexpr int kChunks = 8;
  constexpr int64_t kMinChunkBytes = (int64_t)64 << 20;
  if (p.kernel == FAMLIES_KERNEL_SCALE) return 1;
  const int64_t span_a = p.swapped ? p.span_b : p.span_a, span_b = p.swapped ? p.span_a : p.span_b;
  const int es_a = p.swapped ? p.es_b : p.es_a, es_b = p.swapped ? p.es_a : p.es_b;
  const bool x_is_a = span_a * es_a >= span_b * es_b;
  const famlies_tensor_t* X = x_is_a ? A : B;
  const famlies_tensor_t* Y = x_is_a ? B : A;
  const int64_t span_x = x_is_a ? span_a : span_b, span_y = x_is_a ? span_b : span_a;
  const int es_x = x_is_a ? es_a : es_b, es_y = x_is_a ? es_b : es_a;
  if (span_x * es_x < kChunks * kMinChunkBytes) return 1;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, X->data) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (at.type != cudaMemoryTypeHost) return 1;  // pageable: copies would not overlap
  // the outermost mode: chunks along it must be disjoint ranges of memory
  int m = 0;
  for (int i = 1; i < X->ndim; ++i)
    if (X->strides[i] > X->strides[m]) m = i;
  const int64_t ext = X->extents[m], st = X->strides[m];
  int64_t rest = 1;
  for (int i = 0; i < X->ndim; ++i)
    if (i != m) rest += (X->extents[i] - 1) * X->strides[i];
  if (ext < 2 || st < rest) return 1;
  cudaStream_t sc = copy_stream();
  if (!sc) return 1;
  const int nch = (int)(ext < kChunks ? ext : kChunks);
  const int iy = find_label(Y, X->labels[m]), ic = find_label(C, X->labels[m]);

  const int64_t bytes_x = span_x * es_x, bytes_y = span_y * es_y, bytes_c = p.span_c * p.es_c;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  void* dev = nullptr;
  if (cudaMallocAsync(&dev, up(bytes_x) + up(bytes_y) + up(bytes_c) + 256, s) != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_ALLOC;
  }
  char* dx = (char*)dev;
  char* dy = dx + up(bytes_x);
  char* dc = dy + up(bytes_y);
  int64_t entries_c = 1;
  for (int i = 0; i < C->ndim; ++i) entries_c *= C->extents[i];
  const bool copy_c_in = beta != 0.0 || entries_c != p.span_c;
  std::vector<cudaEvent_t> ev(nch + 1, nullptr);
  for (auto& e : ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  cudaError_t e = cudaSuccess;
  int rc = FAMLIES_OK;
  // All host-to-device copies go in order on the copy stream (one copy
  // engine serves them in that order): the smaller input and C first, which
  // every chunk needs, then X's chunks; chunk i's contraction waits for its
  // copy only.  The copy stream starts once the workspace exists.
  e = cudaEventRecord(ev[nch], s);
  if (!e) e = cudaStreamWaitEvent(sc, ev[nch], 0);
  if (!e && bytes_y) e = cudaMemcpyAsync(dy, Y->data, bytes_y, cudaMemcpyHostToDevice, sc);
  if (!e && copy_c_in) e = cudaMemcpyAsync(dc, C->data, bytes_c, cudaMemcpyHostToDevice, sc);
  for (int i = 0; i < nch && !e; ++i) {
    const int64_t e0 = ext * i / nch, e1 = ext * (i + 1) / nch;
    const int64_t off = e0 * st * es_x, nb = ((e1 - e0 - 1) * st + rest) * es_x;
    e = cudaMemcpyAsync(dx + off, (const char*)X->data + off, nb, cudaMemcpyHostToDevice, sc);
    if (!e) e = cudaEventRecord(ev[i], sc);
  }
  int64_t ex_x[FAMLIES_MAX_NDIM], ex_y[FAMLIES_MAX_NDIM], ex_c[FAMLIES_MAX_NDIM];
  for (int i = 0; i < nch && !e && !rc; ++i) {
    const int64_t e0 = ext * i / nch, e1 = ext * (i + 1) / nch;
    famlies_tensor_t xi = *X, yi = *Y, ci = *C;
    std::memcpy(ex_x, X->extents, sizeof(int64_t) * X->ndim);
    std::memcpy(ex_y, Y->extents, sizeof(int64_t) * Y->ndim);
    std::memcpy(ex_c, C->extents, sizeof(int64_t) * C->ndim);
    ex_x[m] = e1 - e0;
    xi.extents = ex_x;
    xi.data = dx + e0 * st * es_x;
    yi.data = dy;
    if (iy >= 0) {
      ex_y[iy] = e1 - e0;
      yi.data = dy + e0 * Y->strides[iy] * es_y;
    }
    yi.extents = ex_y;
    ci.data = dc;
    if (ic >= 0) {
      ex_c[ic] = e1 - e0;
      ci.data = dc + e0 * C->strides[ic] * p.es_c;
    }
    ci.extents = ex_c;
    xi.size_bytes = yi.size_bytes = ci.size_bytes = 0;
    const double bi = (ic >= 0 || i == 0) ? beta : 1.0;  // a contracted label accumulates
    e = cudaStreamWaitEvent(s, ev[i], 0);
    if (e) break;
    Plan pc;
    rc = make_plan(alpha, x_is_a ? &xi : &yi, x_is_a ? &yi : &xi, &ci, dtype, opt, &pc);
    if (!rc) rc = run_plan(pc, alpha, bi, s, opt, nullptr);
  }
  if (!e && !rc) e = cudaMemcpyAsync(C->data, dc, bytes_c, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(dev, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaError_t e3 = cudaStreamSynchronize(sc);
  for (auto& v : ev) cudaEventDestroy(v);
  if (rc) return rc;
  if (e != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_CUDA;
  }
  return FAMLIES_OK;
}

}  // namespace

int famlies_contract_host(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
                          double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                          void* stream, const famlies_options_t* opt) {
  Plan p;
  int rc = make_plan(alpha, A, B, C, dtype, opt, &p);
  if (rc) return rc;
  if (p.kernel == FAMLIES_KERNEL_NONE) return FAMLIES_OK;
  if ((rc = check_device())) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = contract_host_chunked(alpha, A, B, beta, C, dtype, s, opt, p)) != 1) return rc;
  // Spans in the caller's operand order (the plan may have swapped roles).
  const int64_t span_a = p.swapped ? p.span_b : p.span_a;
  const int64_t span_b = p.swapped ? p.span_a : p.span_b;
  const bool reads_ab = p.kernel != FAMLIES_KERNEL_SCALE;
  const int64_t bytes_a = reads_ab ? span_a * p.es_a : 0;
  const int64_t bytes_b = reads_ab ? span_b * p.es_b : 0;
  const int64_t bytes_c = p.span_c * p.es_c;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  void* dev = nullptr;
  if (cudaMallocAsync(&dev, up(bytes_a) + up(bytes_b) + up(bytes_c) + 256, s) != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_ALLOC;
  }
  char* da = (char*)dev;
  char* db = da + up(bytes_a);
  char* dc = db + up(bytes_b);
  int64_t entries_c = 1;
  for (int i = 0; i < C->ndim; ++i) entries_c *= C->extents[i];
  // C is copied in when beta reads it, or when its span has gaps that the
  // copy back must not overwrite with undefined bytes.
  const bool copy_c_in = beta != 0.0 || entries_c != p.span_c;
  cudaError_t e = cudaSuccess;
  if (bytes_a) e = cudaMemcpyAsync(da, A->data, bytes_a, cudaMemcpyHostToDevice, s);
  if (!e && bytes_b) e = cudaMemcpyAsync(db, B->data, bytes_b, cudaMemcpyHostToDevice, s);
  if (!e && copy_c_in) e = cudaMemcpyAsync(dc, C->data, bytes_c, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    famlies_tensor_t a2 = *A, b2 = *B, c2 = *C;
    a2.data = da;
    b2.data = db;
    c2.data = dc;
    a2.size_bytes = b2.size_bytes = c2.size_bytes = 0;
    Plan p2;
    rc = make_plan(alpha, &a2, &b2, &c2, dtype, opt, &p2);
    if (!rc) rc = run_plan(p2, alpha, beta, s, opt, nullptr);
    if (!rc) e = cudaMemcpyAsync(C->data, dc, bytes_c, cudaMemcpyDeviceToHost, s);
  }
  cudaFreeAsync(dev, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (rc) return rc;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_CUDA;
  }
  return FAMLIES_OK;
}

int famlies_contract_batched(int64_t count, const double* alpha, const famlies_tensor_t* A,
                             const famlies_tensor_t* B, const double* beta,
                             const famlies_tensor_t* C, famlies_dtype_t dtype, void* stream,
                             int use_graph) {
  if (count < 0 || (count > 0 && (!alpha || !beta || !A || !B || !C)))
    return FAMLIES_ERR_INVALID_ARG;
  std::vector<Plan> plans((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    int rc = make_plan(alpha[i], &A[i], &B[i], &C[i], dtype, nullptr, &plans[i]);
    if (rc) return rc;
    // bf16 problems stay on the packed kernel, which the grouped launch runs
    if (plans[i].kernel == FAMLIES_KERNEL_TC_BF16_DIRECT) plans[i].kernel = FAMLIES_KERNEL_TC_BF16;
  }
  if (count == 0) return FAMLIES_OK;
  int rc = check_device();
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // problems of the packed tensor-core kernels go through one grouped launch
  // per stage; the rest (empty, scale-only, CUDA-core) one by one
  std::vector<const Plan*> grouped;
  std::vector<double> ga, gb;
  for (int64_t i = 0; i < count; ++i) {
    const int k = plans[i].kernel;
    if (k == FAMLIES_KERNEL_TC_EMU || k == FAMLIES_KERNEL_TC_BF16 || k == FAMLIES_KERNEL_TC_TF32X3) {
      grouped.push_back(&plans[i]);
      ga.push_back(alpha[i]);
      gb.push_back(beta[i]);
    } else if ((rc = run_plan(plans[i], alpha[i], beta[i], s, nullptr, nullptr))) {
      return rc;
    }
  }
  int* status = device_status_ptr();
  if (!status) return FAMLIES_ERR_CUDA;
  return run_grouped(grouped, ga, gb, s, use_graph != 0, status, env_wait_limit());
}

int famlies_device_status(void* stream) {
  if (check_device()) return FAMLIES_ERR_NO_DEVICE;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_CUDA;
  }
  int v = 0;
  if (read_clear_status(&v)) return FAMLIES_ERR_CUDA;
  return v;
}

}  // extern "C"
