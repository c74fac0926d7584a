// famlies_contract_noalloc: the CUDA-core (fp64 / fp32) contraction for
// callers that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc / cudaMallocAsync is not
// available or not allowed -- for example a host that pre-reserves all
// device memory for its own pool and forbids other allocations, a real-time
// loop that may not take the allocator's locks or risk an out-of-memory
// failure mid-run, or an embedding that hands the library only the input
// and output buffers.  The regular entry points take stream-ordered
// workspace for their offset tables; this one keeps them in a fixed device
// array that is part of the library image instead.
//
// The array: kScratchEntries int64 entries (1 MiB) in file-scope device
// memory, present on every GPU that loads the library until the process
// exits.  A call needs 2*(m + n + k) + 3*batch entries (the offset tables of
// its fused label classes); larger calls are rejected with
// FAMLIES_ERR_SCRATCH before anything is launched.
//
// Sharing: every call on a device uses the same array, and the offset-table
// kernel rewrites every entry a call reads before the contraction kernel
// reads it, so nothing has to start at zero.  Two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// the array and may compute wrong results: order such calls on one stream
// or with events.
//
// Set-up: the first call on each device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture on the device.
#include <cstdlib>
#include <mutex>

#include <cuda_runtime.h>

#include "device.h"
#include "plan.h"

using namespace famlies;

namespace {

constexpr int64_t kScratchEntries = (int64_t)1 << 17;  // 1 MiB of int64 offsets
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int64_t g_noalloc_scratch[kScratchEntries];

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device
// pointer).  Returns nullptr when there is no usable device.
int64_t* scratch_address() {
  static std::mutex mu;
  static int64_t* addr[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = (int64_t*)p;
  }
  return addr[dev];
}

bool is_sm103() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return major == 10 && minor == 3;
}

}  // namespace

extern "C" FAMLIES_API int famlies_contract_noalloc(double alpha, const famlies_tensor_t* A,
                                                    const famlies_tensor_t* B, double beta,
                                                    const famlies_tensor_t* C,
                                                    famlies_dtype_t dtype, void* stream) {
  if (dtype != FAMLIES_F64 && dtype != FAMLIES_F32) return FAMLIES_ERR_UNSUPPORTED;
  famlies_options_t opt = {};
  opt.kernel = 1;  // the CUDA-core kernels: their only scratch is the offset tables
  Plan p;
  int rc = make_plan(alpha, A, B, C, dtype, &opt, &p);
  if (rc) return rc;
  if (p.kernel == FAMLIES_KERNEL_NONE) return FAMLIES_OK;
  if (table_entries(p) > kScratchEntries) return FAMLIES_ERR_SCRATCH;
  if (!is_sm103()) return FAMLIES_ERR_NO_DEVICE;
  int64_t* scratch = scratch_address();
  int* status = device_status_ptr();
  if (!scratch || !status) return FAMLIES_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Tables t;
  if (launch_tables(p, scratch, &t, s) != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_CUDA;
  }
  cudaError_t err;
  if (p.kernel == FAMLIES_KERNEL_SCALE) {
    err = launch_scale(p, t, beta, s);
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
    g.wait_limit = (int64_t)1 << 26;
    g.status = status;
    err = launch_simt(p, g, nullptr, s);
  }
  if (err != cudaSuccess) {
    cudaGetLastError();
    return FAMLIES_ERR_CUDA;
  }
  return FAMLIES_OK;
}
