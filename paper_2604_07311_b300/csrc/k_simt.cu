// CUDA-core kernels: offset tables, C := beta*C, and the fp64 / fp32 SIMT
// contraction (the native-fp64 path and a forced-SIMT fp32 path).
//
// The SIMT contraction stages a BM x BK tile of A and a BN x BK tile of B
// into shared memory straight from the strided tensors through the offset
// tables (block-scatter vectors, Sec. 2.3 of the paper): threads are laid
// along whichever index is unit-stride in that operand so that the gathers
// coalesce.  Each thread then owns a TM x TN register block of C, updated
// with fused multiply-adds, and the epilogue applies alpha/beta and scatters
// to C's strided layout.  Native fp64 on B300 is bound by the fp64 pipe, not
// by memory, so this simple register-blocked form reaches that pipe's rate.
#include <cstdint>

#include "device.h"

namespace famlies {

// Device status word: FAMLIES_OK, or the first error a kernel recorded
// (kernels get its address through GemmArgs::status).
__device__ int g_famlies_status = 0;

int* device_status_ptr() {
  static int* ptr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!ptr[dev] && cudaGetSymbolAddress((void**)&ptr[dev], g_famlies_status) != cudaSuccess) {
    cudaGetLastError();
    ptr[dev] = nullptr;
  }
  return ptr[dev];
}

int read_clear_status(int* value) {
  int zero = 0;
  if (cudaMemcpyFromSymbol(value, g_famlies_status, sizeof(int)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_famlies_status, &zero, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

// ---------------------------------------------------------------- tables
struct TableJobs {
  TableJob j[9];
};

__global__ void k_tables(TableJobs jobs) {
  const TableJob& J = jobs.j[blockIdx.y];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < J.total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i, off = 0;
    for (int d = 0; d < J.n; ++d) {
      int64_t e = J.ext[d];
      off += (r % e) * J.st[d];
      r /= e;
    }
    J.out[i] = off;
  }
}

cudaError_t launch_tables(const Plan& p, int64_t* ws, Tables* t, cudaStream_t s) {
  TableJobs jobs;
  const ClassModes* cls[9] = {&p.M, &p.M, &p.N, &p.N, &p.K, &p.K, &p.L, &p.L, &p.L};
  const int which[9] = {0, 2, 1, 2, 0, 1, 0, 1, 2};  // sa, sc, sb, sc, sa, sb, sa, sb, sc
  int64_t* ptr[9];
  int64_t off = 0, maxn = 1;
  for (int i = 0; i < 9; ++i) {
    TableJob& J = jobs.j[i];
    const ClassModes& cm = *cls[i];
    J.n = cm.n;
    for (int d = 0; d < cm.n; ++d) {
      J.ext[d] = cm.m[d].ext;
      J.st[d] = which[i] == 0 ? cm.m[d].sa : (which[i] == 1 ? cm.m[d].sb : cm.m[d].sc);
    }
    J.total = cm.total();
    J.out = ws + off;
    ptr[i] = ws + off;
    off += J.total;
    maxn = J.total > maxn ? J.total : maxn;
  }
  t->am = ptr[0]; t->cm = ptr[1]; t->bn = ptr[2]; t->cn = ptr[3];
  t->ak = ptr[4]; t->bk = ptr[5]; t->al = ptr[6]; t->bl = ptr[7]; t->cl = ptr[8];
  int64_t blocks = (maxn + 255) / 256;
  dim3 grid((unsigned)(blocks > 1024 ? 1024 : blocks), 9);
  k_tables<<<grid, 256, 0, s>>>(jobs);
  return cudaGetLastError();
}

// The nine table jobs of one plan, writing into ws (same order and
// placement as launch_tables); fills *t with the table addresses.
void plan_table_jobs(const Plan& p, int64_t* ws, TableJob jobs[9], Tables* t) {
  const ClassModes* cls[9] = {&p.M, &p.M, &p.N, &p.N, &p.K, &p.K, &p.L, &p.L, &p.L};
  const int which[9] = {0, 2, 1, 2, 0, 1, 0, 1, 2};
  int64_t* ptr[9];
  int64_t off = 0;
  for (int i = 0; i < 9; ++i) {
    TableJob& J = jobs[i];
    const ClassModes& cm = *cls[i];
    J.n = cm.n;
    for (int d = 0; d < cm.n; ++d) {
      J.ext[d] = cm.m[d].ext;
      J.st[d] = which[i] == 0 ? cm.m[d].sa : (which[i] == 1 ? cm.m[d].sb : cm.m[d].sc);
    }
    J.total = cm.total();
    J.out = ws + off;
    ptr[i] = ws + off;
    off += J.total;
  }
  t->am = ptr[0]; t->cm = ptr[1]; t->bn = ptr[2]; t->cn = ptr[3];
  t->ak = ptr[4]; t->bk = ptr[5]; t->al = ptr[6]; t->bl = ptr[7]; t->cl = ptr[8];
}

// Many problems' tables in one launch: blockIdx.y walks the job list.
__global__ void k_tables_grouped(const TableJob* __restrict__ jobs, int64_t njobs) {
  for (int64_t j = blockIdx.y; j < njobs; j += gridDim.y) {
    const TableJob J = jobs[j];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < J.total;
         i += (int64_t)gridDim.x * blockDim.x) {
      int64_t r = i, off = 0;
      for (int d = 0; d < J.n; ++d) {
        int64_t e = J.ext[d];
        off += (r % e) * J.st[d];
        r /= e;
      }
      J.out[i] = off;
    }
  }
}

cudaError_t launch_tables_grouped(const TableJob* jobs, int64_t njobs, int64_t max_total,
                                  cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  const int64_t bx = (max_total + 255) / 256;
  dim3 grid((unsigned)(bx > 64 ? 64 : (bx < 1 ? 1 : bx)),
            (unsigned)(njobs > 32768 ? 32768 : njobs));
  k_tables_grouped<<<grid, 256, 0, s>>>(jobs, njobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- C := beta*C
template <typename T>
__global__ void k_scale(T* __restrict__ c, Tables t, int64_t m, int64_t n, int64_t l, T beta, int tri) {
  const int64_t total = m * n * l;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t im = i % m, r = i / m;
    int64_t in = r % n, il = r / n;
    if (!tri_keep(tri, im, in)) continue;  // outside the updated triangle
    T* p = c + t.cm[im] + t.cn[in] + t.cl[il];
    *p = beta == T(0) ? T(0) : beta * *p;  // beta == 0: C is not read
  }
}

cudaError_t launch_scale(const Plan& p, const Tables& t, double beta, cudaStream_t s) {
  int64_t total = p.m * p.n * p.l;
  int64_t blocks = (total + 255) / 256;
  int grid = (int)(blocks > 4 * 148 * 8 ? 4 * 148 * 8 : blocks);
  if (grid < 1) grid = 1;
  if (p.es_c == 8)
    k_scale<double><<<grid, 256, 0, s>>>((double*)p.c, t, p.m, p.n, p.l, beta, p.tri);
  else
    k_scale<float><<<grid, 256, 0, s>>>((float*)p.c, t, p.m, p.n, p.l, (float)beta, p.tri);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- SIMT GEMM
// 256 threads; thread (tx, ty) owns rows ty + i*(BM/TM) and columns
// tx + j*(BN/TN) of the tile (interleaved so shared-memory reads of a warp
// hit distinct banks).
// GEN: the launch has a generated operand (band, Khatri-Rao) or a triangle
// of C; plain contractions run the GEN = false instantiation, which has
// neither the extra loads nor the checks.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool GEN>
__global__ void __launch_bounds__(256) k_simt(GemmArgs g) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const T* __restrict__ A = (const T*)g.a;
  const T* __restrict__ B = (const T*)g.b;
  T* __restrict__ C = (T*)g.c;
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t tiles_m = (g.m + BM - 1) / BM, tiles_n = (g.n + BN - 1) / BN;
  const int64_t ntiles = tiles_m * tiles_n * g.l;
  const T alpha = (T)g.alpha, beta = (T)g.beta;
  // split K (blockIdx.y of gridDim.y): this block's k range; its partial
  // results go to g.part for k_simt_reduce
  const int64_t kbeg = g.k * blockIdx.y / gridDim.y, kend = g.k * (blockIdx.y + 1) / gridDim.y;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t tm = tile % tiles_m, rest = tile / tiles_m;
    const int64_t tn = rest % tiles_n, il = rest / tiles_n;
    const int64_t m0 = tm * BM, n0 = tn * BN;
    // a tile wholly outside the updated triangle has nothing to do
    if (GEN && (g.tri == 1 ? m0 + BM - 1 < n0 : (g.tri == 2 && m0 > n0 + BN - 1))) continue;
    const int64_t al = g.t.al[il], bl = g.t.bl[il], cl = g.t.cl[il];
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        int mm, kk;
        if (g.a_contig == 2) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
        const int64_t gm = m0 + mm, gk = k0 + kk;
        As[kk][mm] = (gm < g.m && gk < kend)
                         ? ((GEN && g.band_op == 1)  ? band_at<T>(A, al + g.t.am[gm], g.t.ak, 0, gk, g.k, g.band)
                            : (GEN && g.krp_op == 1) ? krp_at<T>(g.krp, gm, g.t.ak[gk])
                                                     : A[al + g.t.am[gm] + g.t.ak[gk]])
                         : T(0);
      }
      for (int e = tid; e < BN * BK; e += 256) {
        int nn, kk;
        if (g.b_contig == 2) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
        const int64_t gn = n0 + nn, gk = k0 + kk;
        Bs[kk][nn] = (gn < g.n && gk < kend)
                         ? ((GEN && g.band_op == 2)  ? band_at<T>(B, bl + g.t.bn[gn], g.t.bk, 0, gk, g.k, g.band)
                            : (GEN && g.krp_op == 2) ? krp_at<T>(g.krp, gn, g.t.bk[gk])
                                                     : B[bl + g.t.bn[gn] + g.t.bk[gk]])
                         : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < BK; ++kk) {
        T ra[TM], rb[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) ra[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
        for (int j = 0; j < TN; ++j) rb[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(ra[i], rb[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty + i * (BM / TM);
      if (gm >= g.m) continue;
      const int64_t crow = cl + g.t.cm[gm];
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gn = n0 + tx + j * (BN / TN);
        if (gn >= g.n || (GEN && !tri_keep(g.tri, gm, gn))) continue;
        if (g.part) {  // a split's partial result, summed by k_simt_reduce
          ((T*)g.part)[(((size_t)blockIdx.y * g.l + il) * g.n + gn) * g.m + gm] = acc[i][j];
          continue;
        }
        T* p = C + crow + g.t.cn[gn];
        T v = alpha * acc[i][j];
        if (beta != T(0)) v = fma(beta, *p, v);
        *p = v;
      }
    }
  }
}

// Split-K reduction of the CUDA-core kernel: C = alpha * (sum of the
// splits' partial results, in split order) + beta * C, inside the triangle.
template <typename T>
__global__ void __launch_bounds__(256) k_simt_reduce(GemmArgs g, int splits) {
  const int64_t total = g.m * g.n * g.l;
  const T* P = (const T*)g.part;
  T* C = (T*)g.c;
  const T alpha = (T)g.alpha, beta = (T)g.beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t im = i % g.m, r = i / g.m;
    const int64_t in = r % g.n, il = r / g.n;
    if (!tri_keep(g.tri, im, in)) continue;
    T acc = T(0);
    for (int sp = 0; sp < splits; ++sp) acc += P[(size_t)sp * total + i];
    T* p = C + g.t.cl[il] + g.t.cm[im] + g.t.cn[in];
    T v = alpha * acc;
    if (beta != T(0)) v = fma(beta, *p, v);
    *p = v;
  }
}

namespace {

// Tile shape and grid of the CUDA-core kernel, and its K splits: a launch
// with fewer tiles than SMs splits K (at least 32 per split, two of the
// kernel's 16-deep k steps) so that every SM gets work: at B300's fp64 rate
// (~8 GFLOP/s per SM) a 64 x 64 tile with k = 256 alone takes ~0.25 ms.
struct SimtShape {
  int bm, bn, blocks_per_sm;
  int64_t tiles;
  int splits;
};

SimtShape simt_shape(const Plan& p) {
  SimtShape sh;
  sh.bm = sh.bn = p.es_a == 8 ? 64 : 128;
  sh.blocks_per_sm = p.es_a == 8 ? 8 : 4;
  sh.tiles = ((p.m + sh.bm - 1) / sh.bm) * ((p.n + sh.bn - 1) / sh.bn) * p.l;
  const int64_t sms = num_sms();
  int64_t sp = 1;
  if (sh.tiles < sms) {
    sp = (2 * sms + sh.tiles - 1) / sh.tiles;
    const int64_t kmax = p.k / 32;
    if (sp > kmax) sp = kmax;
    if (sp > 64) sp = 64;
    if (sp < 1) sp = 1;
  }
  sh.splits = (int)sp;
  return sh;
}

}  // namespace

int64_t simt_workspace_bytes(const Plan& p) {
  const SimtShape sh = simt_shape(p);
  return sh.splits > 1 ? (int64_t)sh.splits * p.m * p.n * p.l * p.es_c : 0;
}

cudaError_t launch_simt(const Plan& p, const GemmArgs& g0, void* ws, cudaStream_t s) {
  const int sms = num_sms();
  const SimtShape sh = simt_shape(p);
  GemmArgs g = g0;
  const int splits = ws ? sh.splits : 1;
  g.part = splits > 1 ? ws : nullptr;
  const int64_t cap = (int64_t)sms * sh.blocks_per_sm;
  const dim3 grid((unsigned)(sh.tiles < cap ? sh.tiles : cap), (unsigned)splits);
  const bool gen = g.band_op || g.krp_op || g.tri;
  mark_begin(g, s);
  if (p.es_a == 8) {
    if (gen) k_simt<double, 64, 64, 16, 4, 4, true><<<grid, 256, 0, s>>>(g);
    else k_simt<double, 64, 64, 16, 4, 4, false><<<grid, 256, 0, s>>>(g);
  } else {
    if (gen) k_simt<float, 128, 128, 16, 8, 8, true><<<grid, 256, 0, s>>>(g);
    else k_simt<float, 128, 128, 16, 8, 8, false><<<grid, 256, 0, s>>>(g);
  }
  mark_end(g, s);
  if (splits > 1) {
    const int64_t total = p.m * p.n * p.l, blocks = (total + 255) / 256;
    const int rg = (int)(blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8);
    if (p.es_a == 8)
      k_simt_reduce<double><<<rg, 256, 0, s>>>(g, splits);
    else
      k_simt_reduce<float><<<rg, 256, 0, s>>>(g, splits);
  }
  return cudaGetLastError();
}

}  // namespace famlies
