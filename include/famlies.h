/*
 * famlies.h -- C ABI of the B300 dense tensor-contraction library.
 *
 * The one operation is the general dense tensor contraction
 *
 *     C[c] := alpha * sum_{k} A[a(c,k)] * B[b(c,k)] + beta * C[c]
 *
 * over integer index labels, with every tensor in an arbitrary strided
 * layout.  The paper asks for tensor contraction computed by fusing the data
 * reorganisation into the level-3 product instead of converting tensors to
 * matrices first (Sec. 1, "Challenges", last item; Sec. 2.3 "Supporting
 * tensor computations", block-scatter mapping), for arbitrarily strided
 * local layouts (Girder 2, "Providing flexibility in data layout"), for
 * transposition expressed as a change of strides (Sec. 2.1 "Variations on
 * functionality"), for mixed/new precisions such as bf16 (Sec. 1.5
 * "Supporting new and mixed precisions"), and for bounds checking with
 * graceful error recovery (Girder 1, "Code safety").  GEMM is the case of
 * one label per class.
 *
 * Label semantics.  A label in C and in exactly one of A, B is a free index
 * (class M if in A, class N if in B); a label in A and B but not in C is
 * contracted (class K); a label in all three is a batch index.  A label that
 * appears in only one tensor, or twice in one tensor, is rejected
 * (FAMLIES_ERR_LABEL).  Extents of a label must agree across tensors.
 *
 * Conventions (BLAS-style).  alpha == 0, or an empty contracted extent:
 * C := beta * C and A, B are not read.  beta == 0: C is not read, so NaN or
 * Inf already in C is overwritten.  Otherwise Inf/NaN in A or B propagate
 * as IEEE arithmetic gives them (the paper adopts consistent NaN/Inf
 * propagation, Sec. 1.5 "BLIS and TBLIS").  An empty free extent is a no-op.
 *
 * Memory.  Every data pointer is a DEVICE pointer on the current CUDA device
 * unless the entry point says otherwise; the caller owns all buffers and the
 * library keeps no pointer after the call returns.  Work is enqueued on the
 * caller's stream (a cudaStream_t passed as void*; NULL is the legacy
 * default stream) and runs asynchronously; temporary workspace is taken
 * from the stream-ordered allocator on that stream and released on it.
 *
 * Errors.  Every entry point returns FAMLIES_OK (0) or a negative
 * FAMLIES_ERR_* code; host-side errors are reported before anything is
 * launched.  Kernels never trap: a kernel whose bounded wait expires
 * records FAMLIES_ERR_DEVICE_TIMEOUT in a device status word, which
 * famlies_device_status() reads.  No C++ exception crosses this ABI.
 */
#ifndef FAMLIES_H
#define FAMLIES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FAMLIES_MAX_NDIM 8

#if defined(__GNUC__)
#define FAMLIES_API __attribute__((visibility("default")))
#else
#define FAMLIES_API
#endif

/* Storage and arithmetic of one call.
 *   F64      A, B, C fp64; native fp64 fused multiply-add.
 *   F64_EMU  A, B, C fp64; each operand is split into `slices` bf16 slices
 *            of 8-bit integer digits (per row / column power-of-two
 *            scaling), the slice products run on the tensor cores with
 *            exact fp32 accumulation, recombination and the alpha/beta
 *            update run in fp64.  6 slices reach fp64-level relative error
 *            (a few 1e-14); 7 go below the native fp64 product's error.
 *   F32      A, B, C fp32; tensor cores with a three-term split of each
 *            operand into tf32 high and low parts (fp32-level accuracy).
 *   BF16     A, B bf16, C fp32; bf16 products with fp32 accumulation.
 * alpha and beta are always passed as double and rounded to the
 * accumulation type (fp32 for F32/BF16). */
typedef enum {
  FAMLIES_F64 = 0,
  FAMLIES_F64_EMU = 1,
  FAMLIES_F32 = 2,
  FAMLIES_BF16 = 3
} famlies_dtype_t;

/* One tensor operand.
 *   ndim       0..FAMLIES_MAX_NDIM modes (0 = scalar).
 *   extents    ndim extents, each >= 0 (may be NULL when ndim == 0).
 *   strides    ndim strides in ELEMENTS, each >= 0.  Stride 0 (broadcast)
 *              is allowed in A and B; C's modes of extent > 1 must not
 *              overlap (FAMLIES_ERR_UNSUPPORTED otherwise).
 *   labels     ndim distinct integer labels.
 *   data       element (i_0..i_{n-1}) is at data + sum_d i_d*strides[d]
 *              (in elements of the operand's storage type).
 *   size_bytes optional size of the allocation starting at data; when > 0
 *              every reachable element must lie inside it
 *              (FAMLIES_ERR_OUT_OF_BOUNDS otherwise).  0 = unchecked. */
typedef struct {
  int32_t ndim;
  const int64_t* extents;
  const int64_t* strides;
  const int32_t* labels;
  void* data;
  int64_t size_bytes;
} famlies_tensor_t;

/* Return codes. */
#define FAMLIES_OK 0
#define FAMLIES_ERR_INVALID_ARG (-1)     /* null pointer, ndim, negative extent/stride, dtype */
#define FAMLIES_ERR_LABEL (-2)           /* label in one tensor only, or repeated in a tensor */
#define FAMLIES_ERR_EXTENT_MISMATCH (-3) /* same label, different extents */
#define FAMLIES_ERR_ALIAS (-4)           /* C's memory range overlaps A's or B's */
#define FAMLIES_ERR_OUT_OF_BOUNDS (-5)   /* reachable element beyond size_bytes */
#define FAMLIES_ERR_UNSUPPORTED (-6)     /* e.g. self-overlapping C, a class too large */
#define FAMLIES_ERR_ALLOC (-7)           /* workspace allocation failed */
#define FAMLIES_ERR_CUDA (-8)            /* a CUDA runtime call failed */
#define FAMLIES_ERR_DEVICE_TIMEOUT (-9)  /* a kernel's bounded wait expired (asynchronous) */
#define FAMLIES_ERR_NO_DEVICE (-10)      /* no usable sm_100-family device */
#define FAMLIES_ERR_SCRATCH (-11)        /* call too large for famlies_contract_noalloc's fixed scratch */

/* Optional knobs for famlies_contract_ex (zero-initialise for defaults).
 *   slices      F64_EMU: number of bf16 slices per operand, 2..7 (default 6).
 *   kernel      0 = automatic; 1 = the SIMT (CUDA-core) kernel (F64, F32);
 *               2 = the packed TMA tensor-core kernel (F32, BF16, F64_EMU);
 *               3 = the tensor-core kernel that gathers operand tiles
 *               element by element straight from the strided tensors (F32,
 *               BF16); 4 = the direct bf16 kernel (BF16): tiles staged
 *               straight from the caller's tensors, by TMA where the
 *               strides allow it and by gather warps otherwise, no pack;
 *               5 = the same with both operands gathered (diagnostics).
 *               Automatic BF16 takes 4 whenever the call fits it (each
 *               label class at most two modes after fusion, at most one
 *               batch mode, each operand unit-stride along a free or a
 *               contracted mode, k <= 16384) and 2 otherwise.  A choice
 *               the dtype or the call has no kernel for returns
 *               FAMLIES_ERR_UNSUPPORTED.
 *   tile_n      tensor-core tile width (64, 128 or 256, or 192 for the
 *               direct bf16 kernel; 0 = automatic).
 *   ctas_per_mma 0 or 1 = one SM per tensor-core MMA (the default); 2 =
 *               CTA pairs where the product supports them: the fp64
 *               split's packed product with 256 x 256 tiles (cta_group::2,
 *               each SM of a pair staging 128 rows of A and 128 columns of
 *               B), for single problems without batch labels or triangle,
 *               k > 512 and at least as many pair tiles as pairs of SMs
 *               that fit at once; other calls run on one SM per MMA.
 *               Results are the same either way (integer-exact products).
 *   wait_limit  iteration cap of every bounded wait (0 = default).
 *   stall_test  testing only (0 in normal use): nonzero makes the
 *               tensor-core product kernels first wait, bounded by
 *               wait_limit, on a barrier phase that nothing completes, so
 *               the call's kernels stop early and the device status reads
 *               FAMLIES_ERR_DEVICE_TIMEOUT; C is then left unspecified.
 *   events      optional pair of cudaEvent_t handles created by the caller
 *               (NULL = none): the library records events[0] on the call's
 *               stream immediately before the main product kernel and
 *               events[1] immediately after it, so the caller can time that
 *               kernel alone.  The library never synchronises on them. */
typedef struct {
  int32_t slices;
  int32_t kernel;
  int32_t tile_n;
  int32_t stall_test;
  int64_t wait_limit;
  void* events[2];
  int32_t ctas_per_mma;
  int32_t reserved32;
  int64_t reserved;
} famlies_options_t;

/* What the planner decided for a call (filled by famlies_plan and, when
 * non-NULL, by famlies_contract_ex).  m, n, k, batch are the products of
 * the extents of each label class; *_modes count the classes' modes after
 * index fusion (adjacent modes whose strides chain in every operand that
 * holds them are merged); swapped = 1 when the kernel treats B as its row
 * operand so that C's unit-stride mode lies along the rows; kernel is the
 * path chosen (see FAMLIES_KERNEL_*); launches counts the kernels the call
 * launched; cached = 1 when the call reused the workspace and offset tables
 * of an earlier call with the same shapes, strides, dtype, knobs and stream
 * (the plan cache; it then launched one kernel fewer: no table build);
 * ctas_per_mma = 2 when the product ran on CTA pairs (one tensor-core MMA
 * over two SMs' shared memory, the fp64 split's 256 x 256 tiles; set by
 * famlies_contract_ex when options ask for pairs and the call supports
 * them, 1 otherwise and from famlies_plan).
 * The plan cache keeps up to 16 such workspaces of at most 256 MB each,
 * the least recently used one that no call is holding freed when a new one
 * is needed, once the last call that used it has finished on its stream (an
 * event recorded after that call's kernels; a host wait when the eviction
 * happens while it is still queued); it is bypassed while the stream is
 * being captured into a graph
 * and turned off by the environment variable FAMLIES_PLAN_CACHE=0.  Calls
 * that share an entry are ordered by their (common) stream. */
typedef struct {
  int64_t m, n, k, batch;
  int32_t m_modes, n_modes, k_modes, batch_modes;
  int32_t swapped;
  int32_t kernel;
  int32_t launches;
  int32_t slices;
  int32_t a_contig; /* 0 none, 1 unit stride along the row class, 2 along k */
  int32_t b_contig;
  int32_t c_contig; /* 0 none, 1 along rows, 2 along columns */
  int32_t cached;   /* 1: served by the plan cache (see above) */
  int32_t ctas_per_mma; /* 2: the product ran on CTA pairs (see above) */
} famlies_plan_info_t;

#define FAMLIES_KERNEL_NONE 0      /* nothing to do (empty C) */
#define FAMLIES_KERNEL_SCALE 1     /* C := beta*C only */
#define FAMLIES_KERNEL_SIMT_F64 2  /* fp64 CUDA-core kernel */
#define FAMLIES_KERNEL_SIMT_F32 3  /* fp32 CUDA-core kernel */
#define FAMLIES_KERNEL_TC_BF16 4   /* pack + TMA-fed tcgen05 bf16 product */
#define FAMLIES_KERNEL_TC_TF32X3 5 /* pack (tf32 hi/lo split) + TMA-fed tcgen05 three-term product */
#define FAMLIES_KERNEL_TC_EMU 6    /* fp64 slice split + tcgen05 slice products + fp64 recombination */
#define FAMLIES_KERNEL_TC_BF16_GATHER 7   /* tcgen05 bf16, tiles gathered straight from strided A, B */
#define FAMLIES_KERNEL_TC_TF32X3_GATHER 8 /* tcgen05 three-term tf32, tiles gathered straight */
#define FAMLIES_KERNEL_TC_BF16_DIRECT 9   /* tcgen05 bf16, tiles staged straight from the strided
                                             tensors by multi-mode TMA boxes or gather warps */

/* C := alpha*contract(A,B) + beta*C on `stream`.  Asynchronous: returns
 * after enqueueing.  Host-side validation errors return before any launch. */
FAMLIES_API int famlies_contract(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
                     double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                     void* stream);

/* famlies_contract with knobs (opt may be NULL) and a plan report (info may
 * be NULL). */
FAMLIES_API int famlies_contract_ex(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
                        double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                        void* stream, const famlies_options_t* opt,
                        famlies_plan_info_t* info);

/* Same operation on HOST buffers (pageable or pinned): the library copies
 * the reachable span of A, B (and C when beta != 0) to device workspace on
 * `stream`, contracts, copies C back and synchronises the stream before
 * returning.  size_bytes, when set, bounds the host spans as above. */
FAMLIES_API int famlies_contract_host(double alpha, const famlies_tensor_t* A, const famlies_tensor_t* B,
                          double beta, const famlies_tensor_t* C, famlies_dtype_t dtype,
                          void* stream, const famlies_options_t* opt);

/* count independent contractions (alpha[i], A[i], B[i], beta[i], C[i]) of
 * one dtype (the blocks of a block-sparse contraction, Sec. 2.3,
 * "tensor-of-tensors" tiling).  Problems of the tensor-core dtypes (F64_EMU,
 * BF16, F32) run as one grouped persistent launch per kernel stage over a
 * device tile list ordered longest-first, each problem with its own tile
 * width; the set is cut, in order, into chunks of at most 4 GB of slice
 * workspace (environment FAMLIES_BATCH_WORKSPACE_MB overrides), which run
 * one after the other.  F64 problems, and problems with alpha == 0 or an
 * empty contracted extent, run one by one.  The tile width is tuned on the
 * first call for a shape class by timing the candidates with C redirected
 * to scratch (FAMLIES_AUTOTUNE=0 disables this) and kept for the process;
 * FAMLIES_TUNE_CACHE=<path> also keeps the tuned widths in that JSON file
 * (one object, shape-class key -> width), read on the first grouped call
 * and rewritten whenever a new class is tuned.  fp64-split tiles leave
 * their int64 sums in per-tile slots (at most 2 GB per chunk, counted in its
 * workspace) that a finishing kernel converts after the chunk's product
 * (FAMLIES_GROUP_DEFER=0, or slots above that size: each tile finishes
 * inside the product instead).  Every C[i] must be
 * disjoint from every A[j], B[j] and from every other C[j] (not checked
 * across problems).  When use_graph is non-zero the whole call is captured
 * once into a CUDA graph, cached by the problem set (device, pointers,
 * shapes, strides, scalars) and replayed on later calls with the same set;
 * each cached set keeps its workspace allocated (at most four sets, least
 * recently used evicted), and replays read the operands' current contents.
 * Asynchronous. */
FAMLIES_API int famlies_contract_batched(int64_t count, const double* alpha, const famlies_tensor_t* A,
                             const famlies_tensor_t* B, const double* beta,
                             const famlies_tensor_t* C, famlies_dtype_t dtype, void* stream,
                             int use_graph);

/* Host-only planning: validates the descriptors and reports the plan
 * without touching any device (data pointers are not dereferenced; C/A/B
 * alias checks use the pointer values). */
FAMLIES_API int famlies_plan(const famlies_tensor_t* A, const famlies_tensor_t* B,
                 const famlies_tensor_t* C, famlies_dtype_t dtype,
                 const famlies_options_t* opt, famlies_plan_info_t* info);

/* Static English text for a return code (never NULL). */
FAMLIES_API const char* famlies_error_string(int code);

/* Synchronises `stream`, then returns and clears the device status word of
 * the current device: FAMLIES_OK, or FAMLIES_ERR_DEVICE_TIMEOUT when some
 * kernel's bounded wait expired since the last call. */
FAMLIES_API int famlies_device_status(void* stream);

/* Library ABI version (major*10000 + minor*100 + patch). */
FAMLIES_API int famlies_version(void);

/* The paper has no counterpart to this entry point: it is a library service
 * for callers that cannot allocate device memory (a host whose memory pool
 * owns the whole device, a real-time loop that may not enter the allocator,
 * an embedding that only hands over its input and output buffers).
 *
 * Same operation and conventions as famlies_contract for dtype F64 or F32
 * (other dtypes: FAMLIES_ERR_UNSUPPORTED), computed by the CUDA-core
 * kernels; it allocates nothing.  Its only scratch, the offset tables, lives
 * in a fixed 1 MiB device array built into the library (2^17 int64 entries,
 * held on every GPU that loads the library until the process exits).  A
 * call needs 2*(m + n + k) + 3*batch entries, where m, n, k and batch are
 * the products of the extents of its label classes (famlies_plan reports
 * them); a larger call returns FAMLIES_ERR_SCRATCH and launches nothing.
 * Every call on a device shares the array and rewrites the part it reads,
 * so calls whose kernels may overlap on the GPU (unordered streams) race
 * and must be ordered by the caller.  The first call on a device looks up
 * the array's device address with that device current; make it before any
 * stream capture on that device.  Asynchronous on `stream`. */
FAMLIES_API int famlies_contract_noalloc(double alpha, const famlies_tensor_t* A,
                                         const famlies_tensor_t* B, double beta,
                                         const famlies_tensor_t* C, famlies_dtype_t dtype,
                                         void* stream);

/* Contraction with a symmetric dense operand (Sec. 3, "tensor contraction
 * with general and symmetric dense tensors").  A is symmetric under the
 * exchange of its first and second halves of modes,
 *   A[x_1..x_h, y_1..y_h] = A[y_1..y_h, x_1..x_h],
 * both halves with the same extents.  With p and q the fused indices of the
 * two halves (first mode fastest, 0 <= p, q < n = product of a half's
 * extents), only the elements with p >= q are stored, column by column:
 * element (p, q) at data[q * n - q * (q - 1) / 2 + (p - q)], n (n + 1) / 2
 * elements in all (LAPACK's lower packed storage of the n x n matrix).
 * Same operation and conventions as famlies_contract_ex with A expanded;
 * A is read once (half the bytes of its dense form).
 * Supported: dtype F64_EMU, with one half of A's modes contracted and the
 * other free (each half fusing into one index) and no batch label; other
 * cases return FAMLIES_ERR_UNSUPPORTED.  A's size_bytes (0 = unchecked)
 * is checked against the packed size; the aliasing check uses the packed
 * range.  Options as for famlies_contract_ex (the kernel choice is fixed). */
typedef struct {
  int32_t ndim;            /* even, 2..FAMLIES_MAX_NDIM */
  const int64_t* extents;  /* ndim; extents[i] == extents[i + ndim/2] */
  const int32_t* labels;   /* ndim distinct labels */
  const void* data;        /* device pointer, packed lower triangle */
  int64_t size_bytes;
} famlies_symtensor_t;

FAMLIES_API int famlies_contract_sym(double alpha, const famlies_symtensor_t* A,
                                     const famlies_tensor_t* B, double beta,
                                     const famlies_tensor_t* C, famlies_dtype_t dtype, void* stream,
                                     const famlies_options_t* opt, famlies_plan_info_t* info);

/* Sandwiched product with a tridiagonal middle factor (Sec. 3, "Beyond
 * LAPACK functionality": the update C := C - A T A^T of skew-symmetric
 * factorisations, a GEMMT that updates one triangle of C, with T A^T formed
 * while the operand is packed instead of in a workspace):
 *   C[i,j] := beta * C[i,j] + alpha * sum_{p,q} A[i,p] T[p,q] A[j,q]
 * for i >= j only; the strictly upper triangle of C is neither read nor
 * written.  A is n x k, element (i,p) at A[i*rs_a + p*cs_a]; C is n x n,
 * element (i,j) at C[i*rs_c + j*cs_c] (strides in elements, >= 0).
 * T is k x k tridiagonal, given by device vectors:
 *   T[p+1,p] = t_sub[p] (k-1 entries), T[p,p] = t_diag[p] (k entries),
 *   T[p,p+1] = t_sup[p] (k-1 entries);
 * t_diag == NULL means a zero diagonal, t_sup == NULL means t_sup = -t_sub
 * (T skew-symmetric).  Only the three diagonals are multiplied (a banded
 * T: no 0 * Inf from entries off the band).  dtype: FAMLIES_F64 (native
 * CUDA cores), FAMLIES_F64_EMU or FAMLIES_F32 (tensor cores); A, C and the
 * vectors hold the dtype's elements (fp64 or fp32); BF16 returns
 * FAMLIES_ERR_UNSUPPORTED.  Error codes, options (kernel choice fixed by the
 * dtype) and info as for famlies_contract_ex; C must not overlap A. */
FAMLIES_API int famlies_gemmt_tridiag(int64_t n, int64_t k, double alpha, const void* A, int64_t rs_a,
                                      int64_t cs_a, const void* t_sub, const void* t_diag,
                                      const void* t_sup, double beta, void* C, int64_t rs_c,
                                      int64_t cs_c, famlies_dtype_t dtype, void* stream,
                                      const famlies_options_t* opt, famlies_plan_info_t* info);

/* A matrix operand: element (i, j) at data[i * rs + j * cs] (strides in
 * elements, >= 0), rows x cols. */
typedef struct {
  const void* data;
  int64_t rows, cols;
  int64_t rs, cs;
} famlies_matrix_t;

/* Matricised tensor times Khatri-Rao product, the inner contraction of
 * CP-ALS (Sec. 3, Girder 5: CP-ALS among the tensor factorisations):
 *   M[i, r] := beta * M[i, r]
 *            + alpha * sum over the other modes of X[.., i (mode `mode`), ..]
 *                      * prod_{m != mode} U[m][i_m, r]
 * X is an N-way tensor (2 <= N <= FAMLIES_MAX_NDIM; its labels are
 * ignored), U an array of N factor matrices (U[m] is X->extents[m] x R;
 * U[mode] is ignored), M is X->extents[mode] x R, R = M->cols.  The
 * Khatri-Rao product of the factors is never stored: its elements are
 * formed (products in increasing m) as the operand is packed.  dtype:
 * FAMLIES_F64 (native), FAMLIES_F64_EMU, FAMLIES_F32; all operands hold the
 * dtype's elements; BF16 returns FAMLIES_ERR_UNSUPPORTED.  M must not
 * overlap X or a factor (FAMLIES_ERR_ALIAS).  Error codes, options (kernel
 * choice fixed by the dtype) and info as for famlies_contract_ex. */
FAMLIES_API int famlies_mttkrp(double alpha, const famlies_tensor_t* X, int32_t mode,
                               const famlies_matrix_t* U, double beta, const famlies_matrix_t* M,
                               famlies_dtype_t dtype, void* stream, const famlies_options_t* opt,
                               famlies_plan_info_t* info);

/* Contraction networks: a pre-ordered sequence of tensor contractions run
 * through the same planner and kernels (Sec. 3, Girder 5, tensor contraction
 * networks).  `tensors` lists every tensor of the network; step i computes
 *   tensors[c] := alpha * contract(tensors[a], tensors[b]) + beta * tensors[c]
 * over the tensors' own labels, like famlies_contract_ex, in the given order
 * on `stream` with one dtype and one options block (NULL: defaults).
 * A tensor whose `data` is NULL is an intermediate: the library allocates
 * it dense (first mode fastest; its `strides` are ignored) from the
 * stream-ordered pool before the first step and frees it after the last,
 * all on `stream`; intermediates never reach the caller.  Ownership of every
 * other tensor stays with the caller.
 * Errors, found before anything is launched: an index out of range or a
 * step whose c equals its a or b, an intermediate read before a step writes
 * it or first written with beta != 0 (FAMLIES_ERR_INVALID_ARG); dtype BF16
 * with an intermediate (its products are fp32, its operands bf16:
 * FAMLIES_ERR_UNSUPPORTED); any error a step's planning reports.  An
 * allocation failure returns FAMLIES_ERR_ALLOC; a launch failure stops the
 * sequence with FAMLIES_ERR_CUDA (earlier steps have run). */
typedef struct {
  int32_t a, b, c;   /* indices into the tensor list */
  int32_t reserved;  /* 0 */
  double alpha, beta;
} famlies_step_t;

FAMLIES_API int famlies_network(const famlies_tensor_t* tensors, int32_t ntensors,
                                const famlies_step_t* steps, int32_t nsteps, famlies_dtype_t dtype,
                                void* stream, const famlies_options_t* opt);

#ifdef __cplusplus
}
#endif

#endif /* FAMLIES_H */
