"""B300-native dense tensor contraction: C := alpha*contract(A, B) + beta*C.

Python face of the C ABI in ``include/famlies.h``.  Importing this package
does not load the CUDA library; the first call does, and raises
``FamliesError`` if it is missing.  ``inputs`` (seeded synthetic workloads)
imports nothing from here.
"""
from __future__ import annotations

import threading

from ._lib import (BF16, DTYPES, F32, F64, F64_EMU, KERNELS, Desc, FamliesError, PlanInfo,
                   desc_numpy, desc_torch, load, options, check, error_string)

__all__ = ["contract", "contract_host", "contract_batched", "contract_network", "contract_sym", "gemmt_tridiag", "mttkrp", "plan", "device_status",
           "FamliesError", "F64", "F64_EMU", "F32", "BF16", "lib_path", "Contract", "contract_autograd"]


def lib_path() -> str:
    from ._lib import LIB_PATH
    return LIB_PATH


def _dtype_code(dtype, A, C):
    import torch
    if dtype is not None:
        return DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    if A.dtype == torch.float64:
        return F64
    if A.dtype == torch.float32:
        return F32
    if A.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported dtype {A.dtype}")


def _stream_handle(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def contract(alpha, A, la, B, lb, beta, C, lc, dtype=None, stream=None, *, slices=0, kernel=0,
             tile_n=0, wait_limit=0, events=None, return_info=False, stall_test=0, ctas_per_mma=0):
    """C := alpha * contract(A, B) + beta * C on the GPU, in place on C.

    A, B, C are CUDA torch tensors (any non-negative strides); la, lb, lc are
    integer labels, one per mode.  dtype: 'f64', 'f64_emu', 'f32', 'bf16' or
    None (from A's dtype).  Enqueued on `stream` (default: torch's current
    stream); asynchronous like any CUDA op.
    """
    lib = load()
    code = _dtype_code(dtype, A, C)
    da, db, dc = _desc_reused(0, A, la), _desc_reused(1, B, lb), _desc_reused(2, C, lc)
    info = PlanInfo() if return_info else None
    if slices or kernel or tile_n or wait_limit or events is not None or stall_test or ctas_per_mma:
        opt = options(slices, kernel, tile_n, wait_limit, events, stall_test, ctas_per_mma)
    else:
        opt = None
    check(lib.famlies_contract_ex(float(alpha), da.ref, db.ref, float(beta), dc.ref, code,
                                  _stream_handle(stream), opt, info))
    return (C, info.as_dict()) if return_info else C


_tls = threading.local()


def _desc_reused(pos, x, labels):
    """Descriptor of torch view x as operand `pos` of a call: the ctypes arrays of
    a (position, shape, strides, labels) signature are built once per thread and
    reused, only the data pointer and the size are rewritten."""
    cache = getattr(_tls, "descs", None)
    if cache is None:
        cache = _tls.descs = {}
    key = (pos, tuple(x.shape), x.stride(), tuple(int(v) for v in labels))
    d = cache.get(key)
    if d is None:
        if len(cache) > 512:
            cache.clear()
        d = cache[key] = Desc(key[1], key[2], key[3], 0, 0)
    d.t.data = x.data_ptr()
    d.t.size_bytes = max(x.untyped_storage().nbytes() - x.storage_offset() * x.element_size(), 0)
    return d


def contract_host(alpha, A, la, B, lb, beta, C, lc, dtype="f64", stream=None, *, slices=0, kernel=0):
    """Same operation on host numpy arrays (copies in, contracts, copies C back; synchronous)."""
    lib = load()
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    da, db, dc = desc_numpy(A, la), desc_numpy(B, lb), desc_numpy(C, lc)
    opt = options(slices, kernel)
    check(lib.famlies_contract_host(float(alpha), da.ref, db.ref, float(beta), dc.ref, code,
                                    _stream_handle(stream) if stream is not None else None, opt))
    return C


def plan(A_shape, A_strides, la, B_shape, B_strides, lb, C_shape, C_strides, lc, dtype="f64",
         pointers=(0x10000, 0x20000000, 0x40000000), slices=0, kernel=0, tile_n=0, ctas_per_mma=0):
    """Host-only plan report (no device needed): classes, fusion, role swap."""
    lib = load()
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    da = Desc(A_shape, A_strides, la, pointers[0])
    db = Desc(B_shape, B_strides, lb, pointers[1])
    dc = Desc(C_shape, C_strides, lc, pointers[2])
    info = PlanInfo()
    check(lib.famlies_plan(da.ref, db.ref, dc.ref, code,
                           options(slices, kernel, tile_n=tile_n, ctas_per_mma=ctas_per_mma), info))
    return info.as_dict()


def contract_batched(alpha, As, las, Bs, lbs, beta, Cs, lcs, dtype=None, stream=None, use_graph=True):
    """count independent contractions in one grouped launch (lists of tensors/labels)."""
    import ctypes
    lib = load()
    n = len(As)
    if not (len(Bs) == len(Cs) == len(las) == len(lbs) == len(lcs) == n):
        raise ValueError("one entry per problem")
    code = _dtype_code(dtype, As[0], Cs[0]) if n else F64
    from ._lib import desc_array_torch
    ta, keep_a = desc_array_torch(As, las)
    tb, keep_b = desc_array_torch(Bs, lbs)
    tc, keep_c = desc_array_torch(Cs, lcs)
    al = [alpha] * n if not hasattr(alpha, "__len__") else list(alpha)
    be = [beta] * n if not hasattr(beta, "__len__") else list(beta)
    aa = (ctypes.c_double * max(n, 1))(*al)
    bb = (ctypes.c_double * max(n, 1))(*be)
    check(lib.famlies_contract_batched(n, aa, ta, tb, bb, tc, code, _stream_handle(stream),
                                       1 if use_graph else 0))
    return Cs


def contract_network(tensors, steps, dtype="f64", stream=None, *, slices=0, kernel=0):
    """A pre-ordered sequence of contractions through the library, in one call.

    tensors: list of (tensor, labels) for caller tensors (CUDA torch tensors,
    any strides) or (shape, labels) for intermediates, which the library
    allocates dense on the device and frees at the end.  steps: list of
    (a, b, c, alpha, beta): tensors[c] := alpha * contract(tensors[a],
    tensors[b]) + beta * tensors[c], run in order on `stream`.
    """
    import ctypes
    from ._lib import Step, TensorDesc
    lib = load()
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    descs = []
    for x, labels in tensors:
        if hasattr(x, "data_ptr"):
            descs.append(desc_torch(x, labels))
        else:
            shape = tuple(int(e) for e in x)
            descs.append(Desc(shape, (0,) * len(shape), labels, 0))
    n = len(descs)
    tt = (TensorDesc * max(n, 1))(*[d.t for d in descs])
    ss = (Step * max(len(steps), 1))(*[Step(int(a), int(b), int(c), 0, float(al), float(be))
                                       for a, b, c, al, be in steps])
    check(lib.famlies_network(tt, n, ss, len(steps), code, _stream_handle(stream), options(slices, kernel)))


def contract_sym(alpha, Ap, extents, la, B, lb, beta, C, lc, dtype="f64_emu", stream=None, *, slices=0,
                 wait_limit=0, events=None, return_info=False):
    """C := alpha * contract(A, B) + beta * C with A symmetric, in place on C.

    A[x, y] = A[y, x] for the first and second halves x, y of its modes
    (`extents` lists all of them, both halves alike).  Ap is a 1-D CUDA
    tensor holding the lower triangle of A as an n x n matrix (n = product
    of a half's extents; fused indices first mode fastest), column by column:
    n (n + 1) / 2 elements.  B and C as for `contract`.
    """
    import ctypes
    from ._lib import SymTensorDesc
    lib = load()
    code = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    nd = len(extents)
    if len(la) != nd:
        raise ValueError("one label per mode of A")
    e = (ctypes.c_int64 * max(nd, 1))(*[int(x) for x in extents])
    lab = (ctypes.c_int32 * max(nd, 1))(*[int(x) for x in la])
    if Ap.dim() != 1 or Ap.stride(0) != 1:
        raise ValueError("Ap must be a contiguous 1-D tensor")
    sa = SymTensorDesc(nd, e, lab, ctypes.c_void_p(Ap.data_ptr()), Ap.numel() * Ap.element_size())
    db, dc = desc_torch(B, lb), desc_torch(C, lc)
    info = PlanInfo()
    opt = options(slices, 0, 0, wait_limit, events)
    check(lib.famlies_contract_sym(float(alpha), ctypes.byref(sa), db.ref, float(beta), dc.ref, code,
                                   _stream_handle(stream), opt, info))
    return (C, info.as_dict()) if return_info else C


def gemmt_tridiag(alpha, A, t_sub, t_diag, t_sup, beta, C, dtype=None, stream=None, *, slices=0,
                  wait_limit=0, events=None, return_info=False):
    """C := beta * C + alpha * A T A^T on the lower triangle of C (i >= j).

    A: (n, k) CUDA tensor, C: (n, n), any non-negative strides.  T is k x k
    tridiagonal: t_sub (k-1), t_diag (k) and t_sup (k-1) are contiguous 1-D
    CUDA tensors of A's dtype, or None (t_diag None: zero diagonal; t_sup
    None: t_sup = -t_sub, T skew-symmetric).  dtype 'f64', 'f64_emu' or
    'f32' (None: from A).  The strictly upper triangle of C is untouched.
    """
    lib = load()
    code = _dtype_code(dtype, A, C)
    if A.dim() != 2 or C.dim() != 2 or C.shape[0] != C.shape[1] or C.shape[0] != A.shape[0]:
        raise ValueError("A must be (n, k) and C (n, n)")

    def vec(v, length):
        if v is None:
            return None
        if v.dim() != 1 or v.numel() < length or (v.numel() > 1 and v.stride(0) != 1):
            raise ValueError("band vectors must be contiguous 1-D tensors of the right length")
        return v.data_ptr()
    n, k = A.shape
    info = PlanInfo()
    opt = options(slices, 0, 0, wait_limit, events)
    check(lib.famlies_gemmt_tridiag(int(n), int(k), float(alpha), A.data_ptr(), A.stride(0), A.stride(1),
                                    vec(t_sub, k - 1), vec(t_diag, k), vec(t_sup, k - 1), float(beta),
                                    C.data_ptr(), C.stride(0), C.stride(1), code, _stream_handle(stream),
                                    opt, info))
    return (C, info.as_dict()) if return_info else C


def mttkrp(alpha, X, mode, factors, beta, M, dtype=None, stream=None, *, slices=0, wait_limit=0,
           events=None, return_info=False):
    """M := beta * M + alpha * X_(mode) (Khatri-Rao product of the other factors).

    X: N-way CUDA tensor (any non-negative strides); factors: N entries, the
    (I_m, R) CUDA matrices for m != mode (factors[mode] is ignored, may be
    None); M: (I_mode, R).  dtype 'f64', 'f64_emu' or 'f32' (None: from X).
    """
    import ctypes
    from ._lib import MatrixDesc
    lib = load()
    code = _dtype_code(dtype, X, M)
    if M.dim() != 2 or len(factors) != X.dim():
        raise ValueError("M must be (I_mode, R) and factors one per mode of X")
    mats = []
    for m, u in enumerate(factors):
        if m == mode or u is None:
            mats.append(MatrixDesc(None, 0, 0, 0, 0))
        else:
            mats.append(MatrixDesc(u.data_ptr(), u.shape[0], u.shape[1], u.stride(0), u.stride(1)))
    arr = (MatrixDesc * len(mats))(*mats)
    md = MatrixDesc(M.data_ptr(), M.shape[0], M.shape[1], M.stride(0), M.stride(1))
    dx = desc_torch(X, list(range(1, X.dim() + 1)))
    info = PlanInfo()
    opt = options(slices, 0, 0, wait_limit, events)
    check(lib.famlies_mttkrp(float(alpha), dx.ref, int(mode), arr, float(beta), ctypes.byref(md), code,
                             _stream_handle(stream), opt, info))
    return (M, info.as_dict()) if return_info else M


def contract_noalloc(alpha, A, la, B, lb, beta, C, lc, dtype=None, stream=None):
    """C := alpha * contract(A, B) + beta * C without any device allocation.

    For callers that may not allocate device memory: fp64 or fp32 tensors,
    computed by the CUDA-core kernels with their offset tables in the
    library's fixed 1 MiB scratch array (calls needing more raise
    FamliesError -11).  Calls sharing a device must not overlap on the GPU.
    """
    import ctypes
    lib = load()
    f = lib.famlies_contract_noalloc
    T = ctypes.POINTER(_TensorDesc)
    f.argtypes = [ctypes.c_double, T, T, ctypes.c_double, T, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    code = _dtype_code(dtype, A, C)
    da, db, dc = desc_torch(A, la), desc_torch(B, lb), desc_torch(C, lc)
    check(f(float(alpha), da.ref, db.ref, float(beta), dc.ref, code, _stream_handle(stream)))
    return C


from ._lib import TensorDesc as _TensorDesc  # noqa: E402


def device_status(stream=None) -> int:
    """Synchronises and returns/clears the device status word (0 or -9 timeout)."""
    return int(load().famlies_device_status(_stream_handle(stream)))


def __getattr__(name):
    if name in ("Contract", "contract_autograd"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
