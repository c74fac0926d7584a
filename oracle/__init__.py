"""FP64 CPU oracle for C := alpha * contract(A, B) + beta * C.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  It shares no code with the
CUDA path (``paper_2604_07311_b300``) and never imports it.

The arithmetic lives in ``oracle.c`` (plain nested loops, fp64, one fma per
term; see its header for the definition it follows: Einstein summation over
labels with general strides, Sec. 1 "Challenges" and Sec. 2.3 of the paper,
strided layouts from Girder 2).  This module only builds that file with gcc
and marshals numpy views into it.

Parity status per function (what pins it, see tests/test_oracle.py):
  contract  -- pinned: exact integer brute force (Python ints), numpy.einsum
               as a second formulation, closed forms (identity, all-ones,
               rank-1, Kronecker), invariants, special cases.
  entries   -- pinned: agrees with contract; Dot2 mode checked against exact
               rational arithmetic (fractions.Fraction).
  gemmt_tridiag -- pinned: exact integer brute force over the dense T
               (Python ints), closed forms (A = identity gives T's lower
               triangle, A = a permutation gives the permuted T, k = 1 gives
               a scaled outer product), the exact zero diagonal of A T A^T
               for skew-symmetric T, the untouched upper triangle, and the
               alpha = 0 / beta = 0 conventions.
  mttkrp    -- pinned: exact integer brute force over every index tuple
               (Python ints), the rank-one closed form (X an outer product
               of vectors gives products of dot products), the two-way case
               (X U or X^T U), R = 1 with all-ones factors (a mode sum).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ERRORS = {0: "ok", -1: "invalid argument", -2: "bad label set", -3: "extent mismatch"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
             "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        dp = ctypes.c_void_p
        tens = [ctypes.c_int, i64p, i64p, i32p, dp]
        lib.oracle_contract.argtypes = [ctypes.c_double, *tens, *tens, ctypes.c_double, *tens, ctypes.c_int]
        lib.oracle_contract.restype = ctypes.c_int
        lib.oracle_entries.argtypes = [ctypes.c_double, *tens, *tens, ctypes.c_double, *tens,
                                       ctypes.c_int64, i64p, ctypes.c_int, dp]
        lib.oracle_entries.restype = ctypes.c_int
        _lib = lib
    return _lib


def _i64(xs):
    arr = (ctypes.c_int64 * max(1, len(xs)))(*[int(x) for x in xs])
    return arr


def _i32(xs):
    return (ctypes.c_int32 * max(1, len(xs)))(*[int(x) for x in xs])


def _view_args(x: np.ndarray, labels):
    if x.dtype != np.float64:
        raise TypeError("oracle operands are float64 arrays")
    if len(labels) != x.ndim:
        raise ValueError("one label per mode")
    strides = []
    for s in x.strides:
        if s < 0 or s % 8:
            raise ValueError("non-negative element strides only")
        strides.append(s // 8)
    keep = (_i64(x.shape), _i64(strides), _i32(labels))
    return keep, [x.ndim, keep[0], keep[1], keep[2], ctypes.c_void_p(x.__array_interface__["data"][0])]


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def contract(alpha, A, la, B, lb, beta, C, lc, threads: int | None = None) -> np.ndarray:
    """C := alpha * sum_K A*B + beta * C, in place on the float64 view C.

    A, B, C are numpy float64 arrays (views with any non-negative strides);
    la, lb, lc are sequences of integer labels, one per mode.
    """
    lib = _load()
    ka, aa = _view_args(A, la)
    kb, ab = _view_args(B, lb)
    kc, ac = _view_args(C, lc)
    rc = lib.oracle_contract(float(alpha), *aa, *ab, float(beta), *ac,
                             int(threads or default_threads()))
    if rc:
        raise OracleError(rc)
    return C


def entries(alpha, A, la, B, lb, beta, C, lc, index, dot2: bool = False) -> np.ndarray:
    """Selected entries of alpha*contract(A,B) + beta*C (C itself untouched).

    index: int array of shape (n, C.ndim), multi-indices into C.
    dot2:  use the compensated dot product (Ogita, Rump, Oishi 2005, Alg. 5.3).
    """
    lib = _load()
    ka, aa = _view_args(A, la)
    kb, ab = _view_args(B, lb)
    kc, ac = _view_args(C, lc)
    idx = np.asarray(index, dtype=np.int64)
    idx = np.ascontiguousarray(idx.reshape(idx.shape[0] if idx.ndim == 2 else -1, C.ndim))
    out = np.empty(idx.shape[0], dtype=np.float64)
    rc = lib.oracle_entries(float(alpha), *aa, *ab, float(beta), *ac, idx.shape[0],
                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            1 if dot2 else 0, out.ctypes.data)
    if rc:
        raise OracleError(rc)
    return out


def gemmt_tridiag(alpha, A, sub, diag, sup, beta, C) -> np.ndarray:
    """Lower triangle of C := beta * C + alpha * A T A^T, in place on C (n x n).

    The sandwiched product of the paper's skew-symmetric factorisations
    (Sec. 3, "Beyond LAPACK functionality"), evaluated in the two steps the
    paper names for it: B = T A^T with T tridiagonal (T[p+1,p] = sub[p],
    T[p,p] = diag[p], T[p,p+1] = sup[p]; diag None: zero diagonal; sup
    None: sup = -sub, T skew-symmetric), then the GEMMT update C := beta C
    + alpha A B of the entries i >= j only.  T is a band: only its three
    diagonals multiply.  alpha == 0: A is not read; beta == 0: C is not read
    (BLAS conventions).  A is n x k; all float64.
    """
    A = np.asarray(A, dtype=np.float64)
    n, k = A.shape
    low = np.tril(np.ones((n, n), dtype=bool))
    if alpha == 0.0 or k == 0 or n == 0:
        C[low] = 0.0 if beta == 0.0 else beta * C[low]
        return C
    sub = np.zeros(0) if sub is None else np.asarray(sub, dtype=np.float64)
    sup = -sub if sup is None else np.asarray(sup, dtype=np.float64)
    B = np.zeros((k, n))
    for p in range(k):  # row p of T A^T: the band of T's row p against A's columns
        if p > 0:
            B[p] += sub[p - 1] * A[:, p - 1]
        if diag is not None:
            B[p] += diag[p] * A[:, p]
        if p + 1 < k:
            B[p] += sup[p] * A[:, p + 1]
    full = A @ B
    C[low] = alpha * full[low] if beta == 0.0 else alpha * full[low] + beta * C[low]
    return C


def khatri_rao(U, mode, N) -> np.ndarray:
    """KR[i_a, i_b, ..., r] = U[a][i_a, r] * U[b][i_b, r] * ... over the modes
    a < b < ... other than `mode` (of N), multiplied left to right: the
    Khatri-Rao product of the factors as an (N-1)+1-way array."""
    KR = None
    for j, m in enumerate(m for m in range(N) if m != mode):
        f = np.asarray(U[m], dtype=np.float64)
        f = f.reshape((1,) * j + f.shape)
        KR = f if KR is None else KR[..., None, :] * f
    return KR


def mttkrp(alpha, X, mode, U, beta, M) -> np.ndarray:
    """M := beta * M + alpha * X_(mode) KR, in place on M (I_mode x R).

    The matricised-tensor-times-Khatri-Rao-product of CP-ALS (Sec. 3,
    Girder 5): KR[(i_m)_{m != mode}, r] = prod over m != mode, in increasing
    m, of U[m][i_m, r], and M[i, r] = sum over the other modes of
    X[..., i, ...] KR[..., r].  The Khatri-Rao product is formed explicitly
    (broadcast products), then contracted with X by numpy.tensordot.
    alpha == 0: X and the factors are not read; beta == 0: M is not read.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.ndim
    R = M.shape[1]
    if alpha == 0.0 or X.size == 0:
        M[...] = 0.0 if beta == 0.0 else beta * M
        return M
    others = [m for m in range(N) if m != mode]
    KR = khatri_rao(U, mode, N)
    prod = np.tensordot(X, KR, axes=(others, list(range(len(others)))))
    M[...] = alpha * prod if beta == 0.0 else alpha * prod + beta * M
    return M
