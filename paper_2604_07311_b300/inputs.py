"""Seeded synthetic inputs shaped like the paper's tensor workloads.

This module holds only random-number generation and tensor shapes/strides:
no contraction arithmetic.  It is the one module that both the oracle-side
tests and the CUDA-side tests/benchmark use, so that both see the same
inputs.  It imports neither the oracle nor the CUDA binding.

Every generator draws in float64 from ``numpy.random.default_rng(seed)``
(PCG64) and returns plain numpy buffers plus descriptors.  Callers cast to
the device dtype themselves.  The workloads stand in for the quantum
chemistry contractions the paper names as a driving application (Sec. 1.4,
"Project Motivation"; Sec. 2.3): no real integrals or amplitudes are used.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20260000


def L(s: str) -> list[int]:
    """Labels from a string of index letters: 'acik' -> [97, 99, 105, 107]."""
    return [ord(ch) for ch in s]


@dataclass
class Operand:
    """One tensor: a flat float64 buffer plus (extents, strides, labels).

    Strides are in elements; element (i0, i1, ...) lives at
    buf[sum(i_d * strides[d])].
    """
    buf: np.ndarray
    extents: tuple
    strides: tuple
    labels: list

    def view(self) -> np.ndarray:
        """numpy view of the buffer with this operand's shape and strides."""
        return np.lib.stride_tricks.as_strided(
            self.buf, shape=self.extents, strides=tuple(8 * s for s in self.strides),
            writeable=True)

    @property
    def span(self) -> int:
        """Number of elements from the first to one past the last reachable."""
        if any(e == 0 for e in self.extents):
            return 0
        return 1 + sum((e - 1) * s for e, s in zip(self.extents, self.strides))


@dataclass
class Problem:
    name: str
    alpha: float
    A: Operand
    B: Operand
    beta: float
    C: Operand
    meta: dict = field(default_factory=dict)

    @property
    def flops(self) -> int:
        """2 * product of all distinct label extents (the algorithmic count)."""
        ext = {}
        for op in (self.A, self.B, self.C):
            for lab, e in zip(op.labels, op.extents):
                ext[lab] = e
        n = 1
        for e in ext.values():
            n *= e
        return 2 * n


def colmajor_strides(extents, lead_pad: int = 0) -> tuple:
    """Column-major strides; lead_pad adds padding to the first mode's stride."""
    st, acc = [], 1
    for d, e in enumerate(extents):
        st.append(acc)
        acc *= (e + lead_pad) if d == 0 else e
    return tuple(st)


def _operand(values: np.ndarray, extents, labels, lead_pad: int = 0, rng=None) -> Operand:
    """Lay `values` (an array of shape `extents`) out column-major in a buffer."""
    strides = colmajor_strides(extents, lead_pad)
    span = 1 + sum((e - 1) * s for e, s in zip(extents, strides)) if all(extents) else 0
    buf = np.zeros(max(span, 1), dtype=np.float64)
    if lead_pad and rng is not None:
        buf[:] = rng.uniform(-1.0, 1.0, size=buf.shape)  # junk in the padding
    op = Operand(buf, tuple(extents), strides, list(labels))
    if span:
        op.view()[...] = values
    return op


def packed_lower(M: np.ndarray) -> np.ndarray:
    """Lower triangle of a square matrix, column by column (LAPACK's lower
    packed storage): M[p, q], p >= q, lands at q * n - q * (q - 1) / 2 + p - q."""
    n = M.shape[0]
    return np.concatenate([M[q:, q] for q in range(n)]) if n else np.zeros(0)


def uniform_operand(rng, extents, labels, lo=-1.0, hi=1.0, lead_pad=0) -> Operand:
    vals = rng.uniform(lo, hi, size=tuple(extents))
    return _operand(vals, extents, labels, lead_pad, rng)


def integer_operand(rng, extents, labels, lo=-4, hi=4, lead_pad=0) -> Operand:
    vals = rng.integers(lo, hi + 1, size=tuple(extents)).astype(np.float64)
    return _operand(vals, extents, labels, lead_pad, rng)


def zeros_operand(extents, labels) -> Operand:
    return _operand(np.zeros(tuple(extents)), extents, labels)


# ---------------------------------------------------------------------------
# Workloads.  Index letters follow the coupled-cluster convention the paper's
# chemistry applications use: a,b,c,d virtual; i,j,k,l,m occupied.
# ---------------------------------------------------------------------------

def four_index(ext: int = 16, seed: int = SEED_BASE + 1, integer: bool = False) -> Problem:
    """C[a,b,i,j] = sum_{c,k} A[a,c,i,k] B[c,k,b,j]; column-major dense.

    ext=16 is the plain fp64 4-index case (16.7M FMA).
    """
    rng = np.random.default_rng(seed)
    gen = integer_operand if integer else uniform_operand
    e = (ext,) * 4
    A = gen(rng, e, L("acik"))
    B = gen(rng, e, L("ckbj"))
    C = zeros_operand(e, L("abij"))
    return Problem("four_index", 1.0, A, B, 0.0, C, {"ext": ext, "seed": seed})


def ladder(v: int = 128, o: int = 32, seed: int = SEED_BASE + 2, with_values: bool = True) -> Problem:
    """Particle-particle ladder C[a,b,i,j] = sum_{c,d} V[a,b,c,d] T[c,d,i,j] + C.

    V is symmetric under (ab)<->(cd) with entries N(0,1)/128: the lower
    triangle (including the diagonal) of the v^2 x v^2 matrix V[(ab),(cd)]
    is drawn and mirrored, so every entry keeps standard deviation 1/128.
    T entries are N(0, 1e-2) read as standard deviation 1e-2; C is U[-1,1]
    and beta = 1.  All column-major dense.
    """
    rng = np.random.default_rng(seed)
    n = v * v
    X = rng.standard_normal((n, n)) / 128.0
    Vm = np.tril(X)
    del X
    Vm += np.tril(Vm, -1).T
    # Vm[p, q] with p = a + v*b (first two modes), q = c + v*d.  Vm is
    # symmetric, so its row-major flattening is also the column-major one.
    Vbuf = Vm.reshape(-1)
    V = Operand(Vbuf, (v, v, v, v), colmajor_strides((v, v, v, v)), L("abcd"))
    T = _operand(rng.standard_normal((v, v, o, o)) * 1e-2, (v, v, o, o), L("cdij"))
    C = _operand(rng.uniform(-1.0, 1.0, size=(v, v, o, o)), (v, v, o, o), L("abij"))
    return Problem("ladder", 1.0, V, T, 1.0, C, {"v": v, "o": o, "seed": seed})


def transpose_free(v: int = 96, o: int = 48, seed: int = SEED_BASE + 3, pad: int = 7,
                   integer: bool = False) -> Problem:
    """C[b,j,a,i] = sum_{c,k} A[a,c,i,k] B[b,k,j,c]; A's mode-1 stride padded.

    A is column-major except that its first mode's stride is v + pad (so
    strides (1, v+pad, (v+pad)*v, (v+pad)*v*o)); B and C are dense.  The
    output modes are permuted relative to both inputs.
    """
    rng = np.random.default_rng(seed)
    gen = integer_operand if integer else uniform_operand
    A = gen(rng, (v, v, o, o), L("acik"), lead_pad=pad)
    B = gen(rng, (v, o, o, v), L("bkjc"))
    C = zeros_operand((v, o, v, o), L("bjai"))
    return Problem("transpose_free", 1.0, A, B, 0.0, C, {"v": v, "o": o, "pad": pad, "seed": seed})


def autograd_problem(i=64, j=64, l=64, k=48, m=48, seed: int = SEED_BASE + 5):
    """A[i,k,m,l], B[k,m,j], T[i,j,l] iid N(0,1) for L = ||contract(A,B) - T||_F^2."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((i, k, m, l))
    B = rng.standard_normal((k, m, j))
    T = rng.standard_normal((i, j, l))
    return {"A": A, "B": B, "T": T, "la": L("ikml"), "lb": L("kmj"), "lc": L("ijl"), "seed": seed}


def block_sparse_extents(nblocks: int = 2000, seed: int = SEED_BASE + 4, choices=None):
    """Per-block extents of the six labels (a,b,c,i,j,k), each from {8,...,96}."""
    rng = np.random.default_rng(seed)
    choices = np.arange(8, 97, 8) if choices is None else np.asarray(choices)
    return rng.choice(choices, size=(nblocks, 6))


def block_sparse(nblocks: int = 2000, seed: int = SEED_BASE + 4, choices=None,
                 integer: bool = False) -> list[Problem]:
    """Independent 4-index blocks C[a,b,i,j] = sum_{c,k} A[a,c,i,k] B[c,k,b,j].

    Each block's six extents are drawn uniformly from {8,16,...,96}.
    """
    ext = block_sparse_extents(nblocks, seed, choices)
    rng = np.random.default_rng(seed + 1000)
    gen = integer_operand if integer else uniform_operand
    out = []
    for bi in range(nblocks):
        a, b, c, i, j, k = (int(x) for x in ext[bi])
        A = gen(rng, (a, c, i, k), L("acik"))
        B = gen(rng, (c, k, b, j), L("ckbj"))
        C = zeros_operand((a, b, i, j), L("abij"))
        out.append(Problem(f"block{bi}", 1.0, A, B, 0.0, C, {"ext": (a, b, c, i, j, k)}))
    return out
