"""GPU parity of the host-buffer entry with pinned inputs large enough that
the library copies the larger input in chunks along its outermost mode and
overlaps each chunk's contraction with the next chunk's copy: a contracted
outermost label (chunks accumulate into C) and a free one (chunks write
disjoint parts of C), against the oracle's compensated sampled sums."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

pytestmark = pytest.mark.gpu


def _pinned(op):
    t = torch.from_numpy(op.buf).pin_memory()
    return W.Operand(t.numpy(), op.extents, op.strides, op.labels), t


def _check(p, dtype, n_samples=256, seed=0):
    A, ta = _pinned(p.A)
    B, tb = _pinned(p.B)
    C, tc = _pinned(p.C)
    C0 = np.array(p.C.view(), copy=True)
    fm.contract_host(p.alpha, A.view(), A.labels, B.view(), B.labels, p.beta, C.view(), C.labels, dtype=dtype)
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, e, size=n_samples) for e in p.C.extents], axis=1)
    want = oracle.entries(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, C0, p.C.labels, idx,
                          dot2=True)
    got = C.view()[tuple(idx.T)]
    return np.linalg.norm(got - want) / np.linalg.norm(want)


def test_contracted_outermost_label_accumulates():
    """Ladder v = 96, o = 24: V (680 MB) is chunked along d, its outermost
    (contracted) mode; beta = 1 with C read once."""
    p = W.ladder(v=96, o=24)
    assert _check(p, "f64_emu") <= 1e-13


def test_free_outermost_label_writes_disjoint_rows():
    """C[i,j] = sum_k A[i,k] B[k,j] with A row-major 8192 x 8192 (537 MB): the
    outermost mode of A is the free i, so each chunk writes its own rows."""
    rng = np.random.default_rng(1300)
    I, K, J = 8192, 8192, 48
    vals = rng.uniform(-1.0, 1.0, size=(I, K))
    A = W.Operand(vals.reshape(-1).copy(), (I, K), (K, 1), [1, 2])
    B = W.uniform_operand(rng, (K, J), [2, 3])
    C = W.uniform_operand(rng, (I, J), [1, 3])
    p = W.Problem("rowmajor", 0.5, A, B, -1.0, C)
    assert _check(p, "f64_emu") <= 1e-13
    assert _check(p, "f64") <= 1e-13
