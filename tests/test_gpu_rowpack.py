"""GPU parity of the one-pass fp64 split (an operand whose k is one
unit-stride mode of length 512..16384: row exponents, Inf/NaN flags and
slices from one read, each row held in registers) against the oracle.
Integer-valued rows scaled by a power of two per row are split exactly
whatever the scale, so those cases compare bit for bit; they pin the
row exponent the kernel reduces across its threads."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _rowmajor(vals, labels, pad=0):
    """A 2-D operand laid out row by row (second index unit-stride), rows
    `pad` elements apart beyond their length."""
    m, k = vals.shape
    ld = k + pad
    buf = np.zeros(m * ld)
    buf.reshape(m, ld)[:, :k] = vals
    return W.Operand(buf, (m, k), (ld, 1), list(labels))


@pytest.mark.parametrize("k", [512, 1000, 4097, 16384])
def test_integer_rows_with_power_of_two_scales_exact(k):
    """A[i, k] row-major (one pass), B column-major (k unit-stride too: one
    pass), each row of A an integer vector times 2^s_i with s_i from -900 to
    900, one row of A holding a NaN and one of B an Inf.  Every product and
    sum is an exact fp64 value, so the result equals the oracle's bit for
    bit."""
    rng = np.random.default_rng(1200 + k)
    m, n = 300, 140
    A = rng.integers(-8, 9, (m, k)).astype(np.float64)
    s = rng.integers(-900, 901, m)
    s[:3] = [0, -1060, 1000]  # a row of subnormals, a row near the top of the range
    A[1] = rng.integers(-3, 4, k).astype(np.float64)
    A = A * np.exp2(s.astype(np.float64))[:, None]
    A[7, k // 3] = np.nan
    B = rng.integers(-8, 9, (k, n)).astype(np.float64) * 0.25
    B[k - 1, 11] = np.inf  # column 11 of B: through B's flags
    C = rng.integers(-8, 9, (m, n)).astype(np.float64)
    Aop = _rowmajor(A, [1, 2])
    Bop = W.Operand(np.asfortranarray(B).reshape(-1, order="F").copy(), (k, n), (1, k), [2, 3])
    Cop = W.Operand(np.asfortranarray(C).reshape(-1, order="F").copy(), (m, n), (1, m), [1, 3])
    p = W.Problem("rowpack_scaled", 2.0, Aop, Bop, -0.5, Cop)
    Cg, info = run_gpu(p, "f64_emu")
    assert info["kernel_name"] == "tc_emu"
    got, want = gpu_dense(Cg), run_oracle(p)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[fin], want[fin])
    if k == 16384:  # both operands one-pass: no exponent pass, no tiled pack
        # tables, two one-pass splits, product (three tiles: K split), split finish, fix-up
        assert info["launches"] + info["cached"] == 6


def test_batched_odd_row_stride():
    """Batched C[i, j, b] = sum_k A[i, k, b] B[k, j, b] with A's rows 2049
    elements apart (odd: 8-byte loads) and k = 2048 unit-stride; B
    column-major.  Uniform values, against the oracle at 1e-13."""
    rng = np.random.default_rng(1210)
    m, k, n, l = 100, 2048, 90, 3
    ld = k + 1
    buf = rng.uniform(-1, 1, m * ld * l + 5)
    A = W.Operand(buf, (m, k, l), (ld, 1, m * ld), [1, 2, 4])
    B = W.uniform_operand(rng, (k, n, l), [2, 3, 4])
    C = W.uniform_operand(rng, (m, n, l), [1, 3, 4])
    p = W.Problem("rowpack_batched", 1.0, A, B, 1.0, C)
    Cg, _ = run_gpu(p, "f64_emu")
    assert rel_frob(gpu_dense(Cg), run_oracle(p)) <= 1e-13


def test_fused_k_modes_and_ragged_rows():
    """A[i, c, d] with (c, d) contiguous (fused to one unit-stride k of
    23 x 45 = 1035, not a multiple of 8: rows of odd length) and B[c, d, j]
    with (c, d) laid out the same way, so both operands split in one pass."""
    rng = np.random.default_rng(1211)
    m, c, d, n = 333, 23, 45, 77
    A = W.Operand(rng.uniform(-1, 1, m * c * d), (m, c, d), (c * d, d, 1), [1, 2, 3])
    B = W.Operand(rng.uniform(-1, 1, c * d * n), (c, d, n), (d, 1, c * d), [2, 3, 4])
    C = W.uniform_operand(rng, (m, n), [1, 4])
    p = W.Problem("rowpack_fused_k", -1.5, A, B, 0.25, C)
    Cg, info = run_gpu(p, "f64_emu")
    # tables, two one-pass splits, product (three tiles: K split in two), split finish, fix-up
    assert info["launches"] + info["cached"] == 6
    assert rel_frob(gpu_dense(Cg), run_oracle(p)) <= 1e-13


@pytest.mark.parametrize("k", [16384, 16385])
def test_at_and_past_the_register_limit(k):
    """k = 16384 is split in one pass (a row fills the 512 threads' registers);
    k = 16385 goes through the exponent pass and the tiled pack.  Both agree
    with the oracle's compensated dot products on sampled entries."""
    rng = np.random.default_rng(1220 + k)
    m, n = 256, 64
    A = _rowmajor(rng.uniform(-1, 1, (m, k)), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.uniform_operand(rng, (m, n), [1, 3])
    p = W.Problem("rowpack_limit", 1.0, A, B, -1.0, C)
    Cg, _ = run_gpu(p, "f64_emu")
    got = gpu_dense(Cg)
    idx = np.stack([rng.integers(0, m, 200), rng.integers(0, n, 200)], axis=1)
    want = oracle.entries(p.alpha, A.view(), A.labels, B.view(), B.labels, p.beta, C.view(), C.labels, idx,
                          dot2=True)
    assert rel_frob(got[idx[:, 0], idx[:, 1]], want) <= 1e-13
    assert fm.device_status() == 0
