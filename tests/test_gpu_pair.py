"""GPU parity of the fp64 split's product on CTA pairs (options
ctas_per_mma = 2; cta_group::2: one tensor-core MMA over two SMs, 256 x 256
output tiles, each CTA staging its 128 rows of A and 128 of the tile's 256
columns of B) against the oracle: every tile split along k and finished by
the separate kernel, no tile split, ragged edges, Inf/NaN rows and columns;
calls the pairs do not support run on one SM per MMA."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _colmajor(vals, labels):
    return W.Operand(np.asfortranarray(vals).reshape(-1, order="F").copy(), vals.shape,
                     tuple(int(np.prod(vals.shape[:i])) for i in range(vals.ndim)), list(labels))


@pytest.mark.parametrize("m,n,k,integer", [
    (19 * 256, 1024, 1024, True),    # 76 pair tiles: every tile split in four
    (37 * 256, 512, 1536, True),     # 74 pair tiles: one whole round, no split
    (19 * 256 + 100, 1000, 777, True),  # ragged rows, columns and k
    (40 * 256, 1024, 4096, False),   # uniform values, against Dot2 on sampled entries
])
def test_pair_product(m, n, k, integer):
    rng = np.random.default_rng(1300 + m + k)
    if integer:
        A = rng.integers(-8, 9, (m, k)).astype(np.float64)
        B = rng.integers(-8, 9, (k, n)).astype(np.float64) * 0.5
        C = rng.integers(-8, 9, (m, n)).astype(np.float64)
    else:
        A, B, C = rng.uniform(-1, 1, (m, k)), rng.uniform(-1, 1, (k, n)), rng.uniform(-1, 1, (m, n))
    p = W.Problem("pair", 1.5, _colmajor(A, [1, 2]), _colmajor(B, [2, 3]), -0.5, _colmajor(C, [1, 3]))
    Cg, info = run_gpu(p, "f64_emu", ctas_per_mma=2)
    assert info["kernel_name"] == "tc_emu"
    got = gpu_dense(Cg)
    if integer:  # every product and sum exact: bit for bit, and the same as one SM per MMA
        assert np.array_equal(got, run_oracle(p))
        C1, info1 = run_gpu(p, "f64_emu")
        assert info1["ctas_per_mma"] == 1 and np.array_equal(gpu_dense(C1), got)
    else:
        idx = np.stack([rng.integers(0, m, 400), rng.integers(0, n, 400)], axis=1)
        want = oracle.entries(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, p.C.view(),
                              p.C.labels, idx, dot2=True)
        assert rel_frob(got[idx[:, 0], idx[:, 1]], want) <= 1e-13
    assert info["ctas_per_mma"] == 2, info
    assert fm.device_status() == 0


def test_pair_nonfinite_rows_and_columns():
    """A NaN in a row of A (second CTA's half of its pair tile) and an Inf in
    a column of B: those rows and columns go to the native fix-up, the rest
    stays exact."""
    rng = np.random.default_rng(1310)
    m, n, k = 19 * 256, 1024, 1024
    A = rng.integers(-8, 9, (m, k)).astype(np.float64)
    A[128 + 37, 5] = np.nan
    B = rng.integers(-8, 9, (k, n)).astype(np.float64)
    B[700, 300] = np.inf
    C = rng.integers(-8, 9, (m, n)).astype(np.float64)
    p = W.Problem("pair_nonfinite", 1.0, _colmajor(A, [1, 2]), _colmajor(B, [2, 3]), 1.0, _colmajor(C, [1, 3]))
    Cg, info = run_gpu(p, "f64_emu", ctas_per_mma=2)
    assert info["ctas_per_mma"] == 2
    got, want = gpu_dense(Cg), run_oracle(p)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[fin], want[fin])


def test_ladder_on_pairs():
    """The CCSD ladder term at v = 80, o = 24 (m = 6400 rows (a, b), n = 576
    columns (i, j), k = 6400: 75 pair tiles), sampled entries against the
    oracle's compensated dot products."""
    p = W.ladder(v=80, o=24)
    Cg, info = run_gpu(p, "f64_emu", ctas_per_mma=2)
    assert info["ctas_per_mma"] == 2
    got = gpu_dense(Cg)
    rng = np.random.default_rng(1320)
    shape = p.C.extents
    idx = np.stack([rng.integers(0, e, 300) for e in shape], axis=1)
    want = oracle.entries(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, p.C.view(),
                          p.C.labels, idx, dot2=True)
    assert rel_frob(got[tuple(idx.T)], want) <= 1e-13


def test_pairs_fall_back_where_unsupported():
    """A batched call (and one with fewer pair tiles than pairs of SMs) asked
    to run on pairs runs on one SM per MMA, with the oracle's result."""
    rng = np.random.default_rng(1330)
    A = W.uniform_operand(rng, (300, 700, 2), [1, 2, 4])
    B = W.uniform_operand(rng, (700, 300, 2), [2, 3, 4])
    C = W.uniform_operand(rng, (300, 300, 2), [1, 3, 4])
    p = W.Problem("pair_batched", 1.0, A, B, 1.0, C)
    Cg, info = run_gpu(p, "f64_emu", ctas_per_mma=2)
    assert info["ctas_per_mma"] == 1
    assert rel_frob(gpu_dense(Cg), run_oracle(p)) <= 1e-13
