"""GPU parity of the tcgen05 paths with gathered operand tiles: bf16 inputs
with fp32 accumulation, and fp32 inputs through the three-term tf32 split."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle, random_label_problem, to_device

pytestmark = pytest.mark.gpu

TOL_BF16 = 2e-2  # relative Frobenius, vs the oracle on the bf16-rounded inputs
TOL_F32 = 1e-5


@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_bf16_transpose_free_reduced(tile_n):
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "bf16", tile_n=tile_n)
    assert info["kernel_name"] == "tc_bf16" and info["swapped"] == 1
    want = run_oracle(p, in_dtype=torch.bfloat16)
    err = rel_frob(gpu_dense(C), want)
    assert err <= TOL_BF16
    assert err <= 1e-5  # fp32 accumulation of exactly-rounded bf16 products


@pytest.mark.parametrize("tile_n", [64, 256])
def test_bf16_integer_exact(tile_n):
    p = W.transpose_free(v=24, o=12, pad=7, integer=True)
    C, _ = run_gpu(p, "bf16", tile_n=tile_n)
    assert np.array_equal(gpu_dense(C), run_oracle(p))


def test_bf16_random_labels_integer_exact():
    rng = np.random.default_rng(300)
    for _ in range(16):
        p = random_label_problem(rng, max_ext=7)
        C, info = run_gpu(p, "bf16")
        want = run_oracle(p)
        assert np.array_equal(gpu_dense(C), want), info


def test_bf16_ragged_gemm_shapes():
    rng = np.random.default_rng(301)
    for m, n, k in [(1, 1, 1), (127, 129, 63), (129, 257, 65), (300, 70, 200), (128, 256, 64)]:
        A = W.uniform_operand(rng, (m, k), [1, 2])
        B = W.uniform_operand(rng, (k, n), [2, 3])
        C = W.uniform_operand(rng, (m, n), [1, 3])
        p = W.Problem("gemm", 0.5, A, B, 2.0, C)
        Cg, _ = run_gpu(p, "bf16")
        want = run_oracle(p, in_dtype=torch.bfloat16, out_dtype=torch.float32)
        assert rel_frob(gpu_dense(Cg), want) <= 1e-5, (m, n, k)


def test_bf16_k_major_operands():
    """Both operands unit-stride along k (vector gathers) and C unit-stride along rows."""
    rng = np.random.default_rng(302)
    m, n, k = 200, 150, 333
    A = W.uniform_operand(rng, (k, m), [2, 1])  # A[k, m]: k fastest
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.zeros_operand((m, n), [1, 3])
    p = W.Problem("kmajor", 1.0, A, B, 0.0, C)
    Cg, info = run_gpu(p, "bf16")
    assert info["a_contig"] == 2 and info["b_contig"] == 2
    want = run_oracle(p, in_dtype=torch.bfloat16)
    assert rel_frob(gpu_dense(Cg), want) <= 1e-5


def test_bf16_full_size_sampled():
    """The v=96, o=48 transpose-free contraction (M=N=K=4608) in the benchmark's
    launch configuration, checked on sampled entries computed one by one."""
    p = W.transpose_free(v=96, o=48, pad=7)
    C, info = run_gpu(p, "bf16")
    assert (info["m"], info["n"], info["k"]) == (4608, 4608, 4608)
    rng = np.random.default_rng(5)
    idx = np.stack([rng.integers(0, e, 512) for e in p.C.extents], axis=1)
    Ar = torch.from_numpy(np.ascontiguousarray(p.A.buf)).to(torch.bfloat16).double().numpy()
    Br = torch.from_numpy(np.ascontiguousarray(p.B.buf)).to(torch.bfloat16).double().numpy()
    Av = np.lib.stride_tricks.as_strided(Ar, p.A.extents, tuple(8 * s for s in p.A.strides))
    Bv = np.lib.stride_tricks.as_strided(Br, p.B.extents, tuple(8 * s for s in p.B.strides))
    want = oracle.entries(1.0, Av, p.A.labels, Bv, p.B.labels, 0.0, np.zeros(p.C.extents),
                          p.C.labels, idx)
    got = gpu_dense(C)[tuple(idx.T)]
    assert rel_frob(got, want) <= 1e-5


def test_tf32x3_reduced_fp32_accuracy():
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "f32", kernel=2)
    assert info["kernel_name"] == "tc_tf32x3"
    want = run_oracle(p, in_dtype=torch.float32)
    assert rel_frob(gpu_dense(C), want) <= TOL_F32


def test_tf32x3_integer_exact_and_ragged():
    p = W.transpose_free(v=24, o=12, pad=7, integer=True)
    C, _ = run_gpu(p, "f32", kernel=2)
    assert np.array_equal(gpu_dense(C), run_oracle(p))
    rng = np.random.default_rng(303)
    for m, n, k in [(1, 1, 1), (129, 65, 37), (256, 130, 100)]:
        A = W.uniform_operand(rng, (m, k), [1, 2])
        B = W.uniform_operand(rng, (k, n), [2, 3])
        Cc = W.uniform_operand(rng, (m, n), [1, 3])
        q = W.Problem("gemm", -1.0, A, B, 0.5, Cc)
        Cg, _ = run_gpu(q, "f32", kernel=2, tile_n=64 if n < 100 else 128)
        want = run_oracle(q, in_dtype=torch.float32, out_dtype=torch.float32)
        assert rel_frob(gpu_dense(Cg), want) <= TOL_F32, (m, n, k)


def test_simt_f32_forced():
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "f32", kernel=1)
    assert info["kernel_name"] == "simt_f32"
    assert rel_frob(gpu_dense(C), run_oracle(p, in_dtype=torch.float32)) <= TOL_F32


def test_bounded_wait_timeout_reports_status_and_context_survives():
    """A wait that runs out (limit of one poll) ends the kernel with a status
    code instead of hanging; the next normal call on the same context works."""
    p = W.transpose_free(v=24, o=12, pad=7)
    assert fm.device_status() == 0
    run_gpu(p, "bf16", wait_limit=1)
    assert fm.device_status() == fm._lib.ERR_DEVICE_TIMEOUT
    assert fm.device_status() == 0  # read clears it
    C, _ = run_gpu(p, "bf16")
    want = run_oracle(p, in_dtype=torch.bfloat16)
    assert rel_frob(gpu_dense(C), want) <= 1e-5
    assert fm.device_status() == 0
