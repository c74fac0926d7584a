"""GPU parity of the tcgen05 bf16 and fp32 (three-term tf32 split) paths, both
the packed TMA-fed kernel and the kernel that gathers operand tiles straight
from the strided tensors."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W
from paper_2604_07311_b300._lib import KERNEL_GATHER, KERNEL_PACKED, KERNEL_SIMT

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle, random_label_problem

pytestmark = pytest.mark.gpu

TOL_BF16 = 2e-2  # relative Frobenius, vs the oracle on the bf16-rounded inputs
TOL_F32 = 1e-5
PATHS = [KERNEL_PACKED, KERNEL_GATHER]
NAMES = {("bf16", KERNEL_PACKED): "tc_bf16", ("bf16", KERNEL_GATHER): "tc_bf16_gather",
         ("f32", KERNEL_PACKED): "tc_tf32x3", ("f32", KERNEL_GATHER): "tc_tf32x3_gather"}


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_bf16_transpose_free_reduced(path, tile_n):
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "bf16", tile_n=tile_n, kernel=path)
    assert info["kernel_name"] == NAMES["bf16", path] and info["swapped"] == 1
    want = run_oracle(p, in_dtype=torch.bfloat16)
    err = rel_frob(gpu_dense(C), want)
    assert err <= TOL_BF16
    assert err <= 1e-5  # fp32 accumulation of exactly-rounded bf16 products


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("tile_n", [64, 256])
def test_bf16_integer_exact(path, tile_n):
    p = W.transpose_free(v=24, o=12, pad=7, integer=True)
    C, _ = run_gpu(p, "bf16", tile_n=tile_n, kernel=path)
    assert np.array_equal(gpu_dense(C), run_oracle(p))


@pytest.mark.parametrize("path", PATHS)
def test_bf16_random_labels_integer_exact(path):
    rng = np.random.default_rng(300)
    for _ in range(16):
        p = random_label_problem(rng, max_ext=7)
        C, info = run_gpu(p, "bf16", kernel=path)
        assert np.array_equal(gpu_dense(C), run_oracle(p)), info


@pytest.mark.parametrize("path", PATHS)
def test_bf16_ragged_gemm_shapes(path):
    rng = np.random.default_rng(301)
    for m, n, k in [(1, 1, 1), (127, 129, 63), (129, 257, 65), (300, 70, 200), (128, 256, 64)]:
        A = W.uniform_operand(rng, (m, k), [1, 2])
        B = W.uniform_operand(rng, (k, n), [2, 3])
        C = W.uniform_operand(rng, (m, n), [1, 3])
        p = W.Problem("gemm", 0.5, A, B, 2.0, C)
        Cg, _ = run_gpu(p, "bf16", kernel=path)
        want = run_oracle(p, in_dtype=torch.bfloat16, out_dtype=torch.float32)
        assert rel_frob(gpu_dense(Cg), want) <= 1e-5, (m, n, k)


@pytest.mark.parametrize("path", PATHS)
def test_bf16_k_major_operands(path):
    """Both operands unit-stride along k and C unit-stride along rows."""
    rng = np.random.default_rng(302)
    m, n, k = 200, 150, 333
    A = W.uniform_operand(rng, (k, m), [2, 1])  # A[k, m]: k fastest
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.zeros_operand((m, n), [1, 3])
    p = W.Problem("kmajor", 1.0, A, B, 0.0, C)
    Cg, info = run_gpu(p, "bf16", kernel=path)
    assert info["a_contig"] == 2 and info["b_contig"] == 2
    assert rel_frob(gpu_dense(Cg), run_oracle(p, in_dtype=torch.bfloat16)) <= 1e-5


@pytest.mark.parametrize("kext", [64, 200, 37])
def test_bf16_k_unit_stride_batched_read_in_place(kext):
    """Operands whose contracted index is unit-stride (and, for k = 64 and
    200, whose rows start on 16-byte boundaries) are read by TMA straight from
    the caller's tensors; k = 37 takes the pack.  C[i,j,b] = sum_k A[k,i,b] B[k,j,b]."""
    rng = np.random.default_rng(305)
    A = W.uniform_operand(rng, (kext, 150, 3), [2, 1, 3])
    B = W.uniform_operand(rng, (kext, 90, 3), [2, 4, 3])
    C = W.uniform_operand(rng, (150, 90, 3), [1, 4, 3])
    p = W.Problem("kmajor_batched", 1.5, A, B, -0.5, C)
    Cg, info = run_gpu(p, "bf16")
    assert info["a_contig"] == 2 and info["b_contig"] == 2 and info["batch"] == 3
    want = run_oracle(p, in_dtype=torch.bfloat16, out_dtype=torch.float32)
    assert rel_frob(gpu_dense(Cg), want) <= 1e-5


def test_bf16_batch_labels():
    """A label in A, B and C (batch): C[i,j,b] = sum_k A[i,k,b] B[k,j,b]."""
    rng = np.random.default_rng(304)
    A = W.uniform_operand(rng, (70, 50, 5), [1, 2, 3])
    B = W.uniform_operand(rng, (50, 90, 5), [2, 4, 3])
    C = W.zeros_operand((70, 90, 5), [1, 4, 3])
    p = W.Problem("batched", 1.0, A, B, 0.0, C)
    for path in PATHS:
        Cg, info = run_gpu(p, "bf16", kernel=path)
        assert info["batch"] == 5
        assert rel_frob(gpu_dense(Cg), run_oracle(p, in_dtype=torch.bfloat16)) <= 1e-5


def _sampled_reference(p, dtype, idx):
    Ar = torch.from_numpy(np.ascontiguousarray(p.A.buf)).to(dtype).double().numpy()
    Br = torch.from_numpy(np.ascontiguousarray(p.B.buf)).to(dtype).double().numpy()
    Av = np.lib.stride_tricks.as_strided(Ar, p.A.extents, tuple(8 * s for s in p.A.strides))
    Bv = np.lib.stride_tricks.as_strided(Br, p.B.extents, tuple(8 * s for s in p.B.strides))
    return oracle.entries(1.0, Av, p.A.labels, Bv, p.B.labels, 0.0, np.zeros(p.C.extents),
                          p.C.labels, idx)


@pytest.mark.parametrize("dtype,tol", [("bf16", 1e-5), ("f32", TOL_F32)])
def test_full_size_transpose_free_sampled(dtype, tol):
    """The v=96, o=48 transpose-free contraction (M=N=K=4608) in the benchmark's
    launch configuration, checked on sampled entries computed one by one."""
    p = W.transpose_free(v=96, o=48, pad=7)
    C, info = run_gpu(p, dtype)
    assert (info["m"], info["n"], info["k"]) == (4608, 4608, 4608)
    rng = np.random.default_rng(5)
    idx = np.stack([rng.integers(0, e, 512) for e in p.C.extents], axis=1)
    want = _sampled_reference(p, torch.bfloat16 if dtype == "bf16" else torch.float32, idx)
    got = gpu_dense(C)[tuple(idx.T)]
    assert rel_frob(got, want) <= tol


@pytest.mark.parametrize("path", PATHS)
def test_tf32x3_reduced_fp32_accuracy(path):
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "f32", kernel=path)
    assert info["kernel_name"] == NAMES["f32", path]
    assert rel_frob(gpu_dense(C), run_oracle(p, in_dtype=torch.float32)) <= TOL_F32


@pytest.mark.parametrize("path", PATHS)
def test_tf32x3_integer_exact_and_ragged(path):
    p = W.transpose_free(v=24, o=12, pad=7, integer=True)
    C, _ = run_gpu(p, "f32", kernel=path)
    assert np.array_equal(gpu_dense(C), run_oracle(p))
    rng = np.random.default_rng(303)
    for m, n, k in [(1, 1, 1), (129, 65, 37), (256, 130, 100)]:
        A = W.uniform_operand(rng, (m, k), [1, 2])
        B = W.uniform_operand(rng, (k, n), [2, 3])
        Cc = W.uniform_operand(rng, (m, n), [1, 3])
        q = W.Problem("gemm", -1.0, A, B, 0.5, Cc)
        Cg, _ = run_gpu(q, "f32", kernel=path, tile_n=64 if n < 100 else 128)
        want = run_oracle(q, in_dtype=torch.float32, out_dtype=torch.float32)
        assert rel_frob(gpu_dense(Cg), want) <= TOL_F32, (m, n, k)


def test_simt_f32_forced():
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "f32", kernel=KERNEL_SIMT)
    assert info["kernel_name"] == "simt_f32"
    assert rel_frob(gpu_dense(C), run_oracle(p, in_dtype=torch.float32)) <= TOL_F32


@pytest.mark.parametrize("path", PATHS)
def test_bounded_wait_timeout_reports_status_and_context_survives(path):
    """A wait that runs out (the test hook makes the MMA issuer wait on a
    barrier phase nothing completes, bounded by 1000 polls) ends the kernels
    with a status code instead of hanging; the next normal call on the same
    context works."""
    p = W.transpose_free(v=24, o=12, pad=7)
    assert fm.device_status() == 0
    run_gpu(p, "bf16", wait_limit=1000, kernel=path, stall_test=1)
    assert fm.device_status() == fm._lib.ERR_DEVICE_TIMEOUT
    assert fm.device_status() == 0  # read clears it
    C, _ = run_gpu(p, "bf16", kernel=path)
    assert rel_frob(gpu_dense(C), run_oracle(p, in_dtype=torch.bfloat16)) <= 1e-5
    assert fm.device_status() == 0


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_split_k_few_tiles(dtype):
    """Two output tiles and a long K: the packed kernel splits K across CTAs
    and sums the partial tiles (with alpha, beta) afterwards; the launch
    count reports the extra reduction."""
    rng = np.random.default_rng(640)
    m, n, k = 200, 64, 8192
    A = W.uniform_operand(rng, (m, k), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.uniform_operand(rng, (m, n), [1, 3])
    p = W.Problem("split_k", 0.75, A, B, -1.5, C)
    Cg, info = run_gpu(p, dtype, kernel=KERNEL_PACKED)
    assert info["launches"] + info["cached"] == 4  # tables + pack + product + split reduction
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    want = run_oracle(p, in_dtype=tdt, out_dtype=torch.float32)
    assert rel_frob(gpu_dense(Cg), want) <= (1e-5 if dtype == "bf16" else TOL_F32)


def test_split_k_integer_exact():
    """Integer-valued bf16 inputs: every partial sum is exact, so splitting K
    changes nothing."""
    rng = np.random.default_rng(641)
    m, n, k = 130, 70, 4096
    A = W.integer_operand(rng, (m, k), [1, 2])
    B = W.integer_operand(rng, (k, n), [2, 3])
    C = W.zeros_operand((m, n), [1, 3])
    p = W.Problem("split_k_int", 1.0, A, B, 0.0, C)
    Cg, info = run_gpu(p, "bf16", kernel=KERNEL_PACKED)
    assert info["launches"] + info["cached"] == 4
    assert np.array_equal(gpu_dense(Cg), run_oracle(p))


def test_split_tail_after_whole_rounds_integer_exact():
    """178 tiles on 148 SMs: one whole round, then the 30-tile tail split
    along K; integer-valued bf16 inputs make every partial sum exact, so
    sampled entries (tail tiles and whole ones) match the oracle exactly."""
    rng = np.random.default_rng(642)
    m, n, k = 89 * 128, 512, 4096
    A = W.integer_operand(rng, (m, k), [1, 2], lo=-2, hi=2)
    B = W.integer_operand(rng, (k, n), [2, 3], lo=-2, hi=2)
    C = W.zeros_operand((m, n), [1, 3])
    p = W.Problem("split_tail", 1.0, A, B, 0.0, C)
    Cg, info = run_gpu(p, "bf16", kernel=KERNEL_PACKED, tile_n=256)
    assert info["launches"] + info["cached"] == 4  # tables + pack + product + split reduction
    got = gpu_dense(Cg)
    rows = np.concatenate([rng.integers(74 * 128, m, 48), rng.integers(0, 74 * 128, 16)])
    idx = np.stack([rows, rng.integers(0, n, rows.size)], axis=1)
    want = oracle.entries(1.0, A.view(), A.labels, B.view(), B.labels, 0.0, C.view(), C.labels, idx)
    assert np.array_equal(got[idx[:, 0], idx[:, 1]], want)
