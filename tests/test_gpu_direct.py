"""GPU parity of the direct bf16 kernel: operand tiles staged straight from the
caller's strided tensors (multi-mode TMA boxes where the strides allow it; a
re-padded copy, or gather warps, otherwise), MN-major or K-major in shared
memory, no pack and no offset tables.  Checked against the FP64 oracle on the
bf16-rounded inputs: bit-exact on integer-valued inputs (every partial sum
is an integer below 2^24, exact in fp32), else within 1e-5 relative
Frobenius (fp32 accumulation of exact bf16 products; the dtype's own bound
is 2e-2)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W
from paper_2604_07311_b300._lib import KERNEL_DIRECT, KERNEL_DIRECT_GATHER, KERNEL_PACKED

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle, random_label_problem, to_device

pytestmark = pytest.mark.gpu

TOL = 1e-5
DIRECT = [KERNEL_DIRECT, KERNEL_DIRECT_GATHER]


@pytest.mark.parametrize("kernel", DIRECT)
@pytest.mark.parametrize("tile_n", [64, 128, 192, 256])
def test_transpose_free_reduced_integer_exact(kernel, tile_n):
    """C[b,j,a,i] = sum_{c,k} A[a,c,i,k] B[b,k,j,c], A's first-mode stride padded
    to 31 (62 bytes: no tensor map can address A, whose rows start on every
    even byte offset mod 16), B read by TMA boxes over (b, k, c, j).  Kernel 4
    first copies A with its strides rounded up to 16 bytes (two launches);
    kernel 5 gathers both operands' tiles in the product (one launch)."""
    p = W.transpose_free(v=24, o=12, pad=7, integer=True)
    C, info = run_gpu(p, "bf16", kernel=kernel, tile_n=tile_n)
    assert info["kernel_name"] == "tc_bf16_direct"
    assert info["launches"] == (2 if kernel == KERNEL_DIRECT else 1)
    assert np.array_equal(gpu_dense(C), run_oracle(p))


@pytest.mark.parametrize("kernel", DIRECT)
def test_transpose_free_unpadded_integer_exact(kernel):
    """The same contraction with dense A: both operands read by TMA boxes (one
    launch) or gathered."""
    p = W.transpose_free(v=24, o=12, pad=0, integer=True)
    C, info = run_gpu(p, "bf16", kernel=kernel)
    assert info["kernel_name"] == "tc_bf16_direct" and info["launches"] == 1
    assert np.array_equal(gpu_dense(C), run_oracle(p))


def test_transpose_free_reduced_default_path():
    p = W.transpose_free(v=24, o=12, pad=7)
    C, info = run_gpu(p, "bf16")
    assert info["kernel_name"] == "tc_bf16_direct" and info["launches"] == 2 and info["swapped"] == 1
    want = run_oracle(p, in_dtype=torch.bfloat16)
    assert rel_frob(gpu_dense(C), want) <= TOL


@pytest.mark.parametrize("kernel", DIRECT)
def test_random_labels_integer_exact(kernel):
    """Random label sets, mode orders and padded strides; calls that fit the
    direct kernel must take it and match exactly."""
    rng = np.random.default_rng(700)
    direct = 0
    for _ in range(80):
        p = random_label_problem(rng, max_ext=9, pad_max=3)
        if p.alpha == 0:  # C := beta * C, no product
            continue
        info = fm.plan(p.A.extents, p.A.strides, p.A.labels, p.B.extents, p.B.strides, p.B.labels,
                       p.C.extents, p.C.strides, p.C.labels, dtype="bf16")
        if info["kernel_name"] != "tc_bf16_direct":
            continue
        direct += 1
        C, info = run_gpu(p, "bf16", kernel=kernel)
        assert info["kernel_name"] == "tc_bf16_direct"
        assert np.array_equal(gpu_dense(C), run_oracle(p)), info
    assert direct >= 15  # 20 of these 80 fit the direct kernel


@pytest.mark.parametrize("kernel", DIRECT)
@pytest.mark.parametrize("layout", ["mn_mn", "k_k", "mn_k", "k_mn"])
def test_gemm_layouts_ragged(kernel, layout):
    """GEMM shapes with ragged edges, each operand unit-stride along its free
    index (MN-major tiles) or along k (K-major tiles)."""
    rng = np.random.default_rng(701)
    for m, n, k in [(1, 1, 1), (127, 129, 63), (129, 257, 65), (300, 70, 200), (128, 256, 64), (40, 520, 777)]:
        la, lb = layout.split("_")
        A = W.uniform_operand(rng, (m, k) if la == "mn" else (k, m), [1, 2] if la == "mn" else [2, 1])
        B = W.uniform_operand(rng, (n, k) if lb == "mn" else (k, n), [3, 2] if lb == "mn" else [2, 3])
        C = W.uniform_operand(rng, (m, n), [1, 3])
        p = W.Problem("gemm", 0.5, A, B, 2.0, C)
        Cg, info = run_gpu(p, "bf16", kernel=kernel)
        assert info["kernel_name"] == "tc_bf16_direct"
        want = run_oracle(p, in_dtype=torch.bfloat16, out_dtype=torch.float32)
        assert rel_frob(gpu_dense(Cg), want) <= TOL, (layout, m, n, k)


@pytest.mark.parametrize("kernel", DIRECT)
def test_batch_and_two_mode_classes(kernel):
    """A batch label and two-mode row, column and contracted classes that do
    not fuse: C[i,l,j,b] = sum_{k,c} A[i,k,l,c,b] B[c,j,k,b]."""
    rng = np.random.default_rng(702)
    ext = {"i": 20, "l": 9, "j": 33, "k": 11, "c": 7, "b": 3}

    def op(labels, pad):
        shape = tuple(ext[x] for x in labels)
        strides = W.colmajor_strides(shape, lead_pad=pad)
        span = 1 + sum((e - 1) * s for e, s in zip(shape, strides))
        return W.Operand(rng.integers(-3, 4, span).astype(np.float64), shape, strides, W.L(labels))
    A, B, C = op("iklcb", 0), op("cjkb", 8), op("iljb", 0)
    p = W.Problem("batched_two_mode", 1.0, A, B, -1.0, C)
    Cg, info = run_gpu(p, "bf16", kernel=kernel)
    assert info["kernel_name"] == "tc_bf16_direct" and info["batch"] == 3
    assert np.array_equal(gpu_dense(Cg), run_oracle(p))


@pytest.mark.parametrize("kernel", DIRECT)
def test_misaligned_bases(kernel):
    """Operands whose first element sits at an odd element offset (2 bytes past
    a 16-byte boundary) cannot be described by a tensor map: re-padded copies
    (kernel 4) or the gather warps (kernel 5) stage them, integer-exact."""
    rng = np.random.default_rng(703)
    m, n, k = 150, 90, 200
    a = torch.from_numpy(rng.integers(-4, 5, m * k + 1).astype(np.float32)).to("cuda", torch.bfloat16)
    b = torch.from_numpy(rng.integers(-4, 5, n * k + 3).astype(np.float32)).to("cuda", torch.bfloat16)
    A = torch.as_strided(a, (m, k), (1, m), 1)
    B = torch.as_strided(b, (k, n), (1, k), 3)
    C = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    _, info = fm.contract(1.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3], dtype="bf16", kernel=kernel,
                          return_info=True)
    assert info["kernel_name"] == "tc_bf16_direct"
    assert info["launches"] == (3 if kernel == KERNEL_DIRECT else 1)
    want = A.double().cpu().numpy() @ B.double().cpu().numpy()
    assert np.array_equal(C.double().cpu().numpy(), want)


def test_beta_zero_overwrites_nan_and_alpha_scales():
    rng = np.random.default_rng(704)
    A = torch.from_numpy(rng.integers(-4, 5, (70, 130)).astype(np.float32)).to("cuda", torch.bfloat16)
    B = torch.from_numpy(rng.integers(-4, 5, (130, 60)).astype(np.float32)).to("cuda", torch.bfloat16)
    C = torch.full((70, 60), float("nan"), dtype=torch.float32, device="cuda")
    _, info = fm.contract(2.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3], dtype="bf16", return_info=True)
    assert info["kernel_name"] == "tc_bf16_direct"
    assert torch.equal(C.double(), 2.0 * (A.double() @ B.double()))


def test_packed_and_direct_agree_bitwise_on_integers():
    p = W.transpose_free(v=24, o=12, pad=7, integer=True)
    Cd, _ = run_gpu(p, "bf16", kernel=KERNEL_DIRECT)
    Cp, _ = run_gpu(p, "bf16", kernel=KERNEL_PACKED)
    assert torch.equal(Cd, Cp)


def test_full_size_transpose_free_direct_sampled():
    """v=96, o=48 (M = N = K = 4608) through the default bf16 path: the direct
    kernel after one re-pad copy of the padded operand, its last round split
    along k; 512 sampled entries computed one by one by the oracle (tail
    tiles and whole ones alike)."""
    p = W.transpose_free(v=96, o=48, pad=7)
    C, info = run_gpu(p, "bf16")
    # re-pad of A, product (648 tiles of 128 x 256: 4 whole rounds, then the
    # 56-tile tail split in two along k), split reduction
    assert info["kernel_name"] == "tc_bf16_direct" and info["launches"] == 3
    assert (info["m"], info["n"], info["k"]) == (4608, 4608, 4608)
    rng = np.random.default_rng(705)
    idx = np.stack([rng.integers(0, e, 512) for e in p.C.extents], axis=1)
    Ar = torch.from_numpy(p.A.buf).to(torch.bfloat16).double().numpy()
    Br = torch.from_numpy(p.B.buf).to(torch.bfloat16).double().numpy()
    Av = np.lib.stride_tricks.as_strided(Ar, p.A.extents, tuple(8 * s for s in p.A.strides))
    Bv = np.lib.stride_tricks.as_strided(Br, p.B.extents, tuple(8 * s for s in p.B.strides))
    want = oracle.entries(1.0, Av, p.A.labels, Bv, p.B.labels, 0.0, np.zeros(p.C.extents), p.C.labels, idx)
    got = gpu_dense(C)[tuple(idx.T)]
    assert rel_frob(got, want) <= TOL


def test_full_size_transpose_free_integer_exact_sampled():
    """The same size with integer-valued inputs in [-4, 4]: every sum is an
    integer of magnitude at most 16 * 4608 < 2^24, so sampled entries match
    exactly."""
    p = W.transpose_free(v=96, o=48, pad=7, integer=True)
    C, info = run_gpu(p, "bf16")
    assert info["kernel_name"] == "tc_bf16_direct"
    rng = np.random.default_rng(706)
    idx = np.stack([rng.integers(0, e, 2048) for e in p.C.extents], axis=1)
    want = oracle.entries(1.0, p.A.view(), p.A.labels, p.B.view(), p.B.labels, 0.0, np.zeros(p.C.extents),
                          p.C.labels, idx)
    assert np.array_equal(gpu_dense(C)[tuple(idx.T)], want)


def test_bounded_wait_timeout_direct():
    p = W.transpose_free(v=24, o=12, pad=7)
    assert fm.device_status() == 0
    run_gpu(p, "bf16", wait_limit=1000, stall_test=1)
    assert fm.device_status() == fm._lib.ERR_DEVICE_TIMEOUT
    assert fm.device_status() == 0
    C, info = run_gpu(p, "bf16")
    assert info["kernel_name"] == "tc_bf16_direct"
    assert rel_frob(gpu_dense(C), run_oracle(p, in_dtype=torch.bfloat16)) <= TOL
    assert fm.device_status() == 0


@pytest.mark.parametrize("kernel", DIRECT)
def test_split_k_few_tiles(kernel):
    """Two output tiles and k = 8192: the tiles' k ranges are split across the
    SMs, every split writes an fp32 partial tile and a reduction sums them in
    split order (deterministic) with alpha and beta."""
    rng = np.random.default_rng(707)
    m, n, k = 200, 64, 8192
    A = W.uniform_operand(rng, (m, k), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.uniform_operand(rng, (m, n), [1, 3])
    p = W.Problem("split_k", 0.75, A, B, -1.5, C)
    Cg, info = run_gpu(p, "bf16", kernel=kernel)
    assert info["kernel_name"] == "tc_bf16_direct" and info["launches"] == 2  # product + reduction
    want = run_oracle(p, in_dtype=torch.bfloat16, out_dtype=torch.float32)
    assert rel_frob(gpu_dense(Cg), want) <= TOL
    Cg2, _ = run_gpu(p, "bf16", kernel=kernel)
    assert torch.equal(Cg, Cg2)  # the split order is fixed


def test_split_tail_integer_exact():
    """178 tiles on 148 SMs (tile width 256): one whole round, then the 30-tile
    tail split along k; integer inputs make every partial sum exact, so
    sampled entries of tail and whole tiles match the oracle exactly."""
    rng = np.random.default_rng(708)
    m, n, k = 89 * 128, 512, 4096
    A = W.integer_operand(rng, (m, k), [1, 2], lo=-2, hi=2)
    B = W.integer_operand(rng, (k, n), [2, 3], lo=-2, hi=2)
    C = W.zeros_operand((m, n), [1, 3])
    p = W.Problem("split_tail", 1.0, A, B, 0.0, C)
    Cg, info = run_gpu(p, "bf16", tile_n=256)
    assert info["kernel_name"] == "tc_bf16_direct" and info["launches"] == 2
    got = gpu_dense(Cg)
    rows = np.concatenate([rng.integers(74 * 128, m, 48), rng.integers(0, 74 * 128, 16)])
    idx = np.stack([rows, rng.integers(0, n, rows.size)], axis=1)
    want = oracle.entries(1.0, A.view(), A.labels, B.view(), B.labels, 0.0, C.view(), C.labels, idx)
    assert np.array_equal(got[idx[:, 0], idx[:, 1]], want)
