"""Many independent contractions in one call (the blocks of a block-sparse
contraction): one grouped launch per stage over a longest-first tile list,
optionally captured in a CUDA graph and replayed.  Every block is checked
against the oracle."""
import numpy as np
import pytest
import torch

import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import OUT_DT, TORCH_DT, gpu_dense, rel_frob, run_oracle, to_device

pytestmark = pytest.mark.gpu

TOL = {"f64_emu": 1e-13, "f64": 1e-13, "f32": 1e-5, "bf16": 1e-5}


def batched_call(blocks, As, Bs, Cs, dtype, use_graph):
    fm.contract_batched([b.alpha for b in blocks], As, [b.A.labels for b in blocks], Bs,
                        [b.B.labels for b in blocks], [b.beta for b in blocks], Cs,
                        [b.C.labels for b in blocks], dtype=dtype, use_graph=use_graph)
    torch.cuda.synchronize()


def run_batch(blocks, dtype, use_graph):
    As = [to_device(b.A, TORCH_DT[dtype]) for b in blocks]
    Bs = [to_device(b.B, TORCH_DT[dtype]) for b in blocks]
    Cs = [to_device(b.C, OUT_DT[dtype]) for b in blocks]
    batched_call(blocks, As, Bs, Cs, dtype, use_graph)
    return As, Bs, Cs


def check(blocks, Cs, dtype, in_dtype=None):
    for b, C in zip(blocks, Cs):
        want = run_oracle(b, in_dtype=in_dtype)
        assert rel_frob(gpu_dense(C), want) <= TOL[dtype], (b.name, b.meta)


@pytest.mark.parametrize("use_graph", [False, True])
def test_block_sparse_emulated_fp64(use_graph):
    blocks = W.block_sparse(nblocks=40, choices=[8, 16, 24, 32, 40])
    _, _, Cs = run_batch(blocks, "f64_emu", use_graph)
    check(blocks, Cs, "f64_emu")
    assert fm.device_status() == 0


def test_block_sparse_integer_exact():
    blocks = W.block_sparse(nblocks=25, choices=[8, 16, 24], integer=True)
    _, _, Cs = run_batch(blocks, "f64_emu", False)
    for b, C in zip(blocks, Cs):
        assert np.array_equal(gpu_dense(C), run_oracle(b)), b.meta


def test_graph_replay_sees_new_values():
    """The second call replays the captured graph; it must read the operands'
    current contents (same addresses, new values) and beta*C."""
    rng = np.random.default_rng(950)
    blocks = W.block_sparse(nblocks=12, choices=[16, 24, 32], seed=77)
    for b in blocks:
        b.beta = 0.5
        b.C.buf[:] = rng.uniform(-1, 1, b.C.buf.shape)
    As, Bs, Cs = run_batch(blocks, "f64_emu", True)
    check(blocks, Cs, "f64_emu")
    firsts = [gpu_dense(C) for C in Cs]  # C now holds the first result: the next C_in
    for b, A in zip(blocks, As):  # new values in place, same addresses
        b.A.buf[:] = rng.uniform(-1, 1, b.A.buf.shape)
        A.copy_(to_device(b.A, torch.float64))
    batched_call(blocks, As, Bs, Cs, "f64_emu", True)
    for b, C, first in zip(blocks, Cs, firsts):
        b.C.view()[...] = first
        assert rel_frob(gpu_dense(C), run_oracle(b)) <= 1e-13


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_block_sparse_bf16_and_fp32(dtype):
    blocks = W.block_sparse(nblocks=30, choices=[8, 16, 24, 32, 48], seed=78)
    _, _, Cs = run_batch(blocks, dtype, dtype == "f32")
    check(blocks, Cs, dtype, in_dtype=TORCH_DT[dtype])


def test_mixed_batch_scale_only_and_empty():
    rng = np.random.default_rng(951)
    blocks = W.block_sparse(nblocks=6, choices=[8, 16], seed=79)
    # one block with an empty contracted extent, one with alpha = 0
    A = W.uniform_operand(rng, (5, 0), [1, 2])
    B = W.uniform_operand(rng, (0, 7), [2, 3])
    C = W.uniform_operand(rng, (5, 7), [1, 3])
    blocks.append(W.Problem("emptyk", 1.0, A, B, 2.0, C))
    blocks[0].alpha = 0.0
    blocks[0].beta = -1.0
    blocks[0].C.buf[:] = rng.uniform(-1, 1, blocks[0].C.buf.shape)
    _, _, Cs = run_batch(blocks, "f64_emu", False)
    check(blocks, Cs, "f64_emu")
    # the fp64 CUDA-core path runs block by block inside the same call
    _, _, Cs = run_batch(blocks[1:6], "f64", False)
    check(blocks[1:6], Cs, "f64")


def _gemm_block(rng, m, n, k, batch, name):
    """C[i,j(,z)] = sum_k A[i,k(,z)] B[k,j(,z)] with an optional batch label z."""
    lz = [9] if batch else []
    ez = (batch,) if batch else ()
    A = W.uniform_operand(rng, (m, k) + ez, [1, 2] + lz)
    B = W.uniform_operand(rng, (k, n) + ez, [2, 3] + lz)
    C = W.uniform_operand(rng, (m, n) + ez, [1, 3] + lz)
    return W.Problem(name, 1.25, A, B, -0.75, C)


@pytest.mark.parametrize("dtype", ["f64_emu", "bf16"])
def test_mixed_widths_and_batch_labels_in_one_group(dtype):
    """Blocks whose column counts call for tile widths 64, 128 and 256 share
    one grouped launch; some carry a batch label."""
    rng = np.random.default_rng(952)
    shapes = [(130, 40, 70, 0), (257, 100, 33, 3), (64, 300, 129, 0), (9, 17, 5, 2),
              (200, 256, 64, 0), (140, 129, 200, 4)]
    blocks = [_gemm_block(rng, m, n, k, z, f"g{i}") for i, (m, n, k, z) in enumerate(shapes)]
    _, _, Cs = run_batch(blocks, dtype, False)
    for b, C in zip(blocks, Cs):
        want = run_oracle(b, in_dtype=TORCH_DT[dtype], out_dtype=OUT_DT[dtype])
        assert rel_frob(gpu_dense(C), want) <= TOL[dtype], b.name


def test_graph_cache_rekeys_on_new_pointers():
    """A different problem set (new output buffers) builds its own graph; the
    cached one keeps working for the original set."""
    rng = np.random.default_rng(953)
    blocks = [_gemm_block(rng, 96, 80, 48, 0, f"h{i}") for i in range(5)]
    As, Bs, Cs = run_batch(blocks, "f64_emu", True)
    check(blocks, Cs, "f64_emu")
    Cs2 = [to_device(b.C, torch.float64) for b in blocks]
    batched_call(blocks, As, Bs, Cs2, "f64_emu", True)
    check(blocks, Cs2, "f64_emu")
    Cs3 = [to_device(b.C, torch.float64) for b in blocks]
    for C3, C in zip(Cs3, Cs):
        C.copy_(C3)
    batched_call(blocks, As, Bs, Cs, "f64_emu", True)  # the first set again: replay
    check(blocks, Cs, "f64_emu")


def test_long_k_block_uses_exact_fine_sums_in_the_grouped_launch():
    """A block with K = 2^18 next to a small one in one grouped launch: the
    schedule keeps a second, exact int64 sum for the fine diagonals (per-CTA
    slots twice as wide); sampled entries of the long block match the
    oracle's compensated sums, the small block matches the oracle."""
    import oracle
    rng = np.random.default_rng(1800)
    K = 1 << 18
    A1 = W.uniform_operand(rng, (64, K), [1, 2])
    B1 = W.uniform_operand(rng, (K, 48), [2, 3])
    C1 = W.zeros_operand((64, 48), [1, 3])
    A2 = W.uniform_operand(rng, (100, 70), [1, 2])
    B2 = W.uniform_operand(rng, (70, 90), [2, 3])
    C2 = W.uniform_operand(rng, (100, 90), [1, 3])
    dev = [to_device(x, torch.float64) for x in (A1, B1, C1, A2, B2, C2)]
    fm.contract_batched(1.0, [dev[0], dev[3]], [[1, 2], [1, 2]], [dev[1], dev[4]], [[2, 3], [2, 3]], 0.5,
                        [dev[2], dev[5]], [[1, 3], [1, 3]], dtype="f64_emu")
    torch.cuda.synchronize()
    idx = np.stack([rng.integers(0, 64, size=256), rng.integers(0, 48, size=256)], axis=1)
    want = oracle.entries(1.0, A1.view(), [1, 2], B1.view(), [2, 3], 0.5, C1.view(), [1, 3], idx, dot2=True)
    got = gpu_dense(dev[2])[idx[:, 0], idx[:, 1]]
    assert rel_frob(got, want) <= 1e-13
    p2 = W.Problem("small", 1.0, A2, B2, 0.5, C2)
    assert rel_frob(gpu_dense(dev[5]), run_oracle(p2)) <= 1e-13
