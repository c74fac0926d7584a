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
