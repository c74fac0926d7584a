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


def test_full_block_sparse_configuration_sampled_dot2():
    """The full configuration: 2000 blocks of the four-index pattern, each of
    the six extents drawn from {8, 16, ..., 96} (7.5e13 flops).  Its literal
    inputs would take ~350 GB, so every block's A and B are column-major views
    into one shared random pool at seeded offsets (read-only: sharing is
    harmless); each C has its own storage (~114 GB).  One grouped call under a
    CUDA graph; 32 entries of each of 64 blocks, the largest included, against
    the oracle's compensated (Dot2) sums, within 1e-13 relative Frobenius."""
    import oracle
    torch.cuda.empty_cache()
    nblocks = 2000
    ext = W.block_sparse_extents(nblocks=nblocks)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    pool = torch.rand(1 << 28, device="cuda", dtype=torch.float64, generator=gen)
    offs = np.random.default_rng(W.SEED_BASE + 40).integers(0, (1 << 28) - 96 ** 4, size=(nblocks, 2))
    As, Bs, Cs = [], [], []
    la, lb, lc = W.L("acik"), W.L("ckbj"), W.L("abij")
    for bi, (a, b, c, i, j, k) in enumerate(map(int, e) for e in ext):
        As.append(torch.as_strided(pool, (a, c, i, k), W.colmajor_strides((a, c, i, k)), int(offs[bi, 0])))
        Bs.append(torch.as_strided(pool, (c, k, b, j), W.colmajor_strides((c, k, b, j)), int(offs[bi, 1])))
        Cs.append(torch.full((j, i, b, a), float("nan"), device="cuda", dtype=torch.float64).permute(3, 2, 1, 0))
    fm.contract_batched(1.0, As, [la] * nblocks, Bs, [lb] * nblocks, 0.0, Cs, [lc] * nblocks,
                        dtype="f64_emu", use_graph=True)
    torch.cuda.synchronize()
    assert fm.device_status() == 0
    sizes = np.array([float(np.prod(e)) for e in ext])
    pick = sorted(set([int(np.argmax(sizes))] +
                      [int(x) for x in np.random.default_rng(960).choice(nblocks, 63, replace=False)]))
    assert len(pick) >= 50
    pool_h = pool.cpu().numpy()
    rng = np.random.default_rng(961)
    num = den = 0.0
    for bi in pick:
        Ah = np.lib.stride_tricks.as_strided(pool_h[int(offs[bi, 0]):], tuple(As[bi].shape),
                                             tuple(8 * x for x in As[bi].stride()))
        Bh = np.lib.stride_tricks.as_strided(pool_h[int(offs[bi, 1]):], tuple(Bs[bi].shape),
                                             tuple(8 * x for x in Bs[bi].stride()))
        got = Cs[bi].cpu().numpy()
        idx = np.stack([rng.integers(0, e, 32) for e in got.shape], axis=1)
        want = oracle.entries(1.0, Ah, la, Bh, lb, 0.0, np.zeros(got.shape), lc, idx, dot2=True)
        g = got[tuple(idx.T)]
        assert np.all(np.isfinite(g)), bi  # beta = 0: the NaN C held is overwritten
        num += float(np.sum((g - want) ** 2))
        den += float(np.sum(want ** 2))
        assert rel_frob(g, want) <= 1e-13, (bi, ext[bi])
    assert (num / den) ** 0.5 <= 1e-13
    del As, Bs, Cs, pool
    torch.cuda.empty_cache()
