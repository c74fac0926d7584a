"""GPU invariants of the contraction (the label system and the alpha/beta
update of Sec. 2.1's "variations on functionality": transposition and
relabelling are changes of description, not of the result): relabelling,
permuting an operand's modes (same memory), swapping the operands, scaling
by powers of two, and GEMM as the two-label case against torch.matmul (a
library cross-check next to the oracle)."""
import numpy as np
import pytest
import torch

import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import rel_frob, to_device

pytestmark = pytest.mark.gpu

DTYPES = {"f64": (torch.float64, torch.float64), "f64_emu": (torch.float64, torch.float64),
          "f32": (torch.float32, torch.float32), "bf16": (torch.bfloat16, torch.float32)}


def _problem(dtype, seed=1500):
    rng = np.random.default_rng(seed)
    tin, tout = DTYPES[dtype]
    A = to_device(W.uniform_operand(rng, (40, 30, 50), W.L("aik")), tin)   # A[a,i,k]
    B = to_device(W.uniform_operand(rng, (50, 30, 60), W.L("kij")), tin)   # B[k,i,j]
    C = to_device(W.uniform_operand(rng, (40, 60, 30), W.L("aji")), tout)  # C[a,j,i] (i batch)
    return A, B, C


def _run(alpha, A, la, B, lb, beta, C, lc, dtype):
    out = C.clone()
    fm.contract(alpha, A, la, B, lb, beta, out, lc, dtype=dtype)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("dtype", ["f64", "f64_emu", "f32", "bf16"])
def test_relabel_permute_and_swap_give_identical_results(dtype):
    A, B, C = _problem(dtype)
    la, lb, lc = W.L("aik"), W.L("kij"), W.L("aji")
    base = _run(1.5, A, la, B, lb, 0.5, C, lc, dtype)
    # a bijective renaming of the labels
    ren = {ord("a"): 7, ord("i"): 3, ord("k"): 11, ord("j"): 5}
    r = lambda ls: [ren[x] for x in ls]
    assert torch.equal(_run(1.5, A, r(la), B, r(lb), 0.5, C, r(lc), dtype), base)
    # A's modes permuted in its descriptor (same memory, same element -> label map)
    Ap = A.permute(2, 0, 1)
    assert torch.equal(_run(1.5, Ap, [la[2], la[0], la[1]], B, lb, 0.5, C, lc, dtype), base)
    # the operands swapped
    assert torch.equal(_run(1.5, B, lb, A, la, 0.5, C, lc, dtype), base)


@pytest.mark.parametrize("dtype", ["f64", "f64_emu", "f32", "bf16"])
def test_powers_of_two_scale_exactly(dtype):
    """alpha = 8 gives 8 x the alpha = 1 result bit for bit (beta = 0), and
    beta = 1/2 on C equals beta = 1 on C/2."""
    A, B, C = _problem(dtype, seed=1501)
    la, lb, lc = W.L("aik"), W.L("kij"), W.L("aji")
    one = _run(1.0, A, la, B, lb, 0.0, C, lc, dtype)
    eight = _run(8.0, A, la, B, lb, 0.0, C, lc, dtype)
    assert torch.equal(eight, 8 * one)
    half = _run(1.0, A, la, B, lb, 0.5, C, lc, dtype)
    assert torch.equal(half, _run(1.0, A, la, B, lb, 1.0, C / 2, lc, dtype))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-14), ("f64_emu", 1e-14), ("f32", 1e-5)])
@pytest.mark.parametrize("m,n,k", [(300, 200, 500), (1024, 1024, 1024)])
def test_gemm_against_torch_matmul(dtype, tol, m, n, k):
    tin, _ = DTYPES[dtype]
    g = torch.Generator(device="cuda")
    g.manual_seed(m + n + k)
    A = torch.rand(m, k, device="cuda", dtype=torch.float64, generator=g).to(tin)
    B = torch.rand(k, n, device="cuda", dtype=torch.float64, generator=g).to(tin)
    C = torch.zeros(m, n, device="cuda", dtype=tin)
    fm.contract(1.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3], dtype=dtype)
    want = A.double() @ B.double()
    assert rel_frob(C.double().cpu().numpy(), want.cpu().numpy()) <= tol
