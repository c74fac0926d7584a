"""GPU parity of contraction networks (a pre-ordered sequence of contractions
in one library call, intermediates allocated and freed by the library) against
the oracle applied step by step."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, to_device

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64_emu": 1e-13, "f32": 1e-5}
DT = {"f64": torch.float64, "f64_emu": torch.float64, "f32": torch.float32}


def _oracle_step(alpha, A, la, B, lb, beta, C, lc):
    C = np.array(C, copy=True)
    oracle.contract(alpha, A, la, B, lb, beta, C, lc)
    return C


@pytest.mark.parametrize("dtype", ["f64", "f64_emu", "f32"])
def test_chain_through_an_intermediate(dtype):
    """D[i,l] = 0.5 * sum_{j,k} A[i,j] B[j,k] C[k,l] - D as two steps; the
    product A B lives only on the device."""
    rng = np.random.default_rng(700)
    ext = {1: 150, 2: 70, 3: 90, 4: 130}
    A = W.uniform_operand(rng, (ext[1], ext[2]), [1, 2])
    B = W.uniform_operand(rng, (ext[2], ext[3]), [2, 3])
    Cm = W.uniform_operand(rng, (ext[3], ext[4]), [3, 4])
    D = W.uniform_operand(rng, (ext[1], ext[4]), [1, 4])
    Ad, Bd, Cd, Dd = (to_device(x, DT[dtype]) for x in (A, B, Cm, D))
    tensors = [(Ad, [1, 2]), (Bd, [2, 3]), ((ext[1], ext[3]), [1, 3]), (Cd, [3, 4]), (Dd, [1, 4])]
    steps = [(0, 1, 2, 1.0, 0.0), (2, 3, 4, 0.5, -1.0)]
    fm.contract_network(tensors, steps, dtype=dtype)
    torch.cuda.synchronize()
    X = _oracle_step(1.0, A.view(), [1, 2], B.view(), [2, 3], 0.0, np.zeros((ext[1], ext[3])), [1, 3])
    want = _oracle_step(0.5, X, [1, 3], Cm.view(), [3, 4], -1.0, D.view(), [1, 4])
    assert rel_frob(gpu_dense(Dd), want) <= TOL[dtype]
    assert fm.device_status() == 0


def test_ladder_terms_accumulate_into_one_result():
    """R[a,b,i,j] = sum_{c,d} V[a,b,c,d] X[c,d,i,j] + R, with the
    intermediate X[c,d,i,j] = sum_{k,l} T[c,d,k,l] Y[k,l,i,j], then a second
    term R += 0.25 * sum_{c,d} V[a,b,c,d] T[c,d,i,j] into the same result
    (emulated fp64)."""
    rng = np.random.default_rng(701)
    v, o = 12, 6
    V = W.uniform_operand(rng, (v, v, v, v), W.L("abcd"))
    T = W.uniform_operand(rng, (v, v, o, o), W.L("cdkl"))
    Y = W.uniform_operand(rng, (o, o, o, o), W.L("klij"))
    R = W.uniform_operand(rng, (v, v, o, o), W.L("abij"))
    Vd, Td, Yd, Rd = (to_device(x, torch.float64) for x in (V, T, Y, R))
    tensors = [(Vd, W.L("abcd")), (Td, W.L("cdkl")), (Yd, W.L("klij")), ((v, v, o, o), W.L("cdij")),
               (Rd, W.L("abij")), (Td, W.L("cdij"))]
    steps = [(1, 2, 3, 1.0, 0.0), (0, 3, 4, 1.0, 1.0), (0, 5, 4, 0.25, 1.0)]
    fm.contract_network(tensors, steps, dtype="f64_emu")
    torch.cuda.synchronize()
    X = _oracle_step(1.0, T.view(), W.L("cdkl"), Y.view(), W.L("klij"), 0.0, np.zeros((v, v, o, o)),
                     W.L("cdij"))
    R1 = _oracle_step(1.0, V.view(), W.L("abcd"), X, W.L("cdij"), 1.0, R.view(), W.L("abij"))
    want = _oracle_step(0.25, V.view(), W.L("abcd"), T.view(), W.L("cdij"), 1.0, R1, W.L("abij"))
    assert rel_frob(gpu_dense(Rd), want) <= 1e-13


def test_planning_error_launches_nothing():
    """A step whose labels do not match (extent mismatch) is found while the
    whole sequence is planned: no step runs, the output keeps its values."""
    rng = np.random.default_rng(702)
    A = to_device(W.uniform_operand(rng, (8, 9), [1, 2]), torch.float64)
    B = to_device(W.uniform_operand(rng, (9, 10), [2, 3]), torch.float64)
    C = to_device(W.uniform_operand(rng, (8, 10), [1, 3]), torch.float64)
    bad = to_device(W.uniform_operand(rng, (11, 10), [1, 3]), torch.float64)  # label 1: 11 != 8
    before = C.clone()
    with pytest.raises(fm.FamliesError) as e:
        fm.contract_network([(A, [1, 2]), (B, [2, 3]), (C, [1, 3]), (bad, [1, 3])],
                            [(0, 1, 2, 1.0, 0.0), (0, 1, 3, 1.0, 0.0)], dtype="f64")
    assert e.value.code == -3  # FAMLIES_ERR_EXTENT_MISMATCH
    torch.cuda.synchronize()
    assert torch.equal(C, before)


def test_empty_network_and_single_step():
    """No steps: nothing runs; one step equals the plain contraction."""
    rng = np.random.default_rng(703)
    A = W.uniform_operand(rng, (20, 30), [1, 2])
    B = W.uniform_operand(rng, (30, 25), [2, 3])
    C = W.uniform_operand(rng, (20, 25), [1, 3])
    Ad, Bd, Cd = (to_device(x, torch.float64) for x in (A, B, C))
    before = Cd.clone()
    fm.contract_network([(Ad, [1, 2]), (Bd, [2, 3]), (Cd, [1, 3])], [], dtype="f64_emu")
    torch.cuda.synchronize()
    assert torch.equal(Cd, before)
    fm.contract_network([(Ad, [1, 2]), (Bd, [2, 3]), (Cd, [1, 3])], [(0, 1, 2, 2.0, -1.0)], dtype="f64_emu")
    torch.cuda.synchronize()
    want = _oracle_step(2.0, A.view(), [1, 2], B.view(), [2, 3], -1.0, C.view(), [1, 3])
    assert rel_frob(gpu_dense(Cd), want) <= 1e-13


@pytest.mark.parametrize("x_first", ["i", "k"])
@pytest.mark.parametrize("j", [200, 600])
@pytest.mark.parametrize("nan", [False, True])
def test_fused_exponents_match_separate_calls_bitwise(x_first, j, nan):
    """X = A B then D = X C - D (emulated fp64): the consumer's rows of X are
    the producer's rows (X listed i first) or its columns (k first), so the
    producer's finish records the consumer's row exponents and Inf/NaN flags
    and the consumer skips its exponent scan of X.  The exponents are the
    ones the scan would find, so the result is bit-identical to two separate
    calls.  k = 200 finishes the producer's tiles in a separate kernel, k =
    600 inside the product; a NaN in A sends rows through the native fix-up,
    which records its values too."""
    rng = np.random.default_rng(710 + j)
    ni, nk, nl = 300, 260, 150
    A = W.uniform_operand(rng, (ni, j), [1, 2])
    if nan:
        A.buf[5 + ni * 7] = np.nan
    B = W.uniform_operand(rng, (j, nk), [2, 3])
    Cm = W.uniform_operand(rng, (nk, nl), [3, 4])
    D = W.uniform_operand(rng, (ni, nl), [1, 4])
    Ad, Bd, Cd = (to_device(x, torch.float64) for x in (A, B, Cm))
    D1, D2 = to_device(D, torch.float64), to_device(D, torch.float64)
    lx = [1, 3] if x_first == "i" else [3, 1]
    shape = (ni, nk) if x_first == "i" else (nk, ni)
    tensors = [(Ad, [1, 2]), (Bd, [2, 3]), (shape, lx), (Cd, [3, 4]), (D1, [1, 4])]
    fm.contract_network(tensors, [(0, 1, 2, 1.0, 0.0), (2, 3, 4, 1.0, -1.0)], dtype="f64_emu")
    X = torch.empty(shape[::-1], dtype=torch.float64, device="cuda").t()  # first mode fastest, as the library lays it
    fm.contract(1.0, Ad, [1, 2], Bd, [2, 3], 0.0, X, lx, dtype="f64_emu")
    fm.contract(1.0, X, lx, Cd, [3, 4], -1.0, D2, [1, 4], dtype="f64_emu")
    torch.cuda.synchronize()
    g1, g2 = gpu_dense(D1), gpu_dense(D2)
    assert np.array_equal(g1, g2, equal_nan=True)
    Xo = _oracle_step(1.0, A.view(), [1, 2], B.view(), [2, 3], 0.0, np.zeros(shape), lx)
    want = _oracle_step(1.0, Xo, lx, Cm.view(), [3, 4], -1.0, D.view(), [1, 4])
    assert np.array_equal(np.isnan(g1), np.isnan(want))
    fin = np.isfinite(want)
    assert rel_frob(g1[fin], want[fin]) <= TOL["f64_emu"]
    assert fm.device_status() == 0
