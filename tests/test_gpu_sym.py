"""GPU parity of contractions with a symmetric operand stored as a packed
lower triangle (Sec. 3: contraction with symmetric dense tensors) against the
oracle applied to the dense expansion of the same operand."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, to_device

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _sym_dense(rng, half):
    """A symmetric tensor with halves of extents `half`: the n x n matrix of
    its fused indices (first mode fastest) has N(0,1) entries, mirrored."""
    n = int(np.prod(half))
    X = rng.standard_normal((n, n))
    M = np.tril(X) + np.tril(X, -1).T
    ext = tuple(half) + tuple(half)
    # M[p, q] with p the first half's fused index: column-major flattening
    dense = M.reshape(-1, order="F").reshape(ext, order="F")
    return M, dense


def _run(alpha, M, ext, la, B, lb, beta, C, lc, **kw):
    Ap = torch.from_numpy(W.packed_lower(M)).to("cuda")
    Bd, Cd = to_device(B, torch.float64), to_device(C, torch.float64)
    _, info = fm.contract_sym(alpha, Ap, ext, la, Bd, lb, beta, Cd, lc, return_info=True, **kw)
    torch.cuda.synchronize()
    return gpu_dense(Cd), info


def _want(alpha, dense, la, B, lb, beta, C, lc):
    Cv = np.array(C.view(), copy=True)
    oracle.contract(alpha, dense, la, B.view(), lb, beta, Cv, lc)
    return Cv


@pytest.mark.parametrize("v,o", [(12, 6), (13, 5), (24, 8)])
def test_ladder_with_packed_v(v, o):
    """C[a,b,i,j] = sum_{c,d} V[a,b,c,d] T[c,d,i,j] + C with V read packed;
    v = 13 leaves ragged 64-row blocks of the triangle."""
    rng = np.random.default_rng(800 + v)
    M, Vd = _sym_dense(rng, (v, v))
    T = W.uniform_operand(rng, (v, v, o, o), W.L("cdij"))
    C = W.uniform_operand(rng, (v, v, o, o), W.L("abij"))
    got, info = _run(1.0, M, (v, v, v, v), W.L("abcd"), T, W.L("cdij"), 1.0, C, W.L("abij"))
    want = _want(1.0, Vd, W.L("abcd"), T, W.L("cdij"), 1.0, C, W.L("abij"))
    assert info["kernel_name"] == "tc_emu"
    assert rel_frob(got, want) <= TOL
    assert fm.device_status() == 0


def test_contracted_first_half():
    """R[c,d,i,j] = sum_{a,b} V[a,b,c,d] T[a,b,i,j]: the free half of V is
    its second one (rows at stride n in the dense expansion)."""
    rng = np.random.default_rng(810)
    v, o = 14, 6
    M, Vd = _sym_dense(rng, (v, v))
    T = W.uniform_operand(rng, (v, v, o, o), W.L("abij"))
    C = W.uniform_operand(rng, (v, v, o, o), W.L("cdij"))
    got, _ = _run(0.5, M, (v, v, v, v), W.L("abcd"), T, W.L("abij"), -1.0, C, W.L("cdij"))
    want = _want(0.5, Vd, W.L("abcd"), T, W.L("abij"), -1.0, C, W.L("cdij"))
    assert rel_frob(got, want) <= TOL


def test_symmetric_operand_as_column_operand():
    """C[i,j,a,b] = sum_{c,d} T[i,j,c,d] V[a,b,c,d]: C's unit-stride mode
    belongs to T, so the kernel takes T as its row operand and V as its
    column operand."""
    rng = np.random.default_rng(820)
    v, o = 12, 7
    M, Vd = _sym_dense(rng, (v, v))
    T = W.uniform_operand(rng, (o, o, v, v), W.L("ijcd"))
    C = W.uniform_operand(rng, (o, o, v, v), W.L("ijab"))
    got, info = _run(1.0, M, (v, v, v, v), W.L("abcd"), T, W.L("ijcd"), 1.0, C, W.L("ijab"))
    want = _want(1.0, Vd, W.L("abcd"), T, W.L("ijcd"), 1.0, C, W.L("ijab"))
    assert info["swapped"] == 1
    assert rel_frob(got, want) <= TOL


def test_halves_of_mixed_extents_and_a_matrix():
    """Halves (5, 7) | (5, 7) (n = 35), and a plain symmetric matrix
    (two modes, C = A B with A symmetric)."""
    rng = np.random.default_rng(830)
    M, Vd = _sym_dense(rng, (5, 7))
    T = W.uniform_operand(rng, (5, 7, 9), W.L("cdj"))
    C = W.zeros_operand((5, 7, 9), W.L("abj"))
    got, _ = _run(1.0, M, (5, 7, 5, 7), W.L("abcd"), T, W.L("cdj"), 0.0, C, W.L("abj"))
    assert rel_frob(got, _want(1.0, Vd, W.L("abcd"), T, W.L("cdj"), 0.0, C, W.L("abj"))) <= TOL
    M2, A2 = _sym_dense(rng, (150,))
    B2 = W.uniform_operand(rng, (150, 70), [2, 3])
    C2 = W.uniform_operand(rng, (150, 70), [1, 3])
    got, _ = _run(2.0, M2, (150, 150), [1, 2], B2, [2, 3], 0.5, C2, [1, 3])
    assert rel_frob(got, _want(2.0, A2, [1, 2], B2, [2, 3], 0.5, C2, [1, 3])) <= TOL


def test_long_k_few_tiles_splits_k():
    """n = 1600 rows and k, 16 columns: 13 tiles, so K is split across the
    SMs (partial sums per tile, then the finishing kernel)."""
    rng = np.random.default_rng(840)
    v, o = 40, 4
    M, Vd = _sym_dense(rng, (v, v))
    T = W.uniform_operand(rng, (v, v, o, o), W.L("cdij"))
    C = W.uniform_operand(rng, (v, v, o, o), W.L("abij"))
    got, info = _run(1.0, M, (v, v, v, v), W.L("abcd"), T, W.L("cdij"), 1.0, C, W.L("abij"))
    want = _want(1.0, Vd, W.L("abcd"), T, W.L("cdij"), 1.0, C, W.L("abij"))
    # tables, V's exponent scan, its reduction and pack, T's one-pass split
    # (k unit-stride), product, split finish, fix-up
    assert info["launches"] + info["cached"] == 8
    assert rel_frob(got, want) <= TOL


def test_nan_in_the_triangle_reaches_both_mirrored_rows():
    """A NaN stored once at (p, q), p > q, stands for A[p, q] and A[q, p]: the
    fix-up recomputes rows p and q natively, and the NaN pattern and the
    finite entries match the oracle on the dense expansion."""
    rng = np.random.default_rng(850)
    v, o = 12, 5
    M, Vd = _sym_dense(rng, (v, v))
    p, q = 100, 7
    M[p, q] = M[q, p] = np.nan
    Vd = M.reshape(-1, order="F").reshape((v,) * 4, order="F")
    T = W.uniform_operand(rng, (v, v, o, o), W.L("cdij"))
    C = W.uniform_operand(rng, (v, v, o, o), W.L("abij"))
    got, _ = _run(1.0, M, (v, v, v, v), W.L("abcd"), T, W.L("cdij"), 1.0, C, W.L("abij"))
    want = _want(1.0, Vd, W.L("abcd"), T, W.L("cdij"), 1.0, C, W.L("abij"))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.isnan(want).any()
    fin = ~np.isnan(want)
    assert rel_frob(got[fin], want[fin]) <= TOL


def test_full_size_ladder_packed_matches_dense_bit_for_bit():
    """v = 128, o = 32 (the benchmark's ladder): V read from its packed
    triangle gives the same slices, exponents and tile order as dense V, so
    the result is bit-identical to the dense path's (which the full-size
    sampled test checks against the oracle), and sampled entries match the
    oracle."""
    p = W.ladder(v=128, o=32)
    n = 128 * 128
    M = p.A.buf.reshape(n, n)  # symmetric: either flattening
    Ap = torch.from_numpy(W.packed_lower(M)).cuda()
    T = to_device(p.B, torch.float64)
    Cs = to_device(p.C, torch.float64)
    Cd = to_device(p.C, torch.float64)
    Vd = to_device(p.A, torch.float64)
    fm.contract_sym(p.alpha, Ap, p.A.extents, p.A.labels, T, p.B.labels, p.beta, Cs, p.C.labels)
    fm.contract(p.alpha, Vd, p.A.labels, T, p.B.labels, p.beta, Cd, p.C.labels, dtype="f64_emu")
    torch.cuda.synchronize()
    assert torch.equal(Cs, Cd)
    rng = np.random.default_rng(860)
    idx = np.stack([rng.integers(0, e, size=256) for e in p.C.extents], axis=1)
    want = oracle.entries(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, p.C.view(),
                          p.C.labels, idx, dot2=True)
    got = Cs.cpu().numpy()[tuple(idx.T)]
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_degenerate_symmetric_operands():
    """n = 1 (a 1 x 1 triangle) and an empty free extent of B (nothing to
    write)."""
    rng = np.random.default_rng(870)
    M, Vd = _sym_dense(rng, (1,))
    B = W.uniform_operand(rng, (1, 9), [2, 3])
    C = W.uniform_operand(rng, (1, 9), [1, 3])
    got, _ = _run(2.0, M, (1, 1), [1, 2], B, [2, 3], 0.5, C, [1, 3])
    assert rel_frob(got, _want(2.0, Vd, [1, 2], B, [2, 3], 0.5, C, [1, 3])) <= TOL
    Ap = torch.from_numpy(W.packed_lower(M)).cuda()
    Bd = torch.empty(1, 0, dtype=torch.float64, device="cuda")
    Cd = torch.empty(1, 0, dtype=torch.float64, device="cuda")
    fm.contract_sym(1.0, Ap, (1, 1), [1, 2], Bd, [2, 3], 0.0, Cd, [1, 3])
    torch.cuda.synchronize()
