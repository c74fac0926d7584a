"""Pins for the FP64 oracle, against things other than the oracle itself.

Each test checks the oracle against an independent formulation or a fact
fixed by the mathematics: exact integer brute force in Python ints, numpy's
einsum, closed forms (identity, all-ones, rank-1, Kronecker operands),
invariants (relabelling, A<->B swap, power-of-two scaling, linearity), the
BLAS conventions for alpha == 0 / beta == 0, empty extents, IEEE propagation
of Inf/NaN (Sec. 1.5 "BLIS and TBLIS": consistent NaN/Inf handling), exact
rationals for the compensated mode, and hand-worked golden values.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2604_07311_b300 import inputs as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.txt")


# ------------------------------------------------------------------ helpers
def strided(rng, shape, pad_max=2, perm=None, integer=True):
    """A float64 view with random padded strides and a random mode order in memory."""
    nd = len(shape)
    perm = list(rng.permutation(nd)) if perm is None else perm
    pads = [int(rng.integers(0, pad_max + 1)) for _ in range(nd)]
    strides = [0] * nd
    acc = 1
    for d in perm:  # memory order
        strides[d] = acc
        acc *= shape[d] + pads[d]
    size = max(acc, 1)
    buf = rng.integers(-4, 5, size=size).astype(np.float64) if integer else rng.uniform(-1, 1, size)
    v = np.lib.stride_tricks.as_strided(buf, shape=tuple(shape), strides=tuple(8 * s for s in strides))
    return v, buf


def brute_force_exact(alpha, A, la, B, lb, beta, C, lc):
    """Python-int Einstein sum; independent of the oracle's code."""
    ext = {}
    for arr, labs in ((A, la), (B, lb), (C, lc)):
        for lab, e in zip(labs, arr.shape):
            ext[lab] = e
    labels = sorted(ext)
    out = {}
    for cidx in itertools.product(*[range(e) for e in C.shape]):
        out[cidx] = Fraction(beta) * Fraction(C[cidx]) if beta != 0 else Fraction(0)
    acc = {k: Fraction(0) for k in out}
    for vals in itertools.product(*[range(ext[l]) for l in labels]):
        asg = dict(zip(labels, vals))
        ai = tuple(asg[l] for l in la)
        bi = tuple(asg[l] for l in lb)
        ci = tuple(asg[l] for l in lc)
        acc[ci] += Fraction(A[ai]) * Fraction(B[bi])
    res = np.empty(C.shape)
    for k in out:
        res[k] = float(out[k] + Fraction(alpha) * acc[k]) if alpha != 0 else float(out[k])
    return res


def random_problem(rng, integer=True, max_ext=3, batch=True):
    """Random label sets: M (A,C), N (B,C), K (A,B), batch (A,B,C)."""
    names = iter(range(100, 200))
    nm, nn, nk = (int(rng.integers(0, 3)) for _ in range(3))
    nl = int(rng.integers(0, 2)) if batch else 0
    M = [next(names) for _ in range(nm)]
    N = [next(names) for _ in range(nn)]
    K = [next(names) for _ in range(nk)]
    Lb = [next(names) for _ in range(nl)]
    ext = {l: int(rng.integers(1, max_ext + 1)) for l in M + N + K + Lb}
    la = list(rng.permutation(M + K + Lb)) if M + K + Lb else []
    lb = list(rng.permutation(N + K + Lb)) if N + K + Lb else []
    lc = list(rng.permutation(M + N + Lb)) if M + N + Lb else []
    la, lb, lc = [int(x) for x in la], [int(x) for x in lb], [int(x) for x in lc]
    A, _ = strided(rng, [ext[l] for l in la], integer=integer)
    B, _ = strided(rng, [ext[l] for l in lb], integer=integer)
    C, _ = strided(rng, [ext[l] for l in lc], integer=integer)
    return A, la, B, lb, C, lc


def einsum_ref(alpha, A, la, B, lb, beta, C, lc):
    sym = {}
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    for lab in list(la) + list(lb) + list(lc):
        if lab not in sym:
            sym[lab] = next(letters)
    spec = "".join(sym[l] for l in la) + "," + "".join(sym[l] for l in lb) + "->" + "".join(sym[l] for l in lc)
    return alpha * np.einsum(spec, A, B) + beta * C


# ------------------------------------------------------------------ pins
def test_bruteforce_exact_integer_random_labels():
    rng = np.random.default_rng(11)
    for trial in range(60):
        A, la, B, lb, C, lc = random_problem(rng)
        alpha, beta = float(rng.integers(-3, 4)), float(rng.integers(-3, 4))
        want = brute_force_exact(alpha, A, la, B, lb, beta, C, lc)
        got = C.copy()
        oracle.contract(alpha, A, la, B, lb, beta, got, lc, threads=3)
        assert np.array_equal(got, want), (trial, la, lb, lc)


def test_einsum_second_formulation_float():
    rng = np.random.default_rng(12)
    for trial in range(40):
        A, la, B, lb, C, lc = random_problem(rng, integer=False, max_ext=5)
        want = einsum_ref(0.75, A, la, B, lb, -1.25, C, lc)
        got = C.copy()
        oracle.contract(0.75, A, la, B, lb, -1.25, got, lc)
        scale = np.abs(want).max() if want.size else 1.0
        assert np.allclose(got, want, rtol=0, atol=1e-14 * max(scale, 1.0)), trial


def test_golden_hand_examples():
    blocks, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "name":
            cur = {"name": vals[0]}
            blocks.append(cur)
        else:
            cur[key] = vals
    assert len(blocks) == 2
    for b in blocks:
        lab = lambda k: [ord(c) for c in b[k]]
        ext = lambda k: tuple(int(x) for x in b[k])
        A = np.array([float(x) for x in b["A"]]).reshape(ext("extents_A"), order="F")
        B = np.array([float(x) for x in b["B"]]).reshape(ext("extents_B"), order="F")
        want = np.array([float(x) for x in b["C"]]).reshape(ext("extents_C"), order="F")
        C = np.asfortranarray(np.zeros(ext("extents_C")))
        oracle.contract(1.0, np.asfortranarray(A), lab("labels_A"), np.asfortranarray(B),
                        lab("labels_B"), 0.0, C, lab("labels_C"))
        assert np.array_equal(C, want), b["name"]


def test_gemm_identity_and_all_ones():
    rng = np.random.default_rng(13)
    m, k = 7, 9
    A = rng.uniform(-1, 1, (m, k))
    I = np.eye(k)
    C = np.zeros((m, k))
    oracle.contract(1.0, A, [1, 2], I, [2, 3], 0.0, C, [1, 3])
    assert np.array_equal(C, A)  # A * I == A exactly
    # all-ones operands: every entry is the product of the contracted extents
    A1 = np.ones((3, 4, 5, 6))
    B1 = np.ones((4, 6, 2))
    C1 = np.zeros((3, 5, 2))
    oracle.contract(1.0, A1, [1, 2, 3, 4], B1, [2, 4, 5], 0.0, C1, [1, 3, 5])
    assert np.all(C1 == 24.0)


def test_rank1_closed_form():
    """A = u(x)v(x)w(x)x, B = p(x)q(x)r(x)s  =>  C[a,b,i,j] = (v.p)(x.q) u_a r_b w_i s_j."""
    rng = np.random.default_rng(14)
    e = {"a": 3, "b": 4, "c": 5, "i": 2, "j": 3, "k": 4}
    vec = {n: rng.integers(-3, 4, size=e[n2]).astype(float) for n, n2 in
           zip("uvwxpqrs", "acikckbj")}
    A = np.einsum("a,c,i,k->acik", vec["u"], vec["v"], vec["w"], vec["x"])
    B = np.einsum("c,k,b,j->ckbj", vec["p"], vec["q"], vec["r"], vec["s"])
    C = np.zeros((e["a"], e["b"], e["i"], e["j"]))
    oracle.contract(1.0, A, W.L("acik"), B, W.L("ckbj"), 0.0, C, W.L("abij"))
    coef = float(vec["v"] @ vec["p"]) * float(vec["x"] @ vec["q"])
    want = coef * np.einsum("a,b,i,j->abij", vec["u"], vec["r"], vec["w"], vec["s"])
    assert np.array_equal(C, want)


def test_kronecker_operand_returns_A():
    """B[c,k,b,j] = delta_cb delta_kj  =>  C[a,b,i,j] = A[a,b,i,j] bit-exactly."""
    rng = np.random.default_rng(15)
    n = 5
    A = rng.uniform(-1, 1, (n, n, 3, 4))  # a c i k
    B = np.einsum("cb,kj->ckbj", np.eye(n), np.eye(4))
    C = np.zeros((n, n, 3, 4))
    oracle.contract(1.0, A, W.L("acik"), B, W.L("ckbj"), 0.0, C, W.L("abij"))
    assert np.array_equal(C, A)


def test_relabel_and_permutation_invariance():
    rng = np.random.default_rng(16)
    for trial in range(20):
        A, la, B, lb, C, lc = random_problem(rng)
        ref = C.copy()
        oracle.contract(1.0, A, la, B, lb, 0.0, ref, lc)
        # permute the modes of A (with their strides and labels) and of C
        pa = rng.permutation(A.ndim)
        pc = rng.permutation(C.ndim)
        Ap = A.transpose(pa)
        lap = [la[i] for i in pa]
        Cp = np.zeros(tuple(C.shape[i] for i in pc))
        lcp = [lc[i] for i in pc]
        oracle.contract(1.0, Ap, lap, B, lb, 0.0, Cp, lcp)
        assert np.array_equal(Cp, ref.transpose(pc))
        # swap the operands
        Cs = np.zeros(C.shape)
        oracle.contract(1.0, B, lb, A, la, 0.0, Cs, lc)
        assert np.array_equal(Cs, ref)
        # renaming labels consistently changes nothing
        ren = {l: 1000 + 7 * l for l in set(la) | set(lb) | set(lc)}
        Cr = np.zeros(C.shape)
        oracle.contract(1.0, A, [ren[l] for l in la], B, [ren[l] for l in lb], 0.0, Cr,
                        [ren[l] for l in lc])
        assert np.array_equal(Cr, ref)


def test_power_of_two_scaling_and_linearity():
    p = W.four_index(ext=6, seed=99)
    A, B = p.A.view(), p.B.view()
    rng = np.random.default_rng(17)
    C0 = rng.uniform(-1, 1, (6, 6, 6, 6))
    base = C0.copy()
    oracle.contract(1.0, A, p.A.labels, B, p.B.labels, 1.0, base, p.C.labels)
    scaled = C0.copy()
    oracle.contract(4.0, A, p.A.labels, B, p.B.labels, 4.0, scaled, p.C.labels)
    assert np.array_equal(scaled, 4.0 * base)  # powers of two scale exactly
    c1 = np.zeros(C0.shape)
    c2 = np.zeros(C0.shape)
    c3 = np.zeros(C0.shape)
    oracle.contract(0.3, A, p.A.labels, B, p.B.labels, 0.0, c1, p.C.labels)
    oracle.contract(0.9, A, p.A.labels, B, p.B.labels, 0.0, c2, p.C.labels)
    oracle.contract(1.2, A, p.A.labels, B, p.B.labels, 0.0, c3, p.C.labels)
    assert np.allclose(c3, c1 + c2, rtol=0, atol=1e-13)


def test_alpha_zero_and_beta_zero_conventions():
    A = np.full((3, 4), np.nan)
    B = np.full((4, 2), np.nan)
    C = np.arange(6.0).reshape(3, 2)
    got = C.copy()
    oracle.contract(0.0, A, [1, 2], B, [2, 3], 2.0, got, [1, 3])
    assert np.array_equal(got, 2.0 * C)  # A, B not read
    A = np.ones((3, 4))
    B = np.ones((4, 2))
    got = np.full((3, 2), np.nan)
    oracle.contract(1.0, A, [1, 2], B, [2, 3], 0.0, got, [1, 3])
    assert np.array_equal(got, np.full((3, 2), 4.0))  # C not read


def test_empty_extents_and_scalar_output():
    C = np.arange(6.0).reshape(3, 2)
    got = C.copy()
    oracle.contract(1.0, np.ones((3, 0)), [1, 2], np.ones((0, 2)), [2, 3], 3.0, got, [1, 3])
    assert np.array_equal(got, 3.0 * C)  # empty K: C := beta*C
    empty = np.zeros((0, 2))
    oracle.contract(1.0, np.ones((0, 4)), [1, 2], np.ones((4, 2)), [2, 3], 1.0, empty, [1, 3])
    rng = np.random.default_rng(18)
    a = rng.integers(-4, 5, (3, 4)).astype(float)
    b = rng.integers(-4, 5, (4, 3)).astype(float)
    s = np.zeros(())
    oracle.contract(1.0, a, [1, 2], b, [2, 1], 0.0, s, [])
    assert s == float(sum(a[i, j] * b[j, i] for i in range(3) for j in range(4)))


def test_error_codes():
    A = np.ones((2, 3))
    B = np.ones((3, 4))
    C = np.zeros((2, 4))
    with pytest.raises(oracle.OracleError) as e:
        oracle.contract(1.0, A, [1, 9], B, [2, 3], 0.0, C, [1, 3])  # 9 only in A
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.contract(1.0, A, [1, 1], B, [1, 3], 0.0, C, [1, 3])  # repeated in A
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError) as e:
        oracle.contract(1.0, A, [1, 2], np.ones((5, 4)), [2, 3], 0.0, C, [1, 3])
    assert e.value.code == -3


def test_ieee_inf_nan_propagation():
    rng = np.random.default_rng(19)
    A = rng.uniform(-1, 1, (4, 5))
    B = rng.uniform(-1, 1, (5, 3))
    B[2, 1] = 0.0
    A[1, 2] = np.inf
    A[3, 0] = np.nan
    C = np.zeros((4, 3))
    oracle.contract(1.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3])
    # row 1: inf * (nonzero) -> +-inf, except column 1 where inf*0 = nan
    assert np.isinf(C[1, 0]) and np.isinf(C[1, 2]) and np.isnan(C[1, 1])
    assert np.all(np.isnan(C[3]))
    assert np.all(np.isfinite(C[[0, 2]]))


def test_entries_match_contract_and_dot2_is_accurate():
    p = W.four_index(ext=5, seed=21)
    A, B = p.A.view(), p.B.view()
    rng = np.random.default_rng(22)
    C0 = rng.uniform(-1, 1, (5, 5, 5, 5))
    full = C0.copy()
    oracle.contract(0.5, A, p.A.labels, B, p.B.labels, 2.0, full, p.C.labels)
    idx = rng.integers(0, 5, size=(30, 4))
    e = oracle.entries(0.5, A, p.A.labels, B, p.B.labels, 2.0, C0, p.C.labels, idx)
    assert np.array_equal(e, full[tuple(idx.T)])
    # Dot2 against exact rational arithmetic on an ill-conditioned dot product
    n = 400
    x = rng.uniform(-1, 1, n) * np.exp2(rng.integers(-20, 20, n))
    y = rng.uniform(-1, 1, n)
    x = np.concatenate([x, -x])  # heavy cancellation
    y = np.concatenate([y, y * (1 + 1e-9)])
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
    s = np.zeros(())
    d2 = oracle.entries(1.0, x, [1], y, [1], 0.0, s, [], np.zeros((1, 0), dtype=np.int64), dot2=True)[0]
    plain = oracle.entries(1.0, x, [1], y, [1], 0.0, s, [], np.zeros((1, 0), dtype=np.int64))[0]
    u = 2.0 ** -53
    absdot = float(sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(x, y)))
    gamma = lambda k: k * u / (1 - k * u)
    # Ogita-Rump-Oishi Prop. 5.5: |res - exact| <= u|exact| + gamma_n^2 sum|x_i y_i|
    assert abs(Fraction(d2) - exact) <= Fraction(u) * abs(exact) + Fraction(gamma(2 * n) ** 2 * absdot)
    # plain recursive sum: |res - exact| <= gamma_n sum|x_i y_i|
    assert abs(Fraction(plain) - exact) <= Fraction(gamma(2 * n) * absdot)
    assert abs(Fraction(d2) - exact) < abs(Fraction(plain) - exact) or plain == float(exact)


def test_planted_transpose_is_caught():
    """A plausible oracle bug (a transposed operand) must fail the einsum pin."""
    rng = np.random.default_rng(23)
    A = rng.uniform(-1, 1, (4, 4))
    B = rng.uniform(-1, 1, (4, 4))
    want = einsum_ref(1.0, A, [1, 2], B, [2, 3], 0.0, np.zeros((4, 4)), [1, 3])
    wrong = np.zeros((4, 4))
    oracle.contract(1.0, A.T, [1, 2], B, [2, 3], 0.0, wrong, [1, 3])  # the planted mistake
    assert not np.allclose(wrong, want)


def test_workload_generators_shapes():
    p = W.transpose_free(v=6, o=3, pad=7)
    assert p.A.strides == (1, 13, 13 * 6, 13 * 6 * 3)
    assert p.flops == 2 * 6 ** 3 * 3 ** 3
    lad = W.ladder(v=4, o=2)
    V = lad.A.view()
    assert np.array_equal(V, V.transpose(2, 3, 0, 1))  # (ab)<->(cd) symmetry
    blocks = W.block_sparse(nblocks=5)
    assert all(set(b.meta["ext"]) <= set(range(8, 97, 8)) for b in blocks)


# ---------------------------------------------------------------------------
# Sandwiched product C := beta C + alpha A T A^T, lower triangle (gemmt_tridiag)
# ---------------------------------------------------------------------------

def _dense_tridiag(k, sub, diag, sup):
    T = [[0] * k for _ in range(k)]
    for p in range(k):
        if diag is not None:
            T[p][p] = diag[p]
        if p + 1 < k:
            T[p + 1][p] = sub[p]
            T[p][p + 1] = -sub[p] if sup is None else sup[p]
    return T


@pytest.mark.parametrize("n,k,skew", [(5, 4, True), (6, 7, False), (3, 1, False), (4, 2, True)])
def test_gemmt_bruteforce_exact_integer(n, k, skew):
    """Every (p, q) of the dense T summed in Python integers (off-band zeros
    included): the oracle's banded two-step evaluation is exact on small
    integers."""
    rng = np.random.default_rng(900 + n * 10 + k)
    A = rng.integers(-3, 4, size=(n, k))
    sub = rng.integers(-3, 4, size=max(k - 1, 0))
    diag = None if skew else rng.integers(-3, 4, size=k)
    sup = None if skew else rng.integers(-3, 4, size=max(k - 1, 0))
    C0 = rng.integers(-5, 6, size=(n, n)).astype(np.float64)
    alpha, beta = -1, 2
    T = _dense_tridiag(k, [int(x) for x in sub], None if diag is None else [int(x) for x in diag],
                       None if sup is None else [int(x) for x in sup])
    want = C0.copy()
    for i in range(n):
        for j in range(i + 1):
            s = sum(int(A[i, p]) * T[p][q] * int(A[j, q]) for p in range(k) for q in range(k))
            want[i, j] = alpha * s + beta * C0[i, j]
    got = oracle.gemmt_tridiag(alpha, A.astype(np.float64), sub, diag, sup, beta, C0.copy())
    assert np.array_equal(got, want)


def test_gemmt_identity_gives_lower_triangle_of_T():
    """A = I: A T A^T = T, so C's lower triangle becomes T's: the diagonal
    and the subdiagonal, never the superdiagonal (a swapped sub/sup or a
    transposed product fails here)."""
    k = 6
    sub = np.arange(1.0, k)
    diag = np.arange(10.0, 10.0 + k)
    sup = -np.arange(100.0, 100.0 + k - 1)
    C = np.full((k, k), 7.0)
    oracle.gemmt_tridiag(1.0, np.eye(k), sub, diag, sup, 0.0, C)
    for i in range(k):
        for j in range(k):
            if i < j:
                assert C[i, j] == 7.0  # upper triangle untouched
            elif i == j:
                assert C[i, j] == diag[i]
            elif i == j + 1:
                assert C[i, j] == sub[j]
            else:
                assert C[i, j] == 0.0


def test_gemmt_permutation_permutes_T():
    """A = the permutation matrix of pi: (A T A^T)[i, j] = T[pi(i), pi(j)]."""
    k = 7
    rng = np.random.default_rng(910)
    pi = rng.permutation(k)
    P = np.zeros((k, k))
    P[np.arange(k), pi] = 1.0
    sub, diag, sup = rng.standard_normal(k - 1), rng.standard_normal(k), rng.standard_normal(k - 1)
    T = np.array(_dense_tridiag(k, list(sub), list(diag), list(sup)), dtype=np.float64)
    C = np.zeros((k, k))
    oracle.gemmt_tridiag(1.0, P, sub, diag, sup, 0.0, C)
    for i in range(k):
        for j in range(i + 1):
            assert C[i, j] == T[pi[i], pi[j]]


def test_gemmt_k1_outer_product_and_skew_zero_diagonal():
    """k = 1: C = beta C + alpha d a a^T (lower).  Skew-symmetric T with
    integer A: A T A^T is skew-symmetric, so its diagonal is exactly 0."""
    a = np.array([[1.0], [-2.0], [3.0]])
    C = np.ones((3, 3))
    oracle.gemmt_tridiag(2.0, a, None, np.array([5.0]), None, 1.0, C)
    want = np.tril(1.0 + 10.0 * (a @ a.T)) + np.triu(np.ones((3, 3)), 1)
    assert np.array_equal(C, want)
    rng = np.random.default_rng(920)
    A = rng.integers(-9, 10, size=(8, 11)).astype(np.float64)
    sub = rng.integers(-9, 10, size=10).astype(np.float64)
    C = np.zeros((8, 8))
    oracle.gemmt_tridiag(1.0, A, sub, None, None, 0.0, C)
    assert np.all(np.diag(C) == 0.0)
    assert np.any(np.tril(C, -1) != 0.0)


def test_gemmt_alpha_beta_conventions():
    """alpha == 0 reads no A (NaN in A ignored), beta == 0 reads no C (NaN in
    C overwritten); the strictly upper triangle is never touched."""
    A = np.full((4, 3), np.nan)
    C = np.arange(16.0).reshape(4, 4)
    C0 = C.copy()
    oracle.gemmt_tridiag(0.0, A, np.ones(2), None, None, 0.5, C)
    assert np.array_equal(np.tril(C), 0.5 * np.tril(C0))
    assert np.array_equal(np.triu(C, 1), np.triu(C0, 1))
    A = np.ones((4, 3))
    C = np.full((4, 4), np.nan)
    oracle.gemmt_tridiag(1.0, A, np.ones(2), None, np.ones(2), 0.0, C)
    iu = np.triu_indices(4, 1)
    assert not np.isnan(np.tril(C)).any()
    assert np.isnan(C[iu]).all()


# ---------------------------------------------------------------------------
# Matricised tensor times Khatri-Rao product (mttkrp)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,mode", [((3, 4, 5), 0), ((3, 4, 5), 1), ((3, 4, 5), 2), ((2, 3, 2, 3), 2)])
def test_mttkrp_bruteforce_exact_integer(shape, mode):
    """Every index tuple of X summed in Python integers."""
    rng = np.random.default_rng(1100 + sum(shape) + mode)
    R = 3
    X = rng.integers(-3, 4, size=shape)
    U = [rng.integers(-3, 4, size=(e, R)) for e in shape]
    M0 = rng.integers(-5, 6, size=(shape[mode], R)).astype(np.float64)
    want = M0.copy()
    for i in range(shape[mode]):
        for r in range(R):
            s = 0
            for idx in itertools.product(*[range(e) for e in shape]):
                if idx[mode] != i:
                    continue
                t = int(X[idx])
                for m, im in enumerate(idx):
                    if m != mode:
                        t *= int(U[m][im, r])
                s += t
            want[i, r] = 2 * s - 1 * M0[i, r]
    got = oracle.mttkrp(2.0, X.astype(np.float64), mode, [u.astype(np.float64) for u in U], -1.0, M0.copy())
    assert np.array_equal(got, want)


def test_mttkrp_rank_one_closed_form():
    """X = a o b o c (outer product): M[i, r] = a[i] (b . U1[:, r]) (c . U2[:, r])
    for mode 0, and the analogous products for modes 1 and 2."""
    rng = np.random.default_rng(1110)
    a, b, c = rng.standard_normal(6), rng.standard_normal(5), rng.standard_normal(4)
    X = np.einsum("i,j,k->ijk", a, b, c)
    U = [rng.standard_normal((6, 3)), rng.standard_normal((5, 3)), rng.standard_normal((4, 3))]
    vecs = [a, b, c]
    for mode in range(3):
        M = np.zeros((X.shape[mode], 3))
        oracle.mttkrp(1.0, X, mode, U, 0.0, M)
        want = vecs[mode][:, None] * np.prod([vecs[m] @ U[m] for m in range(3) if m != mode], axis=0)[None, :]
        assert np.allclose(M, want, rtol=1e-13, atol=1e-13)


def test_mttkrp_two_way_is_a_matrix_product():
    """N = 2: mode 0 gives X U1, mode 1 gives X^T U0 (a transposed operand
    would fail on the non-square X)."""
    rng = np.random.default_rng(1120)
    X = rng.integers(-4, 5, size=(5, 7)).astype(np.float64)
    U0, U1 = rng.integers(-4, 5, size=(5, 2)).astype(np.float64), rng.integers(-4, 5, size=(7, 2)).astype(np.float64)
    M = np.zeros((5, 2))
    assert np.array_equal(oracle.mttkrp(1.0, X, 0, [None, U1], 0.0, M), X @ U1)
    M = np.zeros((7, 2))
    assert np.array_equal(oracle.mttkrp(1.0, X, 1, [U0, None], 0.0, M), X.T @ U0)


def test_mttkrp_all_ones_factors_sum_the_other_modes():
    """R = 1 and all-ones factors: M[i, 0] is the sum of X over the other modes."""
    rng = np.random.default_rng(1130)
    X = rng.integers(-9, 10, size=(4, 3, 5, 2)).astype(np.float64)
    U = [np.ones((e, 1)) for e in X.shape]
    M = np.zeros((5, 1))
    oracle.mttkrp(1.0, X, 2, U, 0.0, M)
    assert np.array_equal(M[:, 0], X.sum(axis=(0, 1, 3)))
