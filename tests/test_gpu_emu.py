"""GPU parity of the split-precision fp64 path (bf16 integer slices on the
tensor cores, exact fp32 accumulation, fp64 recombination) against the FP64
oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle, random_label_problem, to_device

pytestmark = pytest.mark.gpu

TOL = 1e-13  # relative Frobenius tolerance for fp64 and emulated fp64


def _alpha_part(p, want):
    """alpha*contract(A,B) part of the reference (want - beta*C_in)."""
    return want - p.beta * np.array(p.C.view())


def test_ladder_reduced():
    p = W.ladder(v=32, o=8)
    C, info = run_gpu(p, "f64_emu")
    assert info["kernel_name"] == "tc_emu" and info["slices"] == 6
    want = run_oracle(p)
    got = gpu_dense(C)
    assert rel_frob(got, want) <= TOL
    # stricter: error relative to the contraction term alone
    ab = _alpha_part(p, want)
    assert np.linalg.norm(got - want) / np.linalg.norm(ab) <= 1e-12


@pytest.mark.parametrize("tile_n", [64, 128, 256])
def test_four_index_tiles(tile_n):
    p = W.four_index(ext=16)
    C, _ = run_gpu(p, "f64_emu", tile_n=tile_n)
    assert rel_frob(gpu_dense(C), run_oracle(p)) <= TOL


def test_integer_inputs_exact():
    p = W.four_index(ext=16, integer=True)
    C, _ = run_gpu(p, "f64_emu")
    assert np.array_equal(gpu_dense(C), run_oracle(p))
    rng = np.random.default_rng(400)
    for _ in range(12):
        q = random_label_problem(rng, max_ext=6)
        Cq, info = run_gpu(q, "f64_emu")
        assert np.array_equal(gpu_dense(Cq), run_oracle(q)), info


def test_error_falls_with_slice_count():
    """Each extra 8-bit slice shrinks the truncation error until fp64 rounding
    is reached (the split converges to the exact product).  The reference is
    the oracle's compensated dot product (Dot2, twice the working precision),
    whose own error lies far below fp64 rounding, so the floor is the GPU
    result's final rounding to fp64: about 2^-53 per entry, 4e-16 in relative
    Frobenius norm with margin."""
    rng = np.random.default_rng(401)
    m, n, k = 256, 192, 640
    A = W.uniform_operand(rng, (m, k), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.zeros_operand((m, n), [1, 3])
    p = W.Problem("gemm", 1.0, A, B, 0.0, C)
    idx = np.stack(np.meshgrid(np.arange(m), np.arange(n), indexing="ij"), axis=-1).reshape(-1, 2)
    want = oracle.entries(p.alpha, A.view(), A.labels, B.view(), B.labels, p.beta, C.view(),
                          C.labels, idx, dot2=True).reshape(m, n)
    errs = []
    for s in range(2, 8):
        Cg, info = run_gpu(p, "f64_emu", slices=s)
        assert info["slices"] == s
        errs.append(rel_frob(gpu_dense(Cg), want))
    for a, b in zip(errs, errs[1:]):
        assert b <= max(a / 16, 4e-16), errs  # 4e-16: fp64 rounding floor of the result
    assert errs[-1] <= 4e-16


def test_nonfinite_rows_follow_ieee():
    rng = np.random.default_rng(402)
    m, n, k = 130, 70, 90
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    A[3, 5] = np.inf
    A[100, 0] = np.nan
    B[7, 20] = -np.inf
    B[:, 33] = 0.0
    B[2, 33] = np.inf          # inf * 0 in column 33 for every finite row
    want = np.zeros((m, n))
    oracle.contract(1.0, A, [1, 2], B, [2, 3], 0.0, want, [1, 3])
    C = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    fm.contract(1.0, torch.from_numpy(A).cuda(), [1, 2], torch.from_numpy(B).cuda(), [2, 3], 0.0, C,
                [1, 3], dtype="f64_emu")
    got = C.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isposinf(got), np.isposinf(want))
    assert np.array_equal(np.isneginf(got), np.isneginf(want))
    fin = np.isfinite(want)
    assert rel_frob(got[fin], want[fin]) <= TOL


def test_wide_exponent_range_per_row_scaling():
    rng = np.random.default_rng(403)
    m, n, k = 150, 140, 300
    A = rng.uniform(-1, 1, (m, k)) * np.exp2(rng.integers(-300, 300, (m, 1)))
    B = rng.uniform(-1, 1, (k, n)) * np.exp2(rng.integers(-200, 200, (1, n)))
    want = np.zeros((m, n))
    oracle.contract(1.0, A, [1, 2], B, [2, 3], 0.0, want, [1, 3])
    C = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    fm.contract(1.0, torch.from_numpy(A).cuda(), [1, 2], torch.from_numpy(B).cuda(), [2, 3], 0.0, C,
                [1, 3], dtype="f64_emu")
    got = C.cpu().numpy()
    # every entry carries its own scale 2^(e_m + e_n): compare scale-free
    scale = np.abs(A).max(1)[:, None] * np.abs(B).max(0)[None, :]
    assert np.abs((got - want) / scale).max() <= 1e-13 * np.sqrt(k)


def test_alpha_beta_conventions():
    rng = np.random.default_rng(404)
    A = torch.from_numpy(rng.uniform(-1, 1, (40, 30))).cuda()
    B = torch.from_numpy(rng.uniform(-1, 1, (30, 20))).cuda()
    C = torch.full((40, 20), float("nan"), dtype=torch.float64, device="cuda")
    fm.contract(2.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3], dtype="f64_emu")
    want = 2.0 * (A @ B)
    assert torch.isfinite(C).all()
    assert (C - want).norm() / want.norm() <= TOL
    C0 = torch.from_numpy(rng.uniform(-1, 1, (40, 20))).cuda()
    C = C0.clone()
    fm.contract(0.0, A * float("nan"), [1, 2], B, [2, 3], 0.5, C, [1, 3], dtype="f64_emu")
    assert torch.equal(C, 0.5 * C0)


def test_batch_labels():
    rng = np.random.default_rng(405)
    A = W.uniform_operand(rng, (70, 50, 3), [1, 2, 3])
    B = W.uniform_operand(rng, (50, 90, 3), [2, 4, 3])
    C = W.uniform_operand(rng, (70, 90, 3), [1, 4, 3])
    p = W.Problem("batched", -1.5, A, B, 0.25, C)
    Cg, info = run_gpu(p, "f64_emu")
    assert info["batch"] == 3
    assert rel_frob(gpu_dense(Cg), run_oracle(p)) <= TOL


def test_full_ladder_sampled_dot2():
    """The v=128, o=32 ladder (GEMM 16384 x 1024 x 16384 after fusion) in the
    benchmark's launch configuration; 4096 sampled entries against the
    compensated (Dot2) oracle."""
    p = W.ladder(v=128, o=32)
    C, info = run_gpu(p, "f64_emu")
    assert (info["m"], info["n"], info["k"]) == (16384, 1024, 16384)
    got_all = gpu_dense(C)
    rng = np.random.default_rng(406)
    idx = np.stack([rng.integers(0, e, 4096) for e in p.C.extents], axis=1)
    want = oracle.entries(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta,
                          p.C.view(), p.C.labels, idx, dot2=True)
    got = got_all[tuple(idx.T)]
    assert rel_frob(got, want) <= TOL
    ab = want - p.beta * p.C.view()[tuple(idx.T)]
    assert np.linalg.norm(got - want) / np.linalg.norm(ab) <= 1e-12


def test_long_k_tile_sums_stay_accurate():
    """K = 2^20: the int64 tile sums take a coarser unit (their bound grows
    with K) and round the least significant diagonals; sampled entries still
    meet the fp64 bound against the oracle's compensated dot products."""
    rng = np.random.default_rng(405)
    m, n, k = 130, 66, 1 << 20
    A = W.uniform_operand(rng, (m, k), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.uniform_operand(rng, (m, n), [1, 3])
    p = W.Problem("long_k", 1.0, A, B, 0.5, C)
    Cg, _ = run_gpu(p, "f64_emu")
    got = gpu_dense(Cg)
    idx = np.stack([rng.integers(0, m, 64), rng.integers(0, n, 64)], axis=1)
    want = oracle.entries(p.alpha, A.view(), A.labels, B.view(), B.labels, p.beta, C.view(),
                          C.labels, idx, dot2=True)
    assert rel_frob(got[idx[:, 0], idx[:, 1]], want) <= TOL


def test_split_k_few_tiles_with_nonfinite_row():
    """Two output tiles and K = 16384: the k range is split across CTAs, the
    splits add into one int64 sum per tile (exact, in any order) and a
    finishing kernel writes C; a row holding NaN still goes to the native
    fix-up."""
    rng = np.random.default_rng(406)
    m, n, k = 200, 100, 16384
    A = rng.uniform(-1, 1, (m, k))
    A[17, 5000] = np.nan
    Aop = W.Operand(np.asfortranarray(A).reshape(-1, order="F").copy(), (m, k), (1, m), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.uniform_operand(rng, (m, n), [1, 3])
    p = W.Problem("split_k_emu", -0.5, Aop, B, 2.0, C)
    Cg, info = run_gpu(p, "f64_emu")
    # tables, A's exponents and pack, B's one-pass split (k unit-stride),
    # product, split finish, fix-up
    assert info["launches"] + info["cached"] == 7
    got, want = gpu_dense(Cg), run_oracle(p)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = ~np.isnan(want)
    assert rel_frob(got[fin], want[fin]) <= TOL


def test_split_every_tile_over_several_rounds():
    """178 tiles on 148 SMs: rather than a whole round plus a 30-tile tail,
    every tile splits K in four (712 items, 1.25 rounds of work instead of 2)
    and meets in its int64 slot; sampled entries against the oracle's
    compensated dot products."""
    rng = np.random.default_rng(407)
    m, n, k = 89 * 128, 512, 2048
    A = W.uniform_operand(rng, (m, k), [1, 2])
    B = W.uniform_operand(rng, (k, n), [2, 3])
    C = W.uniform_operand(rng, (m, n), [1, 3])
    p = W.Problem("split_tail_emu", 1.0, A, B, -1.0, C)
    Cg, info = run_gpu(p, "f64_emu", tile_n=256)
    # tables, A's exponents and pack, B's one-pass split, product, split finish, fix-up
    assert info["launches"] + info["cached"] == 7
    got = gpu_dense(Cg)
    rows = np.concatenate([rng.integers(74 * 128, m, 48), rng.integers(0, 74 * 128, 16)])
    idx = np.stack([rows, rng.integers(0, n, rows.size)], axis=1)
    want = oracle.entries(p.alpha, A.view(), A.labels, B.view(), B.labels, p.beta, C.view(),
                          C.labels, idx, dot2=True)
    assert rel_frob(got[idx[:, 0], idx[:, 1]], want) <= TOL


@pytest.mark.parametrize("k,deferred", [(512, True), (513, False)])
def test_short_k_finish_boundary_integer_exact(k, deferred):
    """m = n = 2048 (128 tiles of 128 x 256): up to K = 512 every tile's int64
    sums go to its own slot and a separate kernel finishes them (seven
    launches: tables, A's exponents and pack, B's one-pass split, product,
    finish, fix-up); from K = 513 the tiles finish inside the product (six).  Integer-valued inputs, alpha and beta
    that are not 0 or 1 and a row holding Inf: both sides exact."""
    rng = np.random.default_rng(408 + k)
    m = n = 2048
    A = rng.integers(-4, 5, (m, k)).astype(np.float64)
    A[77, 3] = np.inf
    Aop = W.Operand(np.asfortranarray(A).reshape(-1, order="F").copy(), (m, k), (1, m), [1, 2])
    B = W.Operand(rng.integers(-4, 5, k * n).astype(np.float64), (k, n), (1, k), [2, 3])
    C = W.Operand(rng.integers(-4, 5, m * n).astype(np.float64), (m, n), (1, m), [1, 3])
    p = W.Problem("short_k_boundary", 0.5, Aop, B, -2.0, C)
    Cg, info = run_gpu(p, "f64_emu", tile_n=256)
    assert info["launches"] + info["cached"] == (7 if deferred else 6), info
    got, want = gpu_dense(Cg), run_oracle(p)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    assert np.array_equal(got[fin], want[fin])


@pytest.mark.parametrize("alpha", [2.0 ** -40, -(2.0 ** 30), 2.0 ** -1040, 3.0, -1.0])
@pytest.mark.parametrize("beta", [0.0, 1.0, -0.25])
@pytest.mark.parametrize("k", [200, 520, 4096])
def test_alpha_beta_kinds_exact(alpha, beta, k):
    """alpha = +-2^p goes into the int64 sums' sign and the scaling exponent
    (integer arithmetic), any other alpha (3, or the subnormal 2^-1040) takes
    one multiply; beta 0, 1 and -0.25 each have their own finish.  Integer
    inputs keep every product, sum and scaling exact, so the result equals
    the oracle's bit for bit.  k = 200: the deferred finish (a separate
    kernel); k = 520: whole tiles finished inside the product; k = 4096: K
    split across the SMs, the separate kernel again."""
    rng = np.random.default_rng(420 + k)
    m, n = 300, 200
    A = W.Operand(rng.integers(-6, 7, m * k).astype(np.float64), (m, k), (1, m), [1, 2])
    B = W.Operand(rng.integers(-6, 7, k * n).astype(np.float64), (k, n), (1, k), [2, 3])
    C = W.Operand(rng.integers(-6, 7, m * n).astype(np.float64), (m, n), (1, m), [1, 3])
    p = W.Problem("alpha_beta_kinds", alpha, A, B, beta, C)
    Cg, info = run_gpu(p, "f64_emu")
    assert np.array_equal(gpu_dense(Cg), run_oracle(p))
    # in-product finish: no separate finishing launch (tables, exponents,
    # pack, B's one-pass split, product, fix-up)
    if k == 520:
        assert info["launches"] + info["cached"] == 6
