"""GPU parity of the sandwiched product C := beta C + alpha A T A^T (T
tridiagonal, lower triangle of C only; Sec. 3, "Beyond LAPACK
functionality") against the oracle's two-step evaluation."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm

from gpu_util import rel_frob

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64_emu": 1e-13, "f32": 1e-5}
DT = {"f64": torch.float64, "f64_emu": torch.float64, "f32": torch.float32}


def _case(rng, n, k, skew=True, row_major_a=False, row_major_c=False, dt=torch.float64):
    A = rng.uniform(-1.0, 1.0, size=(n, k))
    sub = rng.uniform(-1.0, 1.0, size=max(k - 1, 0))
    diag = None if skew else rng.uniform(-1.0, 1.0, size=k)
    sup = None if skew else rng.uniform(-1.0, 1.0, size=max(k - 1, 0))
    C = rng.uniform(-1.0, 1.0, size=(n, n))
    # the device sees values rounded to its dtype; the oracle gets the same values
    r = lambda x: None if x is None else torch.from_numpy(x).to(dt).to(torch.float64).numpy()
    A, sub, diag, sup, C = r(A), r(sub), r(diag), r(sup), r(C)
    Ad = torch.from_numpy(A).to("cuda", dt)
    if not row_major_a:
        Ad = Ad.t().contiguous().t()  # column-major: unit stride along i
    Cd = torch.from_numpy(C).to("cuda", dt)
    if not row_major_c:
        Cd = Cd.t().contiguous().t()
    dev = lambda x: None if x is None else torch.from_numpy(x).to("cuda", dt)
    return (A, sub, diag, sup, C), (Ad, dev(sub), dev(diag), dev(sup), Cd)


def _check(host, devs, alpha, beta, dtype):
    A, sub, diag, sup, C = host
    Ad, sd, dd, ud, Cd = devs
    _, info = fm.gemmt_tridiag(alpha, Ad, sd, dd, ud, beta, Cd, dtype=dtype, return_info=True)
    torch.cuda.synchronize()
    got = Cd.to(torch.float64).cpu().numpy()
    want = oracle.gemmt_tridiag(alpha, A, sub, diag, sup, beta, C.copy())
    low = np.tril(np.ones_like(C, dtype=bool))
    assert np.array_equal(got[~low], C[~low])  # strictly upper triangle untouched
    assert rel_frob(got[low], want[low]) <= TOL[dtype]
    assert fm.device_status() == 0
    return info


@pytest.mark.parametrize("dtype", ["f64_emu", "f64", "f32"])
def test_skew_update_ragged(dtype):
    """C := C - A T A^T, T skew-symmetric (the LTL^T update), n and k not
    multiples of any tile."""
    rng = np.random.default_rng(1000)
    host, devs = _case(rng, 300, 201, dt=DT[dtype])
    info = _check(host, devs, -1.0, 1.0, dtype)
    assert info["kernel_name"] == {"f64_emu": "tc_emu", "f64": "simt_f64", "f32": "tc_tf32x3"}[dtype]


@pytest.mark.parametrize("dtype", ["f64_emu", "f64", "f32"])
def test_general_tridiagonal_row_major_c(dtype):
    """A general tridiagonal T (own diagonal and superdiagonal) and a
    row-major C: the planner puts C's unit stride (j) on the kernel's rows,
    so the banded operand becomes the row operand and the kept triangle
    row <= col in the kernel's indices."""
    rng = np.random.default_rng(1001)
    host, devs = _case(rng, 260, 130, skew=False, row_major_c=True, dt=DT[dtype])
    info = _check(host, devs, 0.75, -0.5, dtype)
    assert info["swapped"] == 1


def test_row_major_a_and_many_tiles():
    """A row-major (unit stride along p) and n = 1500: many tiles of the
    triangle over several rounds of the persistent grid."""
    rng = np.random.default_rng(1002)
    host, devs = _case(rng, 1500, 700, row_major_a=True)
    _check(host, devs, -1.0, 1.0, "f64_emu")


@pytest.mark.parametrize("dtype", ["f64_emu", "f32", "f64"])
def test_few_tiles_long_k_splits_k(dtype):
    """n = 200 (two tiles of the triangle), k = 20000: the product splits K
    across the SMs and the finishing kernel writes the triangle."""
    rng = np.random.default_rng(1003)
    host, devs = _case(rng, 200, 20000, dt=DT[dtype])
    info = _check(host, devs, -1.0, 1.0, dtype)
    # tables, tile list, packs (+ exponents), product, split finish (+ fix-up)
    assert info["launches"] + info["cached"] == {"f64_emu": 9, "f32": 6, "f64": 3}[dtype]


def test_nan_in_a_reaches_its_row_and_column():
    """A NaN in row r of A makes row r and column r of A T A^T NaN (through
    the row operand and through T A^T); the fix-up recomputes them natively
    inside the triangle, matching the oracle's NaN pattern."""
    rng = np.random.default_rng(1004)
    host, devs = _case(rng, 150, 90)
    A, sub, diag, sup, C = host
    A[40, 17] = np.nan
    devs[0][40, 17] = float("nan")
    Ad, sd, dd, ud, Cd = devs
    fm.gemmt_tridiag(-1.0, Ad, sd, dd, ud, 1.0, Cd, dtype="f64_emu")
    torch.cuda.synchronize()
    got = Cd.cpu().numpy()
    want = oracle.gemmt_tridiag(-1.0, A, sub, diag, sup, 1.0, C.copy())
    low = np.tril(np.ones_like(C, dtype=bool))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.isnan(want[40, :41]).all() and np.isnan(want[40:, 40]).all()
    fin = low & ~np.isnan(want)
    assert rel_frob(got[fin], want[fin]) <= 1e-13
    assert np.array_equal(got[~low], C[~low])


@pytest.mark.parametrize("dtype", ["f64_emu", "f64"])
def test_scale_only_and_empty(dtype):
    """alpha = 0 (and k = 0) scale the triangle only; beta = 0 overwrites a
    NaN-filled triangle; n = 0 is a no-op."""
    rng = np.random.default_rng(1005)
    host, devs = _case(rng, 70, 30)
    A, sub, diag, sup, C = host
    Ad, sd, dd, ud, Cd = devs
    fm.gemmt_tridiag(0.0, Ad, sd, dd, ud, 0.5, Cd, dtype=dtype)
    torch.cuda.synchronize()
    low = np.tril(np.ones_like(C, dtype=bool))
    got = Cd.cpu().numpy()
    assert np.array_equal(got[low], 0.5 * C[low]) and np.array_equal(got[~low], C[~low])
    Cn = torch.full((70, 70), float("nan"), dtype=torch.float64, device="cuda")
    fm.gemmt_tridiag(1.0, Ad, sd, dd, ud, 0.0, Cn, dtype=dtype)
    want = oracle.gemmt_tridiag(1.0, A, sub, diag, sup, 0.0, np.full((70, 70), np.nan))
    got = Cn.cpu().numpy()
    assert not np.isnan(got[low]).any() and np.isnan(got[~low]).all()
    assert rel_frob(got[low], want[low]) <= 1e-13
    E = torch.empty((0, 5), dtype=torch.float64, device="cuda")
    fm.gemmt_tridiag(1.0, E, sd, dd, ud, 1.0, torch.empty((0, 0), dtype=torch.float64, device="cuda"),
                     dtype=dtype)
    torch.cuda.synchronize()


def test_full_size_panel_update():
    """The benchmark's panel update, n = 16384, k = 256, emulated fp64 in the
    launch configuration the benchmark times, against the oracle on the
    whole lower triangle."""
    rng = np.random.default_rng(1010)
    n, k = 16384, 256
    A = rng.standard_normal((n, k))
    sub = rng.standard_normal(k - 1)
    Ad = torch.from_numpy(A).cuda().t().contiguous().t()
    sd = torch.from_numpy(sub).cuda()
    C = rng.standard_normal((n, n))
    Cd = torch.from_numpy(C).cuda().t().contiguous().t()
    fm.gemmt_tridiag(-1.0, Ad, sd, None, None, 1.0, Cd, dtype="f64_emu")
    torch.cuda.synchronize()
    got = Cd.cpu().numpy()
    del Cd
    want = oracle.gemmt_tridiag(-1.0, A, sub, None, None, 1.0, C.copy())
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.array_equal(got[~low], C[~low])
    assert rel_frob(got[low], want[low]) <= 1e-13
