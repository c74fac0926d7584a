"""GPU parity of the tensor-factorisation inner contractions (Sec. 3, Girder
5: CP-ALS and HOOI): the matricised tensor times Khatri-Rao product with the
Khatri-Rao operand generated while it is packed, and a HOOI projection as a
pre-ordered network of tensor-times-matrix contractions, against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import rel_frob, to_device

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f64_emu": 1e-13, "f32": 1e-5}
DT = {"f64": torch.float64, "f64_emu": torch.float64, "f32": torch.float32}


def _round(x, dt):
    return torch.from_numpy(x).to(dt).to(torch.float64).numpy()


def _run(rng, shape, mode, R, dtype, alpha=1.0, beta=0.5, x_perm=None, m_row_major=False):
    dt = DT[dtype]
    X = _round(rng.uniform(-1.0, 1.0, size=shape), dt)
    U = [_round(rng.uniform(-1.0, 1.0, size=(e, R)), dt) for e in shape]
    M = _round(rng.uniform(-1.0, 1.0, size=(shape[mode], R)), dt)
    Xd = torch.from_numpy(X).to("cuda", dt)
    if x_perm is not None:  # same values, another memory order
        Xd = Xd.permute(*x_perm).contiguous().permute(*[int(i) for i in np.argsort(x_perm)])
    Ud = [torch.from_numpy(u).to("cuda", dt).t().contiguous().t() for u in U]  # column-major factors
    Md = torch.from_numpy(M).to("cuda", dt)
    if not m_row_major:
        Md = Md.t().contiguous().t()
    _, info = fm.mttkrp(alpha, Xd, mode, [None if m == mode else Ud[m] for m in range(len(shape))], beta,
                        Md, dtype=dtype, return_info=True)
    torch.cuda.synchronize()
    want = oracle.mttkrp(alpha, X, mode, U, beta, M.copy())
    return Md.to(torch.float64).cpu().numpy(), want, info


@pytest.mark.parametrize("dtype", ["f64_emu", "f64", "f32"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mttkrp_three_way_every_mode(dtype, mode):
    """A ragged 3-way tensor, each mode in turn (modes 1 and 2 leave the
    other two modes unfusable in X's layout for mode 1)."""
    rng = np.random.default_rng(1200 + mode)
    got, want, info = _run(rng, (70, 45, 33), mode, 20, dtype)
    assert rel_frob(got, want) <= TOL[dtype]
    assert info["kernel_name"] == {"f64_emu": "tc_emu", "f64": "simt_f64", "f32": "tc_tf32x3"}[dtype]
    assert fm.device_status() == 0


def test_mttkrp_four_way_permuted_x_row_major_m():
    """A 4-way X stored in a permuted order and a row-major M (the planner
    puts r on the kernel's rows, so the Khatri-Rao operand is the row
    operand)."""
    rng = np.random.default_rng(1210)
    got, want, info = _run(rng, (12, 9, 14, 11), 2, 33, "f64_emu", alpha=-2.0, beta=1.0,
                           x_perm=(3, 1, 0, 2), m_row_major=True)
    assert info["swapped"] == 1
    assert rel_frob(got, want) <= 1e-13


@pytest.mark.parametrize("dtype", ["f64_emu", "f32"])
def test_mttkrp_tall_k_splits_k(dtype):
    """I_mode = 200 rows, R = 16, the other modes 160 x 150: two tiles with a
    24000-long K, split across the SMs."""
    rng = np.random.default_rng(1220)
    got, want, info = _run(rng, (200, 160, 150), 0, 16, dtype)
    assert rel_frob(got, want) <= TOL[dtype]


def test_mttkrp_nan_in_a_factor_reaches_its_column():
    """A NaN in U[1][j, r] makes column r of the Khatri-Rao operand hold NaN,
    so column r of M is NaN (recomputed natively by the fix-up); the other
    columns match the oracle."""
    rng = np.random.default_rng(1230)
    shape, mode, R = (40, 30, 20), 0, 8
    X = rng.uniform(-1.0, 1.0, size=shape)
    U = [rng.uniform(-1.0, 1.0, size=(e, R)) for e in shape]
    U[1][7, 3] = np.nan
    M = rng.uniform(-1.0, 1.0, size=(40, R))
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda() for u in U]
    Md = torch.from_numpy(M).cuda().t().contiguous().t()
    fm.mttkrp(1.0, Xd, mode, [None, Ud[1], Ud[2]], 1.0, Md, dtype="f64_emu")
    torch.cuda.synchronize()
    got = Md.cpu().numpy()
    want = oracle.mttkrp(1.0, X, mode, U, 1.0, M.copy())
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.isnan(want[:, 3]).all()
    fin = ~np.isnan(want)
    assert rel_frob(got[fin], want[fin]) <= 1e-13


def test_mttkrp_scale_only_and_two_way():
    """alpha = 0 scales M without reading X or the factors; N = 2 is X U."""
    rng = np.random.default_rng(1240)
    M = torch.rand(30, 5, dtype=torch.float64, device="cuda")
    M0 = M.clone()
    X = torch.full((30, 8), float("nan"), dtype=torch.float64, device="cuda")
    U1 = torch.full((8, 5), float("nan"), dtype=torch.float64, device="cuda")
    fm.mttkrp(0.0, X, 0, [None, U1], 0.25, M, dtype="f64_emu")
    torch.cuda.synchronize()
    assert torch.equal(M, 0.25 * M0)
    Xh = rng.uniform(-1, 1, size=(130, 90))
    Uh = rng.uniform(-1, 1, size=(90, 17))
    Md = torch.zeros(130, 17, dtype=torch.float64, device="cuda").t().contiguous().t()
    fm.mttkrp(1.0, torch.from_numpy(Xh).cuda(), 0, [None, torch.from_numpy(Uh).cuda()], 0.0, Md,
              dtype="f64_emu")
    torch.cuda.synchronize()
    assert rel_frob(Md.cpu().numpy(), Xh @ Uh) <= 1e-13


@pytest.mark.parametrize("dtype", ["f64_emu", "f32"])
def test_hooi_projection_as_a_network(dtype):
    """HOOI's inner step for mode 0 of a 3-way tensor: Y[i, q, s] =
    sum_{j,k} X[i,j,k] U1[j,q] U2[k,s] as two tensor-times-matrix
    contractions in one network call (the intermediate kept on the device),
    against the oracle step by step."""
    rng = np.random.default_rng(1250)
    I, J, K, Q, S = 60, 50, 40, 12, 10
    X = W.uniform_operand(rng, (I, J, K), W.L("ijk"))
    U1 = W.uniform_operand(rng, (J, Q), W.L("jq"))
    U2 = W.uniform_operand(rng, (K, S), W.L("ks"))
    Y = W.zeros_operand((I, Q, S), W.L("iqs"))
    dt = DT[dtype]
    Xd, U1d, U2d, Yd = (to_device(t, dt) for t in (X, U1, U2, Y))
    tensors = [(Xd, W.L("ijk")), (U1d, W.L("jq")), ((I, Q, K), W.L("iqk")), (U2d, W.L("ks")),
               (Yd, W.L("iqs"))]
    fm.contract_network(tensors, [(0, 1, 2, 1.0, 0.0), (2, 3, 4, 1.0, 0.0)], dtype=dtype)
    torch.cuda.synchronize()
    T = np.zeros((I, Q, K))
    oracle.contract(1.0, X.view(), W.L("ijk"), U1.view(), W.L("jq"), 0.0, T, W.L("iqk"))
    want = np.zeros((I, Q, S))
    oracle.contract(1.0, T, W.L("iqk"), U2.view(), W.L("ks"), 0.0, want, W.L("iqs"))
    assert rel_frob(Yd.to(torch.float64).cpu().numpy(), want) <= TOL[dtype]


def test_mttkrp_full_size_every_mode_sampled_dot2():
    """The benchmark's shape, X 512^3 fp64 with R = 64 (K = 262144),
    emulated fp64, every mode, on 512 sampled entries of M evaluated by the
    oracle with the compensated dot product over the oracle's Khatri-Rao
    product (a plain fp64 sum of 262144 random-sign terms is itself off by
    ~1e-12 relative)."""
    rng = np.random.default_rng(1260)
    I, R = 512, 64
    X = rng.standard_normal((I, I, I))
    U = [rng.standard_normal((I, R)) for _ in range(3)]
    Xd = torch.from_numpy(X).cuda()
    Ud = [torch.from_numpy(u).cuda().t().contiguous().t() for u in U]
    L = [1, 2, 3]
    for mode in range(3):
        Md = torch.zeros(R, I, dtype=torch.float64, device="cuda").t()
        fm.mttkrp(1.0, Xd, mode, Ud, 0.0, Md, dtype="f64_emu")
        torch.cuda.synchronize()
        KR = oracle.khatri_rao(U, mode, 3)
        others = [m + 1 for m in range(3) if m != mode]
        idx = np.stack([rng.integers(0, I, size=512), rng.integers(0, R, size=512)], axis=1)
        want = oracle.entries(1.0, X, L, KR, others + [9], 0.0, np.zeros((I, R)), [mode + 1, 9], idx,
                              dot2=True)
        got = Md.cpu().numpy()[idx[:, 0], idx[:, 1]]
        assert rel_frob(got, want) <= 1e-13


def test_mttkrp_degenerate_shapes():
    """R = 0 (nothing to write), an empty contracted mode (M := beta M), and
    an extent-1 mode (dropped from the Khatri-Rao digits)."""
    X = torch.rand(5, 0, 4, dtype=torch.float64, device="cuda")
    U = [torch.rand(5, 3, dtype=torch.float64, device="cuda"), torch.rand(0, 3, dtype=torch.float64, device="cuda"),
         torch.rand(4, 3, dtype=torch.float64, device="cuda")]
    M = torch.rand(5, 3, dtype=torch.float64, device="cuda")
    M0 = M.clone()
    fm.mttkrp(1.0, X, 0, U, 0.5, M, dtype="f64_emu")
    torch.cuda.synchronize()
    assert torch.equal(M, 0.5 * M0)
    E = torch.empty(5, 0, dtype=torch.float64, device="cuda")
    X2 = torch.rand(5, 4, 6, dtype=torch.float64, device="cuda")
    fm.mttkrp(1.0, X2, 0, [None, torch.empty(4, 0, dtype=torch.float64, device="cuda"),
                           torch.empty(6, 0, dtype=torch.float64, device="cuda")], 0.0, E, dtype="f64_emu")
    rng = np.random.default_rng(1270)
    Xh = rng.uniform(-1, 1, size=(30, 1, 20))
    Uh = [rng.uniform(-1, 1, size=(e, 7)) for e in (30, 1, 20)]
    Md = torch.zeros(7, 30, dtype=torch.float64, device="cuda").t()
    fm.mttkrp(1.0, torch.from_numpy(Xh).cuda(), 0, [None] + [torch.from_numpy(u).cuda() for u in Uh[1:]], 0.0,
              Md, dtype="f64_emu")
    torch.cuda.synchronize()
    want = oracle.mttkrp(1.0, Xh, 0, Uh, 0.0, np.zeros((30, 7)))
    assert rel_frob(Md.cpu().numpy(), want) <= 1e-13
