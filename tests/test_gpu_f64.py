"""GPU parity of the native-fp64 path against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle, random_label_problem, to_device

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-13  # relative Frobenius tolerance for fp64 results


def test_four_index_ext16_random():
    p = W.four_index(ext=16)
    C, info = run_gpu(p, "f64")
    assert info["kernel_name"] == "simt_f64"
    assert rel_frob(gpu_dense(C), run_oracle(p)) <= TOL_F64


def test_four_index_integer_exact():
    p = W.four_index(ext=16, integer=True)
    C, _ = run_gpu(p, "f64")
    assert np.array_equal(gpu_dense(C), run_oracle(p))


@pytest.mark.parametrize("seed", range(4))
def test_random_labels_integer_exact(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(12):
        p = random_label_problem(rng, max_ext=6)
        C, _ = run_gpu(p, "f64")
        assert np.array_equal(gpu_dense(C), run_oracle(p))


def test_ladder_reduced_beta_one():
    p = W.ladder(v=32, o=8)
    C, info = run_gpu(p, "f64")
    assert (info["m"], info["n"], info["k"]) == (1024, 64, 1024)
    assert rel_frob(gpu_dense(C), run_oracle(p)) <= TOL_F64


def test_ragged_tiles():
    rng = np.random.default_rng(7)
    for m, n, k in [(1, 1, 1), (65, 63, 17), (130, 70, 33), (64, 64, 16)]:
        A = W.uniform_operand(rng, (m, k), [1, 2])
        B = W.uniform_operand(rng, (k, n), [2, 3])
        C = W.uniform_operand(rng, (m, n), [1, 3])
        p = W.Problem("gemm", 1.5, A, B, -0.5, C)
        Cg, _ = run_gpu(p, "f64")
        assert rel_frob(gpu_dense(Cg), run_oracle(p)) <= TOL_F64, (m, n, k)


def test_alpha_zero_beta_zero_empty_and_scalar():
    nan = float("nan")
    A = torch.full((3, 4), nan, dtype=torch.float64, device="cuda")
    B = torch.full((4, 2), nan, dtype=torch.float64, device="cuda")
    C0 = torch.arange(6, dtype=torch.float64, device="cuda").reshape(3, 2)
    C = C0.clone()
    fm.contract(0.0, A, [1, 2], B, [2, 3], 2.0, C, [1, 3])
    assert torch.equal(C, 2 * C0)  # alpha == 0: A, B not read
    A = torch.ones((3, 4), dtype=torch.float64, device="cuda")
    B = torch.ones((4, 2), dtype=torch.float64, device="cuda")
    C = torch.full((3, 2), nan, dtype=torch.float64, device="cuda")
    fm.contract(1.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3])
    assert torch.equal(C, torch.full((3, 2), 4.0, dtype=torch.float64, device="cuda"))
    C = C0.clone()  # empty K: C := beta*C
    fm.contract(1.0, A[:, :0], [1, 2], B[:0], [2, 3], 3.0, C, [1, 3])
    assert torch.equal(C, 3 * C0)
    E = torch.zeros((0, 2), dtype=torch.float64, device="cuda")  # empty M: no-op
    fm.contract(1.0, A[:0], [1, 2], B, [2, 3], 1.0, E, [1, 3])
    a = torch.randint(-4, 5, (3, 4), device="cuda").double()
    b = torch.randint(-4, 5, (4, 3), device="cuda").double()
    s = torch.zeros((), dtype=torch.float64, device="cuda")
    fm.contract(1.0, a, [1, 2], b, [2, 1], 0.0, s, [])
    assert s.item() == float((a * b.T).sum().item())
    torch.cuda.synchronize()


def test_ieee_propagation():
    rng = np.random.default_rng(19)
    A = rng.uniform(-1, 1, (4, 5))
    B = rng.uniform(-1, 1, (5, 3))
    B[2, 1] = 0.0
    A[1, 2] = np.inf
    A[3, 0] = np.nan
    want = np.zeros((4, 3))
    oracle.contract(1.0, A, [1, 2], B, [2, 3], 0.0, want, [1, 3])
    C = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    fm.contract(1.0, torch.from_numpy(A).cuda(), [1, 2], torch.from_numpy(B).cuda(), [2, 3], 0.0, C,
                [1, 3])
    got = C.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    assert np.allclose(got[fin], want[fin], rtol=1e-14, atol=0)


def test_host_buffers_entry_point():
    p = W.four_index(ext=12, seed=5)
    want = run_oracle(p)
    C = np.array(p.C.view(), copy=True)
    fm.contract_host(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, C, p.C.labels,
                     dtype="f64")
    assert rel_frob(C, want) <= TOL_F64


def test_device_status_clean():
    assert fm.device_status() == 0


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5)])
def test_cuda_core_few_tiles_split_k(dtype, tol):
    """100 x 50 outputs (2 tiles) with K = 30000: the CUDA-core kernel splits
    K across the SMs and sums the partial tiles in split order."""
    rng = np.random.default_rng(1400)
    A = W.uniform_operand(rng, (100, 30000), [1, 2])
    B = W.uniform_operand(rng, (30000, 50), [2, 3])
    C = W.uniform_operand(rng, (100, 50), [1, 3])
    p = W.Problem("few_tiles", 0.5, A, B, -2.0, C)
    dt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    got, info = run_gpu(p, dtype, kernel=1)
    assert info["kernel_name"] == ("simt_f64" if dtype == "f64" else "simt_f32")
    assert info["launches"] + info["cached"] == 3  # tables, split product, reduction
    want = run_oracle(p, dt, dt)
    assert rel_frob(gpu_dense(got), want) <= tol
