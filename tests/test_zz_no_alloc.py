"""The no-allocation entry point (famlies_contract_noalloc) against the regular
one and against the oracle.  It serves callers that may not allocate device
memory themselves or through the library (a pre-reserved device pool, a
real-time loop); its offset tables live in a fixed scratch array inside the
library.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes both alone in a
fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import _lib
from paper_2604_07311_b300 import inputs as W

from gpu_util import OUT_DT, TORCH_DT, gpu_dense, rel_frob, random_label_problem, to_device

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-5}  # the relative Frobenius tolerances of the other tests
ERR_SCRATCH = -11


def noalloc_abi(alpha, A, la, B, lb, beta, C, lc, dtype: str) -> int:
    """Calls famlies_contract_noalloc directly through the C ABI."""
    lib = fm.load()
    f = lib.famlies_contract_noalloc
    T = ctypes.POINTER(_lib.TensorDesc)
    f.argtypes = [ctypes.c_double, T, T, ctypes.c_double, T, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    da, db, dc = _lib.desc_torch(A, la), _lib.desc_torch(B, lb), _lib.desc_torch(C, lc)
    return f(float(alpha), da.ref, db.ref, float(beta), dc.ref, _lib.DTYPES[dtype],
             torch.cuda.current_stream().cuda_stream)


def oracle_dense(p: W.Problem, dtype: str) -> np.ndarray:
    """The oracle's result on the inputs as the device holds them."""
    Ar = W.Operand(torch.from_numpy(p.A.buf).to(TORCH_DT[dtype]).double().numpy(), p.A.extents,
                   p.A.strides, p.A.labels)
    Br = W.Operand(torch.from_numpy(p.B.buf).to(TORCH_DT[dtype]).double().numpy(), p.B.extents,
                   p.B.strides, p.B.labels)
    Cr = W.Operand(torch.from_numpy(p.C.buf).to(OUT_DT[dtype]).double().numpy(), p.C.extents,
                   p.C.strides, p.C.labels)
    want = np.array(Cr.view(), copy=True)
    oracle.contract(p.alpha, Ar.view(), p.A.labels, Br.view(), p.B.labels, p.beta, want, p.C.labels)
    return want


def both_paths(p: W.Problem, dtype: str):
    A = to_device(p.A, TORCH_DT[dtype])
    B = to_device(p.B, TORCH_DT[dtype])
    C_ref = to_device(p.C, OUT_DT[dtype])
    C_new = to_device(p.C, OUT_DT[dtype])
    fm.contract(p.alpha, A, p.A.labels, B, p.B.labels, p.beta, C_ref, p.C.labels, dtype=dtype)
    rc = noalloc_abi(p.alpha, A, p.A.labels, B, p.B.labels, p.beta, C_new, p.C.labels, dtype)
    torch.cuda.synchronize()
    assert rc == 0, fm.error_string(rc)
    return gpu_dense(C_new), gpu_dense(C_ref)


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    rng = np.random.default_rng(900)
    cases = [(W.four_index(ext=16), "f64"),
             (W.transpose_free(v=24, o=12, pad=7), "f32"),
             (W.ladder(v=16, o=8), "f64"),
             (random_label_problem(rng, max_ext=6, integer=False), "f64")]
    for p, dtype in cases:
        exact = oracle_dense(p, dtype)
        for _ in range(2):  # two calls in a row share (and rewrite) the scratch array
            got, want = both_paths(p, dtype)
            assert rel_frob(got, want) <= TOL[dtype], (p.name, dtype)
            assert rel_frob(got, exact) <= TOL[dtype], (p.name, dtype)
    assert fm.device_status() == 0


def test_noalloc_rejects_calls_beyond_its_scratch():
    m = 1 << 17  # 2*(m + n + k) offsets exceed the 2^17-entry array
    A = torch.zeros((m, 4), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    C = torch.zeros((m, 2), dtype=torch.float64, device="cuda")
    assert noalloc_abi(1.0, A, [1, 2], B, [2, 3], 0.0, C, [1, 3], "f64") == ERR_SCRATCH
    assert "scratch" in fm.error_string(ERR_SCRATCH)
    Ab = torch.zeros((4, 4), dtype=torch.bfloat16, device="cuda")
    Bb = torch.zeros((4, 4), dtype=torch.bfloat16, device="cuda")
    Cb = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    assert noalloc_abi(1.0, Ab, [1, 2], Bb, [2, 3], 0.0, Cb, [1, 3], "bf16") == -6
