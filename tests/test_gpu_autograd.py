"""Differentiable contraction: forward and adjoints (dA, dB as contractions of
dC with the other operand) against the oracle's gradient and against fp64
central finite differences of L = ||contract(A,B) - T||_F^2."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_07311_b300 import inputs as W
from paper_2604_07311_b300.autograd import contract_autograd

from gpu_util import rel_frob

pytestmark = pytest.mark.gpu


def oracle_grads(Af, la, Bf, lb, Tf, lc):
    C = np.zeros(Tf.shape)
    oracle.contract(1.0, Af, la, Bf, lb, 0.0, C, lc)
    dC = 2.0 * (C - Tf)
    dA = np.zeros(Af.shape)
    dB = np.zeros(Bf.shape)
    oracle.contract(1.0, dC, lc, Bf, lb, 0.0, dA, la)
    oracle.contract(1.0, Af, la, dC, lc, 0.0, dB, lb)
    return C, dA, dB


def test_loss_gradient_fp32_full_size():
    """A[i,k,m,l], B[k,m,j], T[i,j,l] with i=j=l=64, k=m=48; fp32 on the GPU."""
    d = W.autograd_problem()
    la, lb, lc = d["la"], d["lb"], d["lc"]
    A32, B32, T32 = (d[x].astype(np.float32) for x in "ABT")
    Af, Bf, Tf = (x.astype(np.float64) for x in (A32, B32, T32))  # the fp32 values, exactly
    A = torch.from_numpy(A32).cuda().requires_grad_()
    B = torch.from_numpy(B32).cuda().requires_grad_()
    T = torch.from_numpy(T32).cuda()
    C = contract_autograd(A, la, B, lb, lc)
    L = ((C - T) ** 2).sum()
    L.backward()
    torch.cuda.synchronize()
    C_ref, dA_ref, dB_ref = oracle_grads(Af, la, Bf, lb, Tf, lc)
    assert rel_frob(C.detach().double().cpu().numpy(), C_ref) <= 1e-5
    gA = A.grad.double().cpu().numpy()
    gB = B.grad.double().cpu().numpy()
    assert rel_frob(gA, dA_ref) <= 1e-5
    assert rel_frob(gB, dB_ref) <= 1e-5

    # fp64 central differences on 100 entries of A and 100 of B (h = 1e-6).
    # L is quadratic, so the difference quotient equals the derivative up to
    # rounding; only the C entries the perturbed element touches are
    # recomputed, the other terms of L cancel between L+ and L-.
    h = 1e-6
    rng = np.random.default_rng(d["seed"] + 1)
    ni, nk, nm, nl = Af.shape
    nj = Bf.shape[2]

    def partial_loss(X, idx_c):
        c = oracle.entries(1.0, Af, la, Bf, lb, 0.0, np.zeros(Tf.shape), lc, idx_c)
        return float(np.sum((c - Tf[tuple(idx_c.T)]) ** 2))

    for _ in range(100):
        i, k, m, l = (int(rng.integers(0, e)) for e in Af.shape)
        idx_c = np.array([[i, j, l] for j in range(nj)])
        orig = Af[i, k, m, l]
        Af[i, k, m, l] = orig + h
        lp = partial_loss(Af, idx_c)
        Af[i, k, m, l] = orig - h
        lm = partial_loss(Af, idx_c)
        Af[i, k, m, l] = orig
        fd = (lp - lm) / (2 * h)
        g = gA[i, k, m, l]
        assert abs(fd - g) <= 1e-3 * max(abs(g), 1.0), (i, k, m, l, fd, g)
    for _ in range(100):
        k, m, j = (int(rng.integers(0, e)) for e in Bf.shape)
        idx_c = np.array([[i, j, l] for i in range(ni) for l in range(nl)])
        orig = Bf[k, m, j]
        Bf[k, m, j] = orig + h
        lp = partial_loss(Bf, idx_c)
        Bf[k, m, j] = orig - h
        lm = partial_loss(Bf, idx_c)
        Bf[k, m, j] = orig
        fd = (lp - lm) / (2 * h)
        g = gB[k, m, j]
        assert abs(fd - g) <= 1e-3 * max(abs(g), 1.0), (k, m, j, fd, g)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f64_emu", 1e-13)])
def test_gradients_fp64_paths_with_batch_labels(dtype, tol):
    """C[a,b,z] = sum_k A[a,k,z] B[k,b,z] (z a batch label) in fp64 and emulated fp64."""
    rng = np.random.default_rng(901)
    la, lb, lc = [1, 2, 9], [2, 3, 9], [1, 3, 9]
    Af = rng.uniform(-1, 1, (70, 90, 3))
    Bf = rng.uniform(-1, 1, (90, 50, 3))
    Tf = rng.uniform(-1, 1, (70, 50, 3))
    A = torch.from_numpy(Af).cuda().requires_grad_()
    B = torch.from_numpy(Bf).cuda().requires_grad_()
    C = contract_autograd(A, la, B, lb, lc, dtype=dtype)
    L = ((C - torch.from_numpy(Tf).cuda()) ** 2).sum()
    L.backward()
    C_ref, dA_ref, dB_ref = oracle_grads(Af, la, Bf, lb, Tf, lc)
    assert rel_frob(C.detach().cpu().numpy(), C_ref) <= tol
    assert rel_frob(A.grad.cpu().numpy(), dA_ref) <= tol
    assert rel_frob(B.grad.cpu().numpy(), dB_ref) <= tol


def test_gradient_bf16_inputs():
    rng = np.random.default_rng(902)
    la, lb, lc = [1, 2], [2, 3], [1, 3]
    A32 = rng.uniform(-1, 1, (130, 70)).astype(np.float32)
    B32 = rng.uniform(-1, 1, (70, 90)).astype(np.float32)
    A = torch.from_numpy(A32).cuda().bfloat16().requires_grad_()
    B = torch.from_numpy(B32).cuda().bfloat16().requires_grad_()
    C = contract_autograd(A, la, B, lb, lc)
    C.sum().backward()
    Ar = A.detach().double().cpu().numpy()
    Br = B.detach().double().cpu().numpy()
    ones = np.ones((130, 90))
    dA_ref = np.zeros(Ar.shape)
    oracle.contract(1.0, ones, lc, Br, lb, 0.0, dA_ref, la)
    # the gradient itself is stored in bf16: compare at bf16 resolution
    assert rel_frob(A.grad.double().cpu().numpy(), dA_ref) <= 2e-2
