"""Differentiable contraction: torch.autograd.Function over the C ABI.

For C[lc] = sum A[la] * B[lb] (Einstein summation over labels) the adjoints
are again contractions of the same kind, with the output gradient dC in
place of one operand:

    dA[la] = sum dC[lc] * B[lb]      dB[lb] = sum A[la] * dC[lc]

Labels of A that are contracted in the forward pass (in A and B only) are
free in dA and come from B; labels summed in dA are B's free labels (in B
and C only); batch labels stay batch labels.  Both adjoints therefore run
on the library's kernels through the same planner with relabelled
descriptors -- no transpose is materialised.  The paper lists tensor
computations, and fused data re-organisation, as the framework's job
(Sec. 1 "Challenges"; Sec. 2.3); differentiation is the task's addition.
"""
from __future__ import annotations

import torch

from . import contract as _contract

_OUT = {torch.float64: torch.float64, torch.float32: torch.float32, torch.bfloat16: torch.float32}


def _out_shape(la, A, lb, B, lc):
    ext = {}
    for labs, t in ((la, A), (lb, B)):
        for lab, e in zip(labs, t.shape):
            ext[int(lab)] = e
    return tuple(ext[int(l)] for l in lc)


class Contract(torch.autograd.Function):
    """C = contract(A, B) with labels (la, lb) -> lc; dtype as for `contract`."""

    @staticmethod
    def forward(ctx, A, B, la, lb, lc, dtype=None):
        C = torch.empty(_out_shape(la, A, lb, B, lc), dtype=_OUT[A.dtype], device=A.device)
        _contract(1.0, A, la, B, lb, 0.0, C, lc, dtype=dtype)
        ctx.save_for_backward(A, B)
        ctx.labels = (list(la), list(lb), list(lc))
        ctx.dtype = dtype
        return C

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        la, lb, lc = ctx.labels
        dC = dC.to(A.dtype) if A.dtype != torch.bfloat16 else dC.to(torch.bfloat16)
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = torch.empty(A.shape, dtype=_OUT[A.dtype], device=A.device)
            _contract(1.0, dC, lc, B, lb, 0.0, dA, la, dtype=ctx.dtype)
            dA = dA.to(A.dtype)
        if ctx.needs_input_grad[1]:
            dB = torch.empty(B.shape, dtype=_OUT[B.dtype], device=B.device)
            _contract(1.0, A, la, dC, lc, 0.0, dB, lb, dtype=ctx.dtype)
            dB = dB.to(B.dtype)
        return dA, dB, None, None, None, None


def contract_autograd(A, la, B, lb, lc, dtype=None):
    """Differentiable C[lc] = sum A[la] B[lb] on the GPU."""
    return Contract.apply(A, B, list(la), list(lb), list(lc), dtype)
