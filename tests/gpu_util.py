"""Helpers shared by the GPU parity tests: move seeded numpy operands to the
device with their exact strides, run the library through the C ABI, and
compare with the oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

TORCH_DT = {"f64": torch.float64, "f64_emu": torch.float64, "f32": torch.float32,
            "bf16": torch.bfloat16}
OUT_DT = {"f64": torch.float64, "f64_emu": torch.float64, "f32": torch.float32,
          "bf16": torch.float32}


def to_device(op: W.Operand, dtype: torch.dtype) -> torch.Tensor:
    """The operand's whole buffer on the device, viewed with its strides."""
    buf = torch.from_numpy(op.buf).to(device="cuda", dtype=dtype)
    return torch.as_strided(buf, op.extents, op.strides)


def rounded_host(op: W.Operand, dtype: torch.dtype) -> W.Operand:
    """The operand with its values rounded to `dtype` and promoted back to fp64."""
    buf = torch.from_numpy(op.buf).to(dtype).to(torch.float64).numpy()
    return W.Operand(buf, op.extents, op.strides, op.labels)


def run_gpu(p: W.Problem, dtype: str, **kw):
    A = to_device(p.A, TORCH_DT[dtype])
    B = to_device(p.B, TORCH_DT[dtype])
    C = to_device(p.C, OUT_DT[dtype])
    _, info = fm.contract(p.alpha, A, p.A.labels, B, p.B.labels, p.beta, C, p.C.labels,
                          dtype=dtype, return_info=True, **kw)
    torch.cuda.synchronize()
    return C, info


def run_oracle(p: W.Problem, in_dtype: torch.dtype | None = None, out_dtype=None) -> np.ndarray:
    """Oracle result on the (optionally dtype-rounded) inputs, as a dense array."""
    A = rounded_host(p.A, in_dtype) if in_dtype is not None else p.A
    B = rounded_host(p.B, in_dtype) if in_dtype is not None else p.B
    C = rounded_host(p.C, out_dtype) if out_dtype is not None else p.C
    Cv = np.array(C.view(), copy=True)
    oracle.contract(p.alpha, A.view(), p.A.labels, B.view(), p.B.labels, p.beta, Cv, p.C.labels)
    return Cv


def rel_frob(got, want) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want)
    num = np.linalg.norm(got - want)
    return float(num / den) if den > 0 else float(num)


def gpu_dense(C: torch.Tensor) -> np.ndarray:
    return C.detach().to(torch.float64).cpu().numpy()


def random_label_problem(rng, max_ext=5, integer=True, batch=True, pad_max=2) -> W.Problem:
    """Random label sets (M, N, K, batch) with random mode orders and padded strides."""
    names = iter(range(100, 200))
    cls = {c: [next(names) for _ in range(int(rng.integers(0, 3)))] for c in "MNK"}
    cls["L"] = [next(names) for _ in range(int(rng.integers(0, 2)))] if batch else []
    ext = {l: int(rng.integers(1, max_ext + 1)) for v in cls.values() for l in v}

    def mk(labels):
        labels = [int(x) for x in rng.permutation(labels)] if labels else []
        shape = [ext[l] for l in labels]
        order = rng.permutation(len(labels))
        strides = [0] * len(labels)
        acc = 1
        for d in order:
            strides[d] = acc
            acc *= shape[d] + int(rng.integers(0, pad_max + 1))
        buf = (rng.integers(-4, 5, size=max(acc, 1)).astype(np.float64) if integer
               else rng.uniform(-1, 1, size=max(acc, 1)))
        return W.Operand(buf, tuple(shape), tuple(strides), labels)

    A = mk(cls["M"] + cls["K"] + cls["L"])
    B = mk(cls["N"] + cls["K"] + cls["L"])
    C = mk(cls["M"] + cls["N"] + cls["L"])
    alpha = float(rng.integers(-2, 3)) if integer else float(rng.uniform(-2, 2))
    beta = float(rng.integers(-2, 3)) if integer else float(rng.uniform(-2, 2))
    return W.Problem("random", alpha, A, B, beta, C)
