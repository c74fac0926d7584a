"""Small-case sweep on the GPU against the oracle: every combination of
extents from {1, 2, 3, 5, 8, 9} for the free, contracted and batch classes,
operands stored with odd padded strides, in each dtype (bounds and edges of
every kernel path where tiles are mostly empty)."""
import itertools

import numpy as np
import pytest
import torch

import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

EXT = (1, 2, 3, 5, 8, 9)
TOL = {"f64": 1e-13, "f64_emu": 1e-13, "f32": 1e-5, "bf16": 1e-5}
RND = {"f64": None, "f64_emu": None, "f32": torch.float32, "bf16": torch.bfloat16}


def _problem(m, n, k, b, rng):
    """C[m,n,b] = sum_k A[k,m,b] B[n,k,b] with each operand's first stride padded
    by an odd amount."""
    A = W.integer_operand(rng, (k, m, b), [3, 1, 4], lead_pad=int(rng.integers(0, 3)) * 2 + 1)
    B = W.integer_operand(rng, (n, k, b), [2, 3, 4], lead_pad=int(rng.integers(0, 3)) * 2 + 1)
    C = W.integer_operand(rng, (m, n, b), [1, 2, 4], lead_pad=int(rng.integers(0, 3)) * 2 + 1)
    return W.Problem("sweep", 1.0, A, B, 1.0, C)


@pytest.mark.parametrize("dtype", ["f64", "f64_emu", "f32", "bf16"])
def test_small_extent_sweep(dtype):
    rng = np.random.default_rng(1600)
    worst = 0.0
    for m, n, k in itertools.product(EXT, EXT, EXT):
        b = int(rng.choice((1, 2, 3)))
        p = _problem(m, n, k, b, rng)
        got, _ = run_gpu(p, dtype)
        want = run_oracle(p, RND[dtype], torch.float32 if dtype in ("f32", "bf16") else None)
        worst = max(worst, rel_frob(gpu_dense(got), want))
    assert worst <= TOL[dtype]
    assert fm.device_status() == 0


def test_log_switch_prints_the_plan():
    """FAMLIES_LOG=1 prints one line per call on stderr with the chosen path
    and sizes (run in a child process so the switch is read fresh)."""
    import os
    import subprocess
    import sys
    code = ("import torch, paper_2604_07311_b300 as fm\n"
            "A=torch.ones(40,50,dtype=torch.float64,device='cuda'); B=torch.ones(50,60,dtype=torch.float64,device='cuda')\n"
            "C=torch.zeros(40,60,dtype=torch.float64,device='cuda')\n"
            "fm.contract(1.0, A, [1,2], B, [2,3], 0.0, C, [1,3], dtype='f64_emu'); torch.cuda.synchronize()\n"
            "print(float(C[0,0]))\n")
    env = dict(os.environ, FAMLIES_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stderr
    assert "famlies: tc_emu m=60 n=40 k=50 batch=1 modes=1/1/1/0 swapped=1" in r.stderr  # C row-major
    assert r.stdout.strip() == "50.0"
