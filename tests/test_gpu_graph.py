"""A library call captured into a CUDA graph (torch.cuda.graph) and replayed
with new input values in the same buffers: every stage of a contraction is
stream-ordered (stream-ordered workspace, memsets, kernels), so the graph
replays the whole call.  Checked against the oracle after each replay."""
import numpy as np
import pytest
import torch

import oracle
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import rel_frob

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("f64_emu", 1e-13), ("f64", 1e-13), ("f32", 1e-5)])
def test_captured_contraction_replays(dtype, tol):
    dt = torch.float64 if dtype != "f32" else torch.float32
    v, o = 24, 8
    rng = np.random.default_rng(1700)
    V = torch.empty((v, v, v, v), dtype=dt, device="cuda")
    T = torch.empty((v, v, o, o), dtype=dt, device="cuda")
    C = torch.empty((v, v, o, o), dtype=dt, device="cuda")
    lv, lt, lc = W.L("abcd"), W.L("cdij"), W.L("abij")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture (one-time attribute setup)
        fm.contract(1.0, V.normal_(), lv, T.normal_(), lt, 0.0, C.zero_(), lc, dtype=dtype, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fm.contract(0.5, V, lv, T, lt, 1.0, C, lc, dtype=dtype, stream=s)
    for rep in range(3):
        Vh = rng.uniform(-1, 1, size=(v, v, v, v))
        Th = rng.uniform(-1, 1, size=(v, v, o, o))
        Ch = rng.uniform(-1, 1, size=(v, v, o, o))
        V.copy_(torch.from_numpy(Vh))
        T.copy_(torch.from_numpy(Th))
        C.copy_(torch.from_numpy(Ch))
        g.replay()
        torch.cuda.synchronize()
        r = lambda x: torch.from_numpy(x).to(dt).double().numpy()
        want = r(Ch).copy()
        oracle.contract(0.5, r(Vh), lv, r(Th), lt, 1.0, want, lc)
        assert rel_frob(C.double().cpu().numpy(), want) <= tol
    assert fm.device_status() == 0
