"""The plan cache: a repeated call with the same shapes, strides, dtype, knobs
and stream reuses its workspace and offset tables (one kernel fewer: no table
build) and gives bit-identical results; another stream, or a call captured
into a CUDA graph, does not share the entry."""
import numpy as np
import pytest
import torch

import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W

from gpu_util import gpu_dense, rel_frob, run_oracle, to_device

pytestmark = pytest.mark.gpu


def _call(p, dtype, C, stream=None):
    A = to_device(p.A, torch.float32 if dtype == "f32" else torch.float64)
    B = to_device(p.B, torch.float32 if dtype == "f32" else torch.float64)
    _, info = fm.contract(p.alpha, A, p.A.labels, B, p.B.labels, p.beta, C, p.C.labels, dtype=dtype,
                          stream=stream, return_info=True)
    return info


@pytest.mark.parametrize("dtype", ["f32", "f64_emu", "f64"])
def test_repeated_call_reuses_tables(dtype):
    rng = np.random.default_rng(950)
    # a shape no other test uses, so the first call here builds the entry
    A = W.uniform_operand(rng, (37, 29, 53), [1, 2, 3])
    B = W.uniform_operand(rng, (29, 53, 41), [2, 3, 4])
    C = W.uniform_operand(rng, (37, 41), [1, 4])
    p = W.Problem("cache", 1.25, A, B, -0.5, C)
    tout = torch.float32 if dtype == "f32" else torch.float64
    C1, C2 = to_device(p.C, tout), to_device(p.C, tout)
    i1 = _call(p, dtype, C1)
    i2 = _call(p, dtype, C2)
    torch.cuda.synchronize()
    assert i1["cached"] == 0 and i2["cached"] == 1
    assert i2["launches"] == i1["launches"] - 1
    assert torch.equal(C1, C2)
    tin = torch.float32 if dtype == "f32" else None
    want = run_oracle(p, in_dtype=tin, out_dtype=torch.float32 if dtype == "f32" else None)
    assert rel_frob(gpu_dense(C2), want) <= (1e-5 if dtype == "f32" else 1e-13)


def test_other_stream_gets_its_own_entry():
    rng = np.random.default_rng(951)
    A = W.uniform_operand(rng, (31, 47), [1, 2])
    B = W.uniform_operand(rng, (47, 23), [2, 3])
    C = W.zeros_operand((31, 23), [1, 3])
    p = W.Problem("cache_streams", 1.0, A, B, 0.0, C)
    s = torch.cuda.Stream()
    C1, C2 = to_device(p.C, torch.float64), to_device(p.C, torch.float64)
    _call(p, "f64", C1)
    with torch.cuda.stream(s):
        info = _call(p, "f64", C2, stream=s)
    s.synchronize()
    torch.cuda.synchronize()
    assert info["cached"] == 0
    assert torch.equal(C1, C2)


def test_capture_bypasses_the_cache_and_replays():
    rng = np.random.default_rng(952)
    A = W.uniform_operand(rng, (60, 44), [1, 2])
    B = W.uniform_operand(rng, (44, 52), [2, 3])
    C = W.zeros_operand((60, 52), [1, 3])
    p = W.Problem("cache_graph", 1.0, A, B, 0.0, C)
    Ad, Bd = to_device(p.A, torch.float64), to_device(p.B, torch.float64)
    Cd = to_device(p.C, torch.float64)
    fm.contract(1.0, Ad, p.A.labels, Bd, p.B.labels, 0.0, Cd, p.C.labels, dtype="f64_emu")  # cache entry
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            _, info = fm.contract(1.0, Ad, p.A.labels, Bd, p.B.labels, 0.0, Cd, p.C.labels, dtype="f64_emu",
                                  return_info=True)
    assert info["cached"] == 0
    Cd.zero_()
    Ad.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    want = 2.0 * run_oracle(p)
    assert rel_frob(gpu_dense(Cd), want) <= 1e-13


def test_eviction_waits_for_queued_calls():
    """More distinct shapes than the cache holds (16), each call a few
    milliseconds of work, all enqueued before any finishes: an entry is
    evicted while the call that last used its workspace may still be queued,
    so the eviction must wait for that call (the entry's event) before the
    workspace is freed.  Every result against the oracle's compensated sums
    on sampled entries."""
    import oracle
    rng = np.random.default_rng(953)
    probs, outs = [], []
    for t in range(20):
        m, n, k = 1024 + 8 * t, 1024, 8192 + 8 * t  # distinct shapes: distinct entries (< 256 MB each)
        A = W.uniform_operand(rng, (m, k), [1, 2])
        B = W.uniform_operand(rng, (k, n), [2, 3])
        C = W.uniform_operand(rng, (m, n), [1, 3])
        p = W.Problem(f"evict{t}", 1.0, A, B, -1.0, C)
        Ad, Bd, Cd = (to_device(x, torch.float64) for x in (p.A, p.B, p.C))
        probs.append((p, Ad, Bd, Cd))
    torch.cuda.synchronize()
    for p, Ad, Bd, Cd in probs:  # no synchronisation between calls
        fm.contract(p.alpha, Ad, p.A.labels, Bd, p.B.labels, p.beta, Cd, p.C.labels, dtype="f64_emu")
    torch.cuda.synchronize()
    assert fm.device_status() == 0
    for p, _, _, Cd in probs:
        got = gpu_dense(Cd)
        idx = np.stack([rng.integers(0, e, 64) for e in got.shape], axis=1)
        want = oracle.entries(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, p.C.view(),
                              p.C.labels, idx, dot2=True)
        assert rel_frob(got[tuple(idx.T)], want) <= 1e-13, p.name
