"""The library's environment switches, each read once per process: with the
plan cache off (FAMLIES_PLAN_CACHE=0) every call plans, allocates and frees
its own workspace; with the grouped autotuner off (FAMLIES_AUTOTUNE=0) the
grouped launch takes its heuristic tile widths.  Each runs in a child
process and is checked against the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, "tests")
import numpy as np
import torch
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W
from gpu_util import OUT_DT, TORCH_DT, gpu_dense, rel_frob, run_gpu, run_oracle, to_device

# the same single problem three times (with the cache on, the second and
# third calls reuse the first one's plan entry), then a different one
for p in (W.ladder(v=24, o=8), W.ladder(v=24, o=8), W.ladder(v=24, o=8), W.four_index(ext=20)):
    C, info = run_gpu(p, "f64_emu")
    err = rel_frob(gpu_dense(C), run_oracle(p))
    assert err <= 1e-13, (p.name, err)
# a grouped batch, graph and no graph
blocks = W.block_sparse(nblocks=24, choices=[8, 16, 24, 40])
for use_graph in (False, True):
    As = [to_device(b.A, torch.float64) for b in blocks]
    Bs = [to_device(b.B, torch.float64) for b in blocks]
    Cs = [to_device(b.C, torch.float64) for b in blocks]
    fm.contract_batched([b.alpha for b in blocks], As, [b.A.labels for b in blocks], Bs,
                        [b.B.labels for b in blocks], [b.beta for b in blocks], Cs,
                        [b.C.labels for b in blocks], dtype="f64_emu", use_graph=use_graph)
    torch.cuda.synchronize()
    for b, C in zip(blocks, Cs):
        err = rel_frob(gpu_dense(C), run_oracle(b))
        assert err <= 1e-13, (b.name, err)
assert fm.device_status() == 0
print("env child ok")
"""


@pytest.mark.parametrize("env", [{"FAMLIES_PLAN_CACHE": "0"}, {"FAMLIES_AUTOTUNE": "0"}],
                         ids=["plan_cache_off", "autotune_off"])
def test_paths_under_environment_switches(env):
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=dict(os.environ, **env),
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "env child ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


GROUPED_CHILD = r"""
import sys
sys.path.insert(0, "tests")
import torch
import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import inputs as W
from gpu_util import gpu_dense, rel_frob, run_oracle, to_device

blocks = W.block_sparse(nblocks=24, choices=[8, 16, 24, 40])
As = [to_device(b.A, torch.float64) for b in blocks]
Bs = [to_device(b.B, torch.float64) for b in blocks]
Cs = [to_device(b.C, torch.float64) for b in blocks]
fm.contract_batched([b.alpha for b in blocks], As, [b.A.labels for b in blocks], Bs,
                    [b.B.labels for b in blocks], [b.beta for b in blocks], Cs,
                    [b.C.labels for b in blocks], dtype="f64_emu", use_graph=False)
torch.cuda.synchronize()
for b, C in zip(blocks, Cs):
    err = rel_frob(gpu_dense(C), run_oracle(b))
    assert err <= 1e-13, (b.name, err)
assert fm.device_status() == 0
print("grouped child ok")
"""


def test_grouped_tiles_finished_inside_the_product():
    # FAMLIES_GROUP_DEFER=0: the path a chunk takes when its tile slots would
    # pass their size cap
    r = subprocess.run([sys.executable, "-c", GROUPED_CHILD], cwd=ROOT,
                       env=dict(os.environ, FAMLIES_GROUP_DEFER="0"), capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "grouped child ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def _grouped_child(cache_path):
    env = dict(os.environ, FAMLIES_TUNE_CACHE=str(cache_path), FAMLIES_LOG="1")
    r = subprocess.run([sys.executable, "-c", GROUPED_CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "grouped child ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    import re
    widths = re.findall(r"grouped \d+ problems \[([^\]]+)\]: tile width (\d+) \(([a-z ]+)\)", r.stderr)
    assert widths, r.stderr[-4000:]
    return widths


def test_tuned_widths_persist_in_the_cache_file(tmp_path):
    import json
    path = tmp_path / "tune.json"
    # first process: nothing cached, the width is timed and written out
    first = _grouped_child(path)
    assert all(how == "timed now" for _, _, how in first), first
    saved = json.loads(path.read_text())
    for key, width, _ in first:
        assert saved[key] == int(width)
    # a second process takes the file's widths, even one changed by hand
    # (any of the three is correct, only speed differs)
    key, width, _ = first[0]
    other = 64 if int(width) != 64 else 128
    saved[key] = other
    path.write_text(json.dumps(saved))
    second = _grouped_child(path)
    assert (key, str(other), "tuned") in second, second
    # entries with a width that is not a tile width are ignored
    saved[key] = 96
    path.write_text(json.dumps(saved))
    third = _grouped_child(path)
    assert any(k == key and how == "timed now" for k, _, how in third), third
