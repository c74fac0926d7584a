"""The seeded input recipe (inputs.py) against what it states: shapes, mode
orders, strides and padding, the distributions' parameters, the ladder's
symmetry, the block-sparse extent set, determinism per seed, and that the
module holds no arithmetic of the method (it imports neither the library's
compute path nor the oracle)."""
import ast
import os

import numpy as np

from paper_2604_07311_b300 import inputs as W


def test_four_index_layout_and_flops():
    p = W.four_index(ext=6)
    assert p.A.labels == W.L("acik") and p.B.labels == W.L("ckbj") and p.C.labels == W.L("abij")
    assert p.A.extents == (6, 6, 6, 6) and p.A.strides == (1, 6, 36, 216)
    assert (p.alpha, p.beta) == (1.0, 0.0)
    assert not np.any(p.C.view())
    assert p.flops == 2 * 6 ** 6  # six distinct labels
    a = p.A.view()
    assert -1.0 <= a.min() and a.max() <= 1.0


def test_ladder_symmetry_spread_and_shapes():
    v, o = 16, 4
    p = W.ladder(v=v, o=o)
    V = p.A.view()
    assert p.A.labels == W.L("abcd") and p.B.labels == W.L("cdij") and p.C.labels == W.L("abij")
    assert p.A.strides == (1, v, v * v, v ** 3)
    # symmetric under the exchange of its first and second halves of modes
    assert np.array_equal(V, V.transpose(2, 3, 0, 1))
    # entries N(0,1)/128 (65536 of them: the sample deviation within 3 %)
    assert abs(V.std() * 128.0 - 1.0) < 0.03
    assert abs(p.B.view().std() / 1e-2 - 1.0) < 0.1
    assert p.C.view().min() >= -1.0 and p.C.view().max() <= 1.0
    assert (p.alpha, p.beta) == (1.0, 1.0)
    assert p.flops == 2 * v ** 4 * o ** 2


def test_transpose_free_padding_and_permuted_output():
    v, o, pad = 6, 3, 7
    p = W.transpose_free(v=v, o=o, pad=pad)
    assert p.A.labels == W.L("acik") and p.B.labels == W.L("bkjc") and p.C.labels == W.L("bjai")
    assert p.A.extents == (v, v, o, o)
    assert p.A.strides == (1, v + pad, (v + pad) * v, (v + pad) * v * o)
    # the padding holds values the view never shows
    used = np.zeros(p.A.buf.shape, dtype=bool)
    idx = np.indices(p.A.extents).reshape(4, -1)
    used[np.dot(np.array(p.A.strides), idx)] = True
    assert np.any(p.A.buf[~used] != 0.0)
    assert p.B.strides == W.colmajor_strides((v, o, o, v))
    assert p.C.extents == (v, o, v, o) and (p.alpha, p.beta) == (1.0, 0.0)


def test_block_sparse_extents_and_blocks():
    ext = W.block_sparse_extents(nblocks=500)
    assert ext.shape == (500, 6)
    assert set(np.unique(ext)) <= set(range(8, 97, 8)) and len(np.unique(ext)) == 12
    small = W.block_sparse_extents(nblocks=50, choices=[8, 16, 24, 32])
    assert set(np.unique(small)) <= {8, 16, 24, 32}
    blocks = W.block_sparse(nblocks=3, choices=[8, 16])
    for b, e in zip(blocks, W.block_sparse_extents(nblocks=3, choices=[8, 16])):
        a_, b_, c_, i_, j_, k_ = (int(x) for x in e)
        assert b.A.extents == (a_, c_, i_, k_) and b.B.extents == (c_, k_, b_, j_)
        assert b.C.extents == (a_, b_, i_, j_)
        assert b.flops == 2 * a_ * b_ * c_ * i_ * j_ * k_


def test_autograd_problem_shapes():
    d = W.autograd_problem(i=5, j=4, l=3, k=2, m=6)
    assert d["A"].shape == (5, 2, 6, 3) and d["B"].shape == (2, 6, 4) and d["T"].shape == (5, 4, 3)
    assert d["la"] == W.L("ikml") and d["lb"] == W.L("kmj") and d["lc"] == W.L("ijl")


def test_seeded_determinism():
    for make in (lambda s: W.four_index(ext=5, seed=s), lambda s: W.ladder(v=6, o=2, seed=s),
                 lambda s: W.transpose_free(v=5, o=2, seed=s)):
        p, q, r = make(11), make(11), make(12)
        for x, y in ((p.A, q.A), (p.B, q.B), (p.C, q.C)):
            assert np.array_equal(x.buf, y.buf)
        assert not np.array_equal(p.B.buf, r.B.buf)


def test_recipe_module_imports_no_method_code():
    path = os.path.join(os.path.dirname(W.__file__), "inputs.py")
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            names.add((node.module or "").split(".")[0] if node.level == 0 else "." + (node.module or ""))
    assert names <= {"__future__", "dataclasses", "numpy"}, names
