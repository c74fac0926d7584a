"""Host-only checks of the C ABI: the library loads, exports every symbol the
header declares, and the planner (label classes, index fusion, role swap,
validation errors) behaves as specified.  No device is touched."""
import os
import re
import subprocess
import sys

import pytest

import paper_2604_07311_b300 as fm
from paper_2604_07311_b300 import _lib
from paper_2604_07311_b300 import inputs as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_07311_b300 import build
    build.build()


def header_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            text = open(os.path.join(ROOT, "include", name)).read()
            syms |= set(re.findall(r"FAMLIES_API\s+[\w\s\*]+?\b(famlies_\w+)\s*\(", text))
    return syms


def test_library_exports_every_declared_symbol():
    syms = header_symbols()
    assert {"famlies_contract", "famlies_contract_batched", "famlies_plan"} <= syms
    out = subprocess.check_output(["nm", "-D", "--defined-only", _lib.LIB_PATH]).decode()
    exported = set(re.findall(r"\bT\s+(famlies_\w+)", out))
    assert syms <= exported, syms - exported
    lib = fm.load()
    for s in syms:
        assert hasattr(lib, s)
    assert lib.famlies_version() >= 100
    assert "label" in fm.error_string(-2)


def P(prob, dtype="f64", **kw):
    return fm.plan(prob.A.extents, prob.A.strides, prob.A.labels, prob.B.extents, prob.B.strides,
                   prob.B.labels, prob.C.extents, prob.C.strides, prob.C.labels, dtype=dtype, **kw)


def test_plan_four_index():
    info = P(W.four_index(ext=16))
    assert (info["m"], info["n"], info["k"], info["batch"]) == (256, 256, 256, 1)
    assert (info["m_modes"], info["n_modes"], info["k_modes"]) == (2, 2, 2)
    assert info["swapped"] == 0 and info["a_contig"] == 1 and info["b_contig"] == 2
    assert info["kernel_name"] == "simt_f64"


def test_plan_ladder_fuses_to_gemm():
    info = P(W.ladder(v=8, o=4), dtype="f64_emu")
    assert (info["m"], info["n"], info["k"]) == (64, 16, 64)
    assert (info["m_modes"], info["n_modes"], info["k_modes"]) == (1, 1, 1)
    assert info["a_contig"] == 1 and info["b_contig"] == 2 and info["c_contig"] == 1
    assert info["kernel_name"] == "tc_emu" and info["slices"] == 6


def test_plan_transpose_free_swaps_roles():
    info = P(W.transpose_free(v=6, o=3, pad=7), dtype="bf16")
    # C[b,j,a,i]: unit stride on b, an index of B -> B supplies the rows
    assert info["swapped"] == 1
    assert (info["m"], info["n"], info["k"]) == (18, 18, 18)
    assert info["m_modes"] == 2 and info["n_modes"] == 2
    assert info["a_contig"] == 1 and info["b_contig"] == 1 and info["c_contig"] == 1
    # every class has two modes and each operand is unit-stride along a free
    # mode: the direct kernel stages its tiles from the strides (no pack)
    assert info["kernel_name"] == "tc_bf16_direct"
    assert P(W.transpose_free(v=6, o=3, pad=7), dtype="bf16", kernel=2)["kernel_name"] == "tc_bf16"


def test_plan_direct_bf16_selection():
    """The direct bf16 kernel takes a call when every class has at most two
    modes, the batch at most one, each operand has a unit stride along a free
    or a contracted mode and k <= 16384; otherwise the packed kernel does,
    and asking for the direct one is an error."""
    gemm = dict(A_shape=(64, 32), A_strides=(1, 64), la=[1, 2], B_shape=(32, 48), B_strides=(1, 32),
                lb=[2, 3], C_shape=(64, 48), C_strides=(1, 64), lc=[1, 3], dtype="bf16")
    assert fm.plan(**gemm)["kernel_name"] == "tc_bf16_direct"
    long_k = dict(gemm, A_shape=(64, 20000), B_shape=(20000, 48), B_strides=(1, 20000))
    assert fm.plan(**long_k)["kernel_name"] == "tc_bf16"
    # three row modes that do not fuse
    three = dict(gemm, A_shape=(4, 4, 4, 32), A_strides=(1, 5, 25, 125), la=[1, 4, 5, 2],
                 C_shape=(4, 4, 4, 48), C_strides=(1, 4, 16, 64), lc=[1, 4, 5, 3])
    assert fm.plan(**three)["kernel_name"] == "tc_bf16"
    # no unit stride in A at all
    strided = dict(gemm, A_strides=(2, 128))
    assert fm.plan(**strided)["kernel_name"] == "tc_bf16"
    for bad in (long_k, three, strided):
        with pytest.raises(fm.FamliesError) as e:
            fm.plan(**bad, kernel=4)
        assert e.value.code == -6
    with pytest.raises(fm.FamliesError) as e:
        fm.plan(**dict(gemm, dtype="f32"), kernel=4)
    assert e.value.code == -6
    assert fm.plan(**gemm, kernel=5)["kernel_name"] == "tc_bf16_direct"


def test_plan_batch_labels_and_extent_one_modes():
    # C[i,b] = sum_k A[i,k,b] B[k,b,u] with u of extent 1 in B only -> label error;
    # with u in C too: u is an N mode of extent 1 and is dropped.
    info = fm.plan((3, 4, 5), (1, 3, 12), [1, 2, 3], (4, 5, 1), (1, 4, 20), [2, 3, 4],
                   (3, 5, 1), (1, 3, 15), [1, 3, 4])
    assert info["batch"] == 5 and info["batch_modes"] == 1
    assert info["n"] == 1 and info["n_modes"] == 0
    with pytest.raises(fm.FamliesError) as e:
        fm.plan((3, 4, 5), (1, 3, 12), [1, 2, 3], (4, 5, 1), (1, 4, 20), [2, 3, 4],
                (3, 5), (1, 3), [1, 3])
    assert e.value.code == -2


@pytest.mark.parametrize("case,code", [
    ("only_in_a", -2), ("repeat", -2), ("extent", -3), ("neg_extent", -1), ("c_overlap", -6),
    ("bounds", -5), ("alias", -4), ("bad_dtype", -1)])
def test_plan_errors(case, code):
    A = dict(shape=(4, 5), strides=(1, 4), labels=[1, 2])
    B = dict(shape=(5, 6), strides=(1, 5), labels=[2, 3])
    C = dict(shape=(4, 6), strides=(1, 4), labels=[1, 3])
    ptrs = (0x10000, 0x20000000, 0x40000000)
    dtype = "f64"
    if case == "only_in_a":
        A["shape"], A["strides"], A["labels"] = (4, 5, 2), (1, 4, 20), [1, 2, 9]
    elif case == "repeat":
        A["labels"] = [1, 1]
    elif case == "extent":
        B["shape"] = (7, 6)
    elif case == "neg_extent":
        A["shape"] = (-4, 5)
    elif case == "c_overlap":
        C["strides"] = (1, 2)
    elif case == "alias":
        ptrs = (0x10000, 0x20000000, 0x10000 + 8)
    elif case == "bad_dtype":
        dtype = 7
    lib = fm.load()
    da = _lib.Desc(A["shape"], A["strides"], A["labels"], ptrs[0], 152 if case == "bounds" else 0)
    db = _lib.Desc(B["shape"], B["strides"], B["labels"], ptrs[1])
    dc = _lib.Desc(C["shape"], C["strides"], C["labels"], ptrs[2])
    info = _lib.PlanInfo()
    dt = dtype if isinstance(dtype, int) else _lib.DTYPES[dtype]
    rc = lib.famlies_plan(da.ref, db.ref, dc.ref, dt, None, info)
    assert rc == code


def test_no_device_is_reported_not_faked():
    """Without a GPU the compute entry points fail loudly (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = fm.load()
    da = _lib.Desc((4, 5), (1, 4), [1, 2], 0x10000)
    db = _lib.Desc((5, 6), (1, 5), [2, 3], 0x20000000)
    dc = _lib.Desc((4, 6), (1, 4), [1, 3], 0x40000000)
    rc = lib.famlies_contract(1.0, da.ref, db.ref, 0.0, dc.ref, 0, None)
    assert rc == -10


def _net_err(tensors, steps, dtype="f64"):
    with pytest.raises(fm.FamliesError) as e:
        fm.contract_network(tensors, steps, dtype=dtype, stream=0)
    return e.value.code


def test_network_validation_before_any_launch():
    """famlies_network rejects malformed sequences on the host, before it
    touches a device: indices out of range, a step writing one of its own
    operands, an intermediate read before it is written or first written
    with beta != 0, and bf16 intermediates."""
    INVALID, UNSUPPORTED = -1, -6
    t = [((4, 5), [1, 2]), ((5, 6), [2, 3]), ((4, 6), [1, 3])]  # all intermediates
    assert _net_err(t, [(0, 1, 3, 1.0, 0.0)]) == INVALID            # c out of range
    assert _net_err(t, [(0, 1, 0, 1.0, 0.0)]) == INVALID            # c == a
    assert _net_err(t, [(0, 1, 2, 1.0, 0.0)]) == INVALID            # A, B never written
    u = [((4, 5), [1, 2]), ((5, 6), [2, 3]), ((4, 6), [1, 3]), ((6, 7), [3, 4]), ((4, 7), [1, 4])]
    # 2 := 0 * 1 needs 0 and 1 written first; 4 := 2 * 3 with beta != 0 on a fresh 4
    assert _net_err(u, [(0, 1, 2, 1.0, 0.0)]) == INVALID
    assert _net_err(u, [(2, 3, 4, 1.0, 1.0)]) == INVALID
    # bf16 with an intermediate: caller tensors at fake addresses (the check
    # comes before anything is dereferenced)
    import ctypes
    lib = _lib.load()
    descs = [_lib.Desc((4, 5), (1, 4), [1, 2], 0x10000, 40), _lib.Desc((5, 6), (1, 5), [2, 3], 0x20000, 60),
             _lib.Desc((4, 6), (0, 0), [1, 3], 0), _lib.Desc((6, 7), (1, 6), [3, 4], 0x30000, 84),
             _lib.Desc((4, 7), (1, 4), [1, 4], 0x40000, 56)]
    tt = (_lib.TensorDesc * 5)(*[d.t for d in descs])
    ss = (_lib.Step * 2)(_lib.Step(0, 1, 2, 0, 1.0, 0.0), _lib.Step(2, 3, 4, 0, 1.0, 0.0))
    assert lib.famlies_network(tt, 5, ss, 2, fm.BF16, None, None) == UNSUPPORTED


def _sym_rc(ext, la, b, c, dtype=None, size_bytes=0):
    """famlies_contract_sym on descriptors at fake addresses (host checks only)."""
    import ctypes
    lib = _lib.load()
    nd = len(ext)
    e = (ctypes.c_int64 * nd)(*ext)
    lab = (ctypes.c_int32 * nd)(*la)
    a = _lib.SymTensorDesc(nd, e, lab, ctypes.c_void_p(0x10000000), size_bytes)
    info = _lib.PlanInfo()
    return lib.famlies_contract_sym(1.0, ctypes.byref(a), b.ref, 0.0, c.ref,
                                    fm.F64_EMU if dtype is None else dtype, None, None, ctypes.byref(info))


def test_symmetric_operand_validation():
    """famlies_contract_sym checks the symmetric operand on the host: an even
    number of modes with equal halves, the packed size, the dtype, and one
    fused index per half (one contracted, one free)."""
    INVALID, OOB, UNSUPPORTED = -1, -5, -6
    v, o = 4, 3
    B = _lib.Desc((v, v, o), (1, v, v * v), [3, 4, 5], 0x20000000)
    C = _lib.Desc((v, v, o), (1, v, v * v), [1, 2, 5], 0x40000000)
    assert _sym_rc((v, v, v), [1, 2, 3], B, C) == INVALID                     # odd number of modes
    assert _sym_rc((v, v, v, v + 1), [1, 2, 3, 4], B, C) == INVALID           # halves differ
    assert _sym_rc((v, v, v, v), [1, 2, 3, 4], B, C, dtype=fm.F64) == UNSUPPORTED
    n = v * v
    assert _sym_rc((v, v, v, v), [1, 2, 3, 4], B, C, size_bytes=n * (n + 1) // 2 * 8 - 8) == OOB
    # K = (c, d) stored d-fastest in B: the contracted half does not fuse
    Bt = _lib.Desc((v, v, o), (v, 1, v * v), [3, 4, 5], 0x20000000)
    assert _sym_rc((v, v, v, v), [1, 2, 3, 4], Bt, C) == UNSUPPORTED
    # one mode of each half contracted, the others free
    B2 = _lib.Desc((v, v, o), (1, v, v * v), [2, 4, 5], 0x20000000)
    C2 = _lib.Desc((v, v, o), (1, v, v * v), [1, 3, 5], 0x40000000)
    assert _sym_rc((v, v, v, v), [1, 2, 3, 4], B2, C2) == UNSUPPORTED


def test_gemmt_validation():
    """famlies_gemmt_tridiag rejects bad arguments on the host: negative
    sizes or strides, bf16, a missing subdiagonal, and C overlapping A
    (checked by the planner before any device work)."""
    lib = _lib.load()
    opt = _lib.options()
    info = _lib.PlanInfo()
    call = lambda n, k, A, rsa, csa, sub, C, rsc, csc, dt=fm.F64_EMU: lib.famlies_gemmt_tridiag(
        n, k, -1.0, A, rsa, csa, sub, None, None, 1.0, C, rsc, csc, dt, None, opt, info)
    A, C, sub = 0x10000000, 0x20000000, 0x30000000
    assert call(-1, 4, A, 1, 8, sub, C, 1, 8) == -1
    assert call(8, 4, A, -1, 8, sub, C, 1, 8) == -1
    assert call(8, 4, A, 1, 8, sub, C, 1, 8, fm.BF16) == -6
    assert call(8, 4, A, 1, 8, None, C, 1, 8) == -1          # k > 1 needs the subdiagonal
    assert call(8, 4, A, 1, 8, sub, A + 64, 1, 8) == -4     # C overlaps A


def test_mttkrp_validation():
    """famlies_mttkrp checks shapes, dtype and aliasing on the host."""
    import ctypes
    lib = _lib.load()
    X = _lib.Desc((4, 5, 6), (1, 4, 20), [0, 0, 0], 0x10000000)
    M = lambda rows, ptr=0x20000000: _lib.MatrixDesc(ptr, rows, 3, 1, rows)
    U = lambda e, ptr: _lib.MatrixDesc(ptr, e, 3, 1, e)
    us = (_lib.MatrixDesc * 3)(U(4, 0x30000000), U(5, 0x40000000), U(6, 0x50000000))
    info = _lib.PlanInfo()
    call = lambda mode, m, dt=fm.F64_EMU, u=us: lib.famlies_mttkrp(1.0, X.ref, mode, u, 0.0, ctypes.byref(m),
                                                                   dt, None, None, ctypes.byref(info))
    assert call(3, M(4)) == -1                        # mode out of range
    assert call(0, M(5)) == -3                        # M's rows are not X's extent
    assert call(0, M(4), fm.BF16) == -6
    bad = (_lib.MatrixDesc * 3)(U(4, 0x30000000), U(7, 0x40000000), U(6, 0x50000000))
    assert call(0, M(4), u=bad) == -3                 # a factor of the wrong height
    assert call(0, M(4, 0x40000000 + 16)) == -4       # M overlaps a factor
    assert call(0, M(4, 0x10000000 + 64)) == -4       # M overlaps X



def test_oversized_generated_operands_are_rejected():
    """A packed symmetric operand whose size overflows and a Khatri-Rao layout
    whose offsets overflow are refused on the host (UNSUPPORTED)."""
    big = 1 << 31
    B = _lib.Desc((big, 3), (1, big), [2, 3], 0x20000000)
    C = _lib.Desc((big, 3), (1, big), [1, 3], 0x40000000)
    assert _sym_rc((big, big), [1, 2], B, C) == -6
    import ctypes
    lib = _lib.load()
    e = 1 << 21
    X = _lib.Desc((4, e, e, e), (1, 4, 4 * e, 4 * e * e), [0, 0, 0, 0], 0x10000000)
    us = (_lib.MatrixDesc * 4)(*[_lib.MatrixDesc(0x30000000, n, 3, 1, n) for n in (4, e, e, e)])
    M = _lib.MatrixDesc(0x50000000, 4, 3, 1, 4)
    info = _lib.PlanInfo()
    assert lib.famlies_mttkrp(1.0, X.ref, 0, us, 0.0, ctypes.byref(M), fm.F64_EMU, None, None,
                              ctypes.byref(info)) == -6


def test_environment_defaults_for_slices_and_tile_width():
    """FAMLIES_SLICES and FAMLIES_FORCE_TILE fill options left at 0; an
    invalid tile width from the environment is refused like one passed in."""
    code = ("import paper_2604_07311_b300 as fm\n"
            "i = fm.plan((64, 32), (1, 64), [1, 2], (32, 48), (1, 32), [2, 3], (64, 48), (1, 64), [1, 3], "
            "dtype='f64_emu')\n"
            "print(i['slices'])\n"
            "i = fm.plan((64, 32), (1, 64), [1, 2], (32, 48), (1, 32), [2, 3], (64, 48), (1, 64), [1, 3], "
            "dtype='f64_emu', slices=4)\n"
            "print(i['slices'])\n")
    env = dict(os.environ, FAMLIES_SLICES="5")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert r.stdout.split() == ["5", "4"], r.stderr
    env = dict(os.environ, FAMLIES_FORCE_TILE="96")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)
    assert "famlies error -1" in r.stderr


def test_ctypes_structs_match_the_header(tmp_path):
    """Every struct the binding marshals has the header's size and field
    offsets (a C program compiled against include/famlies.h prints them)."""
    pairs = [("famlies_tensor_t", _lib.TensorDesc), ("famlies_symtensor_t", _lib.SymTensorDesc),
             ("famlies_matrix_t", _lib.MatrixDesc), ("famlies_options_t", _lib.Options),
             ("famlies_step_t", _lib.Step), ("famlies_plan_info_t", _lib.PlanInfo)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "famlies.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    import ctypes
    for cname, cls in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_ctas_per_mma_option_is_validated():
    """ctas_per_mma takes 0, 1 or 2; anything else is an invalid argument.  The
    host-only plan reports one CTA per MMA (pairs are decided with the device)."""
    A = ((64, 96), (1, 64), [1, 2])
    B = ((96, 80), (1, 96), [2, 3])
    C = ((64, 80), (1, 64), [1, 3])
    for v in (0, 1, 2):
        info = fm.plan(*A, *B, *C, dtype="f64_emu", ctas_per_mma=v)
        assert info["ctas_per_mma"] == 1
    for v in (-1, 3):
        with pytest.raises(fm.FamliesError) as e:
            fm.plan(*A, *B, *C, dtype="f64_emu", ctas_per_mma=v)
        assert e.value.code == -1  # FAMLIES_ERR_INVALID_ARG


def test_bulk_batch_descriptors_match_single_ones():
    # The grouped call marshals its descriptors in bulk; each must read as the
    # per-tensor descriptor of the same view (any strides, storage offsets,
    # a 0-mode tensor, mixed ranks).
    import torch
    from paper_2604_07311_b300 import _lib
    base = torch.zeros(4000, dtype=torch.float64)
    xs = [base[:24].view(2, 3, 4).permute(2, 0, 1),
          base[100:100 + 60].view(5, 12)[:, 1:7],
          base[7:8].view(()),
          base[1000:].view(-1, 30)[:, ::3],
          torch.zeros(3, 1, 5, dtype=torch.float64).transpose(0, 2)]
    labels = [[1, 2, 3], [4, 5], [], [6, 7], [8, 9, 10]]
    p, keep = _lib.desc_array_torch(xs, labels)
    for i, (x, la) in enumerate(zip(xs, labels)):
        d = _lib.desc_torch(x, la).t
        q = p[i]
        assert (q.ndim, q.data, q.size_bytes) == (d.ndim, d.data, d.size_bytes)
        for m in range(d.ndim):
            assert (q.extents[m], q.strides[m], q.labels[m]) == (d.extents[m], d.strides[m], d.labels[m])
    with pytest.raises(ValueError):
        _lib.desc_array_torch(xs[:2], [[1, 2, 3], [4]])
    with pytest.raises(ValueError):
        _lib.desc_array_torch(xs[:2], [[1, 2], [3, 4, 5]])
