"""ctypes binding of libfamlies.so (include/famlies.h): argument marshalling only.

Every step of a contraction runs in the library's CUDA kernels; this module
converts torch tensors / numpy arrays into ``famlies_tensor_t`` descriptors
and raises ``FamliesError`` on a non-zero return code.  There is no fallback:
if the shared library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfamlies.so")

F64, F64_EMU, F32, BF16 = 0, 1, 2, 3
DTYPES = {"f64": F64, "f64_emu": F64_EMU, "f32": F32, "bf16": BF16}
KERNELS = {0: "none", 1: "scale", 2: "simt_f64", 3: "simt_f32", 4: "tc_bf16", 5: "tc_tf32x3",
           6: "tc_emu", 7: "tc_bf16_gather", 8: "tc_tf32x3_gather", 9: "tc_bf16_direct"}
# option values for `kernel=`: automatic, CUDA-core, packed tensor-core, element-gathered
# tensor-core, direct bf16 (TMA boxes / gather warps), direct bf16 with both operands gathered
KERNEL_AUTO, KERNEL_SIMT, KERNEL_PACKED, KERNEL_GATHER, KERNEL_DIRECT, KERNEL_DIRECT_GATHER = 0, 1, 2, 3, 4, 5
ERR_DEVICE_TIMEOUT = -9

EXPORTS = ["famlies_contract", "famlies_contract_ex", "famlies_contract_host",
           "famlies_contract_batched", "famlies_plan", "famlies_error_string",
           "famlies_device_status", "famlies_version"]


class TensorDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("extents", ctypes.POINTER(ctypes.c_int64)),
                ("strides", ctypes.POINTER(ctypes.c_int64)), ("labels", ctypes.POINTER(ctypes.c_int32)),
                ("data", ctypes.c_void_p), ("size_bytes", ctypes.c_int64)]


def desc_array_torch(xs, labels):
    """famlies_tensor_t descriptors of many torch views at once: all extents,
    strides and labels in three flat arrays and the descriptors in a numpy
    record array laid out like TensorDesc (field offsets from ctypes), so that
    a batch of thousands of tensors costs a few attribute reads per tensor
    instead of a ctypes object each.  Returns (pointer to the first
    descriptor, the arrays to keep alive during the call)."""
    import itertools
    import numpy as np
    n = len(xs)
    shapes = [tuple(x.shape) for x in xs]
    nd = np.fromiter((len(s) for s in shapes), dtype=np.int32, count=n)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(nd, out=off[1:])
    tot = int(off[-1])
    ext = np.fromiter(itertools.chain.from_iterable(shapes), dtype=np.int64, count=tot)
    st = np.fromiter(itertools.chain.from_iterable(x.stride() for x in xs), dtype=np.int64, count=tot)
    nl = np.fromiter((len(la) for la in labels), dtype=np.int32, count=n)
    if not np.array_equal(nl, nd):
        raise ValueError("one label per mode")
    lab = np.fromiter(itertools.chain.from_iterable(labels), dtype=np.int32, count=tot)
    ptr = np.fromiter((x.data_ptr() for x in xs), dtype=np.uint64, count=n)
    size = np.fromiter((x.untyped_storage().nbytes() - x.storage_offset() * x.element_size() for x in xs),
                       dtype=np.int64, count=n)
    names = [f for f, _ in TensorDesc._fields_]
    rec = np.zeros(max(n, 1), dtype=np.dtype({
        "names": names,
        "formats": [np.int32, np.uint64, np.uint64, np.uint64, np.uint64, np.int64],
        "offsets": [getattr(TensorDesc, f).offset for f in names],
        "itemsize": ctypes.sizeof(TensorDesc)}))
    if n:
        rec["ndim"][:n] = nd
        rec["extents"][:n] = ext.ctypes.data + 8 * off[:-1]
        rec["strides"][:n] = st.ctypes.data + 8 * off[:-1]
        rec["labels"][:n] = lab.ctypes.data + 4 * off[:-1]
        rec["data"][:n] = ptr
        rec["size_bytes"][:n] = np.maximum(size, 0)
    return rec.ctypes.data_as(ctypes.POINTER(TensorDesc)), (rec, ext, st, lab)


class SymTensorDesc(ctypes.Structure):
    """famlies_symtensor_t: a symmetric operand stored as a packed lower triangle."""
    _fields_ = [("ndim", ctypes.c_int32), ("extents", ctypes.POINTER(ctypes.c_int64)),
                ("labels", ctypes.POINTER(ctypes.c_int32)), ("data", ctypes.c_void_p),
                ("size_bytes", ctypes.c_int64)]


class MatrixDesc(ctypes.Structure):
    """famlies_matrix_t: element (i, j) at data[i * rs + j * cs]."""
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("rs", ctypes.c_int64), ("cs", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_int32), ("kernel", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("stall_test", ctypes.c_int32), ("wait_limit", ctypes.c_int64),
                ("events", ctypes.c_void_p * 2), ("ctas_per_mma", ctypes.c_int32), ("reserved32", ctypes.c_int32),
                ("reserved", ctypes.c_int64)]


class Step(ctypes.Structure):
    """famlies_step_t: tensors[c] := alpha * contract(tensors[a], tensors[b]) + beta * tensors[c]."""
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("c", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("alpha", ctypes.c_double), ("beta", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("batch", ctypes.c_int64), ("m_modes", ctypes.c_int32), ("n_modes", ctypes.c_int32),
                ("k_modes", ctypes.c_int32), ("batch_modes", ctypes.c_int32),
                ("swapped", ctypes.c_int32), ("kernel", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("slices", ctypes.c_int32), ("a_contig", ctypes.c_int32), ("b_contig", ctypes.c_int32),
                ("c_contig", ctypes.c_int32), ("cached", ctypes.c_int32), ("ctas_per_mma", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["kernel_name"] = KERNELS.get(self.kernel, "?")
        return d


class FamliesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"famlies error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Loads the shared library (raises if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("FAMLIES_LIB", LIB_PATH)
    if not os.path.exists(path):
        raise FamliesError(-8, f"libfamlies.so not built at {path}; run `python -m paper_2604_07311_b300.build`")
    lib = ctypes.CDLL(path)
    T = ctypes.POINTER(TensorDesc)
    vp = ctypes.c_void_p
    d = ctypes.c_double
    lib.famlies_contract.argtypes = [d, T, T, d, T, ctypes.c_int, vp]
    lib.famlies_contract_ex.argtypes = [d, T, T, d, T, ctypes.c_int, vp, ctypes.POINTER(Options),
                                        ctypes.POINTER(PlanInfo)]
    lib.famlies_contract_host.argtypes = [d, T, T, d, T, ctypes.c_int, vp, ctypes.POINTER(Options)]
    lib.famlies_contract_batched.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), T, T,
                                             ctypes.POINTER(ctypes.c_double), T, ctypes.c_int, vp,
                                             ctypes.c_int]
    lib.famlies_plan.argtypes = [T, T, T, ctypes.c_int, ctypes.POINTER(Options), ctypes.POINTER(PlanInfo)]
    lib.famlies_network.argtypes = [T, ctypes.c_int32, ctypes.POINTER(Step), ctypes.c_int32, ctypes.c_int,
                                    vp, ctypes.POINTER(Options)]
    lib.famlies_contract_sym.argtypes = [d, ctypes.POINTER(SymTensorDesc), T, d, T, ctypes.c_int, vp,
                                         ctypes.POINTER(Options), ctypes.POINTER(PlanInfo)]
    i64 = ctypes.c_int64
    lib.famlies_gemmt_tridiag.argtypes = [i64, i64, d, vp, i64, i64, vp, vp, vp, d, vp, i64, i64, ctypes.c_int,
                                          vp, ctypes.POINTER(Options), ctypes.POINTER(PlanInfo)]
    lib.famlies_mttkrp.argtypes = [d, T, ctypes.c_int32, ctypes.POINTER(MatrixDesc), d,
                                   ctypes.POINTER(MatrixDesc), ctypes.c_int, vp, ctypes.POINTER(Options),
                                   ctypes.POINTER(PlanInfo)]
    lib.famlies_error_string.argtypes = [ctypes.c_int]
    lib.famlies_error_string.restype = ctypes.c_char_p
    lib.famlies_device_status.argtypes = [vp]
    for f in ("famlies_contract", "famlies_contract_ex", "famlies_contract_host",
              "famlies_contract_batched", "famlies_plan", "famlies_device_status", "famlies_version",
              "famlies_network", "famlies_contract_sym", "famlies_gemmt_tridiag", "famlies_mttkrp"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def error_string(code: int) -> str:
    return load().famlies_error_string(code).decode()


def check(code: int):
    if code != 0:
        raise FamliesError(code, error_string(code))


class Desc:
    """Owns the ctypes arrays behind one famlies_tensor_t."""

    def __init__(self, shape, strides, labels, data_ptr: int, size_bytes: int = 0):
        n = len(shape)
        if len(strides) != n or len(labels) != n:
            raise ValueError("shape, strides and labels must have one entry per mode")
        self._e = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in shape])
        self._s = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in strides])
        self._l = (ctypes.c_int32 * max(n, 1))(*[int(x) for x in labels])
        self.t = TensorDesc(n, self._e, self._s, self._l, ctypes.c_void_p(int(data_ptr)), int(size_bytes))

    @property
    def ref(self):
        return ctypes.byref(self.t)


def desc_torch(x, labels) -> Desc:
    """Descriptor of a torch tensor view (device pointer, element strides)."""
    st = x.untyped_storage()
    size = st.nbytes() - x.storage_offset() * x.element_size()
    return Desc(tuple(x.shape), tuple(x.stride()), labels, x.data_ptr(), max(size, 0))


def desc_numpy(x, labels) -> Desc:
    """Descriptor of a numpy view (host pointer, element strides)."""
    es = x.itemsize
    if any(s < 0 or s % es for s in x.strides):
        raise ValueError("non-negative element strides only")
    return Desc(x.shape, tuple(s // es for s in x.strides), labels, x.__array_interface__["data"][0])


def options(slices=0, kernel=0, tile_n=0, wait_limit=0, events=None, stall_test=0, ctas_per_mma=0) -> Options:
    """events: optional (begin, end) torch.cuda.Event pair recorded around the product kernel."""
    o = Options()
    o.slices, o.kernel, o.tile_n, o.wait_limit = int(slices), int(kernel), int(tile_n), int(wait_limit)
    o.stall_test = int(stall_test)
    o.ctas_per_mma = int(ctas_per_mma)
    if events is not None:
        for i, ev in enumerate(events):
            if getattr(ev, "cuda_event", 0) == 0:
                ev.record()  # materialises the underlying cudaEvent_t
            o.events[i] = ev.cuda_event
    return o
