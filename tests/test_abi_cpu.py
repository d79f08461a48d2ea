"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/amgd.h declares, and rejects bad arguments on the host before
touching the device."""
import ctypes
import os

import numpy as np
import pytest

from paper_1106_5990_gb300 import _build, amgd, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return amgd.lib()


def test_exports_every_header_symbol(L):
    names = amgd.header_symbols(os.path.join(ROOT, "include", "amgd.h"))
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(amgd.SIGNATURES)


def test_status_strings(L):
    for code in range(0, -10, -1):
        s = amgd.amgd_status_string(code)
        assert s.startswith("AMGD_")
    assert amgd.amgd_status_string(-99) == "unknown status"


def _create(rp, col, val, K=4):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    st = amgd.lib().amgd_create(rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                len(rp) - 1, K, 0, amgd.AMGD_MEM_HOST, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("case,code", [
    ("rp0", amgd.AMGD_ERR_CSR), ("decreasing", amgd.AMGD_ERR_CSR),
    ("col_range", amgd.AMGD_ERR_CSR), ("duplicate", amgd.AMGD_ERR_CSR),
    ("nonfinite", amgd.AMGD_ERR_CSR), ("zero_diag", amgd.AMGD_ERR_ZERO_DIAG),
    ("no_diag", amgd.AMGD_ERR_ZERO_DIAG), ("K0", amgd.AMGD_ERR_UNSUPPORTED),
    ("K65", amgd.AMGD_ERR_UNSUPPORTED)])
def test_create_rejects_bad_input_on_host(L, case, code):
    rp, col, val = inputs.lap1d(6)
    rp, col, val = rp.copy(), col.copy(), val.copy()
    K = 4
    if case == "rp0":
        rp = rp + 1
    elif case == "decreasing":
        rp[3] = rp[2] - 1
    elif case == "col_range":
        col[2] = 6
    elif case == "duplicate":
        col[1] = col[0]
    elif case == "nonfinite":
        val[4] = np.nan
    elif case == "zero_diag":
        val[0] = 0.0
    elif case == "no_diag":
        col[0] = 2      # row 0 becomes (2, 1): no diagonal, no duplicate
        col[0], col[1] = 1, 2
    elif case == "K0":
        K = 0
    elif case == "K65":
        K = 65
    st, h = _create(rp, col, val, K)
    assert st == code, (case, st, amgd.amgd_last_error(None))
    assert not h.value
    assert amgd.amgd_last_error(None)


def _create_batch(mats, K=4):
    nm = len(mats)
    rps = [np.ascontiguousarray(m[0], np.int64) for m in mats]
    cols = [np.ascontiguousarray(m[1], np.int32) for m in mats]
    vals = [np.ascontiguousarray(m[2], np.float64) for m in mats]
    arr = lambda xs: (ctypes.c_void_p * nm)(*[x.ctypes.data for x in xs])
    ns = np.array([len(r) - 1 for r in rps], np.int64)
    h = ctypes.c_void_p()
    st = amgd.lib().amgd_create_batch(nm, arr(rps), arr(cols), arr(vals), ns.ctypes.data, K, 0,
                                      amgd.AMGD_MEM_HOST, ctypes.byref(h))
    return st, h


def test_create_batch_rejects_a_bad_matrix_on_host(L):
    """Every matrix of a batch is validated on the host before any device
    work, and the message names the matrix and the row."""
    good = inputs.lap1d(6)
    rp, col, val = (x.copy() for x in inputs.lap1d(5))
    col[2] = 9
    st, h = _create_batch([good, (rp, col, val)])
    assert st == amgd.AMGD_ERR_CSR and not h.value
    assert "matrix 1" in amgd.amgd_last_error(None)
    rp, col, val = (x.copy() for x in inputs.lap1d(5))
    val[0] = 0.0
    st, h = _create_batch([(rp, col, val), good])
    assert st == amgd.AMGD_ERR_ZERO_DIAG and not h.value
    assert "matrix 0" in amgd.amgd_last_error(None)
    st, h = _create_batch([good, good], K=65)
    assert st == amgd.AMGD_ERR_UNSUPPORTED and not h.value


def test_create_rejects_sizes_beyond_the_abi_on_host(L):
    """0 <= n < 2^31 and nnz < 2^31: the limits are checked before an array
    is read past what the caller passed (row_ptr is read only after n is
    accepted, col and val only after nnz = row_ptr[n] is)."""
    h = ctypes.c_void_p()
    rp = np.array([0, 1], np.int64)
    col = np.zeros(1, np.int32)
    val = np.ones(1)
    args = lambda r, n: (r.ctypes.data, col.ctypes.data, val.ctypes.data, n, 4, 0,
                         amgd.AMGD_MEM_HOST, ctypes.byref(h))
    assert L.amgd_create(*args(rp, -1)) == amgd.AMGD_ERR_ARG
    assert L.amgd_create(*args(rp, 1 << 31)) == amgd.AMGD_ERR_UNSUPPORTED
    assert "2^31" in amgd.amgd_last_error(None)
    big = np.array([0, 1 << 31], np.int64)                     # nnz = 2^31, col never read
    assert L.amgd_create(*args(big, 1)) == amgd.AMGD_ERR_UNSUPPORTED
    neg = np.array([0, -5], np.int64)
    assert L.amgd_create(*args(neg, 1)) == amgd.AMGD_ERR_CSR
    # a batch whose total row count reaches 2^31
    nm = 2
    ptrs = (ctypes.c_void_p * nm)(rp.ctypes.data, rp.ctypes.data)
    cptrs = (ctypes.c_void_p * nm)(col.ctypes.data, col.ctypes.data)
    vptrs = (ctypes.c_void_p * nm)(val.ctypes.data, val.ctypes.data)
    ns = np.array([1 << 30, 1 << 30], np.int64)
    assert L.amgd_create_batch(nm, ptrs, cptrs, vptrs, ns.ctypes.data, 4, 0, amgd.AMGD_MEM_HOST,
                               ctypes.byref(h)) == amgd.AMGD_ERR_UNSUPPORTED
    assert not h.value


def test_null_arguments(L):
    assert L.amgd_create(None, None, None, 0, 4, 0, 0, None) == amgd.AMGD_ERR_ARG
    assert L.amgd_create_batch(0, None, None, None, None, 4, 0, 0, None) == amgd.AMGD_ERR_ARG
    assert L.amgd_destroy(None) == amgd.AMGD_OK
    assert L.amgd_relax(None, 1, 1.0, 0) == amgd.AMGD_ERR_ARG
    assert L.amgd_strength(None, None, None, 0, None, 0) == amgd.AMGD_ERR_ARG


def test_noalloc_rejects_arguments_on_the_host(L):
    """Size and pointer checks of amgd_strength_noalloc run before any CUDA
    call (this machine has no GPU)."""
    P = ctypes.c_void_p(16)          # never dereferenced: every call below fails its checks
    assert L.amgd_strength_noalloc(P, P, P, -1, 0.5, P, P, 0, None) == amgd.AMGD_ERR_ARG
    assert "< 0" in amgd.amgd_last_error(None)
    assert L.amgd_strength_noalloc(P, P, P, 268_435_457, 0.5, P, P, 0, None) == \
        amgd.AMGD_ERR_UNSUPPORTED
    assert "268435456" in amgd.amgd_last_error(None)
    assert L.amgd_strength_noalloc(None, P, P, 4, 0.5, P, P, 0, None) == amgd.AMGD_ERR_ARG
    assert L.amgd_strength_noalloc(P, None, P, 4, 0.5, P, P, 0, None) == amgd.AMGD_ERR_ARG
    assert L.amgd_strength_noalloc(P, P, P, 4, -0.5, P, P, 0, None) == amgd.AMGD_ERR_ARG
    assert L.amgd_strength_noalloc(P, P, P, 4, 0.5, P, None, 3, None) == amgd.AMGD_ERR_ARG
    assert L.amgd_strength_noalloc(P, P, P, 4, 0.5, P, P, -1, None) == amgd.AMGD_ERR_ARG


# entry points whose first argument is not a handle, or that accept a NULL one
_NOT_HANDLE_FIRST = {"amgd_create", "amgd_create_batch", "amgd_destroy", "amgd_strength_noalloc",
                     "amgd_status_string", "amgd_last_error", "amgd_checked_build"}


def test_checked_build_flag(L):
    """The library the tests load by default is the normal build; its
    status text covers the checked build's error code."""
    assert L.amgd_checked_build() == 0
    assert amgd.amgd_status_string(amgd.AMGD_ERR_CHECK).startswith("AMGD_ERR_CHECK")


@pytest.mark.parametrize("name", sorted(set(amgd.SIGNATURES) - _NOT_HANDLE_FIRST))
def test_every_handle_call_rejects_a_null_handle(L, name):
    """A NULL handle is an argument error on the host: no entry point
    dereferences it or reaches the device (this machine has no GPU)."""
    _, argtypes = amgd.SIGNATURES[name]
    args = [None if t is ctypes.c_void_p or t is ctypes.c_char_p else t(0) for t in argtypes]
    assert getattr(L, name)(*args) == amgd.AMGD_ERR_ARG, name


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(amgd, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(amgd, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        amgd.lib()


def test_binding_checks_buffers_before_the_library():
    """The binding hands the library only buffers of the documented dtype and
    length: inputs of another dtype are converted, outputs must match, and a
    short buffer is refused instead of being read or written past its end."""
    torch = pytest.importorskip("torch")
    # inputs: converted (numpy and torch), length checked
    x = amgd.arg_in([1, 2, 3], np.int64, 3, "x")
    assert x.dtype == np.int64 and x.flags["C_CONTIGUOUS"]
    t = amgd.arg_in(torch.arange(6, dtype=torch.int32)[::2], np.float64, 3, "t")
    assert t.dtype == torch.float64 and t.is_contiguous() and t.tolist() == [0.0, 2.0, 4.0]
    same = torch.zeros(4, dtype=torch.float64)
    assert amgd.arg_in(same, np.float64, 4, "same") is same          # no copy when it matches
    with pytest.raises(ValueError):
        amgd.arg_in(np.zeros(2), np.float64, 3, "short")
    with pytest.raises(ValueError):
        amgd.arg_in(torch.zeros(2), np.float64, 3, "short")
    # outputs: must already be right
    out = np.zeros(5, np.int32)
    assert amgd.arg_out(out, np.int32, 5, "out") is out
    for bad in (np.zeros(5, np.int64), np.zeros(10, np.int32)[::2], [0] * 5,
                torch.zeros(5, dtype=torch.int64)):
        with pytest.raises(TypeError):
            amgd.arg_out(bad, np.int32, 5, "out")
    ro = np.zeros(5, np.int32)
    ro.flags.writeable = False
    with pytest.raises(TypeError):
        amgd.arg_out(ro, np.int32, 5, "out")
    with pytest.raises(ValueError):
        amgd.arg_out(np.zeros(4, np.int32), np.int32, 5, "out")
    with pytest.raises(ValueError):
        amgd.arg_out(torch.zeros(4, dtype=torch.int32), np.int32, 5, "out")
    # ptr_mem refuses strided buffers (no assert that -O would strip)
    with pytest.raises(ValueError):
        amgd.ptr_mem(np.zeros(10)[::2])
    with pytest.raises(ValueError):
        amgd.ptr_mem(torch.zeros(10)[::2])
