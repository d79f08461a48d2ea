"""Thin ctypes binding of the C ABI in include/amgd.h (libamgd.so).

Every function here marshals arguments and calls the library; every step of
the strength build runs in the library's CUDA kernels.  The functions keep
the C names (``amgd_create``, ``amgd_relax``, ...) and return the C status;
``check`` turns a status into an exception.  ``Handle`` is a small
convenience wrapper over the same calls that accepts numpy arrays (host
memory) and torch tensors (device or host memory); torch is used only as a
carrier of memory and streams.

The library is loaded from the in-tree build (paper_1106_5990_gb300/_lib);
there is no fallback: if it is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# AMGD_CHECKED=1 loads the checked build (every gather index bounds-tested in
# the kernels; failures reported as AMGD_ERR_CHECK), built by
# _build.build(checked=True)
LIB_PATH = os.path.join(_HERE, "_lib", "libamgd_checked.so" if os.environ.get("AMGD_CHECKED") == "1"
                        else "libamgd.so")

AMGD_OK = 0
AMGD_ERR_ARG = -1
AMGD_ERR_CSR = -2
AMGD_ERR_ZERO_DIAG = -3
AMGD_ERR_CUDA = -4
AMGD_ERR_OOM = -5
AMGD_ERR_STATE = -6
AMGD_ERR_CAPACITY = -7
AMGD_ERR_TIMEOUT = -8
AMGD_ERR_UNSUPPORTED = -9
AMGD_ERR_CHECK = -10

AMGD_MEM_HOST = 0
AMGD_MEM_DEVICE = 1
AMGD_SWEEP_JACOBI = 0
AMGD_SWEEP_MCGS = 1
AMGD_TARGET_RESIDUAL = 0
AMGD_TARGET_PLAIN = 1
AMGD_FP64 = 0
AMGD_FP32 = 1
AMGD_BF16 = 2
AMGD_KERNEL_RELAX = 0
AMGD_KERNEL_EDGE = 1
AMGD_SUM_PLAIN = 0
AMGD_SUM_COMPENSATED = 1

PRECISIONS = {"fp64": AMGD_FP64, "fp32": AMGD_FP32, "bf16": AMGD_BF16}

# name -> (restype, argtypes); mirrors include/amgd.h
_P = ctypes.c_void_p
_i32, _i64, _u64, _f64, _int = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                ctypes.c_double, ctypes.c_int)
SIGNATURES = {
    "amgd_create": (_int, [_P, _P, _P, _i64, _i32, _u64, _int, _P]),
    "amgd_create_batch": (_int, [_i32, _P, _P, _P, _P, _i32, _u64, _int, _P]),
    "amgd_batch_offsets": (_int, [_P, _P, _P]),
    "amgd_sizes": (_int, [_P, _P, _P, _P, _P, _P]),
    "amgd_set_stream": (_int, [_P, _P]),
    "amgd_set_precision": (_int, [_P, _int]),
    "amgd_set_target": (_int, [_P, _int]),
    "amgd_set_summation": (_int, [_P, _int]),
    "amgd_set_matrix_ids": (_int, [_P, _P]),
    "amgd_set_weights": (_int, [_P, _P]),
    "amgd_set_coloring": (_int, [_P, _P, _i32, _int]),
    "amgd_init_vectors": (_int, [_P, _u64]),
    "amgd_set_vectors": (_int, [_P, _P, _int]),
    "amgd_get_vectors": (_int, [_P, _P, _int]),
    "amgd_set_values": (_int, [_P, _P, _int]),
    "amgd_relax": (_int, [_P, _i32, _f64, _int]),
    "amgd_distances": (_int, [_P, _f64, _P, _P, _P, _int]),
    "amgd_strength": (_int, [_P, _P, _P, _i64, _P, _int]),
    "amgd_graph_capture": (_int, [_P, _u64, _i32, _f64, _int, _f64, _P, _P, _i64]),
    "amgd_graph_launch": (_int, [_P]),
    "amgd_set_kernel_shape": (_int, [_P, _int, _int, _int, _int, _int]),
    "amgd_get_kernel_shape": (_int, [_P, _int, _P, _P, _P, _P]),
    "amgd_autotune": (_int, [_P, _int, _f64, ctypes.c_char_p]),
    "amgd_enable_phase_timing": (_int, [_P, _int]),
    "amgd_phase_times": (_int, [_P, _P]),
    "amgd_strength_noalloc": (_int, [_P, _P, _P, _i64, _f64, _P, _P, _i64, _P]),
    "amgd_set_checkpointing": (_int, [_P, _i32]),
    "amgd_set_search_depth": (_int, [_P, _i32]),
    "amgd_ls_interpolation": (_int, [_P, _P, _int, _i32, _f64, _P, _P, _P, _i64, _P, _P, _int]),
    "amgd_distance_pattern": (_int, [_P, _P, _P, _i64, _P, _int]),
    "amgd_cr_stats": (_int, [_P, _P, _P]),
    "amgd_set_values_async": (_int, [_P, _P, _int]),
    "amgd_strength_async": (_int, [_P, _P, _P, _i64, _int]),
    "amgd_sync": (_int, [_P]),
    "amgd_cr_coarsen": (_int, [_P, _P, _int, _P, _int, _int, _f64, _i32, _f64, _f64, _f64, _i32,
                               _u64, _P, _P]),
    "amgd_backward": (_int, [_P, _P, _int, _P, _P, _P]),
    "amgd_backward_scalars": (_int, [_P, _P, _P]),
    "amgd_graph_capture_backward": (_int, [_P, _u64, _i32, _f64, _f64, _P]),
    "amgd_destroy": (_int, [_P]),
    "amgd_status_string": (ctypes.c_char_p, [_int]),
    "amgd_last_error": (ctypes.c_char_p, [_P]),
    "amgd_checked_build": (_int, []),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libamgd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built; run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class AmgdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (amgd_status_string(status), msg))
        self.status = status


def amgd_status_string(status: int) -> str:
    return lib().amgd_status_string(status).decode()


def amgd_last_error(h) -> str:
    return lib().amgd_last_error(h).decode()


def check(status: int, h=None) -> int:
    if status != AMGD_OK:
        raise AmgdError(status, amgd_last_error(h))
    return status


# thin pass-throughs with the C names (pointers as ints)
def _wrap(name):
    def f(*args):
        return getattr(lib(), name)(*args)
    f.__name__ = name
    f.__doc__ = "C ABI %s (include/amgd.h); returns the status." % name
    return f


for _n in SIGNATURES:
    if _n not in ("amgd_status_string", "amgd_last_error"):
        globals()[_n] = _wrap(_n)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def ptr_mem(x):
    """(address, AMGD_MEM_*) of a contiguous numpy array or torch tensor."""
    if x is None:
        return None, AMGD_MEM_HOST
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("the library needs a contiguous tensor")
        return x.data_ptr(), (AMGD_MEM_DEVICE if x.is_cuda else AMGD_MEM_HOST)
    if not isinstance(x, np.ndarray) or not x.flags["C_CONTIGUOUS"]:
        raise ValueError("the library needs a contiguous numpy array")
    return x.ctypes.data, AMGD_MEM_HOST


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _count(x) -> int:
    return x.numel() if _is_torch(x) else x.size


def arg_in(x, dtype, count, name):
    """An input buffer for the library: a contiguous numpy array or torch
    tensor of `dtype` with at least `count` elements.  Another dtype, or a
    non-contiguous layout, is converted (a copy on the same device).  The
    library reads exactly the documented number of elements, so a shorter
    buffer is refused here instead of being read past its end."""
    if _is_torch(x):
        import torch
        td = getattr(torch, np.dtype(dtype).name)
        if x.dtype != td or not x.is_contiguous():
            x = x.to(td).contiguous()
    else:
        x = _host(x, dtype)
    if _count(x) < count:
        raise ValueError("%s: %d elements, the library reads %d" % (name, _count(x), count))
    return x


def arg_out(x, dtype, count, name):
    """An output buffer the library writes: it must already be a contiguous,
    writable numpy array or torch tensor of `dtype` with at least `count`
    elements (a converted copy would not be the caller's buffer)."""
    if _is_torch(x):
        import torch
        td = getattr(torch, np.dtype(dtype).name)
        if x.dtype != td or not x.is_contiguous():
            raise TypeError("%s: expected a contiguous %s tensor, got %s%s"
                            % (name, td, x.dtype, "" if x.is_contiguous() else " (strided)"))
    elif (not isinstance(x, np.ndarray) or x.dtype != np.dtype(dtype)
          or not x.flags["C_CONTIGUOUS"] or not x.flags["WRITEABLE"]):
        raise TypeError("%s: expected a contiguous writable numpy array of %s"
                        % (name, np.dtype(dtype).name))
    if _count(x) < count:
        raise ValueError("%s: %d elements, the library writes up to %d"
                         % (name, _count(x), count))
    return x


class Handle:
    """Owning wrapper of an amgd_handle."""

    def __init__(self, row_ptr, col, val, K: int, seed: int = 0, batch=None):
        L = lib()
        self.h = ctypes.c_void_p()
        if batch is None:
            rp = arg_in(row_ptr, np.int64, 1, "row_ptr")
            n = _count(rp) - 1
            nnz = int(rp[-1])                  # the library reads col and val up to row_ptr[n]
            c = arg_in(col, np.int32, max(nnz, 0), "col")
            v = arg_in(val, np.float64, max(nnz, 0), "val")
            self._keep = (rp, c, v)
            prp, mem = ptr_mem(rp)
            check(L.amgd_create(prp, ptr_mem(c)[0], ptr_mem(v)[0], n, K, seed, mem,
                                ctypes.byref(self.h)))
        else:
            mats = []                          # host arrays (the batch form reads host memory)
            for b, (r, c, v) in enumerate(batch):
                r = arg_in(_host(r, np.int64), np.int64, 1, "row_ptr of matrix %d" % b)
                nnz = max(int(r[-1]), 0)
                mats.append((r, arg_in(_host(c, np.int32), np.int32, nnz, "col of matrix %d" % b),
                             arg_in(_host(v, np.float64), np.float64, nnz,
                                    "val of matrix %d" % b)))
            nmat = len(mats)
            arr = lambda xs: (ctypes.c_void_p * nmat)(*[x.ctypes.data for x in xs])
            rps, cols, vals = arr([m[0] for m in mats]), arr([m[1] for m in mats]), \
                arr([m[2] for m in mats])
            ns = np.array([len(m[0]) - 1 for m in mats], dtype=np.int64)
            self._keep = (mats, ns)
            check(L.amgd_create_batch(nmat, rps, cols, vals, ns.ctypes.data, K, seed,
                                      AMGD_MEM_HOST, ctypes.byref(self.h)))
        n, nnz, E = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        k, nm = ctypes.c_int32(), ctypes.c_int32()
        check(L.amgd_sizes(self.h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(E),
                           ctypes.byref(k), ctypes.byref(nm)), self.h)
        self.n, self.nnz, self.E, self.K, self.nmat = n.value, nnz.value, E.value, k.value, nm.value
        self.nnz_p, self.E_p = self.nnz, self.E       # entries of the fit pattern (G_d)
        self._pending = []        # buffers of asynchronous calls, kept alive until sync()
        self._graph_keep = ()     # buffers a captured graph writes, kept alive with it

    # -- plumbing -------------------------------------------------------------
    def _ck(self, status):
        return check(status, self.h)

    def close(self):
        if self.h:
            lib().amgd_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def offsets(self):
        ro = np.zeros(self.nmat + 1, dtype=np.int64)
        so = np.zeros(self.nmat + 1, dtype=np.int64)
        self._ck(lib().amgd_batch_offsets(self.h, ro.ctypes.data, so.ctypes.data))
        return ro, so

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        s = getattr(stream, "cuda_stream", stream)
        self._ck(lib().amgd_set_stream(self.h, s))

    def set_precision(self, storage):
        storage = PRECISIONS.get(storage, storage)
        self._ck(lib().amgd_set_precision(self.h, storage))

    def set_target(self, target):
        self._ck(lib().amgd_set_target(self.h, target))

    def set_matrix_ids(self, ids):
        """Philox key word 1 of each matrix's start vectors (its index in a larger
        batch that this handle is one shard of); None restores 0..nmat-1."""
        if ids is None:
            self._ck(lib().amgd_set_matrix_ids(self.h, None))
            return
        a = np.ascontiguousarray(ids, dtype=np.int64)
        if a.shape != (self.nmat,):
            raise ValueError("set_matrix_ids: need %d ids" % self.nmat)
        self._ck(lib().amgd_set_matrix_ids(self.h, a.ctypes.data))

    def set_summation(self, mode):
        """AMGD_SUM_COMPENSATED (default) or AMGD_SUM_PLAIN, or "compensated" / "plain"."""
        if isinstance(mode, str):
            mode = {"plain": AMGD_SUM_PLAIN, "compensated": AMGD_SUM_COMPENSATED}[mode]
        self._ck(lib().amgd_set_summation(self.h, mode))

    def set_weights(self, w):
        if w is None:
            self._ck(lib().amgd_set_weights(self.h, None))
        else:
            w = _host(w, np.float64)
            self._ck(lib().amgd_set_weights(self.h, w.ctypes.data))

    def set_coloring(self, color, ncolors=None):
        c = arg_in(color, np.int32, self.n, "color")
        nc = int(c.max()) + 1 if ncolors is None else ncolors
        p, mem = ptr_mem(c)
        self._ck(lib().amgd_set_coloring(self.h, p, nc, mem))

    def init_vectors(self, seed):
        self._ck(lib().amgd_init_vectors(self.h, seed))

    def set_vectors(self, X):
        X = arg_in(X, np.float64, self.n * self.K, "X")
        p, mem = ptr_mem(X)
        self._ck(lib().amgd_set_vectors(self.h, p, mem))

    def get_vectors(self, out=None):
        out = np.empty((self.n, self.K), dtype=np.float64) if out is None else out
        p, mem = ptr_mem(arg_out(out, np.float64, self.n * self.K, "out"))
        self._ck(lib().amgd_get_vectors(self.h, p, mem))
        return out

    def set_values(self, val):
        val = arg_in(val, np.float64, self.nnz, "val")
        p, mem = ptr_mem(val)
        self._ck(lib().amgd_set_values(self.h, p, mem))

    def set_search_depth(self, d):
        """Measure the graph G_d of A^d (d >= 1); per-slot outputs then have
        nnz_p entries in the order of distance_pattern()."""
        self._ck(lib().amgd_set_search_depth(self.h, d))
        nnz_p = ctypes.c_int64()
        self._ck(lib().amgd_distance_pattern(self.h, None, None, 0, ctypes.byref(nnz_p),
                                             AMGD_MEM_HOST))
        self.nnz_p, self.E_p = nnz_p.value, nnz_p.value - self.n

    def distance_pattern(self):
        """(row_ptr int64, col int32) of the current fit pattern (host)."""
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.nnz_p, 1), dtype=np.int32)
        self._ck(lib().amgd_distance_pattern(self.h, rp.ctypes.data, col.ctypes.data,
                                             col.size, None, AMGD_MEM_HOST))
        return rp, col[:self.nnz_p]

    # -- the path -------------------------------------------------------------
    def relax(self, nu, omega, sweep=AMGD_SWEEP_JACOBI):
        self._ck(lib().amgd_relax(self.h, nu, omega, sweep))

    def distances(self, theta, want=("a", "dist", "ls"), out=None):
        """Run the edge pass; return dict of requested per-slot outputs (host numpy
        unless `out` supplies device tensors)."""
        if out is None:
            out = {k: np.empty(self.nnz_p, dtype=np.float64) for k in want}
        for k, v in out.items():
            if k not in ("a", "dist", "ls"):
                raise ValueError("distances: unknown output %r" % k)
            arg_out(v, np.float64, self.nnz_p, k)
        ptrs = [ptr_mem(out.get(k))[0] for k in ("a", "dist", "ls")]
        mems = {ptr_mem(v)[1] for v in out.values()} or {AMGD_MEM_HOST}
        if len(mems) != 1:
            raise ValueError("distances: all outputs must live in the same memory")
        self._ck(lib().amgd_distances(self.h, theta, ptrs[0], ptrs[1], ptrs[2], mems.pop()))
        return out

    def strength(self, s_row_ptr=None, s_col=None):
        """Strength CSR; host numpy by default, or into given device tensors."""
        nnz_s = ctypes.c_int64()
        if s_row_ptr is None:
            s_rp = np.empty(self.n + 1, dtype=np.int64)
            s_col = np.empty(max(self.E_p, 1), dtype=np.int32)
            self._ck(lib().amgd_strength(self.h, s_rp.ctypes.data, s_col.ctypes.data, self.E_p,
                                         ctypes.byref(nnz_s), AMGD_MEM_HOST))
            return s_rp, s_col[:nnz_s.value]
        p_rp, mem = ptr_mem(arg_out(s_row_ptr, np.int64, self.n + 1, "s_row_ptr"))
        p_col, mem2 = ptr_mem(arg_out(s_col, np.int32, 0, "s_col"))
        if mem != mem2:
            raise ValueError("strength: outputs must live in the same memory")
        self._ck(lib().amgd_strength(self.h, p_rp, p_col, _count(s_col), None, mem))
        return s_row_ptr, s_col

    def ls_interpolation(self, coarse, caliber, gamma=1.5):
        """Least-squares interpolation (host numpy): (p_row_ptr, p_col, p_val, ls)."""
        c = arg_in(coarse, np.uint8, self.n, "coarse")
        pc, cmem = ptr_mem(c)
        p_rp = np.empty(self.n + 1, dtype=np.int64)
        ls = np.empty(self.n, dtype=np.float64)
        cap = self.n * caliber
        p_col = np.empty(max(cap, 1), dtype=np.int32)
        p_val = np.empty(max(cap, 1), dtype=np.float64)
        nnz = ctypes.c_int64()
        self._ck(lib().amgd_ls_interpolation(self.h, pc, cmem, caliber, gamma, p_rp.ctypes.data,
                                             p_col.ctypes.data, p_val.ctypes.data, cap,
                                             ctypes.byref(nnz), ls.ctypes.data, AMGD_MEM_HOST))
        return p_rp, p_col[:nnz.value], p_val[:nnz.value], ls

    def cr_coarsen(self, coarse0=None, ls=None, sweep=AMGD_SWEEP_JACOBI, omega=1.0, nu=5,
                   theta=0.5, delta=0.7, tol=0.5, max_sets=20, seed=0):
        """Compatible-relaxation coarsening (host numpy): (coarse mask, rho per
        stage).  ls: LS per slot of the current pattern (numpy or torch), or
        None for the handle's last distances."""
        c = (np.zeros(self.n, dtype=np.uint8) if coarse0 is None
             else np.array(_host(coarse0, np.uint8), dtype=np.uint8, copy=True))
        if c.size < self.n:
            raise ValueError("coarse0: %d elements, the library reads %d" % (c.size, self.n))
        p_ls, ls_mem = None, AMGD_MEM_HOST
        if ls is not None:
            ls = arg_in(ls, np.float64, self.nnz_p, "ls")
            p_ls, ls_mem = ptr_mem(ls)
        rho = np.empty(max_sets + 1, dtype=np.float64)
        m = ctypes.c_int32()
        self._ck(lib().amgd_cr_coarsen(self.h, c.ctypes.data, AMGD_MEM_HOST, p_ls, ls_mem, sweep,
                                       omega, nu, theta, delta, tol, max_sets, seed,
                                       rho.ctypes.data, ctypes.byref(m)))
        return c, rho[:m.value]

    def set_values_async(self, val):
        """Stream-ordered value update (numpy array, pinned torch tensor or
        device tensor); val must stay unchanged until sync()."""
        if _is_torch(val):
            # read by a copy that runs after this call returns: a converted
            # temporary would be freed first, so the tensor must already match
            v = arg_out(val, np.float64, self.nnz, "val")
        else:
            v = arg_in(val, np.float64, self.nnz, "val")
        p, mem = ptr_mem(v)
        self._ck(lib().amgd_set_values_async(self.h, p, mem))
        self._pending.append(v)                  # alive until sync()
        return v

    def strength_async(self, s_rp, s_col):
        """Stream-ordered strength CSR into s_rp (n+1 int64) and s_col (int32,
        its length is the capacity); valid after sync()."""
        p_rp, mem = ptr_mem(arg_out(s_rp, np.int64, self.n + 1, "s_rp"))
        p_col, mem2 = ptr_mem(arg_out(s_col, np.int32, 0, "s_col"))
        if mem != mem2:
            raise ValueError("strength_async: outputs must live in the same memory")
        self._ck(lib().amgd_strength_async(self.h, p_rp, p_col, _count(s_col), mem))
        self._pending.append((s_rp, s_col))

    def sync(self):
        """Wait for the asynchronous work of the handle; raises deferred errors."""
        try:
            self._ck(lib().amgd_sync(self.h))
        finally:
            self._pending.clear()

    def cr_stats(self):
        """(selection rounds, kernel launches) of the last cr_coarsen."""
        r, l = ctypes.c_int32(), ctypes.c_int64()
        self._ck(lib().amgd_cr_stats(self.h, ctypes.byref(r), ctypes.byref(l)))
        return r.value, l.value

    # -- reverse pass ---------------------------------------------------------
    def set_checkpointing(self, every):
        self._ck(lib().amgd_set_checkpointing(self.h, every))

    def backward(self, ls_bar=None, out=None):
        """dL/dval per slot, dL/domega and the built-in loss (ls_bar None) of
        the last recorded relaxation + distances.  ls_bar and out: numpy
        arrays (host) or torch tensors (device or host), nnz float64."""
        if out is None:
            out = np.empty(self.nnz, dtype=np.float64)
        p_out, mem = ptr_mem(arg_out(out, np.float64, self.nnz, "out"))
        p_in = None
        if ls_bar is not None:
            ls_bar = arg_in(ls_bar, np.float64, self.nnz, "ls_bar")
            p_in, mem_in = ptr_mem(ls_bar)
            if mem_in != mem:
                raise ValueError("backward: ls_bar and out must live in the same memory")
        wb, loss = ctypes.c_double(), ctypes.c_double()
        self._ck(lib().amgd_backward(self.h, p_in, mem, p_out, ctypes.byref(wb),
                                     ctypes.byref(loss)))
        return out, wb.value, loss.value

    def backward_scalars(self):
        """(dL/domega, loss) of the last reverse pass (waits for it)."""
        wb, loss = ctypes.c_double(), ctypes.c_double()
        self._ck(lib().amgd_backward_scalars(self.h, ctypes.byref(wb), ctypes.byref(loss)))
        return wb.value, loss.value

    def graph_capture_backward(self, seed, nu, omega, theta, val_bar):
        """Capture forward + reverse pass (built-in loss) into the handle's
        graph; val_bar: device float64 tensor of nnz entries."""
        vb = arg_out(val_bar, np.float64, self.nnz, "val_bar")
        self._ck(lib().amgd_graph_capture_backward(self.h, seed, nu, omega, theta,
                                                   ptr_mem(vb)[0]))
        self._graph_keep = (vb,)

    def graph_capture(self, seed, nu, omega, sweep, theta, s_row_ptr, s_col):
        """Capture a whole build into the handle's CUDA graph; s_row_ptr (n+1
        int64) and s_col (int32, its length is the capacity) are device
        tensors the replays write."""
        rp = arg_out(s_row_ptr, np.int64, self.n + 1, "s_row_ptr")
        col = arg_out(s_col, np.int32, 0, "s_col")
        self._ck(lib().amgd_graph_capture(self.h, seed, nu, omega, sweep, theta,
                                          ptr_mem(rp)[0], ptr_mem(col)[0], _count(col)))
        self._graph_keep = (rp, col)

    def graph_launch(self):
        self._ck(lib().amgd_graph_launch(self.h))

    def set_kernel_shape(self, kernel, G, NV, U, staged=0):
        self._ck(lib().amgd_set_kernel_shape(self.h, kernel, G, NV, U, staged))

    def kernel_shape(self, kernel):
        """(G, NV, U, staged) of a kernel for the current storage."""
        g, nv, u, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._ck(lib().amgd_get_kernel_shape(self.h, kernel, ctypes.byref(g), ctypes.byref(nv),
                                             ctypes.byref(u), ctypes.byref(st)))
        return g.value, nv.value, u.value, st.value

    def autotune(self, sweep=AMGD_SWEEP_JACOBI, omega=1.0, cache_path=None):
        c = cache_path.encode() if cache_path else None
        self._ck(lib().amgd_autotune(self.h, sweep, omega, c))
        return self.kernel_shape(AMGD_KERNEL_RELAX), self.kernel_shape(AMGD_KERNEL_EDGE)

    def enable_phase_timing(self, enable=True):
        self._ck(lib().amgd_enable_phase_timing(self.h, int(enable)))

    def phase_times(self):
        """ms of (vector start, sweeps, distances, strength) of the last replay."""
        ms = (ctypes.c_float * 4)()
        self._ck(lib().amgd_phase_times(self.h, ms))
        return list(ms)


def build(A, K, seed=0, nu=4, omega=2.0 / 3.0, sweep=AMGD_SWEEP_JACOBI, theta=0.5,
          precision="fp64", color=None, target=AMGD_TARGET_RESIDUAL, weights=None, depth=1):
    """The whole strength build in one call: K test vectors from `seed`, nu
    sweeps, the one-point fits and the strength graph (§3, §4.1, §4.2).

    A: a torch sparse CSR tensor (CPU or CUDA; float64 values) or a
    (row_ptr, col, val) triple of numpy arrays.  color: the coloring of the
    multicolor sweep (required for AMGD_SWEEP_MCGS).  Returns (a, dist, S):
    the per-slot fit coefficient and algebraic distance r = 1/LS (in the slot
    order of the pattern: A's, or the graph of A^depth) and S = (s_row_ptr,
    s_col), the strength graph.  Torch CUDA tensors when A is on the GPU,
    numpy arrays otherwise."""
    dev = False
    if _is_torch(A):
        import torch
        dev = A.is_cuda
        rp = A.crow_indices().to(torch.int64).contiguous()
        col = A.col_indices().to(torch.int32).contiguous()
        val = A.values().to(torch.float64).contiguous()
    else:
        rp, col, val = A
    with Handle(rp, col, val, K, seed) as h:
        h.set_precision(precision)
        if target != AMGD_TARGET_RESIDUAL:
            h.set_target(target)
        if weights is not None:
            h.set_weights(weights)
        if color is not None:
            h.set_coloring(color)
        if depth > 1:
            h.set_search_depth(depth)
        h.relax(nu, omega, sweep)
        if dev:
            import torch
            out = {k: torch.empty(h.nnz_p, dtype=torch.float64, device=A.device)
                   for k in ("a", "dist")}
            h.distances(theta, want=("a", "dist"), out=out)
            s_rp = torch.empty(h.n + 1, dtype=torch.int64, device=A.device)
            s_col = torch.empty(max(h.E_p, 1), dtype=torch.int32, device=A.device)
            h.strength(s_rp, s_col)
            torch.cuda.synchronize(A.device)
            S = (s_rp, s_col[: int(s_rp[-1].item())])
        else:
            out = h.distances(theta, want=("a", "dist"))
            S = h.strength()
    return out["a"], out["dist"], S


def header_symbols(header_path: str | None = None) -> list:
    """Names of the functions declared in include/amgd.h."""
    import re
    if header_path is None:
        header_path = os.path.join(os.path.dirname(_HERE), "include", "amgd.h")
    text = open(header_path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(amgd_[a-z_]+)\s*\(", text)))
