"""FP64 CPU oracle for the algebraic-distance strength build (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (``include/amgd.h``,
the CUDA library and its Python binding) never imports, links or calls it.

The arithmetic lives in ``amgd_oracle.c`` (plain C, FP64, one row at a time
in CSR order); this module only compiles it with gcc and marshals numpy
arrays.  Paper passages followed (Brandt, Brannick, Kahl, Livshits, "An
algebraic distances measure of AMG strength of connection"):

* test vectors relaxed on A x = 0 from random starts -- §3, §5.2
* residual-corrected LS target y_i = x_i - r_i / a_ii -- Eqs. (3.2), (4.1)
* one-point LS fit and algebraic distance r_ij = 1/LS_ij -- §4.1, Eq. (4.3)
* strength graph r_ij > theta max_k r_ik -- §4.2, Eq. (4.4)
* least-squares interpolation of a given caliber -- §4.3
* compatible-relaxation coarsening -- §3.2, Eqs. (3.4), (3.5); Algorithm 1
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amgd_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liborc.so")

TARGET_RESIDUAL = 0   # y_i = x_i - r_i / a_ii   (Eqs. (3.2), (4.1), (4.3))
TARGET_PLAIN = 1      # y_i = x_i                (Eq. (3.1))
SWEEP_JACOBI = 0
SWEEP_MCGS = 1


def build_lib(force: bool = False) -> str:
    """Compile amgd_oracle.c into oracle/_lib/liborc.so with gcc (no fusion)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Oracle:
    """The oracle functions bound to one compiled copy of amgd_oracle.c.

    The default instance uses oracle/_lib/liborc.so; tests may load a
    deliberately mutated copy to show that the pins catch a planted mistake.
    """

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, f64, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
        L.orc_philox4x64_10.argtypes = [P, P, P]
        L.orc_philox4x64_10.restype = None
        L.orc_tv_init.argtypes = [i64, i32, u64, u64, P]
        L.orc_tv_init.restype = None
        L.orc_check_csr.argtypes = [i64, P, P, P]
        L.orc_check_csr.restype = ctypes.c_int
        L.orc_jacobi_sweep.argtypes = [i64, P, P, P, i32, f64, P, P]
        L.orc_jacobi_sweep.restype = None
        L.orc_mcgs_sweep.argtypes = [i64, P, P, P, P, i32, i32, f64, P, P]
        L.orc_mcgs_sweep.restype = None
        L.orc_target.argtypes = [i64, P, P, P, i32, i32, P, P]
        L.orc_target.restype = None
        L.orc_edge_ls.argtypes = [i64, P, P, P, i32, P, i32, P, P, P, P]
        L.orc_edge_ls.restype = None
        L.orc_threshold.argtypes = [i64, P, P, P, f64, P, P]
        L.orc_threshold.restype = None
        L.orc_strength_csr.argtypes = [i64, P, P, P, P, P]
        L.orc_strength_csr.restype = i64
        L.orc_adjoint_jacobi.argtypes = [i64, P, P, P, i32, P, i32, P, i32, f64, f64, P, P, P,
                                         P, P]
        L.orc_adjoint_jacobi.restype = ctypes.c_int
        L.orc_distance_graph.argtypes = [i64, P, P, i32, P, P]
        L.orc_distance_graph.restype = i64
        L.orc_edge_ls_graph.argtypes = [i64, P, P, P, P, P, i32, P, i32, P, P, P, P]
        L.orc_edge_ls_graph.restype = None
        L.orc_ls_interp.argtypes = [i64, i32, P, P, P, P, P, P, i32, f64, P, P, P, P, i64]
        L.orc_ls_interp.restype = i64
        L.orc_cr_coarsen.argtypes = [i64, P, P, P, P, P, P, i32, f64, P, i32, i32, f64, f64, f64,
                                     i32, u64, P, P]
        L.orc_cr_coarsen.restype = i32
        self.L = L
        self.path = path

    def philox4x64_10(self, ctr, key) -> np.ndarray:
        c = np.ascontiguousarray(ctr, dtype=np.uint64)
        k = np.ascontiguousarray(key, dtype=np.uint64)
        out = np.zeros(4, dtype=np.uint64)
        self.L.orc_philox4x64_10(_p(c), _p(k), _p(out))
        return out

    def tv_init(self, n: int, K: int, seed: int, stream: int = 0) -> np.ndarray:
        X = np.empty((n, K), dtype=np.float64)
        self.L.orc_tv_init(n, K, seed, stream, _p(X))
        return X

    def check_csr(self, rp, col, val) -> int:
        rp, col, val = _csr(rp, col, val)
        return int(self.L.orc_check_csr(len(rp) - 1, _p(rp), _p(col), _p(val)))

    def jacobi_sweep(self, rp, col, val, X, omega: float) -> np.ndarray:
        rp, col, val = _csr(rp, col, val)
        X = np.ascontiguousarray(X, dtype=np.float64)
        n, K = X.shape
        Xn = np.empty_like(X)
        self.L.orc_jacobi_sweep(n, _p(rp), _p(col), _p(val), K, omega, _p(X), _p(Xn))
        return Xn

    def mcgs_sweep(self, rp, col, val, color, X, omega: float = 1.0) -> np.ndarray:
        rp, col, val = _csr(rp, col, val)
        X = np.ascontiguousarray(X, dtype=np.float64)
        color = np.ascontiguousarray(color, dtype=np.int32)
        ncolors = int(color.max()) + 1 if color.size else 0
        n, K = X.shape
        Xn = np.empty_like(X)
        self.L.orc_mcgs_sweep(n, _p(rp), _p(col), _p(val), _p(color), ncolors, K, omega,
                              _p(X), _p(Xn))
        return Xn

    def relax(self, rp, col, val, X, nu: int, omega: float, sweep: int = SWEEP_JACOBI,
              color=None, keep_all: bool = False):
        """nu sweeps from X; returns the final block (and every iterate if keep_all)."""
        its = [np.ascontiguousarray(X, dtype=np.float64)]
        for _ in range(nu):
            if sweep == SWEEP_JACOBI:
                its.append(self.jacobi_sweep(rp, col, val, its[-1], omega))
            else:
                its.append(self.mcgs_sweep(rp, col, val, color, its[-1], omega))
        return its if keep_all else its[-1]

    def target(self, rp, col, val, X, mode: int = TARGET_RESIDUAL) -> np.ndarray:
        rp, col, val = _csr(rp, col, val)
        X = np.ascontiguousarray(X, dtype=np.float64)
        n, K = X.shape
        Y = np.empty_like(X)
        self.L.orc_target(n, _p(rp), _p(col), _p(val), K, mode, _p(X), _p(Y))
        return Y

    def edge_ls(self, rp, col, val, X, Y, w=None, mode: int = TARGET_RESIDUAL):
        rp, col, val = _csr(rp, col, val)
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        n, K = X.shape
        w = np.ones(K) if w is None else np.ascontiguousarray(w, dtype=np.float64)
        a = np.empty(len(col))
        ls = np.empty(len(col))
        self.L.orc_edge_ls(n, _p(rp), _p(col), _p(val), K, _p(w), mode, _p(X), _p(Y),
                           _p(a), _p(ls))
        return a, ls

    def threshold(self, rp, col, ls, theta: float):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        ls = np.ascontiguousarray(ls, dtype=np.float64)
        n = len(rp) - 1
        flag = np.empty(len(col), dtype=np.uint8)
        count = np.empty(n, dtype=np.int64)
        self.L.orc_threshold(n, _p(rp), _p(col), _p(ls), theta, _p(flag), _p(count))
        return flag, count

    def strength_csr(self, rp, col, flag):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        flag = np.ascontiguousarray(flag, dtype=np.uint8)
        n = len(rp) - 1
        s_rp = np.empty(n + 1, dtype=np.int64)
        s_col = np.empty(max(int(flag.sum()), 1), dtype=np.int32)
        k = self.L.orc_strength_csr(n, _p(rp), _p(col), _p(flag), _p(s_rp), _p(s_col))
        return s_rp, s_col[:k]

    def distance_graph(self, rp, col, d: int):
        """(row_ptr, col) of the graph G_d of A^d (structural, ascending columns)."""
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n = len(rp) - 1
        total = self.L.orc_distance_graph(n, _p(rp), _p(col), d, None, None)
        if total < 0:
            raise MemoryError("oracle distance graph: out of memory")
        prp = np.empty(n + 1, dtype=np.int64)
        pcol = np.empty(max(total, 1), dtype=np.int32)
        self.L.orc_distance_graph(n, _p(rp), _p(col), d, _p(prp), _p(pcol))
        return prp, pcol[:total]

    def edge_ls_graph(self, rp, col, val, prp, pcol, X, Y, w=None, mode: int = TARGET_RESIDUAL):
        rp, col, val = _csr(rp, col, val)
        prp = np.ascontiguousarray(prp, dtype=np.int64)
        pcol = np.ascontiguousarray(pcol, dtype=np.int32)
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        n, K = X.shape
        w = np.ones(K) if w is None else np.ascontiguousarray(w, dtype=np.float64)
        a = np.empty(len(pcol))
        ls = np.empty(len(pcol))
        self.L.orc_edge_ls_graph(n, _p(rp), _p(col), _p(val), _p(prp), _p(pcol), K, _p(w), mode,
                                 _p(X), _p(Y), _p(a), _p(ls))
        return a, ls

    def ls_interp(self, X, Y, prp, pcol, coarse, caliber: int, gamma: float = 1.5, w=None):
        """Least-squares interpolation (§4.3): P as (p_rp, p_col, p_val) and
        the chosen LS per row, from vectors X, targets Y, the neighbourhood
        pattern (prp, pcol) and the coarse mask."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        prp = np.ascontiguousarray(prp, dtype=np.int64)
        pcol = np.ascontiguousarray(pcol, dtype=np.int32)
        coarse = np.ascontiguousarray(coarse, dtype=np.uint8)
        n, K = X.shape
        w = np.ones(K) if w is None else np.ascontiguousarray(w, dtype=np.float64)
        cap = n * max(caliber, 1)
        p_rp = np.empty(n + 1, dtype=np.int64)
        p_col = np.empty(max(cap, 1), dtype=np.int32)
        p_val = np.empty(max(cap, 1), dtype=np.float64)
        ls = np.empty(n, dtype=np.float64)
        total = self.L.orc_ls_interp(n, K, _p(w), _p(X), _p(Y), _p(prp), _p(pcol), _p(coarse),
                                     caliber, gamma, _p(p_rp), _p(p_col), _p(p_val), _p(ls), cap)
        if total < 0:
            raise MemoryError("oracle interpolation: out of memory or capacity")
        return p_rp, p_col[:total], p_val[:total], ls

    def cr_coarsen(self, rp, col, val, prp, pcol, ls, theta: float = 0.5, nu: int = 5,
                   omega: float = 1.0, sweep: int = SWEEP_JACOBI, color=None,
                   delta: float = 0.7, tol: float = 0.5, max_sets: int = 20, seed: int = 0,
                   coarse0=None):
        """Compatible-relaxation coarsening (§3.2, §4.2, Algorithm 1): the
        coarse mask C and the convergence estimate rho_f of every stage, from
        A (F-relaxation), the fit pattern (prp, pcol) and its per-slot LS."""
        rp, col, val = _csr(rp, col, val)
        prp = np.ascontiguousarray(prp, dtype=np.int64)
        pcol = np.ascontiguousarray(pcol, dtype=np.int32)
        ls = np.ascontiguousarray(ls, dtype=np.float64)
        n = len(rp) - 1
        coarse = (np.zeros(n, dtype=np.uint8) if coarse0 is None
                  else np.array(coarse0, dtype=np.uint8, copy=True))
        if sweep == SWEEP_MCGS:
            color = np.ascontiguousarray(color, dtype=np.int32)
            ncol = int(color.max()) + 1 if n else 1
        else:
            color, ncol = np.zeros(max(n, 1), dtype=np.int32), 1
        rho = np.empty(max_sets + 1, dtype=np.float64)
        m = self.L.orc_cr_coarsen(n, _p(rp), _p(col), _p(val), _p(prp), _p(pcol), _p(ls), sweep,
                                  omega, _p(color), ncol, nu, theta, delta, tol, max_sets,
                                  seed, _p(coarse), _p(rho))
        if m < 0:
            raise MemoryError("oracle CR coarsening: out of memory")
        return coarse, rho[:m]

    def build(self, rp, col, val, K: int, seed: int, nu: int, omega: float, theta: float,
              sweep: int = SWEEP_JACOBI, color=None, w=None, mode: int = TARGET_RESIDUAL,
              X0=None, stream: int = 0, d: int = 1):
        """The whole path: X0 -> nu sweeps -> target -> per-edge LS -> threshold -> CSR.
        d > 1: fits, threshold and strength graph over the graph G_d of A^d."""
        n = len(rp) - 1
        X = (self.tv_init(n, K, seed, stream) if X0 is None
             else np.ascontiguousarray(X0, np.float64))
        Xnu = self.relax(rp, col, val, X, nu, omega, sweep, color)
        Y = self.target(rp, col, val, Xnu, mode)
        if d == 1:
            prp, pcol = np.asarray(rp, np.int64), np.asarray(col, np.int32)
            a, ls = self.edge_ls(rp, col, val, Xnu, Y, w, mode)
        else:
            prp, pcol = self.distance_graph(rp, col, d)
            a, ls = self.edge_ls_graph(rp, col, val, prp, pcol, Xnu, Y, w, mode)
        flag, count = self.threshold(prp, pcol, ls, theta)
        s_rp, s_col = self.strength_csr(prp, pcol, flag)
        return dict(X=Xnu, Y=Y, a=a, ls=ls, flag=flag, count=count, s_rp=s_rp, s_col=s_col,
                    prp=prp, pcol=pcol)

    def adjoint_jacobi(self, rp, col, val, X0, nu: int, omega: float, theta: float, w=None,
                       mode: int = TARGET_RESIDUAL, ls_bar=None):
        """Reverse pass through nu Jacobi sweeps, the target and the one-point
        fits.  ls_bar None: the loss is the sum of r^2 = LS^-2 over the kept
        slots with LS > 0.  Returns dict(val_bar, omega_bar, loss, x0_bar)."""
        rp, col, val = _csr(rp, col, val)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        n, K = X0.shape
        w = np.ones(K) if w is None else np.ascontiguousarray(w, dtype=np.float64)
        lsb = None if ls_bar is None else np.ascontiguousarray(ls_bar, dtype=np.float64)
        vb = np.empty(len(col))
        xb = np.empty_like(X0)
        wb = ctypes.c_double()
        loss = ctypes.c_double()
        rc = self.L.orc_adjoint_jacobi(n, _p(rp), _p(col), _p(val), K, _p(w), mode, _p(X0), nu,
                                       omega, theta, None if lsb is None else _p(lsb), _p(vb),
                                       ctypes.byref(wb), ctypes.byref(loss), _p(xb))
        if rc != 0:
            raise MemoryError("oracle adjoint: out of memory")
        return dict(val_bar=vb, omega_bar=wb.value, loss=loss.value, x0_bar=xb)


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(build_lib())
    return _default


def compile_variant(src_text: str, out_path: str) -> Oracle:
    """Compile a (mutated) copy of the oracle source and load it."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", c_path, "-o", out_path, "-lm"])
    return Oracle(out_path)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _csr(rp, col, val):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return rp, col, val


def philox4x64_10(ctr, key):
    return default().philox4x64_10(ctr, key)


def tv_init(n, K, seed, stream=0):
    return default().tv_init(n, K, seed, stream)


def check_csr(rp, col, val):
    return default().check_csr(rp, col, val)


def jacobi_sweep(rp, col, val, X, omega):
    return default().jacobi_sweep(rp, col, val, X, omega)


def mcgs_sweep(rp, col, val, color, X, omega=1.0):
    return default().mcgs_sweep(rp, col, val, color, X, omega)


def relax(rp, col, val, X, nu, omega, sweep=SWEEP_JACOBI, color=None, keep_all=False):
    return default().relax(rp, col, val, X, nu, omega, sweep, color, keep_all)


def target(rp, col, val, X, mode=TARGET_RESIDUAL):
    return default().target(rp, col, val, X, mode)


def edge_ls(rp, col, val, X, Y, w=None, mode=TARGET_RESIDUAL):
    return default().edge_ls(rp, col, val, X, Y, w, mode)


def threshold(rp, col, ls, theta):
    return default().threshold(rp, col, ls, theta)


def strength_csr(rp, col, flag):
    return default().strength_csr(rp, col, flag)


def build(rp, col, val, K, seed, nu, omega, theta, sweep=SWEEP_JACOBI, color=None,
          w=None, mode=TARGET_RESIDUAL, X0=None, stream=0, d=1):
    return default().build(rp, col, val, K, seed, nu, omega, theta, sweep, color, w, mode,
                           X0, stream, d)


def ls_interp(X, Y, prp, pcol, coarse, caliber, gamma=1.5, w=None):
    return default().ls_interp(X, Y, prp, pcol, coarse, caliber, gamma, w)


def cr_coarsen(rp, col, val, prp, pcol, ls, theta=0.5, nu=5, omega=1.0, sweep=SWEEP_JACOBI,
               color=None, delta=0.7, tol=0.5, max_sets=20, seed=0, coarse0=None):
    return default().cr_coarsen(rp, col, val, prp, pcol, ls, theta, nu, omega, sweep, color,
                                delta, tol, max_sets, seed, coarse0)


def distance_graph(rp, col, d):
    return default().distance_graph(rp, col, d)


def edge_ls_graph(rp, col, val, prp, pcol, X, Y, w=None, mode=TARGET_RESIDUAL):
    return default().edge_ls_graph(rp, col, val, prp, pcol, X, Y, w, mode)


def adjoint_jacobi(rp, col, val, X0, nu, omega, theta, w=None, mode=TARGET_RESIDUAL, ls_bar=None):
    return default().adjoint_jacobi(rp, col, val, X0, nu, omega, theta, w, mode, ls_bar)


def strength_loss(rp, col, val, X0, nu, omega, theta, w=None, mode=TARGET_RESIDUAL):
    """(loss, flag): the sum of r^2 = LS^-2 over the kept slots with LS > 0,
    by the forward path alone (Jacobi sweeps)."""
    o = default()
    Xnu = o.relax(rp, col, val, X0, nu, omega, SWEEP_JACOBI)
    Y = o.target(rp, col, val, Xnu, mode)
    a, ls = o.edge_ls(rp, col, val, Xnu, Y, w, mode)
    flag, _ = o.threshold(rp, col, ls, theta)
    keep = (flag == 1) & (ls > 0)
    return float(np.sum(1.0 / ls[keep] ** 2)), flag


def strength_ratio(rp, col, ls) -> np.ndarray:
    """rho_p = m_i / LS_p in [0,1] per off-diagonal slot (0/0 := 1); NaN on the
    diagonal.  rho > theta  <=>  the slot is strong; used to exclude edges whose
    distance lies within a band of theta from strength-set comparisons."""
    rp = np.asarray(rp, dtype=np.int64)
    col = np.asarray(col)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    off = col != rows
    ls_off = np.where(off, ls, np.inf)
    m = np.full(n, np.inf)
    np.minimum.at(m, rows, ls_off)
    mi = m[rows]
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(ls == 0, 1.0, mi / np.where(ls == 0, 1.0, ls))
    rho = np.where(off, rho, np.nan)
    return rho
