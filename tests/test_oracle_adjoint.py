"""Pins of the oracle's reverse pass (Jacobi sweeps -> target -> one-point
fits -> loss on LS).  The paper differentiates nothing, so the reverse pass
is pinned to the mathematics of derivatives:

* central finite differences of the oracle's own forward path, for every
  matrix value, for omega and for every start-vector entry (the kept set is
  checked not to change under the perturbation);
* homogeneity: every stage is unchanged under A -> cA (D^{-1} A and the
  residual-corrected target are scale-free), so L(cA) = L(A) and Euler's
  theorem gives <dL/dA, A> = 0 exactly;
* special cases: with no sweeps and the plain target nothing depends on A or
  omega; the gradient is linear in the upstream dL/dLS.
"""
import math

import numpy as np

import oracle
from paper_1106_5990_gb300 import inputs


def _loss(orc, rp, col, val, X0, nu, omega, theta, w, mode):
    Xnu = orc.relax(rp, col, val, X0, nu, omega, oracle.SWEEP_JACOBI)
    Y = orc.target(rp, col, val, Xnu, mode)
    _, ls = orc.edge_ls(rp, col, val, Xnu, Y, w, mode)
    flag, _ = orc.threshold(rp, col, ls, theta)
    keep = (flag == 1) & (ls > 0)
    return float(np.sum(1.0 / ls[keep] ** 2)), flag


def _case(seed=11, kind="stencil"):
    if kind == "stencil":
        rp, col, val = inputs.aniso2d_9pt(5, 1e-2, math.pi / 6)
    else:   # unsymmetric values and pattern, varying diagonal
        rp, col, val = inputs.random_csr(20, 5.0, seed)
    n = len(rp) - 1
    K = 4
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, K)
    X0 = oracle.default().tv_init(n, K, seed)
    return rp, col, val, X0, w


def pin_adjoint_fd(orc):
    for kind, mode in (("stencil", oracle.TARGET_RESIDUAL), ("stencil", oracle.TARGET_PLAIN),
                       ("random", oracle.TARGET_RESIDUAL)):
        _fd_case(orc, kind, mode)


def _fd_case(orc, kind, mode):
    rp, col, val, X0, w = _case(11, kind)
    nu, omega, theta = 3, 0.7, 0.5
    r = orc.adjoint_jacobi(rp, col, val, X0, nu, omega, theta, w, mode)
    L0, f0 = _loss(orc, rp, col, val, X0, nu, omega, theta, w, mode)
    assert abs(r["loss"] - L0) <= 1e-12 * L0

    def fd(f, h):
        (lp, fp), (lm, fm) = f(h), f(-h)
        assert np.array_equal(fp, f0) and np.array_equal(fm, f0)
        return (lp - lm) / (2 * h)

    g = np.empty(len(val))
    for p in range(len(val)):
        def f(h, p=p):
            v = val.copy()
            v[p] += h
            return _loss(orc, rp, col, v, X0, nu, omega, theta, w, mode)
        g[p] = fd(f, 1e-6 * abs(val[p]))
    assert np.linalg.norm(r["val_bar"] - g) <= 1e-6 * np.linalg.norm(g)

    gw = fd(lambda h: _loss(orc, rp, col, val, X0, nu, omega + h, theta, w, mode), 1e-6)
    assert abs(r["omega_bar"] - gw) <= 1e-6 * abs(gw)

    gx = np.empty_like(X0)
    for i in range(X0.shape[0]):
        for k in range(X0.shape[1]):
            def f(h, i=i, k=k):
                X = X0.copy()
                X[i, k] += h
                return _loss(orc, rp, col, val, X, nu, omega, theta, w, mode)
            gx[i, k] = fd(f, 1e-6)
    assert np.linalg.norm(r["x0_bar"] - gx) <= 1e-6 * np.linalg.norm(gx)


def test_adjoint_matches_finite_differences(orc):
    pin_adjoint_fd(orc)


def pin_adjoint_homogeneity(orc):
    for N, mode in ((12, oracle.TARGET_RESIDUAL), (12, oracle.TARGET_PLAIN)):
        rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
        X0 = oracle.default().tv_init(N * N, 8, 5)
        r = orc.adjoint_jacobi(rp, col, val, X0, 4, 0.8, 0.5, None, mode)
        vb = r["val_bar"]
        assert np.linalg.norm(vb) > 0
        assert abs(vb @ val) <= 1e-12 * np.linalg.norm(vb) * np.linalg.norm(val)


def test_adjoint_homogeneity(orc):
    pin_adjoint_homogeneity(orc)


def pin_adjoint_special_cases(orc):
    rp, col, val, X0, w = _case(3)
    # no sweeps, plain target: LS depends on X0 only
    r = orc.adjoint_jacobi(rp, col, val, X0, 0, 0.7, 0.5, w, oracle.TARGET_PLAIN)
    assert np.all(r["val_bar"] == 0.0) and r["omega_bar"] == 0.0
    assert np.linalg.norm(r["x0_bar"]) > 0
    # no sweeps: omega enters nothing
    r = orc.adjoint_jacobi(rp, col, val, X0, 0, 0.7, 0.5, w, oracle.TARGET_RESIDUAL)
    assert r["omega_bar"] == 0.0 and np.linalg.norm(r["val_bar"]) > 0
    # the built-in loss's gradient equals an explicit upstream gradient, and
    # the result is linear in it
    r = orc.adjoint_jacobi(rp, col, val, X0, 2, 0.7, 0.5, w)
    Xnu = orc.relax(rp, col, val, X0, 2, 0.7, oracle.SWEEP_JACOBI)
    Y = orc.target(rp, col, val, Xnu)
    _, ls = orc.edge_ls(rp, col, val, Xnu, Y, w)
    flag, _ = orc.threshold(rp, col, ls, 0.5)
    lsb = np.where((flag == 1) & (ls > 0), -2.0 / np.where(ls > 0, ls, 1.0) ** 3, 0.0)
    r2 = orc.adjoint_jacobi(rp, col, val, X0, 2, 0.7, 0.5, w, ls_bar=3.0 * lsb)
    assert np.allclose(r2["val_bar"], 3.0 * r["val_bar"], rtol=1e-12, atol=0)
    assert math.isclose(r2["omega_bar"], 3.0 * r["omega_bar"], rel_tol=1e-12)
    assert math.isnan(r2["loss"])


def test_adjoint_special_cases(orc):
    pin_adjoint_special_cases(orc)
