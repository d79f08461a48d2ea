"""Mixed-precision paths (FP32 or BF16 vector storage, FP32 arithmetic)
against the FP64 oracle.

Stage checks feed both sides the same generator-made vectors, exactly
representable in the storage type (multiples of 2^-7 in [-1, 1)), so that
only the mixed arithmetic differs:
  * one sweep: the stored result is within half a storage ulp of the exact
    FP64 sweep plus the FP32 rounding bound of the row sum;
  * distances: LS within 1e-3 relative of the FP64 functional (the accuracy
    bar of the mixed path), flags identical outside |rho - theta| <= 1e-3;
  * cancellation (LS << S_yy): the FP64 fallback keeps LS accurate.
End to end (same seed, every stage mixed): strength sets identical outside a
+-1e-2 band around theta; FP32 storage keeps distances within 1e-3; BF16
storage is reported by its error quantiles (rounding the vectors to BF16
alone moves distances by about 1e-3 end to end).
"""
import math

import numpy as np
import pytest

import oracle
from parity import check_flags, edge_rows, flags_from_strength_fast, ls_scales
from paper_1106_5990_gb300 import inputs

pytestmark = pytest.mark.gpu
amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")

ULP_BITS = {"bf16": 7, "fp32": 23}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()


def grid_vectors(n, K, seed):
    """Vectors on the 2^-7 grid of [-1, 1): exact in BF16 and FP32."""
    g = np.random.default_rng(seed)
    return g.integers(-128, 128, size=(n, K)).astype(np.float64) / 128.0


def ulp(x, prec):
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    return np.where(ax > 0, 2.0 ** (e - ULP_BITS[prec]), 0.0)


CASES = {
    "aniso9_64_rb": (lambda: inputs.aniso2d_9pt(64, 1e-3, math.pi / 6), "redblack64"),
    "jump3d_14": (lambda: inputs.jump3d_7pt(14, 2.0, 2), None),
    "graph_3000": (lambda: inputs.graph_laplacian(3000, 8.0, 4), None),
    "random_2000": (lambda: inputs.random_csr(2000, 7.0, 5), None),
}


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("K", [16, 32])
def test_sweep_stage(prec, case, K):
    make, col_kind = CASES[case]
    rp, col, val = make()
    n = len(rp) - 1
    X = grid_vectors(n, K, 1)
    omega = 1.0 if col_kind else 0.8
    with amgd.Handle(rp, col, val, K, 0) as h:
        h.set_precision(prec)
        h.set_vectors(X)
        assert np.array_equal(h.get_vectors(), X)      # exact in the storage type
        if col_kind:
            color = inputs.red_black(64)
            h.set_coloring(color)
            h.relax(1, omega, amgd.AMGD_SWEEP_MCGS)
            want = oracle.mcgs_sweep(rp, col, val, color, X, omega)
            # magnitude of the terms of every updated value
            S = _term_scale(rp, col, val, np.abs(X), omega)
        else:
            h.relax(1, omega, amgd.AMGD_SWEEP_JACOBI)
            want = oracle.jacobi_sweep(rp, col, val, X, omega)
            S = _term_scale(rp, col, val, np.abs(X), omega)
        got = h.get_vectors()
    deg = np.diff(rp)[:, None]
    base = 0.5 * np.maximum(ulp(want, prec), ulp(got, prec)) + (2 * deg + 8) * 2.0 ** -24 * S
    bound = base
    if col_kind:
        # a row of a later color reads the stored (rounded) new values of
        # earlier colors: their error propagates with weight |omega a_ij / a_ii|
        import scipy.sparse as sp
        color = inputs.red_black(64)
        rows, cols = edge_rows(rp, col)
        diag = val[rows == cols]
        earlier = color[cols] < color[rows]
        B = sp.csr_matrix((np.abs(omega * val[earlier] / diag[rows[earlier]]),
                           (rows[earlier], cols[earlier])), shape=(n, n))
        for _ in range(int(color.max())):
            bound = base + B @ bound
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)


def _term_scale(rp, col, val, absX, omega):
    """|x_i| + |omega/a_ii| sum_p |a_ip| |x_p| per row and component (for the
    red-black sweep the new values are bounded by the same expression of the
    old magnitudes up to one sweep; a factor 4 covers it)."""
    n = len(rp) - 1
    rows, cols = edge_rows(rp, col)
    diag = val[rows == cols]
    acc = np.zeros_like(absX)
    np.add.at(acc, rows, np.abs(val)[:, None] * absX[cols])
    return 4.0 * (absX + np.abs(omega / diag)[:, None] * acc)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("target", [0, 1])
def test_distance_stage(prec, case, target):
    make, _ = CASES[case]
    rp, col, val = make()
    n = len(rp) - 1
    K = 16
    X = grid_vectors(n, K, 2)
    Y = oracle.target(rp, col, val, X, target)
    a_w, ls_w = oracle.edge_ls(rp, col, val, X, Y, None, target)
    flag_w, _ = oracle.threshold(rp, col, ls_w, 0.5)
    with amgd.Handle(rp, col, val, K, 0) as h:
        h.set_precision(prec)
        h.set_target(target)
        h.set_vectors(X)
        out = h.distances(0.5)
        s_rp, s_col = h.strength()
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, sxx = ls_scales(rp, col, X, Y)
    big = ls_w >= 1e-8 * syy
    rel = np.abs(out["ls"] - ls_w) / np.where(big, ls_w, syy)
    assert rel[off].max() <= 1e-3, rel[off].max()
    ascale = np.abs(a_w) + np.sqrt(syy / np.maximum(sxx, 1e-300))
    assert (np.abs(out["a"] - a_w)[off] / ascale[off]).max() <= 1e-3
    flag = flags_from_strength_fast(rp, col, s_rp, s_col)
    check_flags(flag, dict(ls=ls_w, flag=flag_w), rp, col, 0.5, 1e-3)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("target", [0, 1])
def test_cancellation_uses_fp64(prec, target):
    """Rows whose target is nearly proportional to a neighbour: LS/S_yy ~ 1e-10,
    far below what FP32 two-pass sums resolve; the FP64 redo must recover it."""
    n, K = 64, 16
    rp, col, val = inputs.lap1d(n)
    g = np.random.default_rng(7)
    base = g.integers(-128, 128, size=K) / 128.0
    base[0] = 0.0
    # every row a power-of-two multiple of one vector plus a deviation of
    # 2^-20 in the component where that vector is zero: exact in FP32 and BF16
    X = np.stack([base * 2.0 ** (i % 3) * (-1) ** (i // 3) for i in range(n)])
    X[:, 0] = 2.0 ** -20 * np.where(g.random(n) < 0.5, -1.0, 1.0)
    Y = oracle.target(rp, col, val, X, target)
    a_w, ls_w = oracle.edge_ls(rp, col, val, X, Y, None, target)
    with amgd.Handle(rp, col, val, K, 0) as h:
        h.set_precision(prec)
        h.set_target(target)
        h.set_vectors(X)
        assert np.array_equal(h.get_vectors(), X)
        out = h.distances(0.5)
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, _ = ls_scales(rp, col, X, Y)
    q = ls_w[off] / syy[off]
    assert q.min() < 1e-6       # the case really is cancellation-bound
    big = ls_w >= 1e-12 * syy
    rel = np.abs(out["ls"] - ls_w) / np.where(big, ls_w, syy)
    assert rel[off].max() <= 1e-3, rel[off].max()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_cancellation_uses_fp64_colored(prec):
    """The same cancellation-bound rows on a handle whose sweeps reorder the
    rows (a coloring): the FP64 redo of the distance pass that reads the
    sweeps' row order writes every output at its caller slot."""
    n, K = 64, 16
    rp, col, val = inputs.lap1d(n)
    g = np.random.default_rng(8)
    base = g.integers(-128, 128, size=K) / 128.0
    base[0] = 0.0
    X = np.stack([base * 2.0 ** (i % 3) * (-1) ** (i // 3) for i in range(n)])
    X[:, 0] = 2.0 ** -20 * np.where(g.random(n) < 0.5, -1.0, 1.0)
    Y = oracle.target(rp, col, val, X, 0)
    a_w, ls_w = oracle.edge_ls(rp, col, val, X, Y, None, 0)
    flag_w, _ = oracle.threshold(rp, col, ls_w, 0.5)
    with amgd.Handle(rp, col, val, K, 0) as h:
        h.set_precision(prec)
        h.set_coloring(inputs.greedy_coloring(rp, col))
        h.set_vectors(X)
        assert np.array_equal(h.get_vectors(), X)
        out = h.distances(0.5)
        s_rp, s_col = h.strength()
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, _ = ls_scales(rp, col, X, Y)
    big = ls_w >= 1e-12 * syy
    rel = np.abs(out["ls"] - ls_w) / np.where(big, ls_w, syy)
    assert rel[off].max() <= 1e-3, rel[off].max()
    flag = flags_from_strength_fast(rp, col, s_rp, s_col)
    check_flags(flag, dict(ls=ls_w, flag=flag_w), rp, col, 0.5, 1e-3)


def test_compensated_sums_resolve_cancellation():
    """S_yx of a one-point fit as a cancelling sum: plain target (y_i = x_i,
    stored exactly), K = 64 full-precision FP32 components whose products
    with x_j = 1 sum to about 1e-7 of their magnitudes.  The compensated FP32
    sums reproduce the oracle's a_ij = S_yx / S_xx to 1e-5 relative; plain
    FP32 chains lose it (their error is of the size of the sum itself)."""
    n, K = 64, 64
    rp, col, val = inputs.lap1d(n)
    g = np.random.default_rng(11)
    X = np.ones((n, K))
    for i in range(0, n, 2):
        v = g.uniform(-1.0, 1.0, K).astype(np.float32).astype(np.float64)
        v[-1] = np.float32(-(v[:-1].sum()) + 3e-7)          # sum of the row ~ 3e-7
        X[i] = v
    X = X.astype(np.float32).astype(np.float64)
    Y = oracle.target(rp, col, val, X, 1)
    a_w, ls_w = oracle.edge_ls(rp, col, val, X, Y, None, 1)
    rows, cols = edge_rows(rp, col)
    sel = (rows != cols) & (rows % 2 == 0)                   # fits of the cancelling rows
    assert np.all(np.abs(a_w[sel]) < 1e-6)                   # the case really cancels
    err = {}
    for mode in ("compensated", "plain"):
        with amgd.Handle(rp, col, val, K, 0) as h:
            h.set_precision("fp32")
            h.set_target(amgd.AMGD_TARGET_PLAIN)
            h.set_summation(mode)
            h.set_vectors(X)
            out = h.distances(0.5)
        err[mode] = (np.abs(out["a"][sel] - a_w[sel]) / np.abs(a_w[sel])).max()
    print("a_ij relative error: compensated %.2e, plain %.2e" % (err["compensated"], err["plain"]))
    assert err["compensated"] <= 1e-5
    assert err["plain"] >= 1e-3


def _end_to_end(prec, rp, col, val, K, seed, nu, omega, sweep, color, theta=0.5):
    want = oracle.build(rp, col, val, K, seed, nu, omega, theta,
                        oracle.SWEEP_MCGS if sweep else oracle.SWEEP_JACOBI, color)
    with amgd.Handle(rp, col, val, K, seed) as h:
        h.set_precision(prec)
        if color is not None:
            h.set_coloring(color)
        h.relax(nu, omega, sweep)
        out = h.distances(theta)
        s_rp, s_col = h.strength()
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    flag = flags_from_strength_fast(rp, col, s_rp, s_col)
    nband = check_flags(flag, want, rp, col, theta, 1e-2)
    big = want["ls"] > 0
    rel = np.abs(out["ls"] - want["ls"])[off & big] / want["ls"][off & big]
    return rel, nband


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_end_to_end_aniso9_redblack(prec):
    N = 128
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    rel, nband = _end_to_end(prec, rp, col, val, 16, 1, 8, 1.0, amgd.AMGD_SWEEP_MCGS,
                             inputs.red_black(N))
    q50, q99, qmax = np.quantile(rel, [0.5, 0.99, 1.0])
    print("%s end-to-end LS rel err: median %.2e p99 %.2e max %.2e, band edges %d"
          % (prec, q50, q99, qmax, nband))
    if prec == "fp32":
        assert qmax <= 1e-3
    else:
        assert q50 <= 5e-3 and q99 <= 3e-2


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_end_to_end_jump3d_jacobi(prec):
    rp, col, val = inputs.jump3d_7pt(20, 2.0, 2)
    rel, _ = _end_to_end(prec, rp, col, val, 32, 3, 6, 0.8, amgd.AMGD_SWEEP_JACOBI, None)
    if prec == "fp32":
        assert rel.max() <= 1e-3
    else:
        assert np.median(rel) <= 5e-3


def test_mixed_batch_equals_separate():
    mats = [inputs.graph_laplacian(n, 4.0, 5, b) for b, n in enumerate([700, 2222, 99])]
    K, seed = 16, 6
    with amgd.Handle(None, None, None, K, seed, batch=mats) as h:
        h.set_precision("bf16")
        h.init_vectors(seed)
        h.relax(4, 2.0 / 3.0)
        out = h.distances(0.5)
        ro, so = h.offsets()
    for b, (rp, col, val) in enumerate(mats):
        with amgd.Handle(rp, col, val, K, seed) as h1:
            h1.set_vectors(oracle.tv_init(len(rp) - 1, K, seed, b))
            h1.set_precision("bf16")
            h1.relax(4, 2.0 / 3.0)
            o1 = h1.distances(0.5)
        sl = slice(so[b], so[b + 1])
        assert np.array_equal(o1["ls"], out["ls"][sl], equal_nan=True)
        assert np.array_equal(o1["a"], out["a"][sl])
