"""GPU (C-ABI) against the FP64 oracle on the same seeded inputs.

Sizes are small enough for the oracle to finish in seconds but span several
blocks/tiles of every kernel and ragged tails; edge cases cover n = 0, a
single row, rows without off-diagonals, degree-one rows, long rows, K = 1 and
K = 64.
"""
import math

import numpy as np
import pytest

import oracle
from parity import (check_a, check_flags, check_ls, edge_rows, flags_from_strength,
                    flags_from_strength_fast, ls_scales)
from paper_1106_5990_gb300 import inputs

pytestmark = pytest.mark.gpu

amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()
    torch.cuda.init()


MATRICES = {
    "poisson5_37": lambda: inputs.poisson2d_5pt(37),
    "aniso9_40": lambda: inputs.aniso2d_9pt(40, 1e-3, math.pi / 6),
    "aniso7_33": lambda: inputs.aniso2d_7pt(33, 0.1, -math.pi / 4),
    "lap1d_1000": lambda: inputs.lap1d(1000),
    "random_1500": lambda: inputs.random_csr(1500, 6.0, 11),
    "random_sym_900": lambda: inputs.random_csr(900, 5.0, 12, symmetric_pattern=True),
    "jump3d_12": lambda: inputs.jump3d_7pt(12, 2.0, 2),
    "graph_2000": lambda: inputs.graph_laplacian(2000, 8.0, 4),
}


def gpu_build(rp, col, val, K, seed, nu, omega, theta, sweep=0, color=None, w=None,
              target=0, precision="fp64", X0=None, edge_stage=None, edge_u=None):
    with amgd.Handle(rp, col, val, K, seed) as h:
        if precision != "fp64":
            h.set_precision(precision)
        if edge_stage is not None:
            G, NV, U, _ = h.kernel_shape(amgd.AMGD_KERNEL_EDGE)
            h.set_kernel_shape(amgd.AMGD_KERNEL_EDGE, G, NV, edge_u or U, edge_stage)
        if color is not None:
            h.set_coloring(color)
        if w is not None:
            h.set_weights(w)
        if target:
            h.set_target(target)
        if X0 is not None:
            h.set_vectors(X0)
        h.relax(nu, omega, sweep)
        X = h.get_vectors()
        out = h.distances(theta)
        s_rp, s_col = h.strength()
    return dict(X=X, a=out["a"], ls=out["ls"], dist=out["dist"], s_rp=s_rp, s_col=s_col)


def compare_fp64(rp, col, val, got, want, theta, w=None):
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    assert np.array_equal(got["X"], want["X"]), "test vectors differ"
    syy, sxx = ls_scales(rp, col, want["X"], want["Y"], w)
    check_ls(got["ls"], want["ls"], syy, off)
    check_a(got["a"], want["a"], syy, sxx, off)
    assert np.all(np.isnan(got["ls"][~off])) and np.all(got["a"][~off] == 0)
    with np.errstate(divide="ignore"):
        np.testing.assert_array_equal(got["dist"][off], 1.0 / got["ls"][off])
    flag = flags_from_strength(rp, col, got["s_rp"], got["s_col"]) if len(rp) < 5000 else \
        flags_from_strength_fast(rp, col, got["s_rp"], got["s_col"])
    check_flags(flag, want, rp, col, theta, 1e-9)


# --------------------------------------------------------------------------- X0
@pytest.mark.parametrize("K", [1, 2, 3, 5, 8, 16, 17, 32, 33, 64])
def test_x0_fp64_bit_exact(K):
    rp, col, val = inputs.random_csr(777, 4.0, K)
    with amgd.Handle(rp, col, val, K, seed=1234 + K) as h:
        X = h.get_vectors()
        h.init_vectors(99)
        X2 = h.get_vectors()
    assert np.array_equal(X, oracle.tv_init(777, K, 1234 + K))
    assert np.array_equal(X2, oracle.tv_init(777, K, 99))


def test_x0_rounded_storages():
    rp, col, val = inputs.poisson2d_5pt(30)
    want = oracle.tv_init(900, 16, 5)
    with amgd.Handle(rp, col, val, 16, 5) as h:
        h.set_precision("fp32")
        assert np.array_equal(h.get_vectors(), want.astype(np.float32).astype(np.float64))
        h.init_vectors(5)
        assert np.array_equal(h.get_vectors(), want.astype(np.float32).astype(np.float64))
        h.set_precision("bf16")
        h.init_vectors(5)
        got = h.get_vectors()
    ulp = 2.0 ** (np.floor(np.log2(np.abs(want))) - 7)
    assert np.all(np.abs(got - want) <= 0.5 * ulp)


# --------------------------------------------------------------------------- sweeps
@pytest.mark.parametrize("name", list(MATRICES))
@pytest.mark.parametrize("K", [1, 3, 8, 16, 32])
def test_jacobi_sweeps_bit_exact(name, K):
    rp, col, val = MATRICES[name]()
    n = len(rp) - 1
    X0 = oracle.tv_init(n, K, 7)
    want = oracle.relax(rp, col, val, X0, 3, 0.7)
    with amgd.Handle(rp, col, val, K, 7) as h:
        h.relax(3, 0.7, amgd.AMGD_SWEEP_JACOBI)
        assert np.array_equal(h.get_vectors(), want)


@pytest.mark.parametrize("name,coloring", [
    ("aniso9_40", "redblack"), ("poisson5_37", "redblack"), ("random_1500", "greedy"),
    ("random_sym_900", "random3"), ("graph_2000", "greedy"), ("aniso7_33", "redblack")])
@pytest.mark.parametrize("K", [2, 16, 64])
def test_mcgs_sweeps_bit_exact(name, coloring, K):
    rp, col, val = MATRICES[name]()
    n = len(rp) - 1
    if coloring == "redblack":
        color = inputs.red_black(int(round(math.sqrt(n))))
    elif coloring == "greedy":
        color = inputs.greedy_coloring(rp, col)
    else:
        color = np.random.default_rng(3).integers(0, 3, n).astype(np.int32)
    X0 = oracle.tv_init(n, K, 3)
    for omega in (1.0, 1.2):
        want = oracle.relax(rp, col, val, X0, 2, omega, oracle.SWEEP_MCGS, color)
        with amgd.Handle(rp, col, val, K, 3) as h:
            h.set_coloring(color)
            h.relax(2, omega, amgd.AMGD_SWEEP_MCGS)
            assert np.array_equal(h.get_vectors(), want)


def arrow(n):
    """1D Laplacian plus a dense first row and column (row 0 holds every
    column): a row far longer than a gather batch or a tile's CSR lines, next to
    rows of two or three entries.  Diagonally dominant."""
    import scipy.sparse as sp
    i = np.arange(n)
    rows = np.concatenate([i[1:], i[:-1], np.zeros(n - 1, int), i[1:]])
    cols = np.concatenate([i[:-1], i[1:], i[1:], np.zeros(n - 1, int)])
    vals = -np.concatenate([np.ones(2 * (n - 1)), np.full(2 * (n - 1), 0.01)])
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A = A + sp.diags(np.asarray(abs(A).sum(1)).ravel() + 1.0)
    A = sp.csr_matrix(A)
    A.sort_indices()
    return (A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64))


TILE_CASES = {
    "aniso9_40": (lambda: inputs.aniso2d_9pt(40, 1e-3, math.pi / 6), "redblack"),
    "graph_2000": (lambda: inputs.graph_laplacian(2000, 8.0, 4), "greedy"),
    "random_1500": (lambda: inputs.random_csr(1500, 6.0, 11), "greedy"),
    "arrow_3001": (lambda: arrow(3001), "greedy"),
}


def _coloring(rp, col, kind):
    n = len(rp) - 1
    return (inputs.red_black(int(round(math.sqrt(n)))) if kind == "redblack"
            else inputs.greedy_coloring(rp, col))


@pytest.mark.parametrize("U", [4, 8])
@pytest.mark.parametrize("NV", [1, 2])
@pytest.mark.parametrize("case", list(TILE_CASES))
@pytest.mark.parametrize("K", [5, 16, 64])
def test_stage3_sweeps_bit_exact(case, NV, U, K):
    """The persistent relaxation kernel with L2 prefetch (stage 3: each warp
    prefetches the row pointers and CSR lines of its rows one and two tiles
    ahead) equals the oracle bit for bit in FP64, Jacobi and multicolor
    Gauss-Seidel, including a dense row far longer than a gather batch next
    to short rows."""
    make, kind = TILE_CASES[case]
    rp, col, val = make()
    n = len(rp) - 1
    color = _coloring(rp, col, kind)
    X0 = oracle.tv_init(n, K, 5)
    P = 1
    while 2 * P < K:
        P *= 2
    if P % NV:
        pytest.skip("shape does not tile the row")
    with amgd.Handle(rp, col, val, K, 5) as h:
        h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, P // NV, NV, U, 3)
        h.relax(3, 0.7, amgd.AMGD_SWEEP_JACOBI)
        assert np.array_equal(h.get_vectors(), oracle.relax(rp, col, val, X0, 3, 0.7))
    with amgd.Handle(rp, col, val, K, 5) as h:
        h.set_coloring(color)
        h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, P // NV, NV, U, 3)
        h.relax(2, 1.1, amgd.AMGD_SWEEP_MCGS)
        want = oracle.relax(rp, col, val, X0, 2, 1.1, oracle.SWEEP_MCGS, color)
        assert np.array_equal(h.get_vectors(), want)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("case", list(TILE_CASES))
def test_stage3_sweeps_mixed_equal_direct(prec, case):
    """FP32 arithmetic on FP32/BF16 storage: the stage-3 kernel stores the
    same bits as the direct kernel (same FMA chains in the same order)."""
    make, kind = TILE_CASES[case]
    rp, col, val = make()
    color = _coloring(rp, col, kind)
    K = 16
    P = {"fp32": 4, "bf16": 2}[prec]
    got = []
    for shape in [(P, 1, 4, 0), (P, 1, 4, 3), (P // 2, 2, 8, 3)]:
        with amgd.Handle(rp, col, val, K, 6) as h:
            h.set_precision(prec)
            h.set_coloring(color)
            h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, *shape)
            h.relax(3, 1.0, amgd.AMGD_SWEEP_MCGS)
            got.append(h.get_vectors())
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[2])


# --------------------------------------------------------------------------- full build
@pytest.mark.parametrize("name", list(MATRICES))
@pytest.mark.parametrize("K,target", [(8, 0), (16, 0), (16, 1), (5, 0), (33, 0)])
def test_build_fp64_parity(name, K, target):
    rp, col, val = MATRICES[name]()
    theta, nu, omega = 0.5, 4, 2.0 / 3.0
    want = oracle.build(rp, col, val, K, 0, nu, omega, theta, mode=target)
    got = gpu_build(rp, col, val, K, 0, nu, omega, theta, target=target)
    compare_fp64(rp, col, val, got, want, theta)


@pytest.mark.parametrize("edge_stage,edge_u", [(None, None), (3, 8)])
def test_build_fp64_mcgs_weights(edge_stage, edge_u):
    N = 48
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    w = np.random.default_rng(0).uniform(0.5, 2.0, 16)
    for theta in (0.25, 0.5, 0.8):
        want = oracle.build(rp, col, val, 16, 1, 8, 1.0, theta, oracle.SWEEP_MCGS, color, w=w)
        got = gpu_build(rp, col, val, 16, 1, 8, 1.0, theta, 1, color, w=w,
                        edge_stage=edge_stage, edge_u=edge_u)
        compare_fp64(rp, col, val, got, want, theta, w)


def _tile_edge_matrices():
    """Tiles of the edge pass: ragged tile ends, rows without off-diagonals,
    one-off-diagonal rows, and a row longer than a tile's slot capacity
    (a tile of its own) next to short rows."""
    yield "graph_2000", inputs.graph_laplacian(2000, 8.0, 4)
    yield "sparse_graph_isolated", inputs.graph_laplacian(700, 0.4, 9)
    yield "lap1d_1000", inputs.lap1d(1000)
    import scipy.sparse as sp
    n = 5000                       # row 17 couples to every row: 5000 entries
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(4.0 if i != 17 else float(n))
        if i != 17:
            rows += [17, i]; cols += [i, 17]; vals += [-0.5, -0.25]
        if i + 1 < n:
            rows += [i, i + 1]; cols += [i + 1, i]; vals += [-1.0, -1.0]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    yield "one_long_row", (A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data)


@pytest.mark.parametrize("K,target", [(16, 0), (8, 1), (33, 0)])
def test_edge_tile_kernel_matches_oracle(K, target):
    for name, (rp, col, val) in _tile_edge_matrices():
        want = oracle.build(rp, col, val, K, 3, 3, 0.6, 0.5, mode=target)
        got = gpu_build(rp, col, val, K, 3, 3, 0.6, 0.5, target=target, edge_stage=1)
        compare_fp64(rp, col, val, got, want, 0.5)


@pytest.mark.parametrize("K,target,U", [(16, 0, 4), (8, 1, 8), (33, 0, 8), (5, 0, 4), (64, 0, 4)])
def test_edge_warp_kernel_matches_oracle(K, target, U):
    """The warp-staged distance kernel (edge stage 3) against the oracle: runs
    of rows parked in the warp's shared-memory window and, for long rows, not
    parked (graph_2000, the 5000-entry row), ragged last warps, rows without
    off-diagonals and one-off-diagonal rows."""
    for name, (rp, col, val) in _tile_edge_matrices():
        want = oracle.build(rp, col, val, K, 3, 3, 0.6, 0.5, mode=target)
        got = gpu_build(rp, col, val, K, 3, 3, 0.6, 0.5, target=target, edge_stage=3, edge_u=U)
        compare_fp64(rp, col, val, got, want, 0.5)


# --------------------------------------------------------------------------- edge cases
def _one_row_matrices():
    yield "single_row", (np.array([0, 1]), np.array([0], np.int32), np.array([2.0]))
    # rows without off-diagonals interleaved with coupled rows
    rp, col, val = inputs.graph_laplacian(300, 0.4, 9)
    yield "sparse_graph_isolated", (rp, col, val)
    # one long row (dense first row and column)
    n = 700
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(float(n))
        if i > 0:
            rows += [0, i]; cols += [i, 0]; vals += [-1.0, -0.5]
        if 0 < i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(-0.25)
    import scipy.sparse as sp
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    yield "long_row", (A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data)


@pytest.mark.parametrize("K", [1, 2, 64])
def test_edge_case_matrices(K):
    for name, (rp, col, val) in _one_row_matrices():
        for target in (0, 1):
            want = oracle.build(rp, col, val, K, 2, 3, 0.6, 0.5, mode=target)
            got = gpu_build(rp, col, val, K, 2, 3, 0.6, 0.5, target=target)
            if K == 1:
                # k = 1 < caliber: every fit is exact up to rounding (LS ~ 0),
                # distances are rounding noise; compare vectors and LS scale only
                assert np.array_equal(got["X"], want["X"]), name
                rows, cols = edge_rows(rp, col)
                off = rows != cols
                syy, _ = ls_scales(rp, col, want["X"], want["Y"])
                assert np.all(got["ls"][off] <= 1e-28 * syy[off] + 1e-300), name
                continue
            compare_fp64(rp, col, val, got, want, 0.5)


@pytest.mark.parametrize("where", ["cuda", "cpu", "numpy"])
def test_one_call_build(where):
    """amgd.build on a torch sparse CSR tensor (GPU or CPU) or a numpy triple
    equals the oracle's build (FP64)."""
    import torch
    rp, col, val = inputs.aniso2d_9pt(32, 1e-3, math.pi / 6)
    color = inputs.red_black(32)
    want = oracle.build(rp, col, val, 8, 3, 4, 1.0, 0.5, oracle.SWEEP_MCGS, color)
    if where == "numpy":
        A = (rp, col, val)
    else:
        A = torch.sparse_csr_tensor(torch.from_numpy(rp), torch.from_numpy(col.astype(np.int64)),
                                    torch.from_numpy(val), size=(1024, 1024)).to(where)
    a, dist, (s_rp, s_col) = amgd.build(A, 8, seed=3, nu=4, omega=1.0, sweep=amgd.AMGD_SWEEP_MCGS,
                                        theta=0.5, color=color)
    if where == "cuda":
        a, dist, s_rp, s_col = (t.cpu().numpy() for t in (a, dist, s_rp, s_col))
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, sxx = ls_scales(rp, col, want["X"], want["Y"])
    check_a(a, want["a"], syy, sxx, off)
    with np.errstate(divide="ignore"):
        check_ls(1.0 / dist, want["ls"], syy, off)
    check_flags(flags_from_strength(rp, col, s_rp, s_col), want, rp, col, 0.5, 1e-9)


def test_empty_matrix():
    rp = np.zeros(1, np.int64)
    col = np.zeros(0, np.int32)
    val = np.zeros(0)
    with amgd.Handle(rp, col, val, 4, 0) as h:
        assert h.n == 0 and h.E == 0
        h.relax(2, 0.7)
        h.distances(0.5)
        s_rp, s_col = h.strength()
        # coarsening, interpolation and the stream-ordered calls on no rows
        C, rho = h.cr_coarsen(np.zeros(0, np.uint8), ls=np.zeros(0))
        assert len(C) == 0 and list(rho) == [0.0]
        P = h.ls_interpolation(np.zeros(0, np.uint8), 2)
        assert list(P[0]) == [0] and len(P[1]) == 0
        h.set_values_async(val)
        o_rp = np.full(1, -1, np.int64)
        h.sync()
        h.distances(0.5)
        h.strength_async(o_rp, np.zeros(0, np.int32))
        h.sync()
        assert list(o_rp) == [0]
    assert list(s_rp) == [0] and len(s_col) == 0


def test_ragged_tile_boundaries():
    """n around the compaction tile (4096 rows) and warp/block multiples."""
    for n in (4095, 4096, 4097, 8193):
        rp, col, val = inputs.lap1d(n)
        want = oracle.build(rp, col, val, 4, 1, 2, 0.6, 0.5, mode=1)
        got = gpu_build(rp, col, val, 4, 1, 2, 0.6, 0.5, target=1)
        compare_fp64(rp, col, val, got, want, 0.5)


# --------------------------------------------------------------------------- batch, graph
def test_batch_equals_separate_and_oracle():
    mats = [inputs.graph_laplacian(n, 4.0, 5, b) for b, n in enumerate([300, 1111, 57, 2500])]
    K, nu, omega, theta, seed = 16, 4, 2.0 / 3.0, 0.5, 6
    with amgd.Handle(None, None, None, K, seed, batch=mats) as h:
        h.relax(nu, omega)
        out = h.distances(theta)
        s_rp, s_col = h.strength()
        X = h.get_vectors()
        ro, so = h.offsets()
    for b, (rp, col, val) in enumerate(mats):
        want = oracle.build(rp, col, val, K, seed, nu, omega, theta, stream=b)
        sl = slice(so[b], so[b + 1])
        rs = slice(ro[b], ro[b + 1])
        got = dict(X=X[rs], a=out["a"][sl], ls=out["ls"][sl], dist=out["dist"][sl],
                   s_rp=s_rp[ro[b]:ro[b + 1] + 1] - s_rp[ro[b]],
                   s_col=s_col[s_rp[ro[b]]:s_rp[ro[b + 1]]] - ro[b])
        compare_fp64(rp, col, val, got, want, theta)
        # identical to a single-matrix handle keyed by (seed, b): same bits
        with amgd.Handle(rp, col, val, K, seed) as h1:
            h1.set_vectors(oracle.tv_init(len(rp) - 1, K, seed, b))
            h1.relax(nu, omega)
            o1 = h1.distances(theta)
        assert np.array_equal(o1["ls"], got["ls"], equal_nan=True)
        assert np.array_equal(o1["a"], got["a"])


def test_graph_capture_equals_stepwise():
    import torch
    N = 64
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    for prec in ("fp64", "bf16"):
        with amgd.Handle(rp, col, val, 16, 1) as h:
            h.set_precision(prec)
            h.set_coloring(color)
            d_rp = torch.empty(N * N + 1, dtype=torch.int64, device="cuda")
            d_col = torch.empty(h.E, dtype=torch.int32, device="cuda")
            h.graph_capture(1, 8, 1.0, amgd.AMGD_SWEEP_MCGS, 0.5, d_rp, d_col)
            for _ in range(3):
                h.graph_launch()
            torch.cuda.synchronize()
            g_ls = h.distances(0.5)["ls"]   # recomputed from the graph's final vectors
            g_rp, g_col = d_rp.cpu().numpy(), d_col.cpu().numpy()
            h.init_vectors(1)
            h.relax(8, 1.0, amgd.AMGD_SWEEP_MCGS)
            s_ls = h.distances(0.5)["ls"]
            s_rp, s_col = h.strength()
        assert np.array_equal(g_ls, s_ls, equal_nan=True)
        assert np.array_equal(g_rp, s_rp)
        assert np.array_equal(g_col[:g_rp[-1]], s_col)


def test_graph_replay_after_set_values():
    """amgd_set_values writes the new values in place, so a captured build
    replayed afterwards uses them (FP64 against the oracle on the new
    values, host and device sources, colored and plain handles)."""
    import torch
    N = 48
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    rng = np.random.default_rng(3)
    val2 = val * rng.uniform(0.8, 1.25, len(val))
    color = inputs.red_black(N)
    for colored in (False, True):
        sweep = amgd.AMGD_SWEEP_MCGS if colored else amgd.AMGD_SWEEP_JACOBI
        osweep = oracle.SWEEP_MCGS if colored else oracle.SWEEP_JACOBI
        omega = 1.0 if colored else 2.0 / 3.0
        want = oracle.build(rp, col, val2, 16, 2, 5, omega, 0.5, osweep,
                            color if colored else None)
        with amgd.Handle(rp, col, val, 16, 2) as h:
            if colored:
                h.set_coloring(color)
            d_rp = torch.empty(N * N + 1, dtype=torch.int64, device="cuda")
            d_col = torch.empty(h.E, dtype=torch.int32, device="cuda")
            h.graph_capture(2, 5, omega, sweep, 0.5, d_rp, d_col)
            h.graph_launch()
            for src in (val2, torch.from_numpy(val2).cuda()):
                h.set_values(src)
                h.graph_launch()
                torch.cuda.synchronize()
                s_rp = d_rp.cpu().numpy()
                got = dict(X=h.get_vectors(), s_rp=s_rp, s_col=d_col[: s_rp[-1]].cpu().numpy())
                got.update(h.distances(0.5))     # same vectors: the graph's distances
                compare_fp64(rp, col, val2, got, want, 0.5)


# --------------------------------------------------------------------------- API states
def test_state_errors_and_roundtrips():
    rp, col, val = inputs.poisson2d_5pt(20)
    with amgd.Handle(rp, col, val, 8, 0) as h:
        with pytest.raises(amgd.AmgdError) as e:
            h.relax(1, 1.0, amgd.AMGD_SWEEP_MCGS)
        assert e.value.status == amgd.AMGD_ERR_STATE
        with pytest.raises(amgd.AmgdError) as e:
            h.strength()
        assert e.value.status == amgd.AMGD_ERR_STATE
        X = np.random.default_rng(0).uniform(-1, 1, (400, 8))
        h.set_vectors(X)
        assert np.array_equal(h.get_vectors(), X)
        h.set_coloring(inputs.red_black(20))
        assert np.array_equal(h.get_vectors(), X)
        h.set_values(val * 3.0)
        h.relax(2, 1.0, amgd.AMGD_SWEEP_MCGS)
        want = oracle.relax(rp, col, val * 3.0, X, 2, 1.0, oracle.SWEEP_MCGS, inputs.red_black(20))
        assert np.array_equal(h.get_vectors(), want)
        h.distances(0.5)
        s_rp = np.empty(401, np.int64)
        s_col = np.empty(3, np.int32)
        import ctypes
        nnz_s = ctypes.c_int64()
        st = amgd.lib().amgd_strength(h.h, s_rp.ctypes.data, s_col.ctypes.data, 3,
                                      ctypes.byref(nnz_s), amgd.AMGD_MEM_HOST)
        assert st == amgd.AMGD_ERR_CAPACITY and nnz_s.value > 3
        with pytest.raises(amgd.AmgdError):
            h.set_weights(np.array([1.0, -1.0] + [1.0] * 6))
        with pytest.raises(amgd.AmgdError):
            h.set_values(np.where(np.arange(len(val)) == 0, 0.0, val))


# --------------------------------------------------------------------------- shapes, tuner
def _valid_shapes(prec, K):
    V = {"fp64": 2, "fp32": 4, "bf16": 8}[prec]
    P = 1
    while P * V < K:
        P *= 2
    return [(P // nv, nv, u, st) for st in (0, 1, 2, 3) for nv in (1, 2, 4) for u in (4, 8)
            if P % nv == 0 and not (st == 2 and u == 8)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("K", [5, 16, 32])
def test_kernel_shapes_agree(prec, K):
    """Shapes change speed, not results: sweeps are identical bit for bit
    (every component's row sum keeps its order); distances agree to the
    rounding of the K-term sums; strength sets agree outside a tiny band."""
    N = 40
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    ref = None
    staged_ok = 0
    for G, NV, U, st in _valid_shapes(prec, K):
        with amgd.Handle(rp, col, val, K, 4) as h:
            h.set_precision(prec)
            h.set_coloring(color)
            try:
                h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, G, NV, U, st)
            except amgd.AmgdError:
                assert st >= 1, "direct shapes are always available"
                continue          # staged shape beyond the shared-memory limit
            staged_ok += st
            # the edge pass has two kernels: rows (stage 0) and tiles (stage 1)
            h.set_kernel_shape(amgd.AMGD_KERNEL_EDGE, G, NV, U, min(st, 1))
            assert h.kernel_shape(amgd.AMGD_KERNEL_RELAX) == (G, NV, U, st)
            h.relax(3, 1.0, amgd.AMGD_SWEEP_MCGS)
            X = h.get_vectors()
            out = h.distances(0.5)
        if ref is None:
            ref = (X, out["ls"])
            continue
        assert np.array_equal(X, ref[0]), (G, NV, U, st)
        tol = 1e-12 if prec == "fp64" else 2e-5
        off = ~np.isnan(ref[1])
        rel = np.abs(out["ls"][off] - ref[1][off]) / np.maximum(ref[1][off], 1e-300)
        assert rel.max() <= tol, (G, NV, U, rel.max())
    assert staged_ok > 0
    with amgd.Handle(rp, col, val, K, 4) as h:
        h.set_precision(prec)
        with pytest.raises(amgd.AmgdError):
            h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, 3, 1, 4)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_batch_shard_keys(prec):
    """A handle over a subset of a batch, keyed by the matrices' indices in the
    whole batch (amgd_set_matrix_ids), reproduces the whole batch's vectors and
    distances of those matrices bit for bit: the one-GPU share of a batch split
    across GPUs."""
    mats = [inputs.graph_laplacian(n, 4.0, 5, b) for b, n in enumerate([700, 2222, 99, 1500, 333])]
    K, seed = 16, 6
    with amgd.Handle(None, None, None, K, seed, batch=mats) as h:
        h.set_precision(prec)
        h.init_vectors(seed)
        h.relax(3, 2.0 / 3.0)
        Xa = h.get_vectors()
        full = h.distances(0.5)
        ro, so = h.offsets()
    ids = [3, 1, 4]
    with amgd.Handle(None, None, None, K, seed, batch=[mats[b] for b in ids]) as h:
        h.set_matrix_ids(ids)
        h.set_precision(prec)
        h.init_vectors(seed)
        h.relax(3, 2.0 / 3.0)
        Xs = h.get_vectors()
        part = h.distances(0.5)
        ro_s, so_s = h.offsets()
    for k, b in enumerate(ids):
        assert np.array_equal(Xs[ro_s[k]:ro_s[k + 1]], Xa[ro[b]:ro[b + 1]]), b
        assert np.array_equal(part["ls"][so_s[k]:so_s[k + 1]], full["ls"][so[b]:so[b + 1]],
                              equal_nan=True), b
        assert np.array_equal(part["a"][so_s[k]:so_s[k + 1]], full["a"][so[b]:so[b + 1]]), b


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("K", [5, 16, 64])
@pytest.mark.parametrize("mat", ["aniso9_40", "graph_2000"])
def test_edge_inplace_shapes_agree(prec, K, mat):
    """The distance kernels on the sweeps' row order -- the row kernel (edge
    stage 2) and the warp-staged kernel (stage 3), every shape and both
    summation modes -- against the row kernel (stage 0) on the same vectors:
    FP64 within 1e-12 relative, mixed within 2e-5; strength sets identical
    outside a band of 1e-4 around theta.  graph_2000's long rows overflow the
    warp windows of stage 3."""
    if mat == "aniso9_40":
        N = 40
        rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
        color, sweep = inputs.red_black(N), amgd.AMGD_SWEEP_MCGS
    else:
        rp, col, val = MATRICES[mat]()
        color, sweep = None, amgd.AMGD_SWEEP_JACOBI
    V = {"fp64": 2, "fp32": 4, "bf16": 8}[prec]
    P = 1
    while P * V < K:
        P *= 2

    def run(shape, summation="compensated"):
        with amgd.Handle(rp, col, val, K, 4) as h:
            h.set_precision(prec)
            if color is not None:
                h.set_coloring(color)
            h.set_summation(summation)
            h.set_kernel_shape(amgd.AMGD_KERNEL_EDGE, *shape)
            h.relax(3, 1.0 if color is not None else 0.7, sweep)
            out = h.distances(0.5)
            s_rp, s_col = h.strength()
        return out, flags_from_strength(rp, col, s_rp, s_col)

    ref, ref_flag = run((P, 1, 4, 0))
    off = ~np.isnan(ref["ls"])
    ref_w = dict(ls=ref["ls"], flag=ref_flag)
    for stage, us in ((2, (2, 4)), (3, (4, 8))):
        for nv in (1, 2, 4):
            if P % nv:
                continue
            for u in us:
                for summation in ("compensated", "plain"):
                    got, flag = run((P // nv, nv, u, stage), summation)
                    tol = 1e-12 if prec == "fp64" else 2e-5
                    rel = np.abs(got["ls"][off] - ref["ls"][off]) / np.maximum(ref["ls"][off], 1e-300)
                    assert rel.max() <= tol, (stage, nv, u, summation, rel.max())
                    assert np.all(np.isnan(got["ls"][~off])) and np.all(got["a"][~off] == 0)
                    check_flags(flag, ref_w, rp, col, 0.5, 1e-4)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("summation", ["compensated", "plain"])
def test_edge_warp_kernel_weighted_mixed(prec, summation):
    """The warp-staged distance kernel (stage 3) with non-unit LS weights on
    the mixed paths (the weights held in shared memory per block) against the
    row kernel (stage 0) on the same vectors: within 2e-5, strength sets equal
    outside a band of 1e-4 around theta."""
    N = 40
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    w = np.random.default_rng(5).uniform(0.5, 2.0, 16)
    V = {"fp32": 4, "bf16": 8}[prec]
    P = 16 // V

    def run(stage, u):
        with amgd.Handle(rp, col, val, 16, 4) as h:
            h.set_precision(prec)
            h.set_coloring(color)
            h.set_weights(w)
            h.set_summation(summation)
            h.set_kernel_shape(amgd.AMGD_KERNEL_EDGE, P, 1, u, stage)
            h.relax(3, 1.0, amgd.AMGD_SWEEP_MCGS)
            out = h.distances(0.5)
            s_rp, s_col = h.strength()
        return out, flags_from_strength(rp, col, s_rp, s_col)

    ref, ref_flag = run(0, 4)
    got, flag = run(3, 8)
    off = ~np.isnan(ref["ls"])
    rel = np.abs(got["ls"][off] - ref["ls"][off]) / np.maximum(ref["ls"][off], 1e-300)
    assert rel.max() <= 2e-5, rel.max()
    check_flags(flag, dict(ls=ref["ls"], flag=ref_flag), rp, col, 0.5, 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_edge_batch_of_two(prec):
    """The distance pass also compiles a gather batch of 2 (both kernels):
    same distances as the default shape (FP64 against the oracle)."""
    rp, col, val = inputs.aniso2d_9pt(40, 1e-3, math.pi / 6)
    want = oracle.build(rp, col, val, 16, 4, 3, 0.7, 0.5)
    for stage in (0, 1):
        with amgd.Handle(rp, col, val, 16, 4) as h:
            h.set_precision(prec)
            G, NV, _, _ = h.kernel_shape(amgd.AMGD_KERNEL_EDGE)
            h.set_kernel_shape(amgd.AMGD_KERNEL_EDGE, G, NV, 2, stage)
            with pytest.raises(amgd.AmgdError):
                h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, G, NV, 2, 0)
            h.relax(3, 0.7)
            X = h.get_vectors()
            out = h.distances(0.5)
            s_rp, s_col = h.strength()
        if prec == "fp64":
            compare_fp64(rp, col, val, dict(X=X, s_rp=s_rp, s_col=s_col, **out), want, 0.5)
        else:
            off = ~np.isnan(want["ls"])
            rel = np.abs(out["ls"][off] - want["ls"][off]) / want["ls"][off]
            assert np.median(rel) <= 5e-3


def test_autotune_and_cache(tmp_path):
    N = 64
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    cache = str(tmp_path / "tune.txt")
    with amgd.Handle(rp, col, val, 16, 1) as h:
        h.set_precision("bf16")
        h.set_coloring(inputs.red_black(N))
        X0 = h.get_vectors()
        r1 = h.autotune(amgd.AMGD_SWEEP_MCGS, 1.0, cache)
        assert np.array_equal(h.get_vectors(), X0)       # the vectors are kept
        lines = open(cache).read().strip().splitlines()
        assert len(lines) == 1 and "relax=" in lines[0] and "edge=" in lines[0]
        r2 = h.autotune(amgd.AMGD_SWEEP_MCGS, 1.0, cache)   # served from the cache
        assert r2 == r1 and len(open(cache).read().strip().splitlines()) == 1
        h.relax(2, 1.0, amgd.AMGD_SWEEP_MCGS)
        h.distances(0.5)
