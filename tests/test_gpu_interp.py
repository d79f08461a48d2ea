"""Least-squares interpolation (§4.3) on the GPU against the oracle: the
GPU evaluates every candidate set in FP64 with the rounding order of the
definition, so on the same stored vectors (the oracle's relaxed vectors,
rounded to the storage type on the CPU and set on the handle) the chosen
sets, weights and LS values equal the oracle's bit for bit -- for every
storage precision (the vectors are widened exactly), with and without a
coloring, search depth 1 and 2, caliber 1 to 4, gamma 1.5 and 0."""
import math

import numpy as np
import pytest

import oracle
from paper_1106_5990_gb300 import inputs

pytestmark = pytest.mark.gpu
amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()


def _case(name):
    if name == "aniso5_24":
        N = 24
        rp, col, val = inputs.aniso2d_5pt(N, 1e-2)
        coarse = inputs.red_black(N).astype(np.uint8) ^ 1          # red points coarse
        return rp, col, val, coarse, inputs.red_black(N)
    rp, col, val = inputs.random_csr(500, 3.0, 13, symmetric_pattern=True)   # <= 26 candidates at d = 2
    coarse = (np.random.default_rng(1).random(500) < 0.35).astype(np.uint8)
    return rp, col, val, coarse, None


def _stored(X, prec):
    """X rounded to the storage type on the CPU; the values are then exact in
    that type, so the GPU stores them unchanged."""
    if prec == "fp64":
        return X
    t = torch.from_numpy(X).to(torch.bfloat16 if prec == "bf16" else torch.float32)
    return t.to(torch.float64).numpy()


@pytest.mark.parametrize("name", ["aniso5_24", "random_500"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("d,c,gamma", [(1, 2, 1.5), (2, 3, 1.5), (2, 4, 0.0), (2, 1, 1.5)])
def test_interp_matches_oracle(name, prec, d, c, gamma):
    rp, col, val, coarse, color = _case(name)
    n, K = len(rp) - 1, 8
    w = np.random.default_rng(4).uniform(0.5, 2.0, K)
    # the oracle's relaxed vectors, in the storage type; the oracle's pattern
    X0 = oracle.tv_init(n, K, 9)
    if color is not None:
        X = oracle.relax(rp, col, val, X0, 3, 1.0, oracle.SWEEP_MCGS, color)
    else:
        X = oracle.relax(rp, col, val, X0, 3, 0.7)
    X = _stored(X, prec)
    prp, pcol = oracle.distance_graph(rp, col, d)
    with amgd.Handle(rp, col, val, K, 9) as h:
        h.set_precision(prec)
        h.set_weights(w)
        if color is not None:
            h.set_coloring(color)
        h.set_search_depth(d)
        h.set_vectors(X)
        assert np.array_equal(h.get_vectors(), X)
        got = h.ls_interpolation(coarse, c, gamma)
    Y = oracle.target(rp, col, val, X)
    want = oracle.ls_interp(X, Y, prp, pcol, coarse, c, gamma, w)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])
    assert np.array_equal(got[2], want[2])
    assert np.array_equal(got[3], want[3])
    # coarse rows interpolate themselves
    for i in np.nonzero(coarse)[0][:50]:
        assert got[1][got[0][i]:got[0][i + 1]].tolist() == [i]


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_interp_unit_weights_both_kernels(prec):
    """Unit weights (the products by w are exact and skipped) on a pattern
    whose fine rows have from 0 to more than 8 coarse candidates, so that
    one call runs the thread-per-row and the warp-per-row kernels."""
    rp, col, val = inputs.random_csr(1500, 2.5, 21, symmetric_pattern=True)   # m: 0 .. 25
    n, K = len(rp) - 1, 16
    coarse = (np.random.default_rng(3).random(n) < 0.45).astype(np.uint8)
    X = _stored(oracle.relax(rp, col, val, oracle.tv_init(n, K, 2), 2, 0.7), prec)
    prp, pcol = oracle.distance_graph(rp, col, 2)
    rows = np.repeat(np.arange(n), np.diff(prp))
    m = np.bincount(rows[coarse[pcol] == 1], minlength=n)[coarse == 0]
    assert m.max() > 8 and m.min() == 0
    with amgd.Handle(rp, col, val, K, 2) as h:
        h.set_precision(prec)
        h.set_search_depth(2)
        h.set_vectors(X)
        got = h.ls_interpolation(coarse, 2, 1.5)
    Y = oracle.target(rp, col, val, X)
    want = oracle.ls_interp(X, Y, prp, pcol, coarse, 2, 1.5)
    for g, w_ in zip(got, want):
        assert np.array_equal(g, w_)


@pytest.mark.parametrize("depth", [1, 2])
@pytest.mark.parametrize("unit_w", [True, False])
def test_interp_ties_and_exact_fits(unit_w, depth):
    """Plain target with planted structure: coarse candidates that repeat one
    another exactly (ties between sets, singular pairs) and fine rows that
    are exact combinations of two coarse neighbours (LS = 0 up to rounding),
    so that sets whose LS values are equal or nearly equal compete."""
    rp, col, val = inputs.random_csr(800, 3.0, 31, symmetric_pattern=True)
    n, K = len(rp) - 1, 8
    rng = np.random.default_rng(5)
    coarse = (rng.random(n) < 0.45).astype(np.uint8)
    X = rng.integers(-64, 65, size=(n, K)) / 64.0
    base = rng.integers(-64, 65, size=K) / 64.0
    cidx = np.flatnonzero(coarse)
    X[cidx[::3]] = base                                     # a third of the coarse rows equal
    for i in np.flatnonzero(coarse == 0)[::2]:
        nb = [j for j in col[rp[i]:rp[i + 1]] if coarse[j]]
        if len(nb) >= 2:
            X[i] = 0.5 * X[nb[0]] - 0.25 * X[nb[1]]         # exact in FP64
    w = np.ones(K) if unit_w else rng.uniform(0.5, 2.0, K)
    prp, pcol = oracle.distance_graph(rp, col, depth)     # depth 2: rows with > 8 candidates
    with amgd.Handle(rp, col, val, K, 1) as h:
        h.set_target(amgd.AMGD_TARGET_PLAIN)
        h.set_weights(w)
        h.set_search_depth(depth)
        h.set_vectors(X)
        got = h.ls_interpolation(coarse, 3, 1.5)
    Y = oracle.target(rp, col, val, X, oracle.TARGET_PLAIN)
    want = oracle.ls_interp(X, Y, prp, pcol, coarse, 3, 1.5, w)
    for g, w_ in zip(got, want):
        assert np.array_equal(g, w_)


@pytest.mark.parametrize("K", [1, 3, 64])
def test_interp_extreme_K(K):
    """K = 1 (every one-point fit exact, so the penalty decides), an odd K and
    the largest K, on the thread and the warp kernels (search depth 2)."""
    rp, col, val = inputs.random_csr(700, 2.5, 17, symmetric_pattern=True)
    n = len(rp) - 1
    coarse = (np.random.default_rng(8).random(n) < 0.4).astype(np.uint8)
    X = oracle.relax(rp, col, val, oracle.tv_init(n, K, 5), 2, 0.7)
    prp, pcol = oracle.distance_graph(rp, col, 2)
    with amgd.Handle(rp, col, val, K, 5) as h:
        h.set_search_depth(2)
        h.set_vectors(X)
        got = h.ls_interpolation(coarse, 3, 1.5)
    Y = oracle.target(rp, col, val, X)
    want = oracle.ls_interp(X, Y, prp, pcol, coarse, 3, 1.5)
    for g, w_ in zip(got, want):
        assert np.array_equal(g, w_)


def test_interp_too_many_candidates():
    rp, col, val = inputs.graph_laplacian(300, 12.0, 2)
    with amgd.Handle(rp, col, val, 8, 1) as h:
        h.relax(2, 0.7)
        h.set_search_depth(3)
        coarse = np.ones(300, dtype=np.uint8)
        coarse[::7] = 0
        with pytest.raises(amgd.AmgdError) as e:
            h.ls_interpolation(coarse, 2)
        assert e.value.status == amgd.AMGD_ERR_UNSUPPORTED
        with pytest.raises(amgd.AmgdError) as e:
            h.ls_interpolation(coarse, 5)
        assert e.value.status == amgd.AMGD_ERR_ARG
