"""Pins of the oracle's least-squares interpolation (§4.3).

* Brute force: every subset of at most c coarse candidates fitted by a
  weighted numpy.linalg.lstsq, the best per size and the size penalty of
  §4.3 applied in plain Python; the oracle's chosen sets, weights and LS
  match on small random problems (plain and residual targets, weights).
* c = 1 is the best one-point fit of step 4 among the coarse candidates.
* With gamma = 0 the largest admissible size wins, and the chosen LS can
  only decrease as the caliber grows (the minimum over a larger family).
* A fine row that is an exact combination of two coarse candidates is
  reproduced exactly; coarse rows interpolate themselves.
"""
import itertools
import math

import numpy as np

import oracle
from paper_1106_5990_gb300 import inputs


def _problem(seed, n=60, K=6):
    rp, col, val = inputs.random_csr(n, 3.5, seed, symmetric_pattern=True)
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, K))
    coarse = (rng.random(n) < 0.4).astype(np.uint8)
    w = rng.uniform(0.5, 2.0, K)
    return rp, col, val, X, coarse, w


def _brute(X, Y, prp, pcol, coarse, c, gamma, w):
    n, K = X.shape
    sw = np.sqrt(w)
    rows = []
    for i in range(n):
        if coarse[i]:
            rows.append(([i], [1.0], 0.0))
            continue
        y = Y[i]
        cand = [j for j in pcol[prp[i]:prp[i + 1]] if coarse[j]]
        syy = float(np.sum(w * y * y))
        best = {0: ([], [], syy)}
        for m in range(1, min(c, len(cand)) + 1):
            for W in itertools.combinations(cand, m):
                A = (sw[:, None] * X[list(W)].T)
                p, _, rank, _ = np.linalg.lstsq(A, sw * y, rcond=None)
                if rank < m:
                    continue
                ls = float(np.sum(w * (y - X[list(W)].T @ p) ** 2))
                if m not in best or ls < best[m][2]:
                    best[m] = (list(W), list(p), ls)
        chosen = 0
        if syy > 0:
            for m in range(1, c + 1):
                if m in best and best[m][2] / syy < (best[chosen][2] / syy) ** (gamma * (m - chosen)):
                    chosen = m
        rows.append(best[chosen])
    return rows


def _rows(p_rp, p_col, p_val, i):
    return list(p_col[p_rp[i]:p_rp[i + 1]]), list(p_val[p_rp[i]:p_rp[i + 1]])


def pin_interp_brute_force(orc):
    for seed, mode, c, d in ((1, oracle.TARGET_RESIDUAL, 3, 2), (2, oracle.TARGET_PLAIN, 2, 2),
                             (3, oracle.TARGET_RESIDUAL, 3, 1)):
        rp, col, val, X, coarse, w = _problem(seed)
        Y = orc.target(rp, col, val, X, mode)
        prp, pcol = orc.distance_graph(rp, col, d)
        p_rp, p_col, p_val, ls = orc.ls_interp(X, Y, prp, pcol, coarse, c, 1.5, w)
        want = _brute(X, Y, prp, pcol, coarse, c, 1.5, w)
        for i, (W, p, l) in enumerate(want):
            got_c, got_v = _rows(p_rp, p_col, p_val, i)
            assert got_c == W, (seed, i)
            assert np.allclose(got_v, p, rtol=1e-8, atol=1e-10), (seed, i)
            syy = float(np.sum(w * Y[i] ** 2))
            assert abs(ls[i] - l) <= 1e-10 * max(syy, 1e-300), (seed, i)


def test_interp_brute_force(orc):
    pin_interp_brute_force(orc)


def pin_interp_single_point(orc):
    rp, col, val, X, coarse, w = _problem(5)
    Y = orc.target(rp, col, val, X)
    prp, pcol = orc.distance_graph(rp, col, 2)
    p_rp, p_col, p_val, ls = orc.ls_interp(X, Y, prp, pcol, coarse, 1, 1.5, w)
    a, l1 = orc.edge_ls_graph(rp, col, val, prp, pcol, X, Y, w, oracle.TARGET_PLAIN)
    # edge_ls_graph in plain mode fits y_i (given) against every x_j of the pattern
    for i in range(len(rp) - 1):
        if coarse[i]:
            continue
        qs = [q for q in range(prp[i], prp[i + 1]) if coarse[pcol[q]]]
        got_c, got_v = _rows(p_rp, p_col, p_val, i)
        if not qs:
            assert got_c == []
            continue
        q = min(qs, key=lambda q: (l1[q], q))
        assert got_c == [pcol[q]]
        assert abs(got_v[0] - a[q]) <= 1e-10 * (abs(a[q]) + 1)
        assert abs(ls[i] - l1[q]) <= 1e-10 * float(np.sum(w * Y[i] ** 2))


def test_interp_single_point(orc):
    pin_interp_single_point(orc)


def pin_interp_monotone_and_exact(orc):
    rp, col, val, X, coarse, w = _problem(7)
    Y = orc.target(rp, col, val, X)
    prp, pcol = orc.distance_graph(rp, col, 2)
    prev = None
    for c in (1, 2, 3):
        _, _, _, ls = orc.ls_interp(X, Y, prp, pcol, coarse, c, 0.0, w)
        if prev is not None:
            assert np.all(ls <= prev * (1 + 1e-12) + 1e-300)
        prev = ls
    # a fine row built as an exact combination of two coarse candidates
    n = len(rp) - 1
    i = next(i for i in range(n) if not coarse[i] and
             sum(coarse[j] for j in pcol[prp[i]:prp[i + 1]]) >= 2)
    cands = [j for j in pcol[prp[i]:prp[i + 1]] if coarse[j]][:2]
    Y2 = Y.copy()
    Y2[i] = 0.25 * X[cands[0]] - 0.75 * X[cands[1]]
    p_rp, p_col, p_val, ls = orc.ls_interp(X, Y2, prp, pcol, coarse, 2, 1.5, w)
    got_c, got_v = _rows(p_rp, p_col, p_val, i)
    assert got_c == sorted(cands)
    want = dict(zip(cands, (0.25, -0.75)))
    assert np.allclose(got_v, [want[j] for j in got_c], rtol=1e-12, atol=1e-13)
    assert ls[i] <= 1e-24 * float(np.sum(w * Y2[i] ** 2))
    for j in range(n):
        if coarse[j]:
            assert _rows(p_rp, p_col, p_val, j) == ([j], [1.0])
    # exact ties: two candidates with identical vectors -- the first in the
    # ascending candidate order is kept, and the pair is singular (skipped)
    X3 = X.copy()
    X3[cands[1]] = X3[cands[0]]
    Y3 = Y.copy()
    Y3[i] = 0.5 * X3[cands[0]]           # both duplicates fit exactly: an exact tie
    p_rp, p_col, p_val, ls = orc.ls_interp(X3, Y3, prp, pcol, coarse, 1, 1.5, w)
    assert _rows(p_rp, p_col, p_val, i)[0] == [min(cands)]


def test_interp_monotone_and_exact(orc):
    pin_interp_monotone_and_exact(orc)
