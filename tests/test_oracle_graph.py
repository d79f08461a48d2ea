"""Pins of the oracle's search depth d > 1 (§4.1, Eq. (4.2); §4.2).

* The graph G_d is compared with the pattern of the d-th power of A's 0/1
  pattern matrix, computed by dense integer matrix products (numpy), on an
  unsymmetric random matrix and stencils, d = 1, 2, 3.
* The fits over G_d are compared with a library weighted least-squares solve
  (numpy.linalg.lstsq) edge by edge; with d = 1 they reproduce step 4 bit
  for bit; the exact degree-one rule fires only on the single neighbour of A.
"""
import math

import numpy as np
import scipy.sparse as sp

import oracle
from paper_1106_5990_gb300 import inputs


def _pattern_power(rp, col, d):
    n = len(rp) - 1
    B = sp.csr_matrix((np.ones(len(col), dtype=np.int64), col, rp), shape=(n, n)).toarray()
    P = np.eye(n, dtype=np.int64)
    for _ in range(d):
        P = np.minimum(P @ B, 1)        # 0/1 pattern of the product
    return P != 0


def pin_distance_graph_matrix_power(orc):
    cases = [inputs.random_csr(60, 3.0, 7), inputs.aniso2d_9pt(7, 1e-2, math.pi / 6),
             inputs.lap1d(20), inputs.graph_laplacian(80, 2.0, 3)]
    for rp, col, val in cases:
        n = len(rp) - 1
        for d in (1, 2, 3):
            prp, pcol = orc.distance_graph(rp, col, d)
            want = _pattern_power(rp, col, d)
            for i in range(n):
                row = pcol[prp[i]:prp[i + 1]]
                assert np.array_equal(row, np.nonzero(want[i])[0]), (d, i)


def test_distance_graph_matrix_power(orc):
    pin_distance_graph_matrix_power(orc)


def pin_edge_ls_graph(orc):
    rp, col, val = inputs.random_csr(50, 3.0, 4)
    n, K = len(rp) - 1, 6
    rng = np.random.default_rng(2)
    w = rng.uniform(0.5, 2.0, K)
    X = rng.uniform(-1, 1, (n, K))
    for mode in (oracle.TARGET_RESIDUAL, oracle.TARGET_PLAIN):
        Y = orc.target(rp, col, val, X, mode)
        # d = 1 reproduces step 4 exactly
        a1, l1 = orc.edge_ls(rp, col, val, X, Y, w, mode)
        a1g, l1g = orc.edge_ls_graph(rp, col, val, rp, col, X, Y, w, mode)
        assert np.array_equal(a1, a1g) and np.array_equal(l1, l1g, equal_nan=True)
        prp, pcol = orc.distance_graph(rp, col, 2)
        a, ls = orc.edge_ls_graph(rp, col, val, prp, pcol, X, Y, w, mode)
        sw = np.sqrt(w)
        for i in range(n):
            arow = col[rp[i]:rp[i + 1]]
            offA = [j for j in arow if j != i]
            for q in range(prp[i], prp[i + 1]):
                j = pcol[q]
                if j == i:
                    assert a[q] == 0 and math.isnan(ls[q])
                    continue
                if mode == oracle.TARGET_RESIDUAL and len(offA) == 1 and j == offA[0]:
                    p1 = rp[i] + list(arow).index(j)
                    aii = val[rp[i] + list(arow).index(i)]
                    assert a[q] == -val[p1] / aii and ls[q] == 0.0
                    continue
                sol, res, _, _ = np.linalg.lstsq((sw * X[j])[:, None], sw * Y[i], rcond=None)
                lsq = float(np.sum(w * (Y[i] - sol[0] * X[j]) ** 2))
                syy = float(np.sum(w * Y[i] ** 2))
                assert abs(a[q] - sol[0]) <= 1e-12 * (abs(sol[0]) + 1.0)
                assert abs(ls[q] - lsq) <= 1e-12 * syy


def test_edge_ls_graph(orc):
    pin_edge_ls_graph(orc)


def test_build_with_depth(orc):
    """The whole path with d = 2: strength graph over G_2, rows in order,
    kept columns a subset of the row's G_2 neighbours."""
    N = 12
    rp, col, val = inputs.aniso2d_5pt(N, 1e-2)
    r = orc.build(rp, col, val, 8, 0, 6, 2.0 / 3.0, 0.5, d=2)
    prp, pcol = r["prp"], r["pcol"]
    assert len(pcol) > len(col)
    for i in range(N * N):
        kept = set(r["s_col"][r["s_rp"][i]:r["s_rp"][i + 1]].tolist())
        assert kept <= set(pcol[prp[i]:prp[i + 1]].tolist()) - {i}
        assert len(kept) >= 1          # the row's nearest neighbour is always kept
