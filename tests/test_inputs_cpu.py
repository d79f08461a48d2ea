"""The synthetic workloads match their stated recipes (inputs.py): structure
(ascending columns, an explicit diagonal, symmetry), the discretisation
formulas, the coefficient and weight distributions, and the sizes of the
1024 x 1024 and 128^3 grids and of the 64-graph batch."""
import math

import numpy as np
import pytest

from paper_1106_5990_gb300 import inputs


def _dense(rp, col, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return A


def _structure(rp, col, val):
    n = len(rp) - 1
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1) and rp[-1] == len(col) == len(val)
    for i in range(n):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c, i         # ascending, diagonal stored


def test_aniso9_stencil_and_structure():
    eps, alpha, N = 1e-3, math.pi / 6, 7
    rp, col, val = inputs.aniso2d_9pt(N, eps, alpha)
    _structure(rp, col, val)
    A = _dense(rp, col, val, N * N)
    assert np.array_equal(A, A.T)
    a, b, c = inputs.aniso_coefficients(eps, alpha)
    assert abs(a + c - (1 + eps)) <= 1e-15 and abs(a * c - b * b / 4 - eps) <= 1e-15   # rotation
    i = 3 * N + 3                                          # interior point
    want = {(0, 0): 2 * a + 2 * c, (1, 0): -a, (-1, 0): -a, (0, 1): -c, (0, -1): -c,
            (1, 1): -b / 4, (-1, -1): -b / 4, (1, -1): b / 4, (-1, 1): b / 4}
    for (dx, dy), v in want.items():
        assert A[i, i + dy * N + dx] == pytest.approx(v, rel=1e-15, abs=1e-17)
    assert np.count_nonzero(A[i]) == 9


def test_red_black_colors():
    N = 9
    color = inputs.red_black(N).reshape(N, N)
    assert set(np.unique(color)) == {0, 1}
    # a proper coloring of the 5-point graph; the 9-point diagonal neighbours share a color
    assert not (color[:, 1:] == color[:, :-1]).any() and not (color[1:] == color[:-1]).any()
    assert (color[1:, 1:] == color[:-1, :-1]).all()


def test_jump3d_harmonic_faces_and_rows():
    N, sigma, seed = 5, 2.0, 2
    rp, col, val = inputs.jump3d_7pt(N, sigma, seed)
    _structure(rp, col, val)
    n = N ** 3
    A = _dense(rp, col, val, n)
    assert np.array_equal(A, A.T) and np.all(A - np.diag(np.diag(A)) <= 0)
    # the cell coefficients kappa = exp(sigma z), z standard normal from the seeded generator
    kappa = np.exp(sigma * inputs._rng(seed).standard_normal(n))
    for i in range(n):
        iz, rem = divmod(i, N * N)
        iy, ix = divmod(rem, N)
        faces = 0.0
        for d, step in ((ix, 1), (iy, N), (iz, N * N)):
            for s in (-1, 1):
                if 0 <= d + s < N:
                    j = i + s * step
                    h = 2 * kappa[i] * kappa[j] / (kappa[i] + kappa[j])
                    assert A[i, j] == pytest.approx(-h, rel=1e-14)
                    faces += h
                else:
                    faces += 2 * kappa[i]                    # Dirichlet face, ghost at h/2
        assert A[i, i] == pytest.approx(faces, rel=1e-14)
        boundary = any(c in (0, N - 1) for c in (ix, iy, iz))
        rs = A[i].sum()
        assert (rs > 0) if boundary else abs(rs) <= 1e-12 * A[i, i]


def test_graph_laplacian_recipe():
    n, mean_deg, seed = 4000, 8.0, 4
    rp, col, val = inputs.graph_laplacian(n, mean_deg, seed, 3)
    _structure(rp, col, val)
    rows = np.repeat(np.arange(n), np.diff(rp))
    off = rows != col
    # symmetric pattern and values, no self loops, weights lognormal(0, 1)
    key = rows[off].astype(np.int64) * n + col[off]
    tkey = col[off].astype(np.int64) * n + rows[off]
    order, torder = np.argsort(key), np.argsort(tkey)
    assert np.array_equal(key[order], tkey[torder])
    assert np.array_equal(val[off][order], val[off][torder])
    w = -val[off]
    assert np.all(w > 0)
    lw = np.log(w[rows[off] < col[off]])
    assert abs(lw.mean()) < 0.02 and abs(lw.std() - 1.0) < 0.02
    # diagonal = row sum of the weights + 1e-6
    rs = np.bincount(rows[off], weights=w, minlength=n)
    d = val[~off]
    assert np.allclose(d - rs, 1e-6, rtol=0, atol=1e-12 * d.max())
    # Poisson(8) out-degree, symmetrised: mean degree just under 16
    deg = np.diff(rp) - 1
    assert 15.5 < deg.mean() < 16.0
    # the same seed and matrix index reproduce it; another index does not
    rp2, col2, val2 = inputs.graph_laplacian(n, mean_deg, seed, 3)
    assert np.array_equal(col, col2) and np.array_equal(val, val2)
    assert not np.array_equal(inputs.graph_laplacian(n, mean_deg, seed, 4)[0], rp)


def test_batch_sizes():
    s = inputs.batch_sizes(64, 10_000, 500_000, 5)
    assert len(s) == 64 and s.min() >= 10_000 and s.max() <= 500_000
    assert np.array_equal(s, inputs.batch_sizes(64, 10_000, 500_000, 5))
    assert 150_000 < s.mean() < 350_000


def test_workload_sizes():
    rp, col, _ = inputs.jump3d_7pt(128, 2.0, 2)
    n = 128 ** 3
    assert len(rp) - 1 == n and len(col) == 7 * n - 6 * 128 ** 2        # 14,581,760
    rp, col, _ = inputs.poisson2d_5pt(64)
    assert len(col) == 20_224
