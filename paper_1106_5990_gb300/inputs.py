"""Seeded synthetic input matrices (CSR) and colorings.

This module builds the *inputs* of the strength-of-connection build -- sparse
matrices shaped like the paper's test problems and the colorings that fix the
Gauss-Seidel order -- and nothing of the method itself (no relaxation, no
least squares, no thresholding).  Both the CUDA path and the FP64 oracle are
fed from here; neither of them imports the other.

All matrices are returned as ``(row_ptr int64[n+1], col int32[nnz],
val float64[nnz])`` with ascending column indices inside each row and an
explicit diagonal.  They are the negated, h^2-scaled operator A = -h^2 L
(the boundary rows/columns of Dirichlet problems are eliminated), so that
A is positive definite for the diffusion problems.  Algebraic distances do
not change under A -> cA, so the scaling is immaterial to the method.

Workloads (Brandt, Brannick, Kahl, Livshits, §5.1):
* ``aniso2d_7pt``  -- the paper's 7-point discretisation of
  a u_xx + b u_xy + c u_yy (Eqs. (5.2), (5.5), (5.6)); reproduces the worked
  stencil S_A printed in §5.1 for alpha = -pi/4, eps = 0.1.
* ``aniso2d_9pt``  -- the same operator with the centred 4-point cross
  derivative (a 9-point stencil).
* ``poisson2d_5pt``, ``lap1d`` -- isotropic special cases.
* ``jump3d_7pt``   -- cell-centred 3D diffusion with lognormal jumping
  coefficients, harmonic averages on faces.
* ``graph_laplacian`` / ``graph_laplacian_batch`` -- random sparse graph
  Laplacians with Poisson neighbour counts and lognormal edge weights.
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), 0x1106_5990]))


# --------------------------------------------------------------------------
# structured 2D / 3D grids
# --------------------------------------------------------------------------
def stencil2d(N: int, stencil: dict) -> tuple:
    """CSR of a constant-coefficient stencil on the N x N interior grid.

    ``stencil`` maps (dx, dy) -> value; unknown i = iy * N + ix.  Entries that
    fall outside the grid are dropped (homogeneous Dirichlet boundary); exact
    zeros are not stored.
    """
    offs = sorted(((dx, dy) for (dx, dy), v in stencil.items() if v != 0.0),
                  key=lambda t: (t[1], t[0]))
    n = N * N
    iy, ix = np.divmod(np.arange(n, dtype=np.int64), N)
    cols, vals, masks = [], [], []
    for dx, dy in offs:
        jx, jy = ix + dx, iy + dy
        ok = (jx >= 0) & (jx < N) & (jy >= 0) & (jy < N)
        cols.append(jy * N + jx)
        vals.append(np.full(n, float(stencil[(dx, dy)])))
        masks.append(ok)
    C = np.stack(cols, 1)
    V = np.stack(vals, 1)
    M = np.stack(masks, 1)
    cnt = M.sum(1)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    return rp, C[M].astype(np.int32), V[M].astype(np.float64)


def aniso_coefficients(eps: float, alpha: float) -> tuple:
    """a, b, c of Eq. (5.5): a = cos^2 + eps sin^2, b = (1-eps) sin 2alpha,
    c = sin^2 + eps cos^2 (rotation of diag(1, eps) by alpha, Eq. (5.2))."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    a = ca * ca + eps * sa * sa
    b = (1.0 - eps) * math.sin(2.0 * alpha)
    c = sa * sa + eps * ca * ca
    return a, b, c


def aniso7_stencil(eps: float, alpha: float, diag: str = "ne") -> dict:
    """Stencil of -h^2 (a u_xx + b u_xy + c u_yy) with the 7-point cross term.

    diag='ne' uses the lower-left/upper-right neighbours for u_xy (the sum of
    the two one-sided differences of Eq. (5.6)); diag='nw' the mirrored pair.
    """
    a, b, c = aniso_coefficients(eps, alpha)
    if diag == "ne":
        # h^2 * S_xy: centre 1, axis neighbours -1/2, (+1,+1) and (-1,-1) +1/2
        sxy = {(0, 0): 1.0, (1, 0): -0.5, (-1, 0): -0.5, (0, 1): -0.5, (0, -1): -0.5,
               (1, 1): 0.5, (-1, -1): 0.5}
    elif diag == "nw":
        sxy = {(0, 0): -1.0, (1, 0): 0.5, (-1, 0): 0.5, (0, 1): 0.5, (0, -1): 0.5,
               (1, -1): -0.5, (-1, 1): -0.5}
    else:
        raise ValueError(diag)
    st = {(0, 0): 2.0 * a + 2.0 * c, (1, 0): -a, (-1, 0): -a, (0, 1): -c, (0, -1): -c}
    for k, v in sxy.items():
        st[k] = st.get(k, 0.0) - b * v
    return st


def aniso9_stencil(eps: float, alpha: float) -> dict:
    """Stencil of -h^2 (a u_xx + b u_xy + c u_yy), centred cross derivative
    u_xy ~ (u(+1,+1) - u(+1,-1) - u(-1,+1) + u(-1,-1)) / 4h^2."""
    a, b, c = aniso_coefficients(eps, alpha)
    return {(0, 0): 2.0 * a + 2.0 * c, (1, 0): -a, (-1, 0): -a, (0, 1): -c, (0, -1): -c,
            (1, 1): -b / 4.0, (-1, -1): -b / 4.0, (1, -1): b / 4.0, (-1, 1): b / 4.0}


def aniso2d_7pt(N: int, eps: float, alpha: float, diag: str = "ne") -> tuple:
    return stencil2d(N, aniso7_stencil(eps, alpha, diag))


def aniso2d_9pt(N: int, eps: float, alpha: float) -> tuple:
    return stencil2d(N, aniso9_stencil(eps, alpha))


def aniso2d_5pt(N: int, eps: float) -> tuple:
    """Grid-aligned anisotropy u_xx + eps u_yy (alpha = 0)."""
    return stencil2d(N, {(0, 0): 2.0 + 2.0 * eps, (1, 0): -1.0, (-1, 0): -1.0,
                         (0, 1): -eps, (0, -1): -eps})


def poisson2d_5pt(N: int) -> tuple:
    return stencil2d(N, {(0, 0): 4.0, (1, 0): -1.0, (-1, 0): -1.0, (0, 1): -1.0, (0, -1): -1.0})


def lap1d(n: int) -> tuple:
    """Tridiagonal [-1, 2, -1] (Dirichlet)."""
    i = np.arange(n, dtype=np.int64)
    cols, vals, masks = [], [], []
    for d, v in ((-1, -1.0), (0, 2.0), (1, -1.0)):
        j = i + d
        masks.append((j >= 0) & (j < n))
        cols.append(j)
        vals.append(np.full(n, v))
    C, V, M = np.stack(cols, 1), np.stack(vals, 1), np.stack(masks, 1)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(M.sum(1), out=rp[1:])
    return rp, C[M].astype(np.int32), V[M]


def red_black(N: int) -> np.ndarray:
    """Red-black coloring (ix + iy) mod 2 of the N x N grid."""
    iy, ix = np.divmod(np.arange(N * N, dtype=np.int64), N)
    return ((ix + iy) % 2).astype(np.int32)


def jump3d_7pt(N: int, sigma: float, seed: int) -> tuple:
    """Cell-centred 7-point diffusion on N^3 cells of the unit cube.

    Cell coefficient kappa = exp(sigma z), z ~ N(0,1) (lognormal(0, sigma));
    interior face coefficient = harmonic mean 2 k_p k_q / (k_p + k_q); a face
    on the Dirichlet boundary couples to a ghost value at half a cell, giving
    2 k_p on the diagonal.  Unknown i = (iz N + iy) N + ix.
    """
    n = N * N * N
    kappa = np.exp(sigma * _rng(seed).standard_normal(n))
    idx = np.arange(n, dtype=np.int64)
    iz, rem = np.divmod(idx, N * N)
    iy, ix = np.divmod(rem, N)
    diag = np.zeros(n)
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    cols, vals, masks = [], [], []
    for dx, dy, dz in offs:
        if (dx, dy, dz) == (0, 0, 0):
            cols.append(idx)
            vals.append(None)
            masks.append(np.ones(n, dtype=bool))
            continue
        jx, jy, jz = ix + dx, iy + dy, iz + dz
        ok = (jx >= 0) & (jx < N) & (jy >= 0) & (jy < N) & (jz >= 0) & (jz < N)
        j = np.where(ok, (jz * N + jy) * N + jx, 0)
        kf = np.where(ok, 2.0 * kappa * kappa[j] / (kappa + kappa[j]), 2.0 * kappa)
        diag += kf
        cols.append(j)
        vals.append(-kf)
        masks.append(ok)
    vals[3] = diag
    C, V, M = np.stack(cols, 1), np.stack(vals, 1), np.stack(masks, 1)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(M.sum(1), out=rp[1:])
    return rp, C[M].astype(np.int32), V[M]


# --------------------------------------------------------------------------
# random graph Laplacians
# --------------------------------------------------------------------------
def _pair_weight(lo: np.ndarray, hi: np.ndarray, seed: int, mat: int) -> np.ndarray:
    """lognormal(0,1) weight of the undirected pair (lo, hi), keyed on the pair
    so that A is exactly symmetric (splitmix64 hash -> two uniforms ->
    Box-Muller)."""
    def mix(z):
        z = (z + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))
    with np.errstate(over="ignore"):
        key = (lo.astype(np.uint64) << np.uint64(32)) ^ hi.astype(np.uint64)
        key = key ^ (np.uint64(seed) * np.uint64(0xD1B54A32D192ED03)) ^ np.uint64(mat)
        h1 = mix(key)
        h2 = mix(h1 ^ np.uint64(0x632BE59BD9B4E019))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53   # (0, 1]
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return np.exp(z)


def graph_laplacian(n: int, mean_deg: float, seed: int, mat: int = 0,
                    shift: float = 1e-6) -> tuple:
    """Symmetric weighted graph Laplacian plus a diagonal shift.

    Node i draws Poisson(mean_deg) targets uniformly over the other nodes (no
    self loops); the union with the transpose is taken (mean degree about
    2 * mean_deg); each undirected pair gets a lognormal(0,1) weight w; the
    off-diagonal is -w and the diagonal the row sum of w plus ``shift``.
    Isolated nodes keep only their diagonal.
    """
    g = _rng(seed * 1000003 + mat)
    deg = g.poisson(mean_deg, size=n)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = g.integers(0, n - 1, size=src.size, dtype=np.int64)
    dst = dst + (dst >= src)                          # uniform over the others
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    key = np.unique(lo * n + hi)
    lo, hi = np.divmod(key, n)
    w = _pair_weight(lo, hi, seed, mat)
    r = np.concatenate([lo, hi, np.arange(n, dtype=np.int64)])
    c = np.concatenate([hi, lo, np.arange(n, dtype=np.int64)])
    rowsum = np.bincount(lo, weights=w, minlength=n) + np.bincount(hi, weights=w, minlength=n)
    v = np.concatenate([-w, -w, rowsum + shift])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    return rp, c.astype(np.int32), v


def batch_sizes(nmat: int, nmin: int, nmax: int, seed: int) -> np.ndarray:
    return _rng(seed).integers(nmin, nmax + 1, size=nmat)


def graph_laplacian_batch(nmat: int, nmin: int, nmax: int, mean_deg: float,
                          graph_seed: int, size_seed: int) -> list:
    sizes = batch_sizes(nmat, nmin, nmax, size_seed)
    return [graph_laplacian(int(s), mean_deg, graph_seed, b) for b, s in enumerate(sizes)]


# --------------------------------------------------------------------------
# small random matrices for parity cases
# --------------------------------------------------------------------------
def random_csr(n: int, nnz_per_row: float, seed: int, symmetric_pattern: bool = False,
               mixed_sign: bool = True, max_row: int | None = None) -> tuple:
    """Random sparse pattern with an explicit diagonal; off-diagonal values of
    mixed sign (or all negative), diagonal = 1 + row sum of |off-diagonals|.
    Row lengths are Poisson(nnz_per_row - 1) capped at max_row - 1."""
    g = _rng(seed)
    k = g.poisson(max(nnz_per_row - 1.0, 0.0), size=n)
    if max_row is not None:
        k = np.minimum(k, max_row - 1)
    k = np.minimum(k, n - 1)
    rows, cols = [], []
    for i in range(n):
        if k[i] == 0:
            continue
        cand = g.choice(n - 1, size=k[i], replace=False)
        cand = cand + (cand >= i)
        rows.append(np.full(k[i], i))
        cols.append(cand)
    r = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    if symmetric_pattern:
        r, c = np.concatenate([r, c]), np.concatenate([c, r])
        key = np.unique(r * n + c)
        r, c = np.divmod(key, n)
    v = g.uniform(0.1, 1.0, size=r.size)
    if mixed_sign:
        v = v * np.where(g.random(r.size) < 0.7, -1.0, 1.0)
    else:
        v = -v
    absrow = np.bincount(r, weights=np.abs(v), minlength=n)
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, 1.0 + absrow])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    return rp, c.astype(np.int32), v.astype(np.float64)


def greedy_coloring(rp, col) -> np.ndarray:
    """First-fit coloring in index order over the symmetrised pattern of A
    (a proper coloring: no two coupled rows share a color)."""
    rp = np.asarray(rp)
    col = np.asarray(col)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    r = np.concatenate([rows, col])
    c = np.concatenate([col, rows])
    keep = r != c
    r, c = r[keep], c[keep]
    order = np.argsort(r, kind="stable")
    r, c = r[order], c[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=ptr[1:])
    color = np.full(n, -1, dtype=np.int32)
    for i in range(n):
        used = set(color[c[ptr[i]:ptr[i + 1]]].tolist())
        k = 0
        while k in used:
            k += 1
        color[i] = k
    return color
