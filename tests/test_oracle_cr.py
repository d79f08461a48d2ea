"""Pins of the oracle's compatible-relaxation coarsening (§3.2, §4.2, Algorithm 1).

* One stage against a brute force that shares none of the oracle's steps:
  F-relaxation as a dense matrix power (Jacobi) or a dense triangular solve
  (Gauss-Seidel/SOR in color order, which a proper coloring makes equal to
  the multicolor sweep), the convergence estimate in the max norm, the
  candidates, the strength graph restricted to F in numpy, the priorities
  from numpy's Philox4x64-10, and the independent set by parallel rounds of
  local maxima (the same unique set as the greedy order, reached by another
  algorithm).
* For many sweeps the estimate tends to the spectral radius of E_f
  (Eq. (3.5): the limit of ||E_f^nu||^(1/nu)).
* Special cases: an all-coarse start has nothing to relax (rho = 0); a
  diagonal matrix under Jacobi with omega = 1 converges in one sweep (up to
  rounding); C_0 is kept; delta above every estimate adds no set; max_sets
  bounds the stages.
"""
import numpy as np
import scipy.linalg

import oracle
from paper_1106_5990_gb300 import inputs
from test_oracle_pins import numpy_philox_block


def _dense(rp, col, val):
    n = len(rp) - 1
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            A[i, col[p]] = val[p]
    return A


def _u_after(A, coarse, nu, omega, sweep, color):
    """u = E_f^nu 1 on F (0 on C), by dense linear algebra."""
    n = A.shape[0]
    F = np.flatnonzero(coarse == 0)
    u = np.zeros(n)
    if len(F) == 0:
        return u
    Aff = A[np.ix_(F, F)]
    D = np.diag(Aff)
    if sweep == oracle.SWEEP_JACOBI:
        E = np.eye(len(F)) - omega * Aff / D[:, None]
    else:
        order = np.lexsort((F, color[F]))          # color-major, then index
        P = Aff[np.ix_(order, order)]
        L = np.tril(P, -1)
        M = np.diag(np.diag(P)) + omega * L
        Ep = np.eye(len(F)) - omega * scipy.linalg.solve_triangular(M, P, lower=True)
        inv = np.empty_like(order)
        inv[order] = np.arange(len(F))
        E = Ep[np.ix_(inv, inv)]
    uf = np.linalg.matrix_power(E, nu) @ np.ones(len(F))
    u[F] = uf
    return u


def _stage_brute(A, prp, pcol, ls, coarse, nu, omega, sweep, color, theta, delta, tol, seed,
                 stage):
    """(rho, new coarse mask or None when the stage stops) by brute force."""
    n = A.shape[0]
    u = _u_after(A, coarse, nu, omega, sweep, color)
    F = coarse == 0
    if not F.any():
        return 0.0, None
    unorm = np.abs(u[F]).max()
    rho = unorm ** (1.0 / nu)
    if not rho > delta:
        return rho, None
    Z = F & (np.abs(u) / unorm > tol)
    strong = np.zeros(len(pcol), dtype=bool)
    for i in np.flatnonzero(F):
        q = np.arange(prp[i], prp[i + 1])
        j = pcol[q]
        ok = (j != i) & F[j]
        if not ok.any():
            continue
        m = ls[q][ok].min()
        strong[q] = ok & ((ls[q] == 0.0) | (theta * ls[q] < m))
    rows = np.repeat(np.arange(n), np.diff(prp))
    adj = [set() for _ in range(n)]
    lam = np.zeros(n, dtype=np.int64)
    for q in np.flatnonzero(strong):
        i, j = int(rows[q]), int(pcol[q])
        adj[i].add(j)
        adj[j].add(i)
        if Z[i] and Z[j]:
            lam[j] += 1
    key = np.array([int(numpy_philox_block((i, stage, 1, 0), (seed, 0))[0]) for i in range(n)],
                   dtype=np.uint64)
    # rank 0 = first in the greedy order: larger lambda, larger key, smaller index
    order = sorted(range(n), key=lambda v: (-int(lam[v]), -int(key[v]), v))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    undecided = set(np.flatnonzero(Z).tolist())
    chosen = set()
    while undecided:
        maxima = [v for v in undecided
                  if all(rank[v] < rank[w] for w in adj[v] if w in undecided)]
        chosen.update(maxima)
        drop = set(maxima)
        for v in maxima:
            drop.update(w for w in adj[v] if w in undecided)
        undecided -= drop
    new = coarse.copy()
    new[sorted(chosen)] = 1
    return rho, new


def _ls_field(prp, pcol, seed):
    """Per-slot LS values: random positive, a few exact zeros, NaN on the diagonal."""
    rng = np.random.default_rng(seed)
    ls = rng.uniform(0.05, 1.0, len(pcol))
    ls[rng.random(len(pcol)) < 0.05] = 0.0
    rows = np.repeat(np.arange(len(prp) - 1), np.diff(prp))
    ls[pcol == rows] = np.nan
    return ls


def _cases():
    N = 10
    rp, col, val = inputs.aniso2d_5pt(N, 1e-1)
    yield "aniso5_jacobi", rp, col, val, oracle.SWEEP_JACOBI, 2.0 / 3.0, None, 1
    rp2, col2, val2 = inputs.poisson2d_5pt(N)
    yield "poisson5_sor", rp2, col2, val2, oracle.SWEEP_MCGS, 1.2, inputs.red_black(N), 1
    rp3, col3, val3 = inputs.random_csr(90, 4.0, 3, symmetric_pattern=True)
    yield "random_jacobi_d2", rp3, col3, val3, oracle.SWEEP_JACOBI, 0.6, None, 2


def pin_cr_stage_brute_force(orc):
    theta, tol, nu, seed = 0.5, 0.5, 4, 11
    for name, rp, col, val, sweep, omega, color, d in _cases():
        A = _dense(rp, col, val)
        n = A.shape[0]
        prp, pcol = orc.distance_graph(rp, col, d)
        ls = _ls_field(prp, pcol, 5)
        rng = np.random.default_rng(7)
        C0 = (rng.random(n) < 0.15).astype(np.uint8)
        for stage_sets in (1, 2):
            C, rho = orc.cr_coarsen(rp, col, val, prp, pcol, ls, theta, nu, omega, sweep, color,
                                    0.05, tol, stage_sets, seed, C0)
            cur = C0.copy()
            for s in range(len(rho)):
                want_rho, nxt = _stage_brute(A, prp, pcol, ls, cur, nu, omega, sweep, color,
                                             theta, 0.05, tol, seed, s)
                assert abs(rho[s] - want_rho) <= 1e-12 * max(want_rho, 1e-300), (name, s)
                if nxt is None or s == stage_sets:
                    break
                assert nxt.sum() > cur.sum(), (name, s)
                cur = nxt
            assert len(rho) == stage_sets + 1, name
            assert np.array_equal(C, cur), name


def pin_cr_spectral_limit(orc):
    """(||E_f^nu 1||_inf)^(1/nu) -> rho(E_f) as nu grows (Eq. (3.5))."""
    N = 8
    rp, col, val = inputs.poisson2d_5pt(N)
    A = _dense(rp, col, val)
    n = A.shape[0]
    C0 = np.zeros(n, dtype=np.uint8)
    C0[::3] = 1
    F = np.flatnonzero(C0 == 0)
    Aff = A[np.ix_(F, F)]
    omega = 0.8
    E = np.eye(len(F)) - omega * Aff / np.diag(Aff)[:, None]
    want = np.abs(np.linalg.eigvals(E)).max()
    _, rho = orc.cr_coarsen(rp, col, val, rp, col, np.ones(len(col)), 0.5, 400, omega,
                            oracle.SWEEP_JACOBI, None, 10.0, 0.5, 0, 0, C0)
    assert abs(rho[0] - want) <= 1e-2 * want, (rho[0], want)


def pin_cr_red_black_closed_form(orc):
    """C = the red points of a red-black ordering leaves F without F-F
    couplings on the 1D and 2D five-point Laplacians (A_ff is diagonal), so
    one F-relaxation sweep multiplies u by exactly (1 - omega): rho_f =
    |1 - omega| for Jacobi and Gauss-Seidel alike (Eq. (3.5) for a diagonal
    E_f), and with delta above it no set is added."""
    N = 8
    rp2, col2, val2 = inputs.poisson2d_5pt(N)
    red2 = (inputs.red_black(N) == 0).astype(np.uint8)
    rp1, col1, val1 = inputs.lap1d(17)
    red1 = (np.arange(17) % 2 == 0).astype(np.uint8)
    for rp, col, val, C0 in ((rp1, col1, val1, red1), (rp2, col2, val2, red2)):
        ls = np.ones(len(col))
        color = C0.astype(np.int32)           # a proper 2-coloring of these graphs
        for omega in (0.5, 0.8, 1.25):
            for sweep in (oracle.SWEEP_JACOBI, oracle.SWEEP_MCGS):
                C, rho = orc.cr_coarsen(rp, col, val, rp, col, ls, 0.5, 3, omega, sweep,
                                        color if sweep == oracle.SWEEP_MCGS else None,
                                        abs(1 - omega) + 1e-9, 0.5, 5, 0, C0)
                assert len(rho) == 1 and abs(rho[0] - abs(1 - omega)) <= 1e-14, (omega, sweep)
                assert np.array_equal(C, C0)


def pin_cr_special_cases(orc):
    N = 6
    rp, col, val = inputs.poisson2d_5pt(N)
    n = N * N
    ls = np.ones(len(col))
    # all coarse: nothing to relax
    C, rho = orc.cr_coarsen(rp, col, val, rp, col, ls, coarse0=np.ones(n, np.uint8), delta=0.0)
    assert list(rho) == [0.0] and C.all()
    # diagonal matrix, Jacobi with omega = 1: one sweep removes everything up to
    # the rounding of (1 / a_ii) * a_ii
    drp = np.arange(n + 1, dtype=np.int64)
    dcol = np.arange(n, dtype=np.int32)
    dval = np.linspace(1.0, 3.0, n)
    C, rho = orc.cr_coarsen(drp, dcol, dval, drp, dcol, np.full(n, np.nan), omega=1.0, nu=3)
    assert len(rho) == 1 and rho[0] < 1e-15 and not C.any()
    # delta above every estimate: no set is added; C_0 is returned unchanged
    C0 = np.zeros(n, np.uint8)
    C0[[0, 7, 20]] = 1
    C, rho = orc.cr_coarsen(rp, col, val, rp, col, ls, delta=10.0, coarse0=C0)
    assert len(rho) == 1 and np.array_equal(C, C0)
    # max_sets bounds the number of stages; C only grows
    C, rho = orc.cr_coarsen(rp, col, val, rp, col, ls, delta=0.0, max_sets=2, coarse0=C0)
    assert len(rho) == 3 and (C >= C0).all() and C.sum() > C0.sum()


def test_cr_stage_brute_force(orc):
    pin_cr_stage_brute_force(orc)


def test_cr_spectral_limit(orc):
    pin_cr_spectral_limit(orc)


def test_cr_red_black_closed_form(orc):
    pin_cr_red_black_closed_form(orc)


def test_cr_special_cases(orc):
    pin_cr_special_cases(orc)


def test_cr_coarsens_anisotropy_along_strong_direction(orc):
    """On u_xx + eps u_yy with small eps the strong couplings are along x, so
    the first coarse set is an independent set of the x-lines: no two
    x-neighbours are both coarse after one stage."""
    N = 16
    rp, col, val = inputs.aniso2d_5pt(N, 1e-3)
    b = orc.build(rp, col, val, 8, 1, 10, 2.0 / 3.0, 0.5)
    C, rho = orc.cr_coarsen(rp, col, val, rp, col, b["ls"], max_sets=1, delta=0.0)
    grid = C.reshape(N, N)
    assert C.sum() > 0
    assert not (grid[:, 1:] & grid[:, :-1]).any()
