"""Compatible-relaxation coarsening (§3.2, §4.2, Algorithm 1) on the GPU
against the oracle.  The F-relaxation sweeps are FP64 fused multiply-adds in
CSR order, the norm is an exact maximum and the independent set is the one
set that the greedy priority order selects.  Given the same per-slot LS
values (the oracle's), the coarse set and every convergence estimate
therefore equal the oracle's bit for bit.  This holds for Jacobi and
multicolor Gauss-Seidel F-relaxation, search depth 1 and 2, empty and
non-empty C_0, and at the full size of the 1024 x 1024 rotated-anisotropy
workload.  The handle's own FP64 distances give the same result wherever no
LS ratio of a row lies within 1e-9 of theta."""
import math
import time

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


# name: (matrix, coloring or None, omega, search depth)
CASES = {
    "aniso9_48_mcgs": (lambda: inputs.aniso2d_9pt(48, 1e-3, math.pi / 6), 48, 1.0, 1),
    "aniso5_64_jacobi": (lambda: inputs.aniso2d_5pt(64, 1e-2), None, 2.0 / 3.0, 1),
    "random_800_d2": (lambda: inputs.random_csr(800, 4.0, 5, symmetric_pattern=True), None, 0.7, 2),
    "graph_3000": (lambda: inputs.graph_laplacian(3000, 8.0, 4), None, 2.0 / 3.0, 1),
    "jump3d_12": (lambda: inputs.jump3d_7pt(12, 2.0, 2), None, 0.8, 1),
    "aniso5_40_d3": (lambda: inputs.aniso2d_5pt(40, 1e-2), None, 2.0 / 3.0, 3),
}


def _setup(name):
    make, grid, omega, d = CASES[name]
    rp, col, val = make()
    color = inputs.red_black(grid) if grid else None
    sweep = oracle.SWEEP_MCGS if color is not None else oracle.SWEEP_JACOBI
    want = oracle.build(rp, col, val, 8, 3, 4, omega, 0.5, sweep, color, d=d)
    return rp, col, val, color, sweep, omega, d, want


def _c0(n, kind):
    if kind == "empty":
        return np.zeros(n, dtype=np.uint8)
    return (np.random.default_rng(2).random(n) < 0.1).astype(np.uint8)


@pytest.mark.parametrize("c0", ["empty", "random"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_cr_matches_oracle(name, c0):
    rp, col, val, color, sweep, omega, d, want = _setup(name)
    n = len(rp) - 1
    C0 = _c0(n, c0)
    args = dict(theta=0.5, nu=5, omega=omega, delta=0.6, tol=0.5, max_sets=12, seed=17)
    Cw, rw = oracle.cr_coarsen(rp, col, val, want["prp"], want["pcol"], want["ls"], sweep=sweep,
                               color=color, coarse0=C0, **args)
    with amgd.Handle(rp, col, val, 8, 3) as h:
        if color is not None:
            h.set_coloring(color)
        h.set_search_depth(d)
        Cg, rg = h.cr_coarsen(C0, ls=want["ls"], sweep=sweep, **args)
        # the LS from device memory gives the same
        Cd, rd = h.cr_coarsen(C0, ls=torch.from_numpy(want["ls"]).cuda(), sweep=sweep, **args)
    print("%s C0=%s: %d stages, |C| = %d of %d, rho %s" % (name, c0, len(rw), Cw.sum(), n,
                                                          np.round(rw, 3)))
    assert len(rw) >= 2
    assert np.array_equal(rg, rw)
    assert np.array_equal(Cg, Cw)
    assert np.array_equal(Cd, Cw) and np.array_equal(rd, rw)
    assert (Cg >= C0).all()


def test_cr_jacobi_on_colored_handle():
    """A handle with a coloring keeps its matrix in color order; Jacobi
    F-relaxation over that order gives the same coarse set as the oracle."""
    rp, col, val, color, sweep, omega, d, want = _setup("aniso9_48_mcgs")
    args = dict(theta=0.5, nu=4, omega=0.7, delta=0.6, tol=0.5, max_sets=12, seed=9)
    Cw, rw = oracle.cr_coarsen(rp, col, val, rp, col, want["ls"], sweep=oracle.SWEEP_JACOBI,
                               **args)
    with amgd.Handle(rp, col, val, 8, 3) as h:
        h.set_coloring(color)
        Cg, rg = h.cr_coarsen(None, ls=want["ls"], sweep=amgd.AMGD_SWEEP_JACOBI, **args)
    assert len(rw) >= 2
    assert np.array_equal(rg, rw) and np.array_equal(Cg, Cw)


def _band_free(prp, pcol, ls, theta, band=1e-9):
    """No two off-diagonal LS values of a row have a ratio within band of theta."""
    n = len(prp) - 1
    for i in range(n):
        q = np.arange(prp[i], prp[i + 1])
        v = ls[q][pcol[q] != i]
        if len(v) < 2:
            continue
        t = theta * v[:, None]
        if np.any(np.abs(t - v[None, :]) <= band * np.maximum(v[None, :], 1e-300)):
            return False
    return True


@pytest.mark.parametrize("name", ["aniso5_64_jacobi", "random_800_d2"])
def test_cr_own_distances(name):
    rp, col, val, color, sweep, omega, d, want = _setup(name)
    args = dict(theta=0.5, nu=5, omega=omega, delta=0.6, tol=0.5, max_sets=12, seed=17)
    with amgd.Handle(rp, col, val, 8, 3) as h:
        h.set_search_depth(d)
        h.relax(4, omega, sweep)
        ls_gpu = h.distances(0.5, want=("ls",))["ls"]
        Cg, rg = h.cr_coarsen(None, ls=None, sweep=sweep, **args)
        Ce, re_ = h.cr_coarsen(None, ls=ls_gpu, sweep=sweep, **args)
    assert np.array_equal(Cg, Ce) and np.array_equal(rg, re_)
    if _band_free(want["prp"], want["pcol"], want["ls"], 0.5):
        Cw, rw = oracle.cr_coarsen(rp, col, val, want["prp"], want["pcol"], want["ls"],
                                   sweep=sweep, color=color, **args)
        assert np.array_equal(Cg, Cw) and np.array_equal(rg, rw)


def test_cr_full_size_aniso9_1024():
    """The 1024 x 1024 rotated anisotropy (eps = 1e-3, alpha = pi/6), LS from
    8 red-black Gauss-Seidel sweeps on K = 16 vectors; CR with 5 red-black
    F-relaxation sweeps per stage."""
    N, K, seed, nu, theta = 1024, 16, 1, 8, 0.5
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    want = oracle.build(rp, col, val, K, seed, nu, 1.0, theta, oracle.SWEEP_MCGS, color)
    args = dict(theta=theta, nu=5, omega=1.0, delta=0.6, tol=0.5, max_sets=12, seed=5)
    t0 = time.perf_counter()
    Cw, rw = oracle.cr_coarsen(rp, col, val, rp, col, want["ls"], sweep=oracle.SWEEP_MCGS,
                               color=color, **args)
    t_or = time.perf_counter() - t0
    with amgd.Handle(rp, col, val, K, seed) as h:
        h.set_coloring(color)
        h.cr_coarsen(None, ls=want["ls"], sweep=amgd.AMGD_SWEEP_MCGS, **args)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Cg, rg = h.cr_coarsen(None, ls=want["ls"], sweep=amgd.AMGD_SWEEP_MCGS, **args)
        t_gpu = time.perf_counter() - t0
        rounds, launches = h.cr_stats()
    print("CR 1024^2: %d stages, |C| = %d, rho %s; oracle %.2f s, GPU %.1f ms (host LS copy "
          "included); %d selection rounds, %d kernels" % (len(rw), Cw.sum(), np.round(rw, 3),
                                                        t_or, 1e3 * t_gpu, rounds, launches))
    stages = len(rw)
    assert rounds >= 4 * (stages - 1)
    # the sweep weights once; per stage: start, 5 sweeps x 2 colors, norm; per
    # added set: candidates, strength, keys, add, 3 kernels per round and one
    # count per batch of rounds
    lower = 1 + stages * 12 + (stages - 1) * 4 + 3 * rounds
    assert lower < launches <= lower + rounds // 4
    assert np.array_equal(rg, rw)
    assert np.array_equal(Cg, Cw)


def test_interp_full_size_aniso9_1024_bf16():
    """LS interpolation (caliber 2, unit weights) at the full 1024 x 1024 size
    on BF16-stored vectors (the oracle's relaxed vectors rounded on the CPU)
    and the oracle's CR coarse set: P equals the oracle's bit for bit."""
    N, K, seed, nu, theta = 1024, 16, 1, 8, 0.5
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    want = oracle.build(rp, col, val, K, seed, nu, 1.0, theta, oracle.SWEEP_MCGS, color)
    C, _ = oracle.cr_coarsen(rp, col, val, rp, col, want["ls"], theta=theta, nu=5, omega=1.0,
                             sweep=oracle.SWEEP_MCGS, color=color, delta=0.6, tol=0.5,
                             max_sets=12, seed=5)
    X = torch.from_numpy(want["X"]).to(torch.bfloat16).to(torch.float64).numpy()
    Y = oracle.target(rp, col, val, X)
    Pw = oracle.ls_interp(X, Y, rp, col, C, 2, 1.5)
    with amgd.Handle(rp, col, val, K, seed) as h:
        h.set_precision("bf16")
        h.set_coloring(color)
        h.set_vectors(X)
        Pg = h.ls_interpolation(C, 2, 1.5)
    for g, w_ in zip(Pg, Pw):
        assert np.array_equal(g, w_)


def test_cr_then_interpolation():
    """Algorithm 1's coarse set feeds the LS interpolation of §4.3: both GPU
    steps in a row equal both oracle steps in a row."""
    rp, col, val, color, sweep, omega, d, want = _setup("aniso5_64_jacobi")
    n, K = len(rp) - 1, 8
    args = dict(theta=0.5, nu=5, omega=omega, delta=0.6, tol=0.5, max_sets=12, seed=17)
    Cw, _ = oracle.cr_coarsen(rp, col, val, rp, col, want["ls"], sweep=sweep, **args)
    prp2, pcol2 = oracle.distance_graph(rp, col, 2)
    Pw = oracle.ls_interp(want["X"], want["Y"], prp2, pcol2, Cw, 2, 1.5)
    with amgd.Handle(rp, col, val, K, 3) as h:
        h.set_vectors(want["X"])
        Cg, _ = h.cr_coarsen(None, ls=want["ls"], sweep=sweep, **args)
        h.set_search_depth(2)
        Pg = h.ls_interpolation(Cg, 2, 1.5)
    assert np.array_equal(Cg, Cw)
    for g, w_ in zip(Pg, Pw):
        assert np.array_equal(g, w_)


def test_cr_special_cases_and_errors():
    rp, col, val = inputs.poisson2d_5pt(16)
    n = 256
    ls = np.ones(len(col))
    with amgd.Handle(rp, col, val, 4, 1) as h:
        C, rho = h.cr_coarsen(np.ones(n, np.uint8), ls=ls, delta=0.0)
        assert list(rho) == [0.0] and C.all()
        C0 = np.zeros(n, np.uint8)
        C0[[3, 50]] = 1
        C, rho = h.cr_coarsen(C0, ls=ls, delta=10.0)
        assert len(rho) == 1 and np.array_equal(C, C0)
        C, rho = h.cr_coarsen(C0, ls=ls, delta=0.0, max_sets=0)
        assert len(rho) == 1 and np.array_equal(C, C0)
        for kw, status in ((dict(nu=0), amgd.AMGD_ERR_ARG), (dict(max_sets=-1), amgd.AMGD_ERR_ARG),
                           (dict(omega=float("nan")), amgd.AMGD_ERR_ARG),
                           (dict(sweep=amgd.AMGD_SWEEP_MCGS), amgd.AMGD_ERR_STATE),
                           (dict(ls=None), amgd.AMGD_ERR_STATE)):
            full = dict(ls=ls)
            full.update(kw)
            with pytest.raises(amgd.AmgdError) as e:
                h.cr_coarsen(None, **full)
            assert e.value.status == status, kw
    mats = [inputs.graph_laplacian(300, 8.0, 4, 0), inputs.graph_laplacian(200, 8.0, 4, 1)]
    with amgd.Handle(None, None, None, 4, 1, batch=mats) as h:
        with pytest.raises(amgd.AmgdError) as e:
            h.cr_coarsen(None, ls=np.ones(h.nnz))
        assert e.value.status == amgd.AMGD_ERR_UNSUPPORTED
