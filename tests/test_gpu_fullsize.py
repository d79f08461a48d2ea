"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times: autotuned kernel shapes and one captured CUDA graph per
build (vector start, sweeps, distances, strength CSR).

The accuracy contract of the mixed paths is asserted as stated: distances
(LS) within 1e-3 relative of the FP64 oracle's build of the same matrix,
seed and sweeps (where LS is not a cancellation residue, LS >= 1e-6 S_yy),
and the strength set identical outside |rho - theta| <= 1e-2.  FP32 vector
storage meets it end to end; BF16 storage meets it per stage (the oracle's
functional evaluated on the GPU's own final vectors) but not end to end --
rounding every iterate to an 8-bit significand moves the distances by about
2e-3 -- so the end-to-end BF16 checks are strict expected failures.

* 9-point rotated anisotropy, 1024 x 1024, 8 red-black Gauss-Seidel sweeps,
  K = 16: FP64 against the whole oracle build (vectors bit for bit, LS / a
  within the FP64 rules, strength set identical outside |rho - theta| <=
  1e-9); FP32 storage end to end; BF16 storage per stage.
* 3D jump coefficients, 128^3, 6 Jacobi sweeps, K = 32, FP32 storage end to
  end.
* 64 graph Laplacians (16.3 M rows) in one handle: three matrices of the
  batch (first, middle, last; keys (seed, b)) against the oracle, FP64, FP32
  and BF16 storage.
The 512 x 512 reverse-pass workload is covered in test_gpu_adjoint.py.
"""
import math

import numpy as np
import pytest

import oracle
from parity import check_a, check_flags, check_ls, edge_rows, flags_from_strength_fast, ls_scales
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


def graph_build(h, K, seed, nu, omega, sweep, theta):
    """One captured build as the benchmark runs it; returns device outputs."""
    h.autotune(sweep, omega, None)
    d_rp = torch.empty(h.n + 1, dtype=torch.int64, device="cuda")
    d_col = torch.empty(max(h.E, 1), dtype=torch.int32, device="cuda")
    h.graph_capture(seed, nu, omega, sweep, theta, d_rp, d_col)
    h.graph_launch()
    X = torch.empty((h.n, K), dtype=torch.float64, device="cuda")
    h.get_vectors(out=X)
    # the per-slot values of the same pass (same kernel, shape and inputs)
    out = {k: torch.empty(h.nnz, dtype=torch.float64, device="cuda") for k in ("a", "ls")}
    h.distances(theta, want=("a", "ls"), out=out)
    torch.cuda.synchronize()
    return X, out, d_rp, d_col


def _rel_ls(got, want, syy, off):
    big = off & (want >= 1e-6 * syy)
    return np.abs(got[big] - want[big]) / want[big]


E2E_BAR = 1e-3       # distance relative error against the FP64 oracle
BAND = 1e-2          # strength set identical outside |rho - theta| <= BAND
_C2 = {}


def _c2_oracle():
    if "want" not in _C2:
        N, K, seed, nu, omega, theta = 1024, 16, 1, 8, 1.0, 0.5
        rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
        color = inputs.red_black(N)
        want = oracle.build(rp, col, val, K, seed, nu, omega, theta, oracle.SWEEP_MCGS, color)
        _C2.update(mat=(rp, col, val), color=color, want=want)
    return _C2


def _c2_gpu(prec):
    key = "gpu_" + prec
    if key not in _C2:
        c = _c2_oracle()
        rp, col, val = c["mat"]
        K, seed, nu, omega, theta = 16, 1, 8, 1.0, 0.5
        with amgd.Handle(rp, col, val, K, seed) as h:
            h.set_precision(prec)
            h.set_coloring(c["color"])
            X, out, d_rp, d_col = graph_build(h, K, seed, nu, omega, amgd.AMGD_SWEEP_MCGS, theta)
            s_rp = d_rp.cpu().numpy()
            s_col = d_col[: int(s_rp[-1])].cpu().numpy()
            _C2[key] = dict(ls=out["ls"].cpu().numpy(), a=out["a"].cpu().numpy(),
                            X=X.cpu().numpy(),
                            flag=flags_from_strength_fast(rp, col, s_rp, s_col))
    return _C2[key]


def _end_to_end_report(prec, got, want, rp, col, theta):
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, _ = ls_scales(rp, col, want["X"], want["Y"])
    rel = _rel_ls(got["ls"], want["ls"], syy, off)
    rho = oracle.strength_ratio(rp, col, want["ls"])
    wide = off & (np.abs(rho - theta) > BAND) & (got["flag"] != want["flag"])
    print("%s end to end: LS rel err median %.2e p99 %.2e max %.2e; %d of %d edges flip "
          "outside the +-%.0e band" % (prec, np.median(rel), np.quantile(rel, 0.99), rel.max(),
                                        wide.sum(), off.sum(), BAND))
    return rel, wide


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_aniso9_1024_end_to_end(prec):
    c = _c2_oracle()
    rp, col, val = c["mat"]
    want = c["want"]
    got = _c2_gpu(prec)
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, sxx = ls_scales(rp, col, want["X"], want["Y"])
    if prec == "fp64":
        assert np.array_equal(got["X"], want["X"])
        check_ls(got["ls"], want["ls"], syy, off)
        check_a(got["a"], want["a"], syy, sxx, off)
        check_flags(got["flag"], want, rp, col, 0.5, 1e-9)
    else:
        rel, wide = _end_to_end_report(prec, got, want, rp, col, 0.5)
        assert rel.max() <= E2E_BAR
        check_flags(got["flag"], want, rp, col, 0.5, BAND)
        assert wide.sum() == 0


def test_aniso9_1024_bf16_stage():
    """BF16 storage: the distance stage on the GPU's own final (BF16) vectors
    against the oracle's functional on the same vectors (exact in FP64)."""
    c = _c2_oracle()
    rp, col, val = c["mat"]
    got = _c2_gpu("bf16")
    Y = oracle.target(rp, col, val, got["X"])
    a_w, ls_w = oracle.edge_ls(rp, col, val, got["X"], Y)
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, sxx = ls_scales(rp, col, got["X"], Y)
    big = ls_w >= 1e-8 * syy
    rel = (np.abs(got["ls"] - ls_w) / np.where(big, ls_w, syy))[off]
    print("bf16 stage LS rel err: median %.2e max %.2e" % (np.median(rel), rel.max()))
    assert rel.max() <= E2E_BAR
    flag_w, _ = oracle.threshold(rp, col, ls_w, 0.5)
    check_flags(got["flag"], dict(ls=ls_w, flag=flag_w), rp, col, 0.5, BAND)


@pytest.mark.xfail(strict=True, reason="BF16 vector storage misses the 1e-3 end-to-end "
                                       "distance bar (median about 2e-3)")
def test_aniso9_1024_bf16_end_to_end_contract():
    c = _c2_oracle()
    rp, col, _ = c["mat"]
    rel, wide = _end_to_end_report("bf16", _c2_gpu("bf16"), c["want"], rp, col, 0.5)
    assert rel.max() <= E2E_BAR and wide.sum() == 0


def test_jump3d_128_fp32():
    N, K, seed, nu, omega, theta = 128, 32, 3, 6, 0.8, 0.5
    rp, col, val = inputs.jump3d_7pt(N, 2.0, 2)
    want = oracle.build(rp, col, val, K, seed, nu, omega, theta)
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    syy, _ = ls_scales(rp, col, want["X"], want["Y"])
    with amgd.Handle(rp, col, val, K, seed) as h:
        h.set_precision("fp32")
        X, out, d_rp, d_col = graph_build(h, K, seed, nu, omega, amgd.AMGD_SWEEP_JACOBI, theta)
        s_rp = d_rp.cpu().numpy()
        s_col = d_col[: int(s_rp[-1])].cpu().numpy()
        ls = out["ls"].cpu().numpy()
    rel = _rel_ls(ls, want["ls"], syy, off)
    q50, q99 = np.quantile(rel, [0.5, 0.99])
    print("fp32 128^3 end-to-end LS rel err: median %.2e p99 %.2e max %.2e"
          % (q50, q99, rel.max()))
    assert rel.max() <= 1e-3
    flag = flags_from_strength_fast(rp, col, s_rp, s_col)
    check_flags(flag, want, rp, col, theta, 1e-2)


_C4 = {}


def _c4_run(prec):
    """Three matrices of the 64-matrix batch (first, middle, last) from one
    captured batched build: GPU outputs and the oracle's build of each."""
    if prec in _C4:
        return _C4[prec]
    K, seed, nu, omega, theta = 16, 6, 4, 2.0 / 3.0, 0.5
    if "mats" not in _C4:
        _C4["mats"] = inputs.graph_laplacian_batch(64, 10_000, 500_000, 8.0, 4, 5)
        _C4["want"] = {b: oracle.build(*_C4["mats"][b], K, seed, nu, omega, theta, stream=b)
                       for b in (0, 31, 63)}
    mats = _C4["mats"]
    res = {}
    with amgd.Handle(None, None, None, K, seed, batch=mats) as h:
        h.set_precision(prec)
        X, out, d_rp, d_col = graph_build(h, K, seed, nu, omega, amgd.AMGD_SWEEP_JACOBI, theta)
        ro, so = h.offsets()
        s_rp_all = d_rp.cpu().numpy()
        for b in (0, 31, 63):
            rp, col, val = mats[b]
            sl = slice(int(so[b]), int(so[b + 1]))
            r0, r1 = int(ro[b]), int(ro[b + 1])
            # this matrix's part of the strength CSR, in local numbering
            s_rp = s_rp_all[r0:r1 + 1] - s_rp_all[r0]
            s_col = d_col[int(s_rp_all[r0]):int(s_rp_all[r1])].cpu().numpy() - r0
            res[b] = dict(ls=out["ls"][sl].cpu().numpy(), a=out["a"][sl].cpu().numpy(),
                          X=X[r0:r1].cpu().numpy(),
                          flag=flags_from_strength_fast(rp, col, s_rp, s_col))
    _C4[prec] = res
    return res


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_batch_64_sampled(prec):
    got_all = _c4_run(prec)
    for b in (0, 31, 63):
        rp, col, val = _C4["mats"][b]
        want = _C4["want"][b]
        got = got_all[b]
        rows, cols = edge_rows(rp, col)
        off = rows != cols
        syy, sxx = ls_scales(rp, col, want["X"], want["Y"])
        if prec == "fp64":
            assert np.array_equal(got["X"], want["X"]), b
            check_ls(got["ls"], want["ls"], syy, off)
            check_a(got["a"], want["a"], syy, sxx, off)
            check_flags(got["flag"], want, rp, col, 0.5, 1e-9)
        else:
            rel, wide = _end_to_end_report("%s graph %d" % (prec, b), got, want, rp, col, 0.5)
            assert rel.max() <= E2E_BAR, b
            check_flags(got["flag"], want, rp, col, 0.5, BAND)


def test_graph_batch_64_bf16_stage():
    got_all = _c4_run("bf16")
    for b in (0, 31, 63):
        rp, col, val = _C4["mats"][b]
        got = got_all[b]
        Y = oracle.target(rp, col, val, got["X"])
        a_w, ls_w = oracle.edge_ls(rp, col, val, got["X"], Y)
        rows, cols = edge_rows(rp, col)
        off = rows != cols
        syy, _ = ls_scales(rp, col, got["X"], Y)
        big = ls_w >= 1e-8 * syy
        rel = (np.abs(got["ls"] - ls_w) / np.where(big, ls_w, syy))[off]
        assert rel.max() <= E2E_BAR, (b, rel.max())
        flag_w, _ = oracle.threshold(rp, col, ls_w, 0.5)
        check_flags(got["flag"], dict(ls=ls_w, flag=flag_w), rp, col, 0.5, BAND)


@pytest.mark.xfail(strict=True, reason="BF16 vector storage misses the 1e-3 end-to-end "
                                       "distance bar on the graph batch (median about 1e-3)")
def test_graph_batch_64_bf16_end_to_end_contract():
    got_all = _c4_run("bf16")
    ok = True
    for b in (0, 31, 63):
        rp, col, _ = _C4["mats"][b]
        rel, wide = _end_to_end_report("bf16 graph %d" % b, got_all[b], _C4["want"][b], rp, col,
                                       0.5)
        ok = ok and rel.max() <= E2E_BAR and wide.sum() == 0
    assert ok
