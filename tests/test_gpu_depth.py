"""Search depth d > 1 (§4.1, Eq. (4.2); §4.2 M^d) on the GPU against the
FP64 oracle: the pattern of A^d bit for bit, then the whole build with the
FP64 rules of the other parity tests (vectors bit for bit, LS within 1e-12
relative or 1e-12 S_yy, strength set identical outside |rho - theta| <=
1e-9), for both edge kernels, both targets, multicolor and Jacobi sweeps,
rows with a single off-diagonal (the exact rule on G_d), and a BF16 end to
end run within the mixed-path band."""
import math

import numpy as np
import pytest

import oracle
from parity import (check_a, check_flags, check_ls, edge_rows, flags_from_strength,
                    flags_from_strength_fast, ls_scales)
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


MATS = {
    "aniso9_30_rb": (lambda: inputs.aniso2d_9pt(30, 1e-3, -math.pi / 4), "rb30"),
    "random_800": (lambda: inputs.random_csr(800, 4.0, 21), None),
    "lap1d_500": (lambda: inputs.lap1d(500), None),
    "graph_1500": (lambda: inputs.graph_laplacian(1500, 3.0, 8), None),
}


def _build_gpu(rp, col, val, K, seed, nu, omega, theta, d, sweep, color, target, stage,
               prec="fp64"):
    with amgd.Handle(rp, col, val, K, seed) as h:
        h.set_precision(prec)
        if color is not None:
            h.set_coloring(color)
        h.set_target(target)
        h.set_search_depth(d)
        G, NV, U, _ = h.kernel_shape(amgd.AMGD_KERNEL_EDGE)
        h.set_kernel_shape(amgd.AMGD_KERNEL_EDGE, G, NV, U, stage)
        h.relax(nu, omega, sweep)
        X = h.get_vectors()
        out = h.distances(theta)
        s_rp, s_col = h.strength()
        prp, pcol = h.distance_pattern()
    return dict(X=X, a=out["a"], ls=out["ls"], dist=out["dist"], s_rp=s_rp, s_col=s_col,
                prp=prp, pcol=pcol)


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("stage", [0, 1])
def test_depth_fp64_matches_oracle(name, d, stage):
    make, cname = MATS[name]
    rp, col, val = make()
    color = inputs.red_black(30) if cname == "rb30" else None
    sweep = amgd.AMGD_SWEEP_MCGS if color is not None else amgd.AMGD_SWEEP_JACOBI
    osweep = oracle.SWEEP_MCGS if color is not None else oracle.SWEEP_JACOBI
    omega = 1.0 if color is not None else 2.0 / 3.0
    for target in (0, 1):
        want = oracle.build(rp, col, val, 8, 5, 3, omega, 0.5, osweep, color, mode=target, d=d)
        got = _build_gpu(rp, col, val, 8, 5, 3, omega, 0.5, d, sweep, color, target, stage)
        prp, pcol = want["prp"], want["pcol"]
        assert np.array_equal(got["prp"], prp) and np.array_equal(got["pcol"], pcol)
        assert np.array_equal(got["X"], want["X"])
        rows, cols = edge_rows(prp, pcol)
        off = rows != cols
        syy, sxx = ls_scales(prp, pcol, want["X"], want["Y"])
        check_ls(got["ls"], want["ls"], syy, off)
        check_a(got["a"], want["a"], syy, sxx, off)
        assert np.all(np.isnan(got["ls"][~off]))
        flag = flags_from_strength(prp, pcol, got["s_rp"], got["s_col"]) if len(prp) < 5000 \
            else flags_from_strength_fast(prp, pcol, got["s_rp"], got["s_col"])
        check_flags(flag, want, prp, pcol, 0.5, 1e-9)


def test_depth_switch_and_graph():
    rp, col, val = inputs.aniso2d_5pt(40, 1e-2)
    K, seed, nu, omega, theta = 16, 3, 5, 2.0 / 3.0, 0.5
    want1 = oracle.build(rp, col, val, K, seed, nu, omega, theta)
    want2 = oracle.build(rp, col, val, K, seed, nu, omega, theta, d=2)
    with amgd.Handle(rp, col, val, K, seed) as h:
        for d, want in ((2, want2), (1, want1), (2, want2)):
            h.set_search_depth(d)
            h.init_vectors(seed)
            h.relax(nu, omega)
            ls = h.distances(theta, want=("ls",))["ls"]
            off = ~np.isnan(want["ls"])
            assert ls.shape == want["ls"].shape
            assert np.allclose(ls[off], want["ls"][off], rtol=1e-11, atol=0)
        # one captured build at d = 2 equals the eager one
        d_rp = torch.empty(h.n + 1, dtype=torch.int64, device="cuda")
        d_col = torch.empty(h.E_p, dtype=torch.int32, device="cuda")
        h.graph_capture(seed, nu, omega, amgd.AMGD_SWEEP_JACOBI, theta, d_rp, d_col)
        h.graph_launch()
        torch.cuda.synchronize()
        s_rp = d_rp.cpu().numpy()
        assert np.array_equal(s_rp, want2["s_rp"])
        assert np.array_equal(d_col[: s_rp[-1]].cpu().numpy(), want2["s_col"])
        # the reverse pass covers depth 1 only
        h.set_checkpointing(2)
        h.relax(1, omega)
        h.distances(theta, want=())
        with pytest.raises(amgd.AmgdError) as e:
            h.backward()
        assert e.value.status == amgd.AMGD_ERR_UNSUPPORTED


@pytest.mark.parametrize("stage", [0, 1])
def test_depth_bf16_end_to_end(stage):
    N = 64
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 8)
    color = inputs.red_black(N)
    want = oracle.build(rp, col, val, 16, 1, 8, 1.0, 0.5, oracle.SWEEP_MCGS, color, d=2)
    got = _build_gpu(rp, col, val, 16, 1, 8, 1.0, 0.5, 2, amgd.AMGD_SWEEP_MCGS, color, 0, stage,
                     prec="bf16")
    prp, pcol = want["prp"], want["pcol"]
    rows, cols = edge_rows(prp, pcol)
    off = rows != cols
    syy, _ = ls_scales(prp, pcol, want["X"], want["Y"])
    big = off & (want["ls"] >= 1e-6 * syy)
    rel = np.abs(got["ls"][big] - want["ls"][big]) / want["ls"][big]
    print("bf16 d=2 end-to-end LS rel err: median %.2e p99 %.2e" % (np.median(rel),
                                                                   np.quantile(rel, 0.99)))
    assert np.median(rel) <= 5e-3 and np.quantile(rel, 0.99) <= 3e-2
    flag = flags_from_strength(prp, pcol, got["s_rp"], got["s_col"])
    check_flags(flag, want, prp, pcol, 0.5, 3e-2)
