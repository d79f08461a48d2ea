"""Reverse pass on the GPU (amgd_set_checkpointing / amgd_backward) against
the FP64 oracle's reverse pass and against finite differences.

FP64 storage: the forward path is bit-identical to the oracle, so the two
reverse passes differ only in the order of their sums; the gradient with
respect to the values of A must agree normwise to 1e-11 and dL/domega to
1e-11 relative (a few thousand FP64 roundings, each amplified by at most
the loss's own conditioning on these small cases).  The checkpoint interval
changes no bit.  Central differences of the GPU's own FP64 forward loss
agree with the gradient to 1e-5 along random directions (the kept set is
checked not to move).

FP32/BF16 storage: the forward path rounds every iterate to the storage
type; the reverse pass itself computes in FP64 from those stored iterates
(the fits refitted in FP64), so the gradient differs from the oracle's FP64
gradient only through the rounding of the stored trajectory.  FP32 storage
is held to the 1e-5 relative bar of the reverse pass -- against the oracle's
gradient and against central differences of the oracle's loss; BF16 storage
(an 8-bit significand per stored iterate) is reported against a loose bar.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1106_5990_gb300 import inputs
from parity import flags_from_strength

pytestmark = pytest.mark.gpu
amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()


def run_gpu(mat, K, seed, nu, omega, theta, every, prec="fp64", target=0, w=None,
            ls_bar=None, batch=None):
    rp, col, val = mat if batch is None else (None, None, None)
    with amgd.Handle(rp, col, val, K, seed, batch=batch) as h:
        h.set_precision(prec)
        h.set_target(target)
        if w is not None:
            h.set_weights(w)
        h.set_checkpointing(every)
        h.init_vectors(seed)
        X0 = h.get_vectors()
        h.relax(nu, omega, amgd.AMGD_SWEEP_JACOBI)
        d = h.distances(theta, want=("ls",))
        vb, wb, loss = h.backward(ls_bar=ls_bar)
        return dict(X0=X0, ls=d["ls"], val_bar=vb, omega_bar=wb, loss=loss)


def x0(mat, K, seed, batch=None):
    """The oracle's start vectors (never the GPU's): Philox of (seed, matrix id)."""
    if batch is None:
        return oracle.tv_init(len(mat[0]) - 1, K, seed)
    return np.concatenate([oracle.tv_init(len(m[0]) - 1, K, seed, b) for b, m in enumerate(batch)])


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) /
                 max(np.linalg.norm(np.asarray(b)), 1e-300))


def check_fp64(g, o, tol=1e-11):
    assert rel(g["val_bar"], o["val_bar"]) <= tol, rel(g["val_bar"], o["val_bar"])
    assert abs(g["omega_bar"] - o["omega_bar"]) <= tol * abs(o["omega_bar"]) + 1e-300
    if not math.isnan(o["loss"]):
        assert abs(g["loss"] - o["loss"]) <= 1e-12 * o["loss"]


CASES = {
    "aniso5_32": (lambda: inputs.aniso2d_5pt(32, 1e-2), 16, 10, 2.0 / 3.0),
    "aniso9_24": (lambda: inputs.aniso2d_9pt(24, 1e-3, math.pi / 6), 8, 6, 0.8),
    "random_600": (lambda: inputs.random_csr(600, 6.0, 9), 8, 5, 0.6),
    "graph_1500": (lambda: inputs.graph_laplacian(1500, 8.0, 4), 16, 4, 2.0 / 3.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("target", [0, 1])
def test_fp64_matches_oracle(case, target):
    make, K, nu, omega = CASES[case]
    mat = make()
    rng = np.random.default_rng(1)
    w = rng.uniform(0.5, 2.0, K) if case == "random_600" else None
    g = run_gpu(mat, K, 7, nu, omega, 0.5, 2, target=target, w=w)
    assert np.array_equal(g["X0"], x0(mat, K, 7))
    o = oracle.adjoint_jacobi(*mat, x0(mat, K, 7), nu, omega, 0.5, w, target)
    check_fp64(g, o)


def test_checkpoint_interval_changes_no_bit():
    mat = inputs.aniso2d_5pt(32, 1e-2)
    ref = run_gpu(mat, 16, 3, 10, 2.0 / 3.0, 0.5, 1)
    for every in (2, 3, 4, 10, 16):
        g = run_gpu(mat, 16, 3, 10, 2.0 / 3.0, 0.5, every)
        assert np.array_equal(g["val_bar"], ref["val_bar"]), every
        assert g["omega_bar"] == ref["omega_bar"] and g["loss"] == ref["loss"]
    again = run_gpu(mat, 16, 3, 10, 2.0 / 3.0, 0.5, 1)
    assert np.array_equal(again["val_bar"], ref["val_bar"])       # deterministic


def test_no_sweeps_and_upstream_gradient():
    mat = inputs.random_csr(400, 5.0, 2)
    rp, col, val = mat
    g = run_gpu(mat, 8, 4, 0, 0.7, 0.5, 2)
    o = oracle.adjoint_jacobi(rp, col, val, x0(mat, 8, 4), 0, 0.7, 0.5)
    check_fp64(g, o)
    assert g["omega_bar"] == 0.0
    # an explicit dL/dLS, host and device
    lsb = np.random.default_rng(5).standard_normal(len(col))
    g = run_gpu(mat, 8, 4, 3, 0.7, 0.5, 2, ls_bar=lsb)
    o = oracle.adjoint_jacobi(rp, col, val, x0(mat, 8, 4), 3, 0.7, 0.5, ls_bar=lsb)
    check_fp64(g, o)
    assert math.isnan(g["loss"])
    with amgd.Handle(rp, col, val, 8, 4) as h:
        h.set_checkpointing(2)
        h.relax(3, 0.7)
        h.distances(0.5, want=())
        d_lsb = torch.from_numpy(lsb).cuda()
        out = torch.empty(len(col), dtype=torch.float64, device="cuda")
        _, wb, _ = h.backward(ls_bar=d_lsb, out=out)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), o["val_bar"]) <= 1e-11
        assert abs(wb - o["omega_bar"]) <= 1e-11 * abs(o["omega_bar"])


def test_batch_matches_oracle():
    mats = [inputs.graph_laplacian(700, 8.0, 4, 0), inputs.graph_laplacian(1100, 8.0, 4, 1)]
    g = run_gpu(None, 16, 6, 4, 2.0 / 3.0, 0.5, 2, batch=mats)
    # the batch is block diagonal: one oracle call on the concatenation
    ro = np.cumsum([0] + [len(m[0]) - 1 for m in mats])
    so = np.cumsum([0] + [len(m[1]) for m in mats])
    rp = np.concatenate([mats[0][0]] + [m[0][1:] + so[b] for b, m in enumerate(mats) if b > 0])
    col = np.concatenate([m[1] + ro[b] for b, m in enumerate(mats)])
    val = np.concatenate([m[2] for m in mats])
    assert np.array_equal(g["X0"], x0(None, 16, 6, batch=mats))
    o = oracle.adjoint_jacobi(rp, col, val, x0(None, 16, 6, batch=mats), 4, 2.0 / 3.0, 0.5)
    check_fp64(g, o)


def test_finite_differences_of_gpu_forward():
    rp, col, val = inputs.aniso2d_9pt(20, 1e-2, math.pi / 6)
    K, nu, omega, theta = 16, 6, 0.7, 0.5
    with amgd.Handle(rp, col, val, K, 11) as h:
        h.set_checkpointing(2)

        def loss(v, om):
            h.set_values(v)
            h.init_vectors(11)
            h.relax(nu, om)
            ls = h.distances(theta, want=("ls",))["ls"]
            s_rp, s_col = h.strength()
            return ls, (s_rp, s_col)

        ls0, kept0 = loss(val, omega)
        vb, wb, L = h.backward()
        rng = np.random.default_rng(0)
        for trial in range(3):
            d = rng.standard_normal(len(val)) * np.abs(val)
            hstep = 1e-6
            lp, kp = loss(val + hstep * d, omega)
            lm, km = loss(val - hstep * d, omega)
            assert np.array_equal(kp[1], kept0[1]) and np.array_equal(km[1], kept0[1])
            Lp = _loss_from(rp, col, lp, kp)
            Lm = _loss_from(rp, col, lm, km)
            fd = (Lp - Lm) / (2 * hstep)
            assert abs(fd - vb @ d) <= 1e-5 * abs(fd), (fd, vb @ d)
        lp, kp = loss(val, omega + 1e-6)
        lm, km = loss(val, omega - 1e-6)
        assert np.array_equal(kp[1], kept0[1]) and np.array_equal(km[1], kept0[1])
        fd = (_loss_from(rp, col, lp, kp) - _loss_from(rp, col, lm, km)) / 2e-6
        assert abs(fd - wb) <= 1e-5 * abs(fd)


def _loss_from(rp, col, ls, strength):
    """The built-in loss from the GPU's own outputs: sum of LS^-2 over the
    slots its strength graph keeps with LS > 0."""
    flag = flags_from_strength(rp, col, *strength)
    keep = (flag == 1) & (ls > 0)
    return float(np.sum(1.0 / ls[keep] ** 2))


def test_state_errors():
    rp, col, val = inputs.poisson2d_5pt(16)
    with amgd.Handle(rp, col, val, 8, 1) as h:
        h.relax(2, 0.7)
        h.distances(0.5, want=())
        with pytest.raises(amgd.AmgdError) as e:
            h.backward()
        assert e.value.status == amgd.AMGD_ERR_STATE
        h.set_checkpointing(2)
        h.relax(2, 0.7)
        with pytest.raises(amgd.AmgdError) as e:        # no distances after the sweeps
            h.backward()
        assert e.value.status == amgd.AMGD_ERR_STATE
        h.distances(0.5, want=())
        h.backward()
        h.set_values(val)                               # trajectory dropped
        with pytest.raises(amgd.AmgdError) as e:
            h.backward()
        assert e.value.status == amgd.AMGD_ERR_STATE
        h.set_coloring(inputs.red_black(16))
        h.relax(2, 0.7)
        h.distances(0.5, want=())
        with pytest.raises(amgd.AmgdError) as e:
            h.backward()
        assert e.value.status == amgd.AMGD_ERR_UNSUPPORTED


MIXED_BARS = {"fp32": 1e-5, "bf16": 5e-2}


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mixed_against_fp64_oracle(prec):
    mat = inputs.aniso2d_5pt(48, 1e-2)
    g = run_gpu(mat, 16, 7, 10, 2.0 / 3.0, 0.5, 2, prec=prec)
    o = oracle.adjoint_jacobi(*mat, x0(mat, 16, 7), 10, 2.0 / 3.0, 0.5)
    e_v = rel(g["val_bar"], o["val_bar"])
    e_w = abs(g["omega_bar"] - o["omega_bar"]) / abs(o["omega_bar"])
    e_l = abs(g["loss"] - o["loss"]) / o["loss"]
    print("%s: val_bar %.2e omega_bar %.2e loss %.2e" % (prec, e_v, e_w, e_l))
    assert max(e_v, e_w, e_l) <= MIXED_BARS[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_aniso5_512(prec):
    """The 512 x 512 anisotropic 5-point workload (eps = 1e-2, K = 16,
    nu = 10 Jacobi sweeps, omega = 2/3, checkpoints every 2 sweeps) against
    the oracle at full size."""
    mat = inputs.aniso2d_5pt(512, 1e-2)
    g = run_gpu(mat, 16, 7, 10, 2.0 / 3.0, 0.5, 2, prec=prec)
    o = oracle.adjoint_jacobi(*mat, x0(mat, 16, 7), 10, 2.0 / 3.0, 0.5)
    if prec == "fp64":
        check_fp64(g, o)
    else:
        e = rel(g["val_bar"], o["val_bar"])
        print("fp32 full size: val_bar %.2e" % e)
        assert e <= MIXED_BARS["fp32"]


def test_fp32_full_size_against_oracle_finite_differences():
    """The 512 x 512 reverse-pass workload at its own precision (FP32 storage):
    directional derivatives of the GPU gradient against central differences
    of the oracle's FP64 loss at the same (FP32-rounded) start vectors, three
    random directions and omega, each within 1e-5 relative; the kept set is
    checked not to move under the perturbation."""
    rp, col, val = inputs.aniso2d_5pt(512, 1e-2)
    K, seed, nu, omega, theta = 16, 7, 10, 2.0 / 3.0, 0.5
    g = run_gpu((rp, col, val), K, seed, nu, omega, theta, 2, prec="fp32")
    X0 = g["X0"]                                   # the GPU's start vectors (FP32 values)
    L0, f0 = oracle.strength_loss(rp, col, val, X0, nu, omega, theta)
    rng = np.random.default_rng(3)
    hstep = 1e-7
    done = 0
    for trial in range(10):
        d = rng.standard_normal(len(val)) * np.abs(val)
        Lp, fp = oracle.strength_loss(rp, col, val + hstep * d, X0, nu, omega, theta)
        Lm, fm = oracle.strength_loss(rp, col, val - hstep * d, X0, nu, omega, theta)
        if not (np.array_equal(fp, f0) and np.array_equal(fm, f0)):
            continue            # an edge at theta moved: the loss is not differentiable there
        fd = (Lp - Lm) / (2 * hstep)
        print("direction %d: fd %.9e  gpu %.9e  rel %.2e" % (trial, fd, g["val_bar"] @ d,
                                                          abs(fd - g["val_bar"] @ d) / abs(fd)))
        assert abs(fd - g["val_bar"] @ d) <= 1e-5 * abs(fd)
        done += 1
        if done == 3:
            break
    assert done == 3
    Lp, fp = oracle.strength_loss(rp, col, val, X0, nu, omega + hstep, theta)
    Lm, fm = oracle.strength_loss(rp, col, val, X0, nu, omega - hstep, theta)
    assert np.array_equal(fp, f0) and np.array_equal(fm, f0)
    fd = (Lp - Lm) / (2 * hstep)
    assert abs(fd - g["omega_bar"]) <= 1e-5 * abs(fd)
    assert abs(g["loss"] - L0) <= 1e-5 * L0


def test_autograd_function():
    from paper_1106_5990_gb300 import autograd as ag
    rp, col, val = inputs.random_csr(300, 5.0, 3)
    vals = torch.from_numpy(val).cuda().requires_grad_(True)
    omega = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    with amgd.Handle(rp, col, val, 8, 2) as h:
        ls = ag.DistanceFn.apply(vals, omega, h, 2, 4, 0.5, 2)
        off = ~torch.isnan(ls)
        wgt = torch.from_numpy(np.random.default_rng(0).standard_normal(len(col))).cuda()
        (ls[off] * wgt[off]).sum().backward()
        o = oracle.adjoint_jacobi(rp, col, val, oracle.tv_init(300, 8, 2), 4, 0.7, 0.5,
                                  ls_bar=np.where(off.cpu().numpy(), wgt.cpu().numpy(), 0.0))
        assert rel(vals.grad.cpu().numpy(), o["val_bar"]) <= 1e-11
        assert abs(omega.grad.item() - o["omega_bar"]) <= 1e-11 * abs(o["omega_bar"])
        vals.grad = None
        omega.grad = None
        L = ag.strength_loss(h, vals, omega, 2, 4, 0.5, 2)
        L.backward()
        o = oracle.adjoint_jacobi(rp, col, val, oracle.tv_init(300, 8, 2), 4, 0.7, 0.5)
        assert abs(L.item() - o["loss"]) <= 1e-12 * o["loss"]
        assert rel(vals.grad.cpu().numpy(), o["val_bar"]) <= 1e-11


def test_graph_replay_matches_eager():
    rp, col, val = inputs.aniso2d_5pt(40, 1e-2)
    K, nu, omega, theta = 16, 10, 2.0 / 3.0, 0.5
    for prec in ("fp64", "fp32"):
        with amgd.Handle(rp, col, val, K, 7) as h:
            h.set_precision(prec)
            h.set_checkpointing(2)
            h.init_vectors(7)
            h.relax(nu, omega)
            h.distances(theta, want=())
            vb_e, wb_e, L_e = h.backward()
            d_vb = torch.full((len(col),), float("nan"), dtype=torch.float64, device="cuda")
            h.graph_capture_backward(7, nu, omega, theta, d_vb)
            for _ in range(2):
                h.graph_launch()
                wb_g, L_g = h.backward_scalars()
                assert np.array_equal(d_vb.cpu().numpy(), vb_e)
                assert wb_g == wb_e and L_g == L_e
            # the replayed trajectory serves an eager reverse pass as well
            vb2, wb2, _ = h.backward()
            assert np.array_equal(vb2, vb_e) and wb2 == wb_e
