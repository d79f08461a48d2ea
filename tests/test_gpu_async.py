"""Stream-ordered value updates and strength outputs (amgd_set_values_async,
amgd_strength_async, amgd_sync): a pipelined stream of builds gives, for every
matrix of the stream, the strength graph of the synchronous path and of the
oracle; deferred errors and the state guard."""
import numpy as np
import pytest

import oracle
from paper_1106_5990_gb300 import inputs
from parity import check_flags, flags_from_strength

pytestmark = pytest.mark.gpu
amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()


def _variants(rp, col, val, count):
    """Symmetric rescalings of the off-diagonal values (factors in [0.2, 1]),
    the diagonal set to the negated off-diagonal row sum plus 1e-2, so that
    every matrix has its own graph."""
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    out = []
    for t in range(count):
        lo, hi = np.minimum(rows, col), np.maximum(rows, col)
        f = (np.sin(0.37 * lo + 0.11 * hi + t) + 1.5) / 2.5          # symmetric, in [0.2, 1]
        v = val.copy()
        off = rows != col
        v[off] = val[off] * f[off]
        d = rows == col
        rs = np.zeros(n)
        np.add.at(rs, rows[off], -v[off])
        v[d] = rs + 1e-2
        out.append(v)
    return out


def test_async_stream_matches_sync_and_oracle():
    N, K, seed, nu, omega, theta = 40, 8, 2, 4, 2.0 / 3.0, 0.5
    rp, col, val = inputs.aniso2d_5pt(N, 1e-2)
    vals = _variants(rp, col, val, 4)
    n = N * N
    with amgd.Handle(rp, col, val, K, seed) as h:
        d_rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        d_col = torch.empty(h.E, dtype=torch.int32, device="cuda")
        h.graph_capture(seed, nu, omega, amgd.AMGD_SWEEP_JACOBI, theta, d_rp, d_col)
        pins = [torch.from_numpy(v).pin_memory() for v in vals]
        outs = [(torch.empty(n + 1, dtype=torch.int64).pin_memory(),
                 torch.empty(h.E, dtype=torch.int32).pin_memory()) for _ in vals]
        for v, (o_rp, o_col) in zip(pins, outs):
            h.set_values_async(v)
            h.graph_launch()
            h.strength_async(o_rp, o_col)
        h.sync()
        got = [(o_rp.numpy().copy(), o_col.numpy()[: int(o_rp[-1])].copy()) for o_rp, o_col in outs]
        # the synchronous path on the same handle
        sync = []
        for v in vals:
            h.set_values(v)
            h.graph_launch()
            sync.append(h.strength())
    for (g_rp, g_col), (s_rp, s_col), v in zip(got, sync, vals):
        assert np.array_equal(g_rp, s_rp) and np.array_equal(g_col, s_col)
        want = oracle.build(rp, col, v, K, seed, nu, omega, theta)
        check_flags(flags_from_strength(rp, col, g_rp, g_col), want, rp, col, theta, 1e-9)
    # the matrices really differ
    assert not all(np.array_equal(got[0][1], g[1]) for g in got[1:])


def test_async_device_outputs_and_capacity():
    rp, col, val = inputs.poisson2d_5pt(32)
    n = 32 * 32
    with amgd.Handle(rp, col, val, 8, 1) as h:
        h.relax(3, 0.7)
        h.distances(0.5, want=())
        s_rp_ref, s_col_ref = h.strength()
        o_rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        o_col = torch.empty(h.E, dtype=torch.int32, device="cuda")
        h.strength_async(o_rp, o_col)
        h.sync()
        assert np.array_equal(o_rp.cpu().numpy(), s_rp_ref)
        assert np.array_equal(o_col[: len(s_col_ref)].cpu().numpy(), s_col_ref)
        small = torch.empty(max(len(s_col_ref) - 1, 1), dtype=torch.int32).pin_memory()
        rp_h = torch.empty(n + 1, dtype=torch.int64).pin_memory()
        h.strength_async(rp_h, small)
        with pytest.raises(amgd.AmgdError) as e:
            h.sync()
        assert e.value.status == amgd.AMGD_ERR_CAPACITY


def test_async_deferred_value_error_and_state_guard():
    rp, col, val = inputs.poisson2d_5pt(16)
    with amgd.Handle(rp, col, val, 4, 1) as h:
        bad = val.copy()
        bad[5] = np.nan
        h.set_values_async(bad)
        with pytest.raises(amgd.AmgdError) as e:
            h.set_precision("bf16")                  # pending asynchronous work
        assert e.value.status == amgd.AMGD_ERR_STATE
        with pytest.raises(amgd.AmgdError) as e:
            h.sync()
        assert e.value.status == amgd.AMGD_ERR_CSR
        zero = val.copy()
        zero[rp[3] + list(col[rp[3]:rp[4]]).index(3)] = 0.0
        h.set_values_async(zero)
        with pytest.raises(amgd.AmgdError) as e:
            h.sync()
        assert e.value.status == amgd.AMGD_ERR_ZERO_DIAG
        # valid values again: the handle works and the guard is released
        h.set_values_async(val)
        h.sync()
        h.set_precision("bf16")
        h.relax(2, 0.7)
        h.distances(0.5, want=())
        s_rp, s_col = h.strength()
        assert s_rp[-1] == len(s_col) > 0
        with pytest.raises(amgd.AmgdError) as e:
            with amgd.Handle(rp, col, val, 4, 1) as h2:
                h2.strength_async(np.empty(257, np.int64), np.empty(10, np.int32))
        assert e.value.status == amgd.AMGD_ERR_STATE


def test_fp64_copies_follow_mixed_value_updates():
    """Value updates under mixed storage leave the row-permuted FP64 values
    and diagonal (used only by FP64 sweeps and the coarsening) to be refreshed
    when one of those next runs: after updates under FP32 storage, an FP64
    build on the same handle equals one on a fresh handle bit for bit."""
    N, K, seed = 24, 8, 3
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, 0.5)
    color = inputs.red_black(N)
    v1, v2 = _variants(rp, col, val, 2)
    for coloring in (False, True):
        with amgd.Handle(rp, col, val, K, seed) as h:
            if coloring:
                h.set_coloring(color)
            h.set_precision("fp32")
            h.set_values(v1)
            h.set_values_async(torch.from_numpy(v2).pin_memory())
            h.sync()
            h.set_precision("fp64")
            h.init_vectors(seed)
            sweep = amgd.AMGD_SWEEP_MCGS if coloring else amgd.AMGD_SWEEP_JACOBI
            h.relax(3, 0.9, sweep)
            X = h.get_vectors()
            ls = h.distances(0.5)["ls"]
        with amgd.Handle(rp, col, v2, K, seed) as f:
            if coloring:
                f.set_coloring(color)
            f.relax(3, 0.9, sweep)
            assert np.array_equal(X, f.get_vectors()), coloring
            assert np.array_equal(ls, f.distances(0.5)["ls"], equal_nan=True), coloring


def test_coarsening_follows_mixed_value_updates():
    """The coarsening reads the row-permuted FP64 values, which a value update
    under mixed storage leaves to be refreshed: after updates under FP32
    storage on a colored handle, the coarse set and the rates equal those of a
    fresh handle holding the same values."""
    N, K, seed = 32, 8, 3
    rp, col, val = inputs.aniso2d_9pt(N, 1e-2, 0.3)
    color = inputs.red_black(N)
    v1, v2 = _variants(rp, col, val, 2)
    ls = oracle.build(rp, col, v2, K, seed, 3, 1.0, 0.5)["ls"]
    args = dict(sweep=amgd.AMGD_SWEEP_MCGS, nu=3, max_sets=6)
    with amgd.Handle(rp, col, val, K, seed) as h:
        h.set_coloring(color)
        h.set_precision("fp32")
        h.set_values(v1)
        h.set_values_async(torch.from_numpy(v2).pin_memory())
        h.sync()
        C, rho = h.cr_coarsen(None, ls=ls, **args)
    with amgd.Handle(rp, col, v2, K, seed) as f:
        f.set_coloring(color)
        f.set_precision("fp32")
        Cf, rhof = f.cr_coarsen(None, ls=ls, **args)
    assert np.array_equal(C, Cf) and np.array_equal(rho, rhof)
