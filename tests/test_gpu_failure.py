"""Bounded device waits: a staged relaxation kernel whose shared-memory copies
never complete gives up after its wait limit, reports AMGD_ERR_TIMEOUT at the
next synchronising call, and leaves the context usable.

The failure is made without faulting anything: the test hook declares 16
more transaction bytes on the first stage's barrier than the bulk copies
deliver, so that barrier never completes; the copies themselves are real and
land normally, and the limit is shortened to about a millisecond.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1106_5990_gb300 import inputs

pytestmark = pytest.mark.gpu
amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_staged_wait_times_out_and_context_survives(monkeypatch, prec):
    N = 96
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    color = inputs.red_black(N)
    monkeypatch.setenv("AMGD_TEST_STAGING_EXTRA_TX", "16")
    monkeypatch.setenv("AMGD_TEST_WAIT_LIMIT", "2000000")
    with amgd.Handle(rp, col, val, 16, 1) as h:
        h.set_precision(prec)
        h.set_coloring(color)
        G = {"fp64": 8, "bf16": 2}[prec]
        h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, G, 1, 4, 1)
        h.relax(1, 1.0, amgd.AMGD_SWEEP_MCGS)
        with pytest.raises(amgd.AmgdError) as e:
            h.get_vectors()
        assert e.value.status == amgd.AMGD_ERR_TIMEOUT
        # the status was cleared by the report; direct kernels still work
        h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, G, 1, 4, 0)
        h.init_vectors(1)
        h.relax(1, 1.0, amgd.AMGD_SWEEP_MCGS)
        h.get_vectors()
    monkeypatch.delenv("AMGD_TEST_STAGING_EXTRA_TX")
    monkeypatch.delenv("AMGD_TEST_WAIT_LIMIT")
    # a fresh handle on the same context runs the staged kernel correctly
    with amgd.Handle(rp, col, val, 16, 1) as h:
        h.set_coloring(color)
        h.set_kernel_shape(amgd.AMGD_KERNEL_RELAX, 8, 1, 4, 1)
        h.relax(2, 1.0, amgd.AMGD_SWEEP_MCGS)
        want = oracle.relax(rp, col, val, oracle.tv_init(N * N, 16, 1), 2, 1.0,
                            oracle.SWEEP_MCGS, color)
        assert np.array_equal(h.get_vectors(), want)
