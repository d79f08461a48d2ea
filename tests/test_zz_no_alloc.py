"""amgd_strength_noalloc: the strength CSR for callers that cannot allocate.

Callers that run inside a memory pool or arena owning every device
allocation, or that must never take the CUDA driver's allocation lock, cannot use
the handle-based entry points (a handle allocates its buffers).  They get
amgd_strength_noalloc, which works only in caller buffers plus a static
device array of the library.  This file checks, through the C ABI, that two
calls in a row reproduce what the existing entry point (amgd_strength on a
handle) returns for the same distances, and that sizes beyond the static
array are refused before any GPU work.

The file name makes pytest collect it after every other test file.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1106_5990_gb300 import inputs

pytestmark = pytest.mark.gpu
amgd = pytest.importorskip("paper_1106_5990_gb300.amgd")


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1106_5990_gb300 import _build
    _build.build()
    return t


def _reference(torch, rp, col, val, K, seed, theta, color=None):
    """Distances (device) and the strength CSR from the handle-based API."""
    with amgd.Handle(rp, col, val, K, seed) as h:
        if color is not None:
            h.set_coloring(color)
            h.relax(4, 1.0, amgd.AMGD_SWEEP_MCGS)
        else:
            h.relax(4, 2.0 / 3.0, amgd.AMGD_SWEEP_JACOBI)
        ls = torch.empty(h.nnz, dtype=torch.float64, device="cuda")
        h.distances(theta, out={"ls": ls})
        s_rp = torch.empty(h.n + 1, dtype=torch.int64, device="cuda")
        s_col = torch.empty(max(h.E, 1), dtype=torch.int32, device="cuda")
        h.strength(s_rp, s_col)
        torch.cuda.synchronize()
        return ls, s_rp.cpu().numpy(), s_col.cpu().numpy(), h.E


def _noalloc(torch, rp, col, ls, theta, cap, out_rp, out_col):
    d_rp = torch.from_numpy(np.ascontiguousarray(rp, np.int64)).cuda()
    d_col = torch.from_numpy(np.ascontiguousarray(col, np.int32)).cuda()
    n = len(rp) - 1
    st = amgd.lib().amgd_strength_noalloc(d_rp.data_ptr(), d_col.data_ptr(), ls.data_ptr(), n,
                                          theta, out_rp.data_ptr(), out_col.data_ptr(), cap,
                                          None)
    assert st == amgd.AMGD_OK, amgd.amgd_last_error(None)
    torch.cuda.synchronize()
    return out_rp.cpu().numpy(), out_col.cpu().numpy()


def test_noalloc_matches_existing_entry_point_twice(torch):
    # call 1: 9-point anisotropy, 16,384 rows (4 tiles), red-black sweeps
    N = 128
    rp1, col1, val1 = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    ls1, ref_rp1, ref_col1, E1 = _reference(torch, rp1, col1, val1, 16, 1, 0.5,
                                             inputs.red_black(N))
    # call 2: a graph with isolated rows, a different size and theta, into the
    # same output buffers (the static scratch keeps call 1's contents)
    rp2, col2, val2 = inputs.graph_laplacian(9000, 3.0, 4)
    ls2, ref_rp2, ref_col2, E2 = _reference(torch, rp2, col2, val2, 8, 2, 0.3)

    cap = max(E1, E2)
    out_rp = torch.full((max(len(rp1), len(rp2)),), -1, dtype=torch.int64, device="cuda")
    out_col = torch.full((cap,), -1, dtype=torch.int32, device="cuda")

    got_rp, got_col = _noalloc(torch, rp1, col1, ls1, 0.5, cap, out_rp, out_col)
    n1 = len(rp1) - 1
    assert np.array_equal(got_rp[:n1 + 1], ref_rp1)
    assert np.array_equal(got_col[:ref_rp1[-1]], ref_col1[:ref_rp1[-1]])

    got_rp, got_col = _noalloc(torch, rp2, col2, ls2, 0.3, cap, out_rp, out_col)
    n2 = len(rp2) - 1
    assert np.array_equal(got_rp[:n2 + 1], ref_rp2)
    assert np.array_equal(got_col[:ref_rp2[-1]], ref_col2[:ref_rp2[-1]])


def test_noalloc_truncation_empty_and_side_stream(torch):
    """cap below the number of kept edges: the first cap columns are written
    and s_row_ptr still counts every kept edge; n = 0 writes s_row_ptr[0] = 0;
    a call enqueued on a side stream gives the same result."""
    N = 64
    rp, col, val = inputs.aniso2d_9pt(N, 1e-3, math.pi / 6)
    ls, ref_rp, ref_col, _ = _reference(torch, rp, col, val, 16, 3, 0.5, inputs.red_black(N))
    E = int(ref_rp[-1])                                 # kept edges
    cap = E // 3
    out_rp = torch.full((len(rp),), -1, dtype=torch.int64, device="cuda")
    out_col = torch.full((E,), -7, dtype=torch.int32, device="cuda")
    got_rp, got_col = _noalloc(torch, rp, col, ls, 0.5, cap, out_rp, out_col)
    assert np.array_equal(got_rp, ref_rp) and got_rp[-1] == E > cap
    assert np.array_equal(got_col[:cap], ref_col[:cap])
    assert np.all(got_col[cap:] == -7)                 # nothing written past cap

    empty_rp = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    st = amgd.lib().amgd_strength_noalloc(empty_rp.data_ptr(), 0, 0, 0, 0.5,
                                          empty_rp.data_ptr(), 0, 0, None)
    assert st == amgd.AMGD_OK
    torch.cuda.synchronize()
    assert empty_rp.item() == 0

    side = torch.cuda.Stream()
    d_rp = torch.from_numpy(np.ascontiguousarray(rp, np.int64)).cuda()
    d_col = torch.from_numpy(np.ascontiguousarray(col, np.int32)).cuda()
    out_rp.fill_(-1)
    out_col.fill_(-1)
    torch.cuda.synchronize()
    st = amgd.lib().amgd_strength_noalloc(d_rp.data_ptr(), d_col.data_ptr(), ls.data_ptr(),
                                          len(rp) - 1, 0.5, out_rp.data_ptr(),
                                          out_col.data_ptr(), E, side.cuda_stream)
    assert st == amgd.AMGD_OK
    side.synchronize()
    assert np.array_equal(out_rp.cpu().numpy(), ref_rp)
    assert np.array_equal(out_col.cpu().numpy(), ref_col[:E])


def test_noalloc_more_than_1024_tiles(torch):
    """4,206,649 rows (1,028 tiles of 4,096 rows): the scan of the tile
    offsets crosses its 1,024-entry chunk and carries the 64-bit sum."""
    n = 1024 * 4096 + 12345
    rp, col, val = inputs.lap1d(n)
    ls, ref_rp, ref_col, _ = _reference(torch, rp, col, val, 4, 9, 0.5)
    E = int(ref_rp[-1])
    out_rp = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    out_col = torch.full((E,), -1, dtype=torch.int32, device="cuda")
    got_rp, got_col = _noalloc(torch, rp, col, ls, 0.5, E, out_rp, out_col)
    assert np.array_equal(got_rp, ref_rp)
    assert np.array_equal(got_col, ref_col[:E])


def test_noalloc_rejects_sizes_beyond_the_static_array(torch):
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    st = amgd.lib().amgd_strength_noalloc(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                          268_435_457, 0.5, dummy.data_ptr(), dummy.data_ptr(),
                                          0, None)
    assert st == amgd.AMGD_ERR_UNSUPPORTED
    assert "268435456" in amgd.amgd_last_error(None)
