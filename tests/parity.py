"""Comparison rules shared by the GPU parity tests.

FP64 path (same rounding of every row sum as the oracle, different order of
the K-term LS sums):
  * test vectors and targets: bit for bit;
  * LS_ij: relative 1e-12 where LS/S_yy >= 1e-8, else |diff| <= 1e-12 S_yy
    (below that ratio LS is a difference of nearly equal numbers and only an
    absolute bound in units of S_yy is meaningful);
  * a_ij: |diff| <= 1e-12 (|a| + sqrt(S_yy/S_xx));
  * strength flags: identical except where |rho - theta| <= band, rho = m_i/LS.
"""
import numpy as np

import oracle


def edge_rows(rp, col):
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    return rows, np.asarray(col)


def ls_scales(rp, col, X, Y, w=None):
    """S_yy of the row and S_xx of the column of every slot (from oracle data)."""
    rows, cols = edge_rows(rp, col)
    w = np.ones(X.shape[1]) if w is None else np.asarray(w)
    syy = (w * Y * Y).sum(1)[rows]
    sxx = (w * X * X).sum(1)[cols]
    return syy, sxx


def check_ls(got, want, syy, off, rel=1e-12, ratio=1e-8, label="LS"):
    g, w_, s = got[off], want[off], syy[off]
    big = w_ >= ratio * s
    err_rel = np.abs(g[big] - w_[big]) / w_[big]
    err_abs = np.abs(g[~big] - w_[~big]) / np.maximum(s[~big], 1e-300)
    worst = max(err_rel.max(initial=0.0), err_abs.max(initial=0.0))
    assert err_rel.max(initial=0.0) <= rel, "%s relative error %.3e" % (label, err_rel.max())
    assert err_abs.max(initial=0.0) <= rel, "%s floor error %.3e" % (label, err_abs.max())
    return worst


def check_a(got, want, syy, sxx, off, tol=1e-12):
    scale = np.abs(want[off]) + np.sqrt(syy[off] / np.maximum(sxx[off], 1e-300))
    err = np.abs(got[off] - want[off]) / scale
    assert err.max(initial=0.0) <= tol, "a error %.3e" % err.max(initial=0.0)
    return err.max(initial=0.0)


def flags_from_strength(rp, col, s_rp, s_col):
    """Per-slot 0/1 from a strength CSR; asserts that each row's kept columns
    are stored columns of that row, in slot order."""
    n = len(rp) - 1
    flag = np.zeros(len(col), dtype=np.uint8)
    for i in range(n):
        row = col[rp[i]:rp[i + 1]]
        pos = {int(c): k for k, c in enumerate(row)}
        kept = s_col[s_rp[i]:s_rp[i + 1]]
        slots = [pos[int(c)] for c in kept]
        assert slots == sorted(slots) and len(set(slots)) == len(slots), i
        flag[rp[i] + np.array(slots, dtype=np.int64)] = 1
    return flag


def flags_from_strength_fast(rp, col, s_rp, s_col):
    """Vectorised variant for large matrices (same checks)."""
    rp = np.asarray(rp, np.int64)
    n = len(rp) - 1
    rows, cols = edge_rows(rp, col)
    key_all = rows * np.int64(n + 1) + cols
    s_rows = np.repeat(np.arange(n), np.diff(s_rp))
    key_s = s_rows * np.int64(n + 1) + np.asarray(s_col, np.int64)
    idx = np.searchsorted(key_all, key_s) if np.all(np.diff(key_all) > 0) else None
    if idx is None:
        order = np.argsort(key_all, kind="stable")
        pos = np.searchsorted(key_all[order], key_s)
        assert np.all(key_all[order][pos] == key_s)
        slot = order[pos]
    else:
        assert np.all(key_all[idx] == key_s)
        slot = idx
    # slot order inside each row
    same_row = s_rows[1:] == s_rows[:-1]
    assert np.all(slot[1:][same_row] > slot[:-1][same_row])
    flag = np.zeros(len(col), dtype=np.uint8)
    flag[slot] = 1
    return flag


def check_flags(got_flag, want, rp, col, theta, band):
    rho = oracle.strength_ratio(rp, col, want["ls"])
    rows, cols = edge_rows(rp, col)
    off = rows != cols
    outside = off & ~(np.abs(rho - theta) <= band)
    bad = np.nonzero(outside & (got_flag != want["flag"]))[0]
    assert bad.size == 0, "strength differs outside the band at %d slots (first %s)" % (
        bad.size, bad[:5])
    assert np.all(got_flag[~off] == 0)
    return int((off & ~outside).sum())
