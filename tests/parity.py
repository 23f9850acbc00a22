"""Element-wise comparison helpers shared by the GPU parity tests.

A Frobenius-norm ratio over a whole gradient can hide one wrong row (a bad
fix-up of a split row, a wrong tail of a short segment).  These helpers
compare every row i of an FP32 result g against the FP64 oracle's g^o:

    ||g_i - g_i^o|| <= rtol * (||g_i^o|| + max(1e-3 ||g^o||_F / sqrt(rows), a_i))

a_i is the rounding scale of row i: the norm of the row computed with the
absolute values of its terms, divided by sqrt(N_i) for its N_i terms (FP32
rounding of a sum of N terms of that size errs by about u sqrt(N) times the
term size, u = 6e-8).  For the gradient row g_i = sum_j r_ij x_j + lam o_i,
a_i = || sum_j |r_ij| |x_j| + lam |o_i| || / sqrt(N_i).

Why a_i: when a row's exact gradient nearly cancels (a scalar gradient at
rank 1 that sums to almost zero), no FP32 evaluation order resolves it to
1e-5 of its own norm; a plain sequential FP32 sum of the same terms reaches
4e-5 and 3e-4 of the fixed floor alone on the rank-1 test cases.  A dropped
or doubled entry still errs by a whole term |r_ij| ||x_j||, about
a_i / sqrt(N_i), far above 1e-5 a_i for any N_i below 1e10
(tests/test_fp32_rounding_model.py plants both).
"""
import numpy as np


def row_error_ratio(g, go, floor=1e-3, extra=None):
    """Per-row error ||g_i - go_i|| / (||go_i|| + max(floor ||go||_F / sqrt(rows), extra_i))."""
    g = np.asarray(g, dtype=np.float64)
    go = np.asarray(go, dtype=np.float64)
    assert g.shape == go.shape, (g.shape, go.shape)
    if g.size == 0:
        return np.zeros(g.shape[0])
    d = np.linalg.norm(g - go, axis=1)
    fl = np.full(go.shape[0], floor * np.linalg.norm(go) / np.sqrt(go.shape[0]))
    if extra is not None:
        fl = np.maximum(fl, np.asarray(extra, dtype=np.float64))
    scale = np.linalg.norm(go, axis=1) + fl
    return d / np.maximum(scale, 1e-300)


def assert_rows_close(g, go, rtol=1e-5, floor=1e-3, what="gradient", extra=None):
    ratio = row_error_ratio(g, go, floor, extra)
    if ratio.size:
        worst = int(np.argmax(ratio))
        assert ratio[worst] <= rtol, f"{what}: row {worst} error ratio {ratio[worst]:.3e} > {rtol:.1e}"
    return float(ratio.max()) if ratio.size else 0.0


def grad_rounding_scales(ix, r, W, H, lam):
    """Rounding scales a_i of the gradient rows (internal orientation of the
    oracle index ix): (for gW = R H + lam W, for gH = R^T W + lam H)."""
    absR = ix.sparse(np.abs(np.asarray(r, dtype=np.float64)))
    W = np.asarray(W, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    aW = np.asarray(absR @ np.abs(H)) + abs(lam) * np.abs(W)
    aH = np.asarray(absR.T @ np.abs(W)) + abs(lam) * np.abs(H)
    dW = np.maximum(np.diff(ix.row_ptr), 1)
    dH = np.maximum(np.diff(ix.col_ptr), 1)
    return np.linalg.norm(aW, axis=1) / np.sqrt(dW), np.linalg.norm(aH, axis=1) / np.sqrt(dH)
