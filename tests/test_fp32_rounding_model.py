"""The per-row gradient tolerance against a model of the kernel's FP32
arithmetic (CPU): the residual of every entry as an FP32 dot product, each
gradient row accumulated in FP32 one entry after another in segments of at
most 1,024 entries, the segments' partial sums added in entry order, then
lam times the own row, on the shapes, seeds and ranks of the GPU parity
test (Eq. "mf": g_W = R H + lam W, g_H = R^T W + lam H).

It shows what the criterion of tests/parity.py rests on: such an FP32
evaluation stays far inside ||g_i - g_i^o|| <= 1e-5 (||g_i^o|| +
max(1e-3 ||g^o||_F / sqrt(rows), a_i)), while without the rounding scale a_i
of each row the rank-1 rows, whose sums nearly cancel, would not (no FP32
summation order resolves them to 1e-5 of their own norm)."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config, random_factors
from parity import grad_rounding_scales, row_error_ratio

SEG = 1024


def _fp32_rows(ptr, other_idx, own, other, r32, lam):
    """FP32 g_i = sum_e r_e other[other_idx[e]] + lam own_i, entries of row i in
    order, in segments of at most SEG entries whose sums are added in order."""
    rows = own.shape[0]
    deg = np.diff(ptr)
    row_of = np.repeat(np.arange(rows), deg)
    pos = np.arange(ptr[-1]) - np.repeat(ptr[:-1], deg)
    seg_in_row = pos // SEG
    nseg_row = (deg + SEG - 1) // SEG
    seg_base = np.concatenate([[0], np.cumsum(nseg_row)[:-1]])
    seg = seg_base[row_of] + seg_in_row
    part = np.zeros((int(nseg_row.sum()), own.shape[1]), np.float32)
    np.add.at(part, seg, r32[:, None] * other[other_idx])       # sequential, in entry order
    g = np.zeros_like(own)
    seg_row = np.repeat(np.arange(rows), nseg_row)
    np.add.at(g, seg_row, part)                                 # segments in order
    return g + np.float32(lam) * own


@pytest.mark.parametrize("k", [1, 8, 64])
@pytest.mark.parametrize("shape", [(3000, 700, 150_000), (20_000, 2_500, 400_000)])
def test_fp32_order_meets_the_per_row_criterion(shape, k):
    m, n, nnz = shape
    p = named_config("small", m=m, n=n, nnz=nnz, seed=7, k_max=127)
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    W, H = random_factors(p.m, p.n, k, seed=k, scale=0.4)
    Wi, Hi = (H, W) if ix.transposed else (W, H)
    lam = p.lam
    # FP32 residual in CSR order, and its CSC-order copy
    ri = ix.rows_of_entries()
    r32 = (np.einsum("ek,ek->e", Wi[ri], Hi[ix.col]).astype(np.float32)
           - ix.val.astype(np.float32))
    gW = _fp32_rows(ix.row_ptr, ix.col, Wi, Hi, r32, lam)
    gH = _fp32_rows(ix.col_ptr, ix.row, Hi, Wi, r32[ix.csc2csr], lam)
    W64, H64 = Wi.astype(np.float64), Hi.astype(np.float64)
    _, _, gWo, gHo, r = O.loss_grad(ix, W64, H64, lam)
    aW, aH = grad_rounding_scales(ix, r, W64, H64, lam)
    worst = max(row_error_ratio(gW, gWo, extra=aW).max(), row_error_ratio(gH, gHo, extra=aH).max())
    assert worst <= 2.5e-6, worst
    if k == 1:
        bare = max(row_error_ratio(gW, gWo).max(), row_error_ratio(gH, gHo).max())
        assert bare > 1e-5, bare


@pytest.mark.parametrize("k", [1, 64])
def test_criterion_catches_a_dropped_or_doubled_entry(k):
    """One entry dropped from (or counted twice in) a row changes the row by
    a whole term |r_e| ||x_j||, about a_i / sqrt(N_i) for a row of N_i terms:
    far above 1e-5 a_i for any N_i below 1e10, so the criterion flags it, on
    the FP32 model's rows, long and short."""
    p = named_config("small", m=20_000, n=2_500, nnz=400_000, seed=7, k_max=127)
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    W, H = random_factors(p.m, p.n, k, seed=k, scale=0.4)
    Wi, Hi = (H, W) if ix.transposed else (W, H)
    ri = ix.rows_of_entries()
    r32 = (np.einsum("ek,ek->e", Wi[ri], Hi[ix.col]).astype(np.float32)
           - ix.val.astype(np.float32))
    gW = _fp32_rows(ix.row_ptr, ix.col, Wi, Hi, r32, p.lam)
    W64, H64 = Wi.astype(np.float64), Hi.astype(np.float64)
    _, _, gWo, _, r = O.loss_grad(ix, W64, H64, p.lam)
    aW, _ = grad_rounding_scales(ix, r, W64, H64, p.lam)
    deg = np.diff(ix.row_ptr)
    rng = np.random.default_rng(k)
    picks = [int(np.argmax(deg)), int(np.argmin(deg))] + list(rng.choice(ix.m, 30, replace=False))
    for i in picks:
        e = int(ix.row_ptr[i] + rng.integers(deg[i]))
        term = r32[e] * Hi[ix.col[e]]
        if not np.any(term):
            continue
        for sign in (-1.0, 1.0):                     # dropped, doubled
            g = gW.copy()
            g[i] += np.float32(sign) * term
            assert row_error_ratio(g, gWo, extra=aW)[i] > 1e-5, (i, deg[i], sign)
