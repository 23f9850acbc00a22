"""BF16-gather precision mode (bm_options.precision = 1).

The gathered factor rows are read as bfloat16 (8-bit mantissa); owned rows,
accumulation and the residual stay FP32.  Errors against FP64 measured at the
recommendation-scale sizes (480,189 x 17,770 at k = 64 and 1,000,990 x
624,961 at k = 127): loss 6e-9 and 3e-8 relative, gradient rows at most
2.3e-3 relative (median 1.6e-3, the bfloat16 rounding 2^-9 of the gathered
rows).  On this test's smaller problem (160,000 entries, errors average
over fewer terms) a bfloat16 model of the gathers (tests/test_bf16_gather_model.py)
gives at most: loss 2.8e-6, gradient 1.6e-3 (Frobenius), per-row ratio 2.1e-3
with the rounding-scale floor of tests/parity.py.  The bounds below are twice those
figures.  A solve in this mode refines its
final iterations in FP32 and must reach the plain FP32 solve's objective
within 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config, random_factors
from tests.parity import assert_rows_close, grad_rounding_scales

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _opts(B, prec):
    o = B.bm_default_options()
    o.precision = prec
    return o


@pytest.mark.parametrize("k", [8, 33, 64])
def test_bf16_loss_grad_error_bounds(B, k):
    p = named_config("small", m=3000, n=900, nnz=160_000, seed=51)
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 64, _opts(B, 1))
    try:
        W, H = random_factors(p.m, p.n, k, seed=k, scale=0.4)
        B.bm_set_factors(h, k, W, H)
        gW, gH = np.empty_like(W), np.empty_like(H)
        f, F = B.bm_loss_grad(h, gW, gH)
        ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
        Wi, Hi = (H, W) if ix.transposed else (W, H)
        fo, Fo, gWo, gHo, r = O.loss_grad(ix, Wi.astype(np.float64), Hi.astype(np.float64), p.lam)
        aW, aH = grad_rounding_scales(ix, r, Wi, Hi, p.lam)
        if ix.transposed:
            gWo, gHo, aW, aH = gHo, gWo, aH, aW
        # bfloat16 rounding of the gathered rows (relative 2^-9) enters every dot product
        assert abs(f - fo) <= 6e-6 * fo
        assert np.linalg.norm(gW - gWo) <= 3.2e-3 * np.linalg.norm(gWo)
        assert np.linalg.norm(gH - gHo) <= 3.2e-3 * np.linalg.norm(gHo)
        assert_rows_close(gW, gWo, 4.2e-3, what="gW (bf16 gathers)", extra=aW)
        assert_rows_close(gH, gHo, 4.2e-3, what="gH (bf16 gathers)", extra=aH)
    finally:
        B.bm_destroy(h)


def test_bf16_solve_matches_fp32_solve(B):
    # lambda = 6 max|A| = 30: the optimum has rank 16 under the cap of 32, so
    # both precisions converge to the same (unique) objective value
    p = named_config("small", m=4000, n=1000, nnz=200_000, seed=52, k_max=32, lam_frac=6.0)
    Fs = []
    for prec in (0, 1):
        h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32, _opts(B, prec))
        try:
            r = B.bm_solve(h, max_outer=300, tol=1e-8)
            assert r["k"] < 32, r
            Wg, Hg = B.bm_get_factors(h, p.m, p.n)
            ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
            Wi, Hi = (Hg, Wg) if ix.transposed else (Wg, Hg)
            Fs.append(O.objective(ix, Wi.astype(np.float64), Hi.astype(np.float64), p.lam))
        finally:
            B.bm_destroy(h)
    assert abs(Fs[1] - Fs[0]) <= 1e-4 * Fs[0], Fs
