"""Panel-ordered work splits of the sparse passes (bm_set_panels, bm_autotune).

Panels reorder the segments of a pass (and cut rows at panel boundaries);
per-row partial sums are still combined in entry order.  Every panel count
must therefore give the oracle's loss, gradients, BM phase and PG step within
the usual FP32 tolerances, and a fixed panel count must be deterministic.
"""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config, random_factors
from tests.parity import assert_rows_close, grad_rounding_scales

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


@pytest.fixture(scope="module")
def prob():
    # m > n (stored transposed) with heavy rows: several segments per row
    return named_config("small", m=20_000, n=2_500, nnz=400_000, seed=61)


def _oracle_grad(p, W, H):
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    Wi, Hi = (H, W) if ix.transposed else (W, H)
    f, F, gW, gH, r = O.loss_grad(ix, Wi.astype(np.float64), Hi.astype(np.float64), p.lam)
    aW, aH = grad_rounding_scales(ix, r, Wi, Hi, p.lam)
    if ix.transposed:
        gW, gH, aW, aH = gH, gW, aH, aW
    return ix, f, F, gW, gH, aW, aH


@pytest.mark.parametrize("panels", [[1, 1, 1, 1, 1], [2, 3, 4, 5, 6], [16, 16, 16, 16, 16], [7, 1, 3, 1, 9]])
def test_loss_grad_any_panels(B, prob, panels):
    p = prob
    k = 33
    W, H = random_factors(p.m, p.n, k, seed=3, scale=0.3)
    _, f_o, F_o, gW_o, gH_o, aW, aH = _oracle_grad(p, W, H)
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 64)
    try:
        B.bm_set_panels(h, panels)
        assert B.bm_get_panels(h) == panels
        B.bm_set_factors(h, k, W, H)
        gW, gH = np.empty_like(W), np.empty_like(H)
        f, F = B.bm_loss_grad(h, gW, gH)
        assert abs(f - f_o) <= RTOL * f_o and abs(F - F_o) <= RTOL * F_o
        assert np.linalg.norm(gW - gW_o) <= RTOL * np.linalg.norm(gW_o)
        assert np.linalg.norm(gH - gH_o) <= RTOL * np.linalg.norm(gH_o)
        assert_rows_close(gW, gW_o, RTOL, what="gW", extra=aW)
        assert_rows_close(gH, gH_o, RTOL, what="gH", extra=aH)
        # a fixed split is deterministic
        gW2, gH2 = np.empty_like(W), np.empty_like(H)
        f2, _ = B.bm_loss_grad(h, gW2, gH2)
        assert f2 == f and np.array_equal(gW2, gW) and np.array_equal(gH2, gH)
    finally:
        B.bm_destroy(h)


def test_bm_phase_and_prox_with_panels_match_natural_split(B, prob):
    p = prob
    k = 8
    W, H = random_factors(p.m, p.n, k, seed=4, scale=0.3)
    out = []
    for panels in ([1, 1, 1, 1, 1], [4, 2, 6, 3, 5]):
        o = B.bm_default_options()
        o.lmsvd_tol = 0.0
        o.lmsvd_imax = 6
        h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32, o)
        try:
            B.bm_set_panels(h, panels)
            B.bm_set_factors(h, k, W, H)
            Fb = B.bm_bm_phase(h, 3)
            info = B.bm_prox_step(h)
            out.append((Fb, info["F"], info["k_new"]))
        finally:
            B.bm_destroy(h)
    (Fb1, Fp1, k1), (Fb2, Fp2, k2) = out
    assert abs(Fb1 - Fb2) <= 1e-5 * Fb1
    assert k1 == k2
    assert abs(Fp1 - Fp2) <= 1e-5 * Fp1


def test_empty_rows_and_columns_with_panels(B):
    # rows and columns without entries, a matrix narrower than the panel count
    rng = np.random.default_rng(5)
    m, n = 40, 9
    rows = rng.integers(0, m // 2, 120).astype(np.int32)
    cols = rng.integers(0, n, 120).astype(np.int32)
    key = np.unique(rows.astype(np.int64) * n + cols)
    rows, cols = (key // n).astype(np.int32), (key % n).astype(np.int32)
    vals = rng.standard_normal(len(rows)).astype(np.float32)
    W, H = random_factors(m, n, 3, seed=6)
    ix = O.build_index(m, n, rows, cols, vals.astype(np.float64))
    Wi, Hi = (H, W) if ix.transposed else (W, H)
    f_o, _, gW_o, gH_o, _ = O.loss_grad(ix, Wi.astype(np.float64), Hi.astype(np.float64), 0.3)
    if ix.transposed:
        gW_o, gH_o = gH_o, gW_o
    h = B.bm_create(m, n, rows, cols, vals, 0.3, 4)
    try:
        B.bm_set_panels(h, [16] * 5)
        B.bm_set_factors(h, 3, W, H)
        gW, gH = np.empty_like(W), np.empty_like(H)
        f, _ = B.bm_loss_grad(h, gW, gH)
        assert abs(f - f_o) <= RTOL * f_o
        assert np.allclose(gW, gW_o, rtol=1e-5, atol=1e-6) and np.allclose(gH, gH_o, rtol=1e-5, atol=1e-6)
    finally:
        B.bm_destroy(h)


def test_set_panels_rejects_bad_counts(B, prob):
    p = prob
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 8)
    try:
        for bad in ([0, 1, 1, 1, 1], [1, 1, 1, 1, B.binding.BM_MAX_PANELS + 1]):
            with pytest.raises(B.BMError):
                B.bm_set_panels(h, bad)
        with pytest.raises(B.BMError):
            B.bm_autotune(h)          # no factors yet
    finally:
        B.bm_destroy(h)


def test_autotune_keeps_results(B, prob):
    p = prob
    o = B.bm_default_options()
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 16, o)
    try:
        B.bm_init(h)
        res = B.bm_autotune(h)
        assert set(res) == set(B.binding.PASS_NAMES)
        for nm, (P, ms, ms1, lay) in res.items():
            assert 1 <= P <= B.binding.BM_MAX_PANELS and ms > 0 and ms1 > 0 and lay in (0, 1)
            assert ms <= ms1 or (P == 1 and lay == B.bm_get_layout(h)[B.binding.PASS_NAMES.index(nm)])
        assert B.bm_get_panels(h) == [res[nm][0] for nm in B.binding.PASS_NAMES]
        assert B.bm_get_layout(h) == [res[nm][3] for nm in B.binding.PASS_NAMES]
        r = B.bm_solve(h, max_outer=5, tol=0.0)
        assert np.isfinite(r["F"])
    finally:
        B.bm_destroy(h)
