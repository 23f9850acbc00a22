"""The bounds of the BF16-gather precision test against a model of that mode
(CPU): every gathered factor row rounded to bfloat16 (round to nearest, ties
to even, on the FP32 bit pattern), owned rows, residuals and accumulation in
FP32, each pass recomputing the residual with its own gathered factor (the
CSR pass gathers H, the CSC pass W), rows accumulated as in
test_fp32_rounding_model.py.  On the GPU test's problem and ranks the model's
errors against the FP64 oracle are at most half of that test's bounds (loss
6e-6, gradients 3.2e-3 in Frobenius norm, 4.2e-3 row by row), and of the size
the bfloat16 rounding 2^-9 predicts."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config, random_factors
from parity import grad_rounding_scales, row_error_ratio
from test_fp32_rounding_model import _fp32_rows


def _bf16(x):
    """Nearest bfloat16 (ties to even) of each FP32 value, returned as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 3.0e38], np.float32)
    y = _bf16(x)
    assert y[0] == 1.0 and y[1] == 1.0 and y[2] == 1.0 + 2.0 ** -6
    assert y[3] == 1.0 and y[4] == -2.5
    rng = np.random.default_rng(0)
    z = rng.standard_normal(10_000).astype(np.float32)
    rel = np.abs(_bf16(z) - z) / np.abs(z)
    assert rel.max() <= 2.0 ** -8 and np.all(_bf16(z).view(np.uint32) & 0xFFFF == 0)


@pytest.mark.parametrize("k", [8, 33, 64])
def test_bf16_gather_model_within_half_the_gpu_bounds(k):
    p = named_config("small", m=3000, n=900, nnz=160_000, seed=51)
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    W, H = random_factors(p.m, p.n, k, seed=k, scale=0.4)
    Wi, Hi = (H, W) if ix.transposed else (W, H)
    Wb, Hb = _bf16(Wi), _bf16(Hi)
    ri = ix.rows_of_entries()
    r_csr = np.einsum("ek,ek->e", Wi[ri], Hb[ix.col]).astype(np.float32) - ix.val.astype(np.float32)
    f = 0.5 * float(np.sum(r_csr.astype(np.float64) ** 2))
    gW = _fp32_rows(ix.row_ptr, ix.col, Wi, Hb, r_csr, p.lam)
    cc = np.repeat(np.arange(ix.n), np.diff(ix.col_ptr))
    r_csc = np.einsum("ek,ek->e", Wb[ix.row], Hi[cc]).astype(np.float32) - ix.cval.astype(np.float32)
    gH = _fp32_rows(ix.col_ptr, ix.row, Hi, Wb, r_csc, p.lam)
    fo, _, gWo, gHo, r = O.loss_grad(ix, Wi.astype(np.float64), Hi.astype(np.float64), p.lam)
    aW, aH = grad_rounding_scales(ix, r, Wi, Hi, p.lam)
    assert abs(f - fo) <= 3e-6 * fo
    for g, go, a in ((gW, gWo, aW), (gH, gHo, aH)):
        fro = np.linalg.norm(g - go) / np.linalg.norm(go)
        assert 2.0 ** -12 <= fro <= 1.6e-3, fro
        assert row_error_ratio(g, go, extra=a).max() <= 2.1e-3
