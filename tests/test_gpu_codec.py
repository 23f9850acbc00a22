"""The one-byte value encoding of the observed values: the library's codes
equal the oracle's definition (bm_oracle.value_codes) byte for byte in CSR
and CSC order, values that do not qualify are left in FP32, and the
loss/gradient passes give bit-identical results with and without it (a code
decodes to exactly the FP32 value)."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config, random_factors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _opts(B, **kw):
    o = B.bm_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _random_problem(m, n, nnz, vals, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(m * n, size=nnz, replace=False)
    rows, cols = np.divmod(idx, n)
    return rows.astype(np.int32), cols.astype(np.int32), vals.astype(np.float32)


@pytest.mark.parametrize("case", ["ratings", "span255", "transposed"])
def test_codes_match_oracle_bytewise(B, case):
    if case == "ratings":
        p = named_config("small", m=900, n=5000, nnz=200_000, seed=13)
        m, n, rows, cols, vals = p.m, p.n, p.rows, p.cols, p.vals
    else:
        m, n = (700, 300) if case == "transposed" else (300, 700)
        rng = np.random.default_rng(3)
        v = rng.integers(-100, 156, size=60_000)
        v[:2] = (-100, 155)
        rows, cols, vals = _random_problem(m, n, v.shape[0], v, 5)
    h = B.bm_create(m, n, rows, cols, vals, 0.5, 8)
    try:
        ix = O.build_index(m, n, rows, cols, vals.astype(np.float64))
        ref = O.value_codes(ix)
        assert ref is not None
        active, off, c_csr, c_csc = B.bm_get_codes(h, ix.nnz)
        assert active and off == ref[0]
        assert np.array_equal(c_csr, ref[1])
        assert np.array_equal(c_csc, ref[2])
    finally:
        B.bm_destroy(h)


def test_values_that_do_not_qualify_stay_fp32(B):
    m, n = 200, 300
    for v in (np.arange(0, 257), np.linspace(0.0, 4.0, 9000)):
        rows, cols, vals = _random_problem(m, n, v.shape[0], v, 7)
        h = B.bm_create(m, n, rows, cols, vals, 0.5, 8)
        try:
            ix = O.build_index(m, n, rows, cols, vals.astype(np.float64))
            assert O.value_codes(ix) is None
            assert not B.bm_get_codes(h)[0]
        finally:
            B.bm_destroy(h)
    p = named_config("small", m=900, n=5000, nnz=200_000, seed=13)
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 8, _opts(B, value_codec=0))
    try:
        assert not B.bm_get_codes(h)[0]
    finally:
        B.bm_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k", [5, 33])
def test_loss_grad_bit_identical_with_codec(B, precision, k):
    p = named_config("small", m=4000, n=900, nnz=180_000, seed=12)     # stored transposed
    W, H = random_factors(p.m, p.n, k, seed=4, scale=0.3)
    out = []
    for codec in (1, 0):
        h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 40, _opts(B, value_codec=codec, precision=precision))
        try:
            assert B.bm_get_codes(h)[0] == bool(codec)
            B.bm_set_factors(h, k, W, H)
            gW = np.empty_like(W)
            gH = np.empty_like(H)
            f, F = B.bm_loss_grad(h, gW, gH)
            Fb = B.bm_bm_phase(h, 2)
            W2, H2 = B.bm_get_factors(h, p.m, p.n)
            out.append((f, F, gW, gH, Fb, W2, H2))
        finally:
            B.bm_destroy(h)
    a, b = out
    assert a[0] == b[0] and a[1] == b[1] and a[4] == b[4]
    for x, y in zip(a[2:4] + a[5:], b[2:4] + b[5:]):
        assert np.array_equal(x, y)
