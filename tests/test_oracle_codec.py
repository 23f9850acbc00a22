"""Pins of the one-byte value encoding in the oracle (bm_oracle.value_codes):
decoding reproduces every observed value exactly in both orders; values that
are not integers, or that span more than 255, are not encoded."""
import numpy as np

from oracle import bm_oracle as O


def _ix(vals, m=30, n=40, seed=0):
    rng = np.random.default_rng(seed)
    idx = rng.choice(m * n, size=vals.shape[0], replace=False)
    rows, cols = np.divmod(idx, n)
    return O.build_index(m, n, rows, cols, vals)


def test_integer_ratings_decode_exactly_in_both_orders():
    rng = np.random.default_rng(1)
    vals = rng.integers(1, 6, size=500).astype(np.float32)
    ix = _ix(vals)
    off, c_csr, c_csc = O.value_codes(ix)
    assert off == 1.0 and c_csr.dtype == np.uint8
    assert np.array_equal(c_csr.astype(np.float64) + off, ix.val)
    assert np.array_equal(c_csc.astype(np.float64) + off, ix.cval)
    # the CSC codes are the CSR codes permuted like the values
    assert np.array_equal(c_csc, c_csr[ix.csc2csr])


def test_full_byte_span_and_negative_offset():
    vals = np.arange(-100, 156, dtype=np.float32)          # span exactly 255
    ix = _ix(vals, m=20, n=20)
    off, c_csr, _ = O.value_codes(ix)
    assert off == -100.0 and c_csr.max() == 255 and c_csr.min() == 0
    assert np.array_equal(c_csr.astype(np.float64) + off, ix.val)


def test_values_that_do_not_qualify():
    assert O.value_codes(_ix(np.arange(0, 257, dtype=np.float32), m=20, n=20)) is None   # span 256
    assert O.value_codes(_ix(np.array([1.0, 2.5, 3.0], np.float32))) is None           # not integral
    assert O.value_codes(_ix(np.array([2.0 ** 24, 2.0 ** 24 + 2], np.float64))) is None  # too large
