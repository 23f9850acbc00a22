"""The arithmetic of the tensor-core Grams' operand splitting (CPU): an FP32
value x is split into bfloat16 slices x1 = RN(x), x2 = RN(x - x1),
x3 = RN(x - x1 - x2); the product of two values is taken as the six slice
products of weight >= 2^-16 (x1 y1, x1 y2, x2 y1, x1 y3, x2 y2, x3 y1), each
an exact FP32 product of two bfloat16 values, which the tensor core sums
with FP32 accumulation.  Checked: the three slices hold x exactly (three
signed 8-bit significands cover the 24 bits of an FP32 value away from the
bottom of the exponent range), each slice product is exact in FP32, and the
six products reproduce x y within 2^-24 relative (an FP32 product's
rounding), where the three leading ones alone leave about 2^-16."""
import numpy as np

from test_bf16_gather_model import _bf16


def _slices(v):
    s1 = _bf16(v)
    r1 = (v - s1).astype(np.float32)
    s2 = _bf16(r1)
    r2 = (r1 - s2).astype(np.float32)
    return s1, s2, _bf16(r2)


def test_three_bfloat16_slices_hold_an_fp32_value_and_six_products_its_products():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200_000) * np.exp(rng.uniform(-20, 20, 200_000))).astype(np.float32)
    y = (rng.standard_normal(200_000) * np.exp(rng.uniform(-20, 20, 200_000))).astype(np.float32)
    x1, x2, x3 = _slices(x)
    y1, y2, y3 = _slices(y)
    X, Y = x.astype(np.float64), y.astype(np.float64)
    assert np.array_equal(x1.astype(np.float64) + x2 + x3, X)
    six = [(x1, y1), (x1, y2), (x2, y1), (x1, y3), (x2, y2), (x3, y1)]
    for a, b in six:
        assert np.array_equal((a * b).astype(np.float64), a.astype(np.float64) * b.astype(np.float64))
    exact = X * Y
    total = sum((a * b).astype(np.float64) for a, b in six)
    assert np.max(np.abs(total - exact) / np.abs(exact)) <= 2.0 ** -24
    lead = sum((a * b).astype(np.float64) for a, b in six[:3])
    assert np.max(np.abs(lead - exact) / np.abs(exact)) >= 2.0 ** -18
