"""GPU parity of the distance-geometry loss/gradient (Eq. "EDM") against the FP64 oracle."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import self_avoiding_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


@pytest.mark.parametrize("n,k,weighted", [(3000, 3, False), (3000, 16, True), (5000, 7, True), (800, 33, False),
                                          (30_000, 16, False)])   # the last: the 30,000-point chain itself
def test_edm_parity(B, n, k, weighted):
    p = self_avoiding_chain(n=n, seed=n + k)
    rng = np.random.default_rng(k)
    V = (p.X_true @ rng.standard_normal((3, k)) * 0.3 + 0.05 * rng.standard_normal((n, k))).astype(np.float32)
    w = rng.uniform(0.5, 2.0, p.npairs).astype(np.float32) if weighted else None
    lam = O.edm_lambda(n, p.d)
    perm = rng.permutation(p.npairs)             # pairs in no particular order, some reversed
    i, j = p.i[perm].copy(), p.j[perm].copy()
    flip = rng.random(p.npairs) < 0.5
    i[flip], j[flip] = j[flip], i[flip]
    d = p.d[perm]
    wp = w[perm] if weighted else None
    h = B.bm_edm_create(n, i, j, d, lam, 64 if k <= 64 else 128, w=wp)
    try:
        B.bm_edm_set_factor(h, k, V)
        gV = np.empty_like(V)
        g = B.bm_edm_loss_grad(h, gV)
        go, grad, _ = O.edm_loss_grad(V.astype(np.float64), p.i, p.j, p.d, w if weighted else 1.0, lam)
        assert abs(g - go) <= 1e-5 * abs(go)
        assert np.linalg.norm(gV - grad) <= 1e-5 * np.linalg.norm(grad)
    finally:
        B.bm_edm_destroy(h)


def test_edm_rejects_bad_pairs(B):
    i = np.array([0, 1], np.int32)
    j = np.array([1, 0], np.int32)
    d = np.array([1.0, 1.0], np.float32)
    with pytest.raises(B.BMError, match="twice"):
        B.bm_edm_create(3, i, j, d, -0.1, 2)
    with pytest.raises(B.BMError, match="range"):
        B.bm_edm_create(3, np.array([0, 2], np.int32), np.array([0, 1], np.int32), d, -0.1, 2)
