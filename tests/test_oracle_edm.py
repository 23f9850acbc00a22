"""Pins of the distance-geometry loss of Eq. "EDM" in the oracle: the dense
evaluation through X = V V^T and <E_ij, X> = X_ii + X_jj - 2 X_ij, central
finite differences, and the symmetric Laplacian form of the gradient."""
import math

import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import self_avoiding_chain


def _case(n=300, k=5, seed=0):
    p = self_avoiding_chain(n=n, seed=seed)
    rng = np.random.default_rng(seed)
    V = p.X_true[:, :3] @ rng.standard_normal((3, k)) * 0.3 + 0.05 * rng.standard_normal((n, k))
    w = rng.uniform(0.5, 2.0, p.npairs)
    return p, V, w


def test_edm_dense_evaluation():
    p, V, w = _case()
    lam = -0.7
    g, grad, r = O.edm_loss_grad(V, p.i, p.j, p.d, w, lam)
    X = V @ V.T
    ii, jj = p.i.astype(int), p.j.astype(int)
    inner = X[ii, ii] + X[jj, jj] - 2 * X[ii, jj]
    g_dense = 0.5 * np.sum(w * (inner - p.d.astype(np.float64) ** 2) ** 2) + lam * np.trace(X)
    assert math.isclose(g, g_dense, rel_tol=1e-12)
    # gradient = 2 (sum w r E_ij + lam I) V with E_ij formed densely
    G = np.zeros((p.n, p.n))
    for a, b, c in zip(ii, jj, w * r):
        G[a, a] += c
        G[b, b] += c
        G[a, b] -= c
        G[b, a] -= c
    assert np.allclose(grad, 2 * (G + lam * np.eye(p.n)) @ V, rtol=1e-11, atol=1e-11)


def test_edm_finite_differences():
    p, V, w = _case(n=200, k=4, seed=1)
    lam = O.edm_lambda(p.n, p.d)
    g, grad, _ = O.edm_loss_grad(V, p.i, p.j, p.d, w, lam)
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(25):
        a, c = rng.integers(p.n), rng.integers(V.shape[1])
        Vp, Vm = V.copy(), V.copy()
        Vp[a, c] += h
        Vm[a, c] -= h
        fd = (O.edm_loss_grad(Vp, p.i, p.j, p.d, w, lam)[0] - O.edm_loss_grad(Vm, p.i, p.j, p.d, w, lam)[0]) / (2 * h)
        # truncation O(h^2) plus rounding of g(V +- h e) divided by 2h
        bound = 1e-7 * max(1.0, abs(grad[a, c])) + 8 * np.finfo(float).eps * abs(g) / (2 * h)
        assert abs(fd - grad[a, c]) <= bound


def test_chain_generator_geometry():
    p = self_avoiding_chain(n=500, seed=4)
    bonds = np.linalg.norm(np.diff(p.X_true, axis=0), axis=1)
    assert np.allclose(bonds, 1.0)
    D = np.linalg.norm(p.X_true[:, None] - p.X_true[None], axis=2)
    iu = np.triu_indices(p.n, 2)
    assert D[iu].min() >= 1.0 - 1e-9                          # non-bonded exclusion
    within = np.argwhere(np.triu(D <= 6.0, 1))
    assert within.shape[0] == p.npairs                          # Omega = all pairs within the cutoff
    dt = D[p.i, p.j]
    assert np.all(np.abs(p.d / dt - 1.0) <= 0.1 + 1e-6)


def test_lambda_of_the_molecular_conformation_setting():
    """Supplement, molecular conformation: lambda = -10 sqrt(n) / sum d_ij^2;
    for n = 4 and d = (1, 2, 2), -10 * 2 / 9."""
    assert O.edm_lambda(4, np.array([1.0, 2.0, 2.0])) == pytest.approx(-20.0 / 9.0, rel=1e-15)
