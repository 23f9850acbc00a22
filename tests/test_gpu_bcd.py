"""GPU parity of the column-block coordinate descent BM solver (the polyMF-SS
form of the paper's matrix completion experiments) against the FP64 oracle in
oracle/bcd_oracle.py: the objective and the factors after whole sweeps,
monotone objective, and Algorithm 1 with this BM phase reaching the oracle's
optimal value."""
import os

import numpy as np
import pytest

from oracle import bcd_oracle as C
from oracle import bm_oracle as O
from synth import named_config, random_factors

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def _internal(ix, W, H):
    W, H = W.astype(np.float64), H.astype(np.float64)
    return (H, W) if ix.transposed else (W, H)


@pytest.mark.parametrize("case,k,epochs", [("tiny", 6, 1), ("tiny", 6, 3), ("zipf_t", 9, 2), ("zipf", 33, 1)])
def test_sweeps_match_oracle(B, case, k, epochs):
    if case == "tiny":
        p = named_config("tiny")
    elif case == "zipf_t":
        p = named_config("small", m=4000, n=900, nnz=180_000, seed=12)     # stored transposed
    else:
        p = named_config("small", m=900, n=5000, nnz=200_000, seed=13)
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 40, _opts(B))
    try:
        W, H = random_factors(p.m, p.n, k, seed=4, scale=0.3)
        B.bm_set_factors(h, k, W, H)
        F = B.bm_bcd_phase(h, epochs)
        Wg, Hg = B.bm_get_factors(h, p.m, p.n)
    finally:
        B.bm_destroy(h)
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    Wi, Hi = _internal(ix, W, H)
    Wo, Ho, Fo = C.bcd_phase(ix, Wi, Hi, p.lam, epochs)
    assert abs(F - Fo[-1]) <= 1e-5 * Fo[-1]
    Wgi, Hgi = _internal(ix, Wg, Hg)
    assert abs(O.objective(ix, Wgi, Hgi, p.lam) - Fo[-1]) <= 1e-5 * Fo[-1]
    assert np.linalg.norm(Wgi - Wo) <= 1e-3 * np.linalg.norm(Wo)
    assert np.linalg.norm(Hgi - Ho) <= 1e-3 * np.linalg.norm(Ho)


def test_objective_nonincreasing_over_sweeps(B):
    p = named_config("small", m=900, n=5000, nnz=200_000, seed=13)
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 40, _opts(B))
    try:
        W, H = random_factors(p.m, p.n, 12, seed=6, scale=0.3)
        B.bm_set_factors(h, 12, W, H)
        F = [B.bm_loss_grad(h)[1]]
        for _ in range(6):
            F.append(B.bm_bcd_phase(h, 1))
        assert all(b <= a * (1 + 1e-6) for a, b in zip(F, F[1:])), F
        assert F[-1] < F[0]
    finally:
        B.bm_destroy(h)


def test_solve_with_column_blocks_reaches_the_oracle_optimum(B):
    """Algorithm 1 with the column-block BM phase on the 500 x 300 planted
    problem: the optimal value (tests/golden/tiny_optimum.txt, written by the
    oracle) does not depend on the BM solver and is reached within 1e-6."""
    F_star = None
    for line in open(os.path.join(GOLDEN, "tiny_optimum.txt")):
        if line.startswith("F_star"):
            F_star = float(line.split()[1])
    p = named_config("tiny")
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 64, _opts(B, bm_solver=1))
    try:
        r = B.bm_solve(h, max_outer=600, tol=0.0, F_target=F_star * (1 + 1e-6))
        assert r["converged"], r
        ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
        Wg, Hg = B.bm_get_factors(h, p.m, p.n)
        Wi, Hi = _internal(ix, Wg, Hg)
        F_chk = O.objective(ix, Wi, Hi, p.lam)
        assert F_star * (1 - 1e-7) <= F_chk <= F_star * (1 + 2e-6)
    finally:
        B.bm_destroy(h)
    with pytest.raises(B.BMError):
        B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 16, _opts(B, bm_solver=2))
