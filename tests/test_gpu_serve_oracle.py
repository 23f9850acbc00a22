"""Serving results checked by the FP64 oracle.

The server hands back every finished solve's factors (keep_factors = 1).  For
each request the oracle
  * re-evaluates the objective of the returned factors in FP64, which must
    equal the objective the server reported, and
  * runs Algorithm 1 to convergence on the same request; the served solution
    must reach that optimal value (FP32 solves within 1e-6 relative, batched
    BF16 solves with FP32 refinement within 1e-4).
The lambda grid {3, 5, 8} max|A| gives optimum ranks below the rank cap, so
every request has one optimal value that all modes must reach.

The single-slot batched run retires each solve and admits the next one into
a fresh batch of one: the freed handle's address is often reused by the next
bm_create, and the server must not run the old batch on the new solve.
"""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import serving_requests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _requests():
    probs, _ = serving_requests(count=6, seed=21, m_range=(300, 1200), n_range=(200, 800),
                                density_range=(0.02, 0.06), rate=None, k_max=32, lam_grid=(3.0, 5.0, 8.0))
    return probs


@pytest.fixture(scope="module")
def optima():
    out = []
    for p in _requests():
        ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
        st, info = O.solve(ix, p.lam, 8, p.k_max, O.Options(), max_outer=600, tol=1e-14)
        out.append((p, ix, info.F_hist[-1], st.W.shape[1]))
    return out


def _serve(B, probs, **kw):
    s = B.bm_server_create(keep_factors=1, **kw)
    try:
        ids = [B.bm_server_submit(s, p.m, p.n, p.rows, p.cols, p.vals, p.lam, p.k_max) for p in probs]
        B.bm_server_drain(s, 600.0)
        res = {r["id"]: r for r in B.bm_server_results(s)}
        out = []
        for i, p in zip(ids, probs):
            r = res[i]
            assert r["status"] == 0, (r, B.binding.lib().bm_server_last_error(s))
            W, H = B.bm_server_factors(s, i, p.m, p.n)
            assert W.shape == (p.m, r["k"]) and H.shape == (p.n, r["k"])
            out.append((r, W, H))
        return out
    finally:
        B.bm_server_destroy(s)


def _check(results, optima, rel_opt, rel_eval):
    for (r, W, H), (p, ix, F_star, k_star) in zip(results, optima):
        W64, H64 = W.astype(np.float64), H.astype(np.float64)
        Wi, Hi = (H64, W64) if ix.transposed else (W64, H64)
        F_chk = O.objective(ix, Wi, Hi, p.lam)           # FP64 objective of the served factors
        assert abs(F_chk - r["F"]) <= rel_eval * F_chk, (r, F_chk)
        assert F_chk >= F_star * (1 - 1e-9), (F_chk, F_star)
        assert F_chk <= F_star * (1 + rel_opt), (r, F_chk, F_star, k_star)


@pytest.mark.parametrize("slots", [1, 3])
def test_batched_fp32_serving_reaches_oracle_optimum(B, optima, slots):
    probs = [o[0] for o in optima]
    res = _serve(B, probs, max_active=slots, precision=0, batched=1, workers=2, max_outer=600, tol=1e-10)
    _check(res, optima, rel_opt=1e-6, rel_eval=1e-6)


def test_batched_bf16_serving_reaches_oracle_optimum(B, optima):
    probs = [o[0] for o in optima]
    res = _serve(B, probs, max_active=4, precision=1, batched=1, workers=2, max_outer=600, tol=1e-10)
    _check(res, optima, rel_opt=1e-4, rel_eval=1e-6)


def test_plain_fp32_serving_reaches_oracle_optimum(B, optima):
    probs = [o[0] for o in optima]
    res = _serve(B, probs, max_active=1, precision=0, batched=0, workers=1, max_outer=600, tol=1e-10)
    _check(res, optima, rel_opt=1e-6, rel_eval=1e-6)
