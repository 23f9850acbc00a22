"""Continuous-batching server: every request completes; each result is the
same alone and in the mix; the batched BF16 server reaches the one-at-a-time
FP32 server's objectives within 1e-4 relative."""
import time

import numpy as np
import pytest

from synth import serving_requests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _requests(count=10, seed=9):
    # lambda in {3, 5, 8} max|A|: optimum ranks 3..29 under the cap of 32, so
    # every request has a unique optimal objective that both modes must reach
    return serving_requests(count=count, seed=seed, m_range=(500, 6000), n_range=(300, 3000),
                            density_range=(0.005, 0.03), rate=200.0, k_max=32, lam_grid=(3.0, 5.0, 8.0))


def _serve(B, probs, arrivals, **kw):
    s = B.bm_server_create(**kw)
    try:
        t0 = time.perf_counter()
        ids = []
        for p, t in zip(probs, arrivals):
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(B.bm_server_submit(s, p.m, p.n, p.rows, p.cols, p.vals, p.lam, p.k_max))
        B.bm_server_drain(s, 600.0)
        res = {r["id"]: r for r in B.bm_server_results(s)}
        out = [res[i] for i in ids]
        assert all(r["status"] == 0 for r in out), (out, B.binding.lib().bm_server_last_error(s))
        return out
    finally:
        B.bm_server_destroy(s)


def test_server_alone_equals_mix_and_modes_agree(B):
    probs, arrivals = _requests()
    mix = _serve(B, probs, arrivals, max_active=8, precision=0, batched=1, workers=4, max_outer=40, tol=1e-7)
    assert all(r["status"] == 0 for r in mix)
    assert all(r["t_done"] >= r["t_start"] >= r["t_submit"] for r in mix)
    # each request alone through the same batched path (a batch of one)
    for p, r in list(zip(probs, mix))[:4]:
        alone = _serve(B, [p], [0.0], max_active=1, precision=0, batched=1, workers=1, max_outer=40, tol=1e-7)[0]
        assert alone["k"] == r["k"] and alone["outer"] == r["outer"]
        assert abs(alone["F"] - r["F"]) <= 1e-6 * abs(r["F"])
    # batched BF16 with FP32 refinement vs one-at-a-time FP32 solves, same requests
    plain = _serve(B, probs, np.zeros(len(probs)), max_active=1, precision=0, batched=0, workers=1,
                   max_outer=400, tol=1e-8)
    bf = _serve(B, probs, np.zeros(len(probs)), max_active=8, precision=1, batched=1, workers=4,
                max_outer=400, tol=1e-8)
    for a, b in zip(plain, bf):
        assert a["status"] == 0 and b["status"] == 0
        assert a["k"] < 32 and b["k"] < 32
        assert abs(a["F"] - b["F"]) <= 1e-4 * abs(a["F"]), (a, b)
