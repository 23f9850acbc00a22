"""The continuous-batching server under many concurrent PG-step workers: 24
requests submitted at once, 16 active solves, 8 host threads driving
different handles.  Every request must complete without error (kernel
attributes shared between host threads are set once, so concurrent launches
of one kernel cannot invalidate each other)."""
import pytest

from synth import serving_requests

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


@pytest.mark.parametrize("precision", [0, 1])
def test_many_workers_complete_every_request(B, precision):
    probs, _ = serving_requests(count=24, seed=4, max_nnz=300_000, k_max=32)
    s = B.bm_server_create(max_active=16, precision=precision, batched=1, workers=8, max_outer=30, tol=1e-6)
    ids = [B.bm_server_submit(s, q.m, q.n, q.rows, q.cols, q.vals, q.lam, q.k_max) for q in probs]
    # bounded wait: a stalled server fails the test instead of hanging it
    B.bm_server_drain(s, 300.0)
    res = {r["id"]: r for r in B.bm_server_results(s)}
    err = B.binding.lib().bm_server_last_error(s)
    B.bm_server_destroy(s)
    assert sorted(res) == sorted(ids)
    assert all(res[i]["status"] == 0 for i in ids), (res, err)
    assert all(res[i]["t_done"] >= res[i]["t_start"] >= res[i]["t_submit"] for i in ids)
