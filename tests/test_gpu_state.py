"""Checkpoint / resume (bm_get_state, bm_set_state): a solve resumed in a new
handle takes the same steps as the uninterrupted one (same kernels in the same
order: identical bits), and damaged or foreign states are rejected."""
import numpy as np
import pytest

from synth import named_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


@pytest.mark.parametrize("name,kw", [("tiny", {}), ("small", dict(m=3000, n=800, nnz=120_000, seed=71))])
def test_resume_equals_uninterrupted(B, name, kw):
    p = named_config(name, **kw)
    a = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32)
    b = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32)
    try:
        B.bm_solve(a, max_outer=4, tol=0.0)
        state = B.bm_get_state(a)
        B.bm_set_state(b, state)
        ra = B.bm_solve(a, max_outer=5, tol=0.0)
        rb = B.bm_solve(b, max_outer=5, tol=0.0)
        assert ra["k"] == rb["k"] and ra["F"] == rb["F"]
        Wa, Ha = B.bm_get_factors(a, p.m, p.n)
        Wb, Hb = B.bm_get_factors(b, p.m, p.n)
        assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
        assert B.bm_get_state(a) == B.bm_get_state(b)
    finally:
        B.bm_destroy(a)
        B.bm_destroy(b)


def test_state_rejects_damaged_or_foreign(B):
    p = named_config("tiny")
    q = named_config("small", m=600, n=400, nnz=20_000, seed=72)
    a = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32)
    c = B.bm_create(q.m, q.n, q.rows, q.cols, q.vals, q.lam, 32)
    try:
        B.bm_solve(a, max_outer=2, tol=0.0)
        st = B.bm_get_state(a)
        for bad in (st[:-4], b"XXXXXXXX" + st[8:], st + b"\\0"):
            with pytest.raises(B.BMError):
                B.bm_set_state(a, bad)
        with pytest.raises(B.BMError):
            B.bm_set_state(c, st)
        B.bm_set_state(a, st)      # the handle stays usable
        assert np.isfinite(B.bm_solve(a, max_outer=1, tol=0.0)["F"])
    finally:
        B.bm_destroy(a)
        B.bm_destroy(c)


def test_state_through_caller_buffers(B):
    """The state written into a caller's (pinned) buffer equals the bytes form
    and restores the same solve as the bytes form does."""
    torch = pytest.importorskip("torch")
    p = named_config("small", m=3000, n=800, nnz=120_000, seed=73)
    a = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32)
    b = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 32)
    try:
        B.bm_solve(a, max_outer=3, tol=0.0)
        ref = B.bm_get_state(a)
        buf = torch.zeros(B.bm_state_size(a) + 4096, dtype=torch.uint8).pin_memory()
        n = B.bm_get_state(a, buf)
        assert n == len(ref) and bytes(buf[:n].numpy().tobytes()) == ref
        with pytest.raises(B.BMError):
            B.bm_get_state(a, np.zeros(n - 1, np.uint8))      # too small
        B.bm_set_state(b, buf, n)
        ra = B.bm_solve(a, max_outer=2, tol=0.0)
        rb = B.bm_solve(b, max_outer=2, tol=0.0)
        assert ra["F"] == rb["F"] and ra["k"] == rb["k"]
    finally:
        B.bm_destroy(a)
        B.bm_destroy(b)
