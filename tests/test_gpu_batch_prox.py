"""Batched PG step (bm_batch_prox_step): every handle's PG step (Eq.
"inexactpg", Algorithm 2) runs on its own host thread and stream, and the
q-wide residual SpMMs of Eq. "ZZ" run as shared launches over the handles'
concatenated segment lists.  Checked over three cycles on problems of
different shapes (one stored transposed) and ranks: each handle's factors
and step results are bit for bit those of bm_prox_step run on its own, the
launches were shared (fewer launches than products), and every reported
objective agrees with the FP64 oracle's evaluation of the returned factors
(Eq. "mf" plus lambda ||X||_* through the balanced factors: FP32 factors,
1e-5)."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from synth import named_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _problems():
    return [named_config("small", m=3000, n=800, nnz=120_000, seed=71),
            named_config("small", m=900, n=5000, nnz=150_000, seed=72),
            named_config("small", m=12_000, n=2_500, nnz=300_000, seed=73),
            named_config("tiny")]


def test_batch_prox_step_matches_individual_and_oracle(B):
    probs = _problems()
    solo, mates = [], []
    try:
        for p in probs:
            for lst in (solo, mates):
                h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 24)
                lst.append(h)
                B.bm_init(h)
        ixs = [O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64)) for p in probs]
        bt = B.bm_batch_create(mates)
        try:
            for cycle in range(3):
                for hs, hm in zip(solo, mates):             # the same BM phase on both sides
                    Fs = B.bm_bm_phase(hs, 3)
                    Fm = B.bm_bm_phase(hm, 3)
                    assert Fs == Fm
                infos = B.bm_batch_prox_step(bt, len(mates))
                for p, ix, hs, hm, im in zip(probs, ixs, solo, mates, infos):
                    i_s = B.bm_prox_step(hs)
                    assert im == i_s, (cycle, im, i_s)
                    Ws, Hs = B.bm_get_factors(hs, p.m, p.n)
                    Wm, Hm = B.bm_get_factors(hm, p.m, p.n)
                    assert np.array_equal(Ws, Wm) and np.array_equal(Hs, Hm), cycle
                    Wi, Hi = (Hm, Wm) if ix.transposed else (Wm, Hm)
                    Fo = O.objective(ix, Wi.astype(np.float64), Hi.astype(np.float64), p.lam)
                    assert abs(im["F"] - Fo) <= 1e-5 * Fo, (cycle, im["F"], Fo)
            products, launches = B.bm_batch_stats(bt)
            assert products > launches >= 1, (products, launches)
        finally:
            B.bm_batch_destroy(bt)
    finally:
        for h in solo + mates:
            B.bm_destroy(h)


def test_batch_prox_step_single_handle_and_rank_zero(B):
    """A batch of one, and a handle at rank 0 (its PG step starts from X = 0)
    beside one of positive rank."""
    p = named_config("tiny")
    q = named_config("small", m=2000, n=600, nnz=60_000, seed=74)
    h0 = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 16)
    h1 = B.bm_create(q.m, q.n, q.rows, q.cols, q.vals, q.lam, 16)
    r0 = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 16)
    r1 = B.bm_create(q.m, q.n, q.rows, q.cols, q.vals, q.lam, 16)
    try:
        B.bm_init(h1)
        B.bm_init(r1)
        bt = B.bm_batch_create([h0, h1])
        try:
            infos = B.bm_batch_prox_step(bt, 2)
            assert infos[0] == B.bm_prox_step(r0) and infos[1] == B.bm_prox_step(r1)
        finally:
            B.bm_batch_destroy(bt)
        one = B.bm_batch_create([h1])
        try:
            i1 = B.bm_batch_prox_step(one, 1)[0]
            assert i1 == B.bm_prox_step(r1)
        finally:
            B.bm_batch_destroy(one)
        for a, b, pp in ((h0, r0, p), (h1, r1, q)):
            Wa, Ha = B.bm_get_factors(a, pp.m, pp.n)
            Wb, Hb = B.bm_get_factors(b, pp.m, pp.n)
            assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    finally:
        for h in (h0, h1, r0, r1):
            B.bm_destroy(h)
