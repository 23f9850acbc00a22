"""Batched BM phase (one launch per sparse pass over all solves, CUDA-graph
replay per epoch) agrees with running each solve's BM phase on its own."""
import numpy as np
import pytest

from synth import named_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _problems():
    return [named_config("small", m=3000, n=800, nnz=120_000, seed=61),
            named_config("small", m=900, n=5000, nnz=150_000, seed=62),
            named_config("small", m=20_000, n=2_500, nnz=400_000, seed=63),
            named_config("tiny")]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_bm_phase_matches_individual(B, prec):
    probs = _problems()
    o = B.bm_default_options()
    o.precision = prec
    solo, mates = [], []
    try:
        for p in probs:
            for lst in (solo, mates):
                h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 24, o)
                lst.append(h)
                B.bm_init(h)
        ks = [B.bm_dims(h)["k"] for h in solo]
        assert ks == [B.bm_dims(h)["k"] for h in mates] and min(ks) >= 1
        bt = B.bm_batch_create(mates)
        try:
            for rep in range(2):                      # second call replays the captured graph
                F_solo = np.array([B.bm_bm_phase(h, 3) for h in solo])
                F_bat = B.bm_batch_bm_phase(bt, len(mates), 3)
                assert np.all(np.abs(F_bat - F_solo) <= 1e-5 * np.abs(F_solo)), (F_bat, F_solo)
            for p, hs, hm in zip(probs, solo, mates):
                Ws, Hs = B.bm_get_factors(hs, p.m, p.n)
                Wm, Hm = B.bm_get_factors(hm, p.m, p.n)
                assert np.linalg.norm(Wm - Ws) <= 1e-3 * np.linalg.norm(Ws)
                assert np.linalg.norm(Hm - Hs) <= 1e-3 * np.linalg.norm(Hs)
                fs, _ = B.bm_loss_grad(hs)
                fm, _ = B.bm_loss_grad(hm)
                assert abs(fm - fs) <= 1e-5 * fs
        finally:
            B.bm_batch_destroy(bt)
    finally:
        for h in solo + mates:
            B.bm_destroy(h)


def test_batch_rejects_bad_sets(B):
    p = named_config("tiny")
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 8)
    try:
        with pytest.raises(B.BMError, match="twice"):
            B.bm_batch_create([h, h])
        bt = B.bm_batch_create([h])
        try:
            with pytest.raises(B.BMError, match="rank"):
                B.bm_batch_bm_phase(bt, 1, 1)           # k = 0 before bm_init
        finally:
            B.bm_batch_destroy(bt)
    finally:
        B.bm_destroy(h)
