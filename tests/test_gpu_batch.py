"""Batched BM phase (one launch per sparse pass over all solves, CUDA-graph
replay per epoch): each problem's objective and factors after the batched
epochs agree with the FP64 oracle's BM phase from the same starting factors
(FP32 gathers: objective within 1e-5; BF16 gathers: within 1e-3, the BF16
rounding of the gathered rows), and with running each solve's BM phase on
its own."""
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
        # the oracle's BM phase from the same starting factors, twice in a row
        ora = []
        for p, h in zip(probs, mates):
            ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
            W0, H0 = B.bm_get_factors(h, p.m, p.n)
            W0, H0 = W0.astype(np.float64), H0.astype(np.float64)
            Wi, Hi = (H0, W0) if ix.transposed else (W0, H0)
            st = O.State(W=Wi, H=Hi, U_prev=np.zeros((ix.m, 0)), U_prev2=None, u=None, psi=0.1,
                         rank_hist=[0, 0], prev_warm_cols=0)
            reps = []
            for _ in range(2):
                st, _ = O.bm_phase(ix, st, p.lam, 3)
                reps.append((O.objective(ix, st.W, st.H, p.lam), st.W, st.H))
            ora.append((ix, reps))
        f_tol = 1e-5 if prec == 0 else 1e-3
        bt = B.bm_batch_create(mates)
        try:
            for rep in range(2):                      # second call replays the captured graph
                F_solo = np.array([B.bm_bm_phase(h, 3) for h in solo])
                F_bat = B.bm_batch_bm_phase(bt, len(mates), 3)
                assert np.all(np.abs(F_bat - F_solo) <= 1e-5 * np.abs(F_solo)), (F_bat, F_solo)
                for p, hm, (ix, reps), Fb in zip(probs, mates, ora, F_bat):
                    Fo, Wo, Ho = reps[rep]
                    assert abs(Fb - Fo) <= f_tol * Fo, (rep, Fb, Fo)
                    Wm, Hm = B.bm_get_factors(hm, p.m, p.n)
                    Wm, Hm = (Hm, Wm) if ix.transposed else (Wm, Hm)
                    Fchk = O.objective(ix, Wm.astype(np.float64), Hm.astype(np.float64), p.lam)
                    assert abs(Fchk - Fb) <= f_tol * Fchk      # reported F is that of the factors
                    if prec == 0 and rep == 0:
                        assert np.linalg.norm(Wm - Wo) <= 1e-3 * np.linalg.norm(Wo)
                        assert np.linalg.norm(Hm - Ho) <= 1e-3 * np.linalg.norm(Ho)
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
