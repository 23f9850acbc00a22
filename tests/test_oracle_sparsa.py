"""Pins of the SpaRSA-step oracle (oracle/sparsa_oracle.py) against dense
evaluations and closed forms: Eq. "trace" and the nuclear norm against the
dense matrices, <dX, dG> against the dense gradient difference, alpha_BB = 1
with full observation, Eq. "back" / Eq. "decrease" re-evaluated densely for
every step (with the flag naming the test that held, and the trial one
reduction earlier failing both), Eq. "proxBB" from the two points where the
PG steps were taken, no backtracking when alpha_max <= 1/L, and the SpaRSA
solve reaching the dense soft-impute optimum."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from oracle import sparsa_oracle as S
from synth import planted_uniform


def _small(m=40, n=60, frac=0.3, rank=3, seed=11, lam=0.5):
    p = planted_uniform(m=m, n=n, rank=rank, frac=frac, noise_sd=0.1, lam=lam, seed=seed)
    return p, O.build_index(p.m, p.n, p.rows, p.cols, p.vals)


def _dense(ix):
    M = np.zeros((ix.m, ix.n))
    mask = np.zeros((ix.m, ix.n), dtype=bool)
    ri = ix.rows_of_entries()
    M[ri, ix.col] = ix.val
    mask[ri, ix.col] = True
    return M, mask


def test_trace_formula_and_nuclear_norm_match_dense():
    rng = np.random.default_rng(0)
    for k1, k0 in ((3, 5), (6, 1), (4, 4)):
        W1, H1 = rng.standard_normal((13, k1)), rng.standard_normal((21, k1))
        W0, H0 = rng.standard_normal((13, k0)), rng.standard_normal((21, k0))
        D = W1 @ H1.T - W0 @ H0.T
        assert abs(S.frob_diff2(W1, H1, W0, H0) - np.sum(D * D)) <= 1e-10 * np.sum(D * D)
        s = np.linalg.svd(W1 @ H1.T, compute_uv=False)
        assert abs(S.nuclear_norm(W1, H1) - s.sum()) <= 1e-10 * s.sum()
    assert S.nuclear_norm(np.zeros((5, 0)), np.zeros((7, 0))) == 0.0


def test_bb_curvature_is_the_dense_gradient_difference():
    """<X_t - X_{t-1}, grad f(X_t) - grad f(X_{t-1})> with dense gradients
    P_Omega(X - A) equals ||r_t - r_{t-1}||^2 used by the oracle."""
    p, ix = _small()
    M, mask = _dense(ix)
    rng = np.random.default_rng(1)
    W1, H1 = rng.standard_normal((ix.m, 4)), rng.standard_normal((ix.n, 4))
    W0, H0 = rng.standard_normal((ix.m, 2)), rng.standard_normal((ix.n, 2))
    X1, X0 = W1 @ H1.T, W0 @ H0.T
    dG = (X1 - M) * mask - (X0 - M) * mask
    curv = np.sum((X1 - X0) * dG)
    r1, r0 = O.residual(ix, W1, H1), O.residual(ix, W0, H0)
    assert abs(curv - np.sum((r1 - r0) ** 2)) <= 1e-10 * curv
    o = S.BbOptions(alpha_min=1e-6, alpha_max=1e6)
    a = S.bb_alpha(W1, H1, r1, S.BbPoint(W0, H0, r0), o, 1.0)
    assert abs(a - np.sum((X1 - X0) ** 2) / curv) <= 1e-10 * a


def test_full_observation_bb_step_is_one_over_lipschitz():
    """Omega = all entries: grad f(X) = X - A, so dG = dX and alpha_BB = 1 = 1/L."""
    rng = np.random.default_rng(2)
    m, n = 9, 14
    A = rng.standard_normal((m, n))
    rows, cols = np.divmod(np.arange(m * n), n)
    ix = O.build_index(m, n, rows, cols, A[rows, cols])
    W1, H1 = rng.standard_normal((ix.m, 3)), rng.standard_normal((ix.n, 3))
    W0, H0 = rng.standard_normal((ix.m, 2)), rng.standard_normal((ix.n, 2))
    r1, r0 = O.residual(ix, W1, H1), O.residual(ix, W0, H0)
    a = S.bb_alpha(W1, H1, r1, S.BbPoint(W0, H0, r0), S.BbOptions(), 1.99)
    assert abs(a - 1.0) <= 1e-12


@pytest.mark.parametrize("delta", [0.995, 0.5])
def test_accepted_steps_satisfy_back_or_decrease_densely(delta):
    """Every accepted step against Eq. "back" / Eq. "decrease" evaluated with
    dense matrices.  With delta = 0.5 the tests part ways (steps accepted by
    Eq. "decrease" alone occur), with the default 0.995 they nearly agree."""
    p, ix = _small(seed=13)
    opt = O.Options(lmsvd_tol=1e-12, lmsvd_imax=200)
    o = S.BbOptions(delta=delta)
    st, _ = O.init_step(ix, p.lam, 4, 20, opt)
    prev = None
    seen_bb = False
    backtracked = by_decrease = 0
    for t in range(6):
        st, _ = O.bm_phase(ix, st, p.lam, 3)
        st1, info, bb, prev = S.prox_step_bb(ix, st, p.lam, 20, opt, o, prev)
        assert bb.accepted_by in (1, 2)
        back, dec = S.dense_check(ix, st, st1, p.lam, bb.alpha, o.delta)
        assert back or dec
        # the flag names the test that held: 1 for Eq. "back", 2 for Eq.
        # "decrease" alone
        assert (bb.accepted_by == 1) == back, (t, bb, back, dec)
        if bb.accepted_by == 2:
            assert dec
        assert abs(bb.alpha - bb.alpha_bb * o.beta ** bb.backtracks) <= 1e-15 * bb.alpha_bb
        # the smallest i: the trial one reduction earlier satisfies neither test
        if bb.backtracks:
            a_prev = bb.alpha / o.beta
            st_prev, _ = O.prox_step(ix, st, p.lam, 20, opt, alpha=a_prev)
            assert not any(S.dense_check(ix, st, st_prev, p.lam, a_prev, o.delta)), (t, bb)
            backtracked += 1
        by_decrease += bb.accepted_by == 2
        seen_bb = seen_bb or (t > 0 and bb.alpha_bb > 1.99)
        st = st1
    assert seen_bb   # the BB value exceeds the fixed step on this sampled problem
    assert backtracked and (by_decrease or delta > 0.9), (backtracked, by_decrease)


def test_bb_step_uses_the_points_where_the_pg_steps_were_taken():
    """Eq. "proxBB" from X_t and X_{t-1}, the last two points where a PG step
    was taken (after their BM phases), as the step ||dX||^2 / <dX, dG> with
    dense gradients P_Omega(X - A), clipped to [alpha_min, alpha_max]; the
    first PG step starts from the fixed step alpha, clipped alike."""
    p, ix = _small(seed=13)
    opt = O.Options(lmsvd_tol=1e-12, lmsvd_imax=200)
    o = S.BbOptions()
    M, mask = _dense(ix)
    st, _ = O.init_step(ix, p.lam, 4, 20, opt)
    st, _ = O.bm_phase(ix, st, p.lam, 3)
    X0 = st.W @ st.H.T
    st1, _, bb0, prev = S.prox_step_bb(ix, st, p.lam, 20, opt, o, None)
    assert bb0.alpha_bb == min(o.alpha_max, max(o.alpha_min, opt.alpha))
    st1, _ = O.bm_phase(ix, st1, p.lam, 3)
    X1 = st1.W @ st1.H.T
    _, _, bb1, _ = S.prox_step_bb(ix, st1, p.lam, 20, opt, o, prev)
    dX = X1 - X0
    dG = np.where(mask, X1 - M, 0.0) - np.where(mask, X0 - M, 0.0)
    expect = min(o.alpha_max, max(o.alpha_min, float(np.sum(dX * dX)) / float(np.sum(dX * dG))))
    assert bb1.alpha_bb == pytest.approx(expect, rel=1e-9)


def test_no_backtracking_when_alpha_at_most_one_over_L():
    """With alpha <= 1/L = 1, Q is a majorisation of F - F(X~) (Eq. "proxgrad"),
    so Eq. "decrease" holds at the first trial."""
    p, ix = _small(seed=17)
    opt = O.Options(alpha=1.0, lmsvd_tol=1e-12, lmsvd_imax=200)
    o = S.BbOptions(alpha_max=1.0)
    st, _ = O.init_step(ix, p.lam, 4, 20, opt)
    prev = None
    for _ in range(4):
        st, _ = O.bm_phase(ix, st, p.lam, 3)
        st, info, bb, prev = S.prox_step_bb(ix, st, p.lam, 20, opt, o, prev)
        assert bb.backtracks == 0 and bb.accepted_by in (1, 2)


def test_sparsa_solve_reaches_the_dense_soft_impute_optimum():
    p, ix = _small(m=40, n=60, frac=0.35, rank=3, seed=21, lam=1.0)
    M, mask = _dense(ix)
    X = np.zeros_like(M)
    for _ in range(20000):
        U, s, Vt = np.linalg.svd(X - (X - M) * mask, full_matrices=False)
        Xn = (U * np.maximum(s - p.lam, 0)) @ Vt
        done = np.linalg.norm(Xn - X) <= 1e-14 * max(1.0, np.linalg.norm(X))
        X = Xn
        if done:
            break
    sX = np.linalg.svd(X, compute_uv=False)
    F_star = 0.5 * np.sum(((X - M) * mask) ** 2) + p.lam * sX.sum()
    st, F, bbs = S.solve_bb(ix, p.lam, 4, 30, O.Options(), S.BbOptions(), max_outer=400, tol=1e-15)
    assert abs(F[-1] - F_star) <= 1e-8 * F_star
    assert st.W.shape[1] == int(np.sum(sX > 1e-8))


def test_sparsa_solve_carries_the_previous_point():
    """The SpaRSA solve's second PG step takes alpha_BB from the points of the
    first and second PG steps, as the step-by-step sequence does."""
    p, ix = _small(seed=13)
    opt = O.Options(lmsvd_tol=1e-12, lmsvd_imax=200)
    o = S.BbOptions()
    _, _, bb_hist = S.solve_bb(ix, p.lam, 4, 20, opt, o, max_outer=2, tol=0.0)
    st, _ = O.init_step(ix, p.lam, 4, 20, opt)
    prev = None
    seq = []
    for _ in range(2):
        st, _ = O.bm_phase(ix, st, p.lam, opt.bm_epochs)
        st, _, bb, prev = S.prox_step_bb(ix, st, p.lam, 20, opt, o, prev)
        seq.append(bb.alpha_bb)
    assert [b.alpha_bb for b in bb_hist] == seq
    assert seq[1] != seq[0]


def test_exhausted_backtracking_keeps_the_last_trial():
    """A step of 1000 (alpha_min = alpha_max) satisfies neither test, nor do
    its two reductions by beta = 0.9: the step ends after max_backtracks
    reductions with flag 0 and keeps the last trial, X_{t+1} at 810 (the
    reading stated in the oracle's notes), and densely neither test holds."""
    p, ix = _small(seed=13)
    opt = O.Options(lmsvd_tol=1e-12, lmsvd_imax=200, alpha=1e3)
    o = S.BbOptions(alpha_min=1e3, alpha_max=1e3, beta=0.9, max_backtracks=2)
    st, _ = O.init_step(ix, p.lam, 4, 20, opt)
    st, _ = O.bm_phase(ix, st, p.lam, 3)
    st1, _, bb, _ = S.prox_step_bb(ix, st, p.lam, 20, opt, o, None)
    assert (bb.accepted_by, bb.backtracks) == (0, 2)
    assert bb.alpha == pytest.approx(810.0, rel=1e-15)
    last, _ = O.prox_step(ix, st, p.lam, 20, opt, alpha=810.0)
    assert np.array_equal(st1.W, last.W) and np.array_equal(st1.H, last.H)
    for a in (1000.0, 900.0, 810.0):
        trial, _ = O.prox_step(ix, st, p.lam, 20, opt, alpha=a)
        assert not any(S.dense_check(ix, st, trial, p.lam, a, o.delta))
