"""Pins of the oracle's rank safeguard (supplement, "Ensuring sufficient
precision in the proximal operation"; Eq. "rt0", "rt0-1", "rt").

The safeguard decides the warm start U^{t,0} of LmSVD:
  * base: orth([U_t, W_t]) after a BM phase that moved the iterate (Eq. rt0),
    orth([U_t, U_{t-1}]) otherwise (Eq. rt0-1);
  * one more column u_t + xi_t (Eq. rt) when rank(X_t) = rank(X_{t-1}) OR
    rank(U^{t-1,0}) <= rank(X_t) + 1 (the explicit "or" form of the trigger),
    with u_t the retained truncated vector projected onto ker(U^_{t,0}^T),
    xi_t in ker([U^_{t,0}, u_t]^T) and ||xi_t|| = psi_t;
  * psi_{t+1} = psi_t / 2 exactly when one value was truncated
    (rank(X_{t+1}) = rank(U^{t,0}) - 1), else psi_{t+1} = psi_t.

The geometric checks below rebuild projections with numpy's QR, not with
the oracle's orth(), and the tiny case is worked out by hand.
"""
import math

import numpy as np

from oracle import bm_oracle as O


def _orthonormal(m, k, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, k)))
    return q


def _state(U, W, rank_hist, prev_warm_cols, u=None, psi=0.1, t=0, U_prev2=None, bm_changed=True):
    return O.State(W=W, H=np.zeros((5, W.shape[1])), U_prev=U, U_prev2=U_prev2, u=u, psi=psi,
                   rank_hist=list(rank_hist), prev_warm_cols=prev_warm_cols, t=t, bm_changed=bm_changed)


def _opt(seed=0, psi0=0.1):
    return O.Options(seed=seed, psi0=psi0)


def _same_span_factor(U, seed):
    """A BM-phase factor W with ran(W) = ran(U): orth([U, W]) adds no column."""
    k = U.shape[1]
    return U @ np.random.default_rng(seed).standard_normal((k, k))


def test_trigger_is_the_or_form():
    """Truth table of the trigger on hand-built states (rank k = 4 throughout)."""
    m, k = 30, 4
    U = _orthonormal(m, k, 1)
    W = _same_span_factor(U, 2)
    u = np.random.default_rng(3).standard_normal(m)
    cases = [
        # (rank_hist, prev_warm_cols, column added?)
        ([3, 4], 9, False),    # rank grew, several values truncated: no column
        ([4, 4], 9, True),     # rank unchanged (first clause alone)
        ([3, 4], 5, True),     # one value truncated: warm cols 5 <= 4 + 1 (second clause alone)
        ([3, 4], 4, True),     # nothing truncated: 4 <= 5
        ([4, 4], 5, True),     # both clauses
        ([5, 4], 6, False),    # rank fell by one, two truncated
    ]
    for hist, pw, added in cases:
        Uh0 = O.warm_start(_state(U, W, hist, pw, u=u), k_max=20, opt=_opt())
        assert Uh0.shape[1] == k + (1 if added else 0), (hist, pw)
        # the base is U itself (W adds no direction)
        assert np.allclose(Uh0[:, :k], U, atol=1e-12)


def test_added_column_geometry():
    """The added column is (u_t + xi_t)/||u_t + xi_t|| with u_t = (I - UU^T)u,
    xi_t orthogonal to U and u_t, ||xi_t|| = psi, and xi_t along the
    counter-generator Gaussian projected off [U, u_t]."""
    m, k, psi, t, seed = 40, 5, 0.1, 3, 7
    U = _orthonormal(m, k, 4)
    W = _same_span_factor(U, 5)
    u = np.random.default_rng(6).standard_normal(m)
    u /= np.linalg.norm(u)
    Uh0 = O.warm_start(_state(U, W, [5, 5], 9, u=u, psi=psi, t=t), k_max=20, opt=_opt(seed=seed))
    assert Uh0.shape[1] == k + 1
    x = Uh0[:, -1]
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    assert np.max(np.abs(U.T @ x)) < 1e-12
    ut = u - U @ (U.T @ u)
    a = float(x @ ut) / float(ut @ ut)          # coefficient of u_t
    xi = x - a * ut                             # the xi part, scaled by the same 1/||u_t + xi_t||
    assert a > 0
    assert abs(float(xi @ ut)) < 1e-12 * np.linalg.norm(ut)
    assert np.max(np.abs(U.T @ xi)) < 1e-12
    assert abs(np.linalg.norm(xi) / a - psi) < 1e-12          # ||xi_t|| = psi_t
    # direction: the Gaussian of stream 1000 + t projected off [U, u_t] (numpy QR)
    g = O.counter_normal(seed, O.STREAM_SAFEGUARD + t, m)
    Qb, _ = np.linalg.qr(np.column_stack([U, ut]))
    gp = g - Qb @ (Qb.T @ g)
    assert np.allclose(xi / np.linalg.norm(xi), gp / np.linalg.norm(gp), atol=1e-12)


def test_column_without_retained_vector_is_unit_random():
    """No truncated vector retained: the column is the unit Gaussian projected off U."""
    m, k, t, seed = 25, 3, 2, 11
    U = _orthonormal(m, k, 8)
    W = _same_span_factor(U, 9)
    Uh0 = O.warm_start(_state(U, W, [3, 3], 3, u=None, t=t), k_max=10, opt=_opt(seed=seed))
    g = O.counter_normal(seed, O.STREAM_SAFEGUARD + t, m)
    gp = g - U @ (U.T @ g)
    assert Uh0.shape[1] == k + 1
    assert np.allclose(Uh0[:, -1], gp / np.linalg.norm(gp), atol=1e-12)


def test_psi_halves_exactly_when_one_value_is_truncated():
    m, n = 6, 7
    st = _state(np.zeros((m, 0)), np.zeros((m, 0)), [2, 2], 3, psi=0.08)
    for warm_cols, k_new, psi_next in [(5, 4, 0.04), (5, 5, 0.08), (5, 3, 0.08), (5, 0, 0.08), (1, 0, 0.04)]:
        res = O.ProxResult(W=np.zeros((m, k_new)), H=np.zeros((n, k_new)), U=np.zeros((m, k_new)),
                           V=np.zeros((n, k_new)), sigma=np.ones(k_new), sigma_hat=np.ones(warm_cols),
                           k_new=k_new, cap_hit=False, eps=0.0, u_trunc=None)
        nxt = O._advance(st, res, warm_cols)
        assert nxt.psi == psi_next, (warm_cols, k_new)
        assert nxt.rank_hist[-2:] == [2, k_new] and nxt.prev_warm_cols == warm_cols and nxt.t == st.t + 1


def test_tiny_case_by_hand():
    """m = 3, U_t = e1, W_t = 2 e1, u = (1, 1, 0)/sqrt 2, psi = 0.1:
    u_t = (0, 1/sqrt 2, 0); xi_t lies along +-e3 (the only direction left), so
    the column is (0, 1/sqrt 2, +-0.1)/sqrt(0.51) = (0, 0.99014754, +-0.14002801),
    the sign that of the Gaussian's third component."""
    e1 = np.array([[1.0], [0.0], [0.0]])
    u = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    Uh0 = O.warm_start(_state(e1, 2.0 * e1, [1, 1], 5, u=u, psi=0.1, t=0), k_max=2, opt=_opt(seed=0))
    sgn = math.copysign(1.0, O.counter_normal(0, O.STREAM_SAFEGUARD, 3)[2])
    assert Uh0.shape == (3, 2)
    assert np.allclose(Uh0[:, 0], [1.0, 0.0, 0.0], atol=1e-15)
    assert np.allclose(Uh0[:, 1], [0.0, 0.99014754, sgn * 0.14002801], atol=1e-8)


def test_base_after_bm_phase_and_without():
    """Eq. rt0 takes W_t; Eq. rt0-1 (BM phase did not move the iterate) takes U_{t-1}."""
    m, k = 30, 3
    U = _orthonormal(m, k, 12)
    W = np.random.default_rng(13).standard_normal((m, k))
    U2 = _orthonormal(m, k, 14)
    no_trig = ([2, 3], 9)
    for changed, second in [(True, W), (False, U2)]:
        Uh0 = O.warm_start(_state(U, W, *no_trig, U_prev2=U2, bm_changed=changed), k_max=20, opt=_opt())
        assert Uh0.shape[1] == 2 * k
        assert np.allclose(Uh0.T @ Uh0, np.eye(2 * k), atol=1e-12)
        Q, _ = np.linalg.qr(Uh0)
        for M in (U, second):
            assert np.linalg.norm(M - Q @ (Q.T @ M)) < 1e-10 * np.linalg.norm(M)
    # without a previous prox, W is used even when the BM phase did not move
    Uh0 = O.warm_start(_state(U, W, *no_trig, U_prev2=None, bm_changed=False), k_max=20, opt=_opt())
    Q, _ = np.linalg.qr(Uh0)
    assert np.linalg.norm(W - Q @ (Q.T @ W)) < 1e-10 * np.linalg.norm(W)


def test_warm_start_is_capped_at_k_max_plus_one():
    m = 20
    U = _orthonormal(m, 6, 15)
    W = np.random.default_rng(16).standard_normal((m, 6))
    Uh0 = O.warm_start(_state(U, W, [6, 6], 3, u=np.ones(m)), k_max=4, opt=_opt())
    assert Uh0.shape[1] == 5 and np.allclose(Uh0, U[:, :5])
    Uh0 = O.warm_start(_state(U[:, :3], W, [6, 6], 3, u=np.ones(m)), k_max=4, opt=_opt())
    assert Uh0.shape[1] == 5          # base 3 + 2 from W; full, so no safeguard column


def test_no_column_when_the_basis_and_u_span_the_whole_space():
    """m = 2, U^ = e_1 and u_t = e_2: no xi_t is orthogonal to [U^, u_t], so
    the safeguard adds no column (and forms no 0/0 on the way)."""
    import warnings
    U = np.array([[1.0], [0.0]])
    W = U * 2.0
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        Uh0 = O.warm_start(_state(U, W, [1, 1], 9, u=np.array([0.0, 3.0])), k_max=3, opt=_opt())
    assert Uh0.shape == (2, 1) and np.allclose(np.abs(Uh0[:, 0]), [1.0, 0.0])
