"""Pins of the oracle's orthonormalisation, LmSVD, exact-SVD/SVT step, PG
state update, initial step and cycle order (Algorithm 1, Algorithm 2, Eq.
"PUi", "orth-W", "nys") against facts that do not come from the oracle:
dense SVDs and eigendecompositions, the block Krylov subspace that the
second Rayleigh-Ritz step of Algorithm 2 spans, the range of the Nystrom
approximation, and closed forms of the singular value soft-threshold with
full observation (where Z = A for alpha = 1)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bm_oracle as O


def _orthonormal(m, k, rng):
    q, r = np.linalg.qr(rng.standard_normal((m, k)))
    return q * np.sign(np.diag(r))


def _angle_residual(U, K):
    """||(I - K K^T) U||_2 for orthonormal K: 0 when ran(U) lies in ran(K)."""
    return np.linalg.norm(U - K @ (K.T @ U), 2)


def _state(W, H, opt):
    U0, _ = O.orth(W, tau=1e-14)
    return O.State(W=W, H=H, U_prev=U0, U_prev2=None, u=None, psi=opt.psi0,
                   rank_hist=[W.shape[1], W.shape[1]], prev_warm_cols=W.shape[1] + 1, t=0,
                   bm_changed=True)


def _full(A):
    m, n = A.shape
    rows, cols = np.divmod(np.arange(m * n), n)
    return O.build_index(m, n, rows, cols, A[rows, cols])


def _low_rank(m, n, sig, rng):
    r = len(sig)
    return (_orthonormal(m, r, rng) * np.asarray(sig)) @ _orthonormal(n, r, rng).T


# ---------------------------------------------------------------- orth (Eq. PUi, orth-W)
def test_orth_is_orthonormal_to_rounding_on_nearly_dependent_columns():
    """Columns at angles of a few 1e-3 (Gram eigenvalues just above tau):
    the result must be orthonormal to rounding, not to eps * cond(Gram)."""
    rng = np.random.default_rng(40)
    m = 200
    B = _orthonormal(m, 8, rng)
    M = np.hstack([B[:, :4], B[:, :4] + 3e-3 * B[:, 4:8]])
    Q, _ = O.orth(M, tau=1e-6)
    assert Q.shape[1] == 8
    assert np.abs(Q.T @ Q - np.eye(8)).max() <= 1e-13
    assert _angle_residual(Q, B) <= 1e-12


def test_orth_keeps_columns_of_any_scale():
    """Eq. "PUi" scales every column to unit norm before the Gram test, so a
    column's length does not decide whether its direction is kept."""
    rng = np.random.default_rng(41)
    B = _orthonormal(50, 3, rng)
    M = B * np.array([1e-4, 1.0, 1e4])
    Q, _ = O.orth(M, tau=1e-6)
    assert Q.shape[1] == 3
    assert _angle_residual(B, Q) <= 1e-12


def test_orth_max_cols_keeps_the_dominant_directions():
    """With unit columns, a cap of j columns keeps the span of the j leading
    left singular vectors of M (numpy's SVD)."""
    rng = np.random.default_rng(42)
    B = _orthonormal(60, 4, rng)
    C = rng.standard_normal((4, 6)) * np.array([[3.0], [1.0], [0.3], [0.1]])
    M = B @ C
    M = M / np.linalg.norm(M, axis=0)
    Q, _ = O.orth(M, tau=1e-6, max_cols=2)
    U, _, _ = np.linalg.svd(M, full_matrices=False)
    assert Q.shape[1] == 2
    assert _angle_residual(Q, U[:, :2]) <= 1e-10


# ---------------------------------------------------------------- LmSVD (Algorithm 2)
def _psd_operator(m, rng, lam=None):
    lam = 0.8 ** np.arange(m) if lam is None else lam
    V = _orthonormal(m, m, rng)
    return (V * lam) @ V.T


def _ritz_top(L, basis, k):
    Q = sla.orth(basis)
    w = np.linalg.eigvalsh(Q.T @ L @ Q)[::-1]
    return w[:k]


@pytest.mark.parametrize("p", [0, 1, 2])
def test_lmsvd_second_step_is_rayleigh_ritz_on_the_block_krylov_space(p):
    """At i = 1 Algorithm 2 optimises over ran(U^{t,1}, U^{t,0}) when p >= 1,
    and U^{t,1} = orth(L(U^{t,0} V)) spans L U0: the Ritz values after two
    Rayleigh-Ritz steps are those of L on span{U0, L U0} (dense, scipy); with
    p = 0 (plain subspace iteration) on span{L U0} alone."""
    rng = np.random.default_rng(43)
    m, k = 40, 4
    L = _psd_operator(m, rng)
    U0 = rng.standard_normal((m, k))
    _, theta, it, _ = O.lmsvd(lambda U: L @ U, U0, p=p, tol=0.0, imax=2, tau=1e-12)
    assert it == 2
    expect = _ritz_top(L, np.hstack([U0, L @ U0]) if p >= 1 else L @ U0, k)
    assert np.allclose(theta, expect, rtol=1e-12, atol=0)
    other = _ritz_top(L, L @ U0 if p >= 1 else np.hstack([U0, L @ U0]), k)
    assert np.abs(other - expect).max() > 1e-4 * expect[0]


def test_lmsvd_stops_at_the_first_small_change_relative_to_theta_1():
    """The stop rule (Algorithm 2: the eigenvalues of successive Rayleigh-Ritz
    matrices differ little), read as max_j |theta_j - theta_j'| <= tol theta_1:
    it holds at the returned iteration and not one iteration earlier.  The
    spectrum makes the trailing Ritz values converge last, so a test relative
    to the smallest one would stop later: the fifth Ritz value is 1e-2 of the
    first and sits on a slowly decaying tail (0.009 * 0.95^j)."""
    rng = np.random.default_rng(44)
    m, k = 60, 5
    lam = np.concatenate([[1.0, 0.5, 0.1, 0.02, 0.01], 0.009 * 0.95 ** np.arange(m - 5)])
    L = _psd_operator(m, rng, lam)
    U0 = rng.standard_normal((m, k))
    tol = 1e-6
    Lop = lambda U: L @ U
    _, th, it, _ = O.lmsvd(Lop, U0, p=1, tol=tol, imax=200, tau=1e-12)
    assert 3 < it < 200
    _, th1, _, _ = O.lmsvd(Lop, U0, p=1, tol=0.0, imax=it - 1, tau=1e-12)
    _, th2, _, _ = O.lmsvd(Lop, U0, p=1, tol=0.0, imax=it - 2, tau=1e-12)
    assert np.abs(th - th1).max() <= tol * th[0]
    assert np.abs(th1 - th2).max() > tol * th1[0]
    # and the trailing values still move by more than tol * theta_k there
    assert np.abs(th - th1).max() > tol * th[-1]


# ---------------------------------------------------------------- PG step with full observation
def _prox_full(A, W, H, lam, k_max, opt):
    ix = _full(A)
    st = _state(W, H, opt)
    st2, info = O.prox_step(ix, st, lam, k_max, opt, alpha=1.0)
    return ix, st, st2, info


def _svt(A, thresh, kcap):
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    k = int(np.sum(s > thresh))
    k = min(k, kcap)
    return (U[:, :k] * (s[:k] - thresh)) @ Vt[:k], U, s, k


def test_prox_caps_the_rank_at_k_max():
    """Six singular values above the threshold and k_max = 4: the step keeps
    exactly the four largest, soft-thresholded (cap_hit), as the dense SVD says."""
    rng = np.random.default_rng(45)
    A = _low_rank(14, 22, [5.0, 4.0, 3.0, 2.0, 1.0, 0.5], rng)
    W = rng.standard_normal((14, 6))
    H = rng.standard_normal((22, 6))
    opt = O.Options(lmsvd_tol=1e-15, lmsvd_imax=300)
    _, _, st2, info = _prox_full(A, W, H, 0.1, 4, opt)
    X, _, _, _ = _svt(A, 0.1, 4)
    assert info.k_new == 4 and info.cap_hit
    assert np.abs(st2.W @ st2.H.T - X).max() <= 1e-9


def test_prox_keeps_small_singular_values_above_the_ritz_cut():
    """Singular values 1 ... 1e-5 and a threshold of 1e-7: the exact prox
    keeps all six.  The cut of Algorithm 2 (J_s) removes s_j <= 1e-6 s_1,
    on the singular values s = sqrt(theta), not on theta = s^2."""
    rng = np.random.default_rng(46)
    sig = [1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5]
    A = _low_rank(12, 20, sig, rng)
    W = rng.standard_normal((12, 8))
    H = rng.standard_normal((20, 8))
    opt = O.Options(lmsvd_tol=1e-15, lmsvd_imax=300)
    _, _, st2, info = _prox_full(A, W, H, 1e-7, 10, opt)
    X, _, _, k = _svt(A, 1e-7, 10)
    assert k == 6 and info.k_new == 6
    assert np.allclose(info.sigma, np.array(sig) - 1e-7, rtol=1e-6, atol=0)
    assert np.abs(st2.W @ st2.H.T - X).max() <= 1e-10


def test_prox_truncated_vector_is_the_next_singular_vector():
    """The safeguard's u_t is the left singular vector of the largest value
    that the threshold removed: with Z = A, A's (k_new + 1)-th one."""
    rng = np.random.default_rng(47)
    A = _low_rank(14, 22, [5.0, 4.0, 3.0, 0.6, 0.3], rng)
    W = rng.standard_normal((14, 6))
    H = rng.standard_normal((22, 6))
    opt = O.Options(lmsvd_tol=1e-15, lmsvd_imax=300)
    _, _, st2, info = _prox_full(A, W, H, 1.0, 8, opt)
    _, U, _, k = _svt(A, 1.0, 8)
    assert k == 3 and info.k_new == 3
    u = st2.u / np.linalg.norm(st2.u)
    assert abs(abs(u @ U[:, 3]) - 1.0) <= 1e-9


def test_state_keeps_the_previous_left_vectors_as_u_t_minus_1():
    """Eq. "rt0-1": the warm start after a PG step with no BM phase between
    uses U_{t-1}; the state after step t+1 holds step t's U_t as U_{t-1}."""
    rng = np.random.default_rng(48)
    A = _low_rank(14, 22, [5.0, 4.0, 3.0, 0.6, 0.3], rng)
    W = rng.standard_normal((14, 6))
    H = rng.standard_normal((22, 6))
    opt = O.Options(lmsvd_tol=1e-12)
    ix, _, st1, _ = _prox_full(A, W, H, 0.5, 8, opt)
    st2, _ = O.prox_step(ix, st1, 0.5, 8, opt, alpha=1.0)
    assert st2.U_prev2 is not None and np.array_equal(st2.U_prev2, st1.U_prev)
    assert not st1.bm_changed and not st2.bm_changed


# ---------------------------------------------------------------- initial step (Eq. nys)
def test_initial_step_spans_the_range_of_the_nystrom_approximation():
    """Sec. "Initialization": Q = orth(A_{-1} G) for the Gaussian G, the
    Nystrom approximation A^ = (A_{-1} Q)(Q^T A_{-1} Q)^+ (A_{-1} Q)^T, and
    U^_0 from its eigendecomposition, so the initial left factor lies in
    ran(A^) = ran(A_{-1} Q) (dense, scipy), with A_{-1} = Z_{-1} Z_{-1}^T and
    Z_{-1} = P_Omega(A) for alpha_{-1} = 1.  A full-rank A keeps this apart
    from ran(Q) (no Nystrom step)."""
    rng = np.random.default_rng(49)
    m, n, k_init = 16, 24, 5
    A = rng.standard_normal((m, n)) * (0.7 ** np.arange(n))
    ix = _full(A)
    opt = O.Options()
    st, info = O.init_step(ix, 0.05, k_init, 10, opt)
    G = O.counter_normal(opt.seed, O.STREAM_INIT_SKETCH, m * k_init).reshape(k_init, m).T
    Am1 = A @ A.T
    Q = sla.orth(Am1 @ G)
    C = Q.T @ Am1 @ Q
    Ahat = (Am1 @ Q) @ np.linalg.pinv(C) @ (Am1 @ Q).T
    K = sla.orth(Ahat, rcond=1e-10)
    assert K.shape[1] == k_init and info.k_new >= 1
    Uw = sla.orth(st.W)
    assert _angle_residual(Uw, K) <= 1e-9
    assert _angle_residual(Uw, Q) > 1e-3


# ---------------------------------------------------------------- Algorithm 1 cycle order
def test_solve_cycle_runs_the_bm_phase_before_the_pg_step():
    """Algorithm 1: each cycle runs the BM phase from (W_t, H_t), then the PG
    step from its result."""
    rng = np.random.default_rng(50)
    A = _low_rank(12, 18, [3.0, 2.0, 1.0], rng) + 0.05 * rng.standard_normal((12, 18))
    mask = rng.random(A.shape) < 0.6
    rows, cols = np.nonzero(mask)
    ix = O.build_index(12, 18, rows, cols, A[rows, cols])
    opt = O.Options()
    lam = 0.3
    st0, _ = O.init_step(ix, lam, 4, 8, opt)
    st_bm, _ = O.bm_phase(ix, st0, lam, opt.bm_epochs)
    st1, _ = O.prox_step(ix, st_bm, lam, 8, opt)
    _, info = O.solve(ix, lam, 4, 8, opt, max_outer=1, tol=0.0)
    assert info.F_hist[1] == O.objective(ix, st1.W, st1.H, lam)
    # the other order reaches a different point
    st_pg, _ = O.prox_step(ix, st0, lam, 8, opt)
    st_b2, _ = O.bm_phase(ix, st_pg, lam, opt.bm_epochs)
    assert O.objective(ix, st_b2.W, st_b2.H, lam) != info.F_hist[1]
