"""GPU parity of Algorithm 1 on the distance-geometry QSDP (Eq. "QSDP" /
Eq. "EDM") against the FP64 oracle in oracle/edm_oracle.py: the BM phase
(PR+ with the exact quartic line search), the initial PG step from X = 0, one
PG step from a given factor (Lemma "PiX", Eq. "proxsym", the rank rule), and
the full solve reaching the oracle's optimum."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from oracle import edm_oracle as E
from synth import self_avoiding_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_2204_14067_gb300 as B
    B.lib()
    return B


def _problem(n, seed, weighted=False):
    p = self_avoiding_chain(n=n, seed=seed)
    w = np.random.default_rng(seed).uniform(0.5, 2.0, p.npairs) if weighted else np.ones(p.npairs)
    i, j, d, w64 = E.pair_arrays(p.i, p.j, p.d, w)
    lam = O.edm_lambda(n, p.d)
    return p, i, j, d, w64, lam


def _handle(B, p, w64, lam, k_max, weighted, opt=None):
    h = B.bm_edm_create(p.n, p.i, p.j, p.d, lam, k_max, w=w64.astype(np.float32) if weighted else None)
    if opt is not None:
        B.bm_edm_set_options(h, opt)
    return h


def _options(B, **kw):
    o = B.bm_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _start(p, k, seed):
    rng = np.random.default_rng(seed)
    V = p.X_true @ rng.standard_normal((3, k)) * 0.5 + 0.05 * rng.standard_normal((p.n, k))
    return E.center(V)


def _gram_rel(Va, Vb):
    Xa, Xb = Va @ Va.T, Vb @ Vb.T
    return np.linalg.norm(Xa - Xb) / max(np.linalg.norm(Xb), 1e-300)


@pytest.mark.parametrize("n,k,weighted", [(2000, 5, False), (3000, 12, True), (700, 33, False)])
def test_bm_phase_matches_oracle(B, n, k, weighted):
    p, i, j, d, w, lam = _problem(n, 40 + k, weighted)
    V0 = _start(p, k, k)
    V32 = V0.astype(np.float32)
    h = _handle(B, p, w, lam, max(k, 16), weighted)
    try:
        B.bm_edm_set_factor(h, k, V32)
        F = B.bm_edm_bm_phase(h, 4)
        Vg = B.bm_edm_get_factor(h, n).astype(np.float64)
    finally:
        B.bm_edm_destroy(h)
    Vo, Fo = E.bm_phase(V32.astype(np.float64), i, j, d, w, lam, 4)
    assert abs(F - Fo[-1]) <= 1e-5 * abs(Fo[-1])
    assert abs(E.objective(Vg, i, j, d, w, lam) - Fo[-1]) <= 1e-5 * abs(Fo[-1])
    assert np.linalg.norm(Vg - Vo) <= 1e-3 * np.linalg.norm(Vo)
    assert np.abs(Vg.sum(axis=0)).max() <= 1e-3 * np.abs(Vg).max() * np.sqrt(n)


def _dense_z(n, i, j, c, V, alpha, lam):
    """Z = V V^T - L_c - alpha lam J as a dense FP64 matrix."""
    J = np.eye(n) - 1.0 / n
    Z = V @ V.T - E.laplacian_apply(n, i, j, c, np.eye(n)) - alpha * lam * J
    return 0.5 * (Z + Z.T)


def _psd_part(Z):
    """P_S+(J Z J) of Lemma "PiX", computed in an orthonormal basis of ker(e^T)
    (so the spectrum holds the n - 1 eigenvalues there, descending)."""
    n = Z.shape[0]
    Qk, _ = np.linalg.qr((np.eye(n) - 1.0 / n)[:, : n - 1])
    ev, U = np.linalg.eigh(Qk.T @ Z @ Qk)
    pos = ev > 0
    Up = Qk @ U[:, pos]
    return (Up * ev[pos]) @ Up.T, ev[::-1]


def _eig_report(V, Z):
    """For V = U diag(sqrt(mu)): max |U^T U - I| and max ||Z u_j - mu_j u_j|| / ||Z||."""
    mu = np.sum(V * V, axis=0)
    U = V / np.sqrt(np.maximum(mu, 1e-300))
    orth = float(np.abs(U.T @ U - np.eye(U.shape[1])).max()) if U.shape[1] else 0.0
    res = float(np.linalg.norm(Z @ U - U * mu, axis=0).max()) / np.linalg.norm(Z, 2) if U.shape[1] else 0.0
    return f"orth {orth:.2e}, eig residual {res:.2e}, mu {np.array2string(mu[:6], precision=6)}"


def _rank_band(mu, rel=1e-6):
    """Ranks consistent with FP32 resolution: eigenvalues within rel * mu_1 of
    zero may fall on either side."""
    tol = rel * max(abs(mu[0]), 1e-300)
    return int(np.sum(mu > tol)), int(np.sum(mu > -tol))


@pytest.mark.parametrize("n,weighted,npos", [(400, False, 12), (800, True, 16)])
def test_initial_pg_step_is_the_exact_projection(B, n, weighted, npos):
    """lambda chosen so that Z_{-1} = alpha L_{w d^2} - alpha lambda J has npos
    positive eigenvalues, fewer than the k_0 computed: X_0 = P_S+(Z_{-1})
    exactly (Lemma "PiX"), compared with the dense FP64 projection."""
    p, i, j, d, w, _ = _problem(n, 70, weighted)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    Ld = E.laplacian_apply(n, i, j, w * d * d, np.eye(n))
    ell = np.linalg.eigvalsh(Ld)[::-1]
    lam = 0.5 * (ell[npos - 1] + ell[npos])
    k_max = 64
    k0 = min(100, int(0.15 * n), k_max)
    opt = _options(B, lmsvd_tol=0.0, lmsvd_imax=150, seed=5)
    h = _handle(B, p, w, lam, k_max, weighted, opt)
    try:
        info = B.bm_edm_init(h)
        Vg = B.bm_edm_get_factor(h, n).astype(np.float64)
    finally:
        B.bm_edm_destroy(h)
    Zd = _dense_z(n, i, j, -alpha * w * d * d, np.zeros((n, 0)), alpha, lam)
    Xd, _ = _psd_part(Zd)
    st, oi = E.init_step(n, i, j, d, w, lam, alpha, k_max, O.Options(lmsvd_tol=0.0, lmsvd_imax=150, seed=5))
    assert info["computed"] == len(oi.mu) == k0
    assert info["rank"] == oi.rank == npos == Vg.shape[1]
    assert info["k_next"] == oi.k_eig_next == npos
    assert not info["all_positive"]
    # FP32 products with Z + sigma J carry errors of order eps32 * theta_1
    # (theta_1 = mu_1 + sigma, the operator's norm on ker(e^T)); X_0 inherits them
    err = np.linalg.norm(Vg @ Vg.T - Xd)
    theta1 = oi.mu[0] + info["sigma"]
    assert err <= 2e-5 * theta1 * np.sqrt(npos), (err, theta1, info, _eig_report(Vg, Zd), _eig_report(st.V, Zd))
    assert np.linalg.norm(st.V @ st.V.T - Xd) <= 1e-7 * np.linalg.norm(Xd)
    Fo = E.objective(st.V, i, j, d, w, lam)
    assert abs(info["F"] - Fo) <= 1e-5 * abs(Fo)


@pytest.mark.parametrize("n,weighted", [(400, False), (800, True)])
def test_initial_pg_step_truncated_matches_oracle(B, n, weighted):
    """The paper's lambda < 0: every computed eigenvalue is positive and X_0
    keeps the leading k_0 eigenpairs; the rank rule then asks for k_0 + n/20.
    The leading eigenvalues (well separated) agree with the oracle's to the
    FP32 resolution of the shifted operator, eps32 * theta_1."""
    p, i, j, d, w, lam = _problem(n, 70, weighted)
    k_max = 64
    opt = _options(B, lmsvd_tol=0.0, lmsvd_imax=100, seed=5)
    h = _handle(B, p, w, lam, k_max, weighted, opt)
    try:
        info = B.bm_edm_init(h)
        Vg = B.bm_edm_get_factor(h, n).astype(np.float64)
    finally:
        B.bm_edm_destroy(h)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    st, oi = E.init_step(n, i, j, d, w, lam, alpha, k_max, O.Options(lmsvd_tol=0.0, lmsvd_imax=100, seed=5))
    assert info["rank"] == oi.rank == len(oi.mu) == Vg.shape[1]
    assert info["all_positive"]
    assert info["k_next"] == oi.k_eig_next == min(k_max, oi.rank + n // 20)
    mu_g = np.sort(np.sum(Vg * Vg, axis=0))[::-1]
    Zd = _dense_z(n, i, j, -alpha * w * d * d, np.zeros((n, 0)), alpha, lam)
    theta1 = oi.mu[0] + info["sigma"]
    assert np.abs(mu_g[:4] - oi.mu[:4]).max() <= 2e-5 * theta1, (info, _eig_report(Vg, Zd), _eig_report(st.V, Zd))
    assert np.abs(Vg.sum(axis=0)).max() <= 1e-3 * np.abs(Vg).max() * np.sqrt(n)


def _near_optimum(n, seed, weighted, cycles):
    p, i, j, d, w, lam = _problem(n, seed, weighted)
    st, F, _ = E.solve(n, i, j, d, w, lam, 40, O.Options(lmsvd_tol=1e-12, lmsvd_imax=200, bm_epochs=200),
                       max_outer=cycles, tol=1e-13)
    return p, i, j, d, w, lam, st.V


@pytest.mark.parametrize("n,weighted,cycles", [(120, False, 10), (200, True, 6)])
def test_pg_step_near_the_optimum_is_the_exact_projection(B, n, weighted, cycles):
    """Near the optimum Z has fewer positive eigenvalues than the k + 1
    computed, so the PG step is the exact projection P_S+(Z) of Lemma "PiX"
    / Eq. "proxsym": compared with the dense FP64 projection and the oracle."""
    p, i, j, d, w, lam, V0 = _near_optimum(n, 17, weighted, cycles)
    k = V0.shape[1]
    k_max = 40
    V32 = np.ascontiguousarray(V0, dtype=np.float32)
    opt = _options(B, lmsvd_tol=0.0, lmsvd_imax=60, seed=9)
    h = _handle(B, p, w, lam, k_max, weighted, opt)
    try:
        B.bm_edm_set_factor(h, k, V32)
        info = B.bm_edm_prox_step(h)
        Vg = B.bm_edm_get_factor(h, n).astype(np.float64)
    finally:
        B.bm_edm_destroy(h)
    V64 = V32.astype(np.float64)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    c = alpha * w * E.residual(V64, i, j, d)
    Xd, ev = _psd_part(_dense_z(n, i, j, c, V64, alpha, lam))
    st2, oi = E.prox_step(E.EdmState(V=V64, U=np.zeros((n, 0)), k_eig=k + 1), i, j, d, w, lam, alpha, k_max,
                          O.Options(lmsvd_tol=0.0, lmsvd_imax=60, seed=9))
    # setup: the eigenvalues left out (k + 2 onwards) are within FP32
    # resolution of zero or negative, so the projection is not truncated
    assert ev[k + 1] <= 1e-6 * ev[0]
    lo, hi = _rank_band(ev[:k + 1])
    assert info["computed"] == len(oi.mu) == k + 1
    assert lo <= info["rank"] <= hi and lo <= oi.rank <= hi
    assert info["k_next"] == max(1, info["rank"])
    err = np.linalg.norm(Vg @ Vg.T - Xd)
    theta1 = ev[0] + info["sigma"]
    assert err <= 2e-5 * theta1 * np.sqrt(k + 1), (err, theta1, info, ev[:k + 2])
    assert err <= 1e-5 * np.linalg.norm(Xd)
    assert np.linalg.norm(st2.V @ st2.V.T - Xd) <= 1e-6 * np.linalg.norm(Xd)
    Fo = E.objective(st2.V, i, j, d, w, lam)
    assert abs(info["F"] - Fo) <= 1e-5 * abs(Fo)
    assert np.abs(Vg.sum(axis=0)).max() <= 1e-3 * np.abs(Vg).max() * np.sqrt(n)


def test_solve_reaches_the_oracle_optimum(B):
    """The QSDP is convex: the GPU solve reaches the oracle's optimal value
    within 1e-6 (the oracle run to a relative change below 1e-11)."""
    n = 120
    p, i, j, d, w, lam = _problem(n, 17)
    k_max = 40
    st, Fo, ranks = E.solve(n, i, j, d, w, lam, k_max,
                            O.Options(lmsvd_tol=1e-12, lmsvd_imax=200, bm_epochs=200), max_outer=60, tol=1e-12)
    F_star = Fo[-1]
    assert abs(Fo[-1] - Fo[-2]) <= 1e-11 * abs(F_star)
    h = _handle(B, p, w, lam, k_max, False, _options(B, lmsvd_tol=1e-7, lmsvd_imax=200, bm_epochs=200))
    try:
        res = B.bm_edm_solve(h, max_outer=80, tol=0.0, F_target=F_star * (1 + 1e-6))
        Vg = B.bm_edm_get_factor(h, n).astype(np.float64)
    finally:
        B.bm_edm_destroy(h)
    assert res["converged"]
    F = E.objective(Vg, i, j, d, w, lam)
    assert abs(res["F"] - F) <= 1e-6 * abs(F)
    # the optimal value is unique; the optimal X need not be (directions D with
    # A(D) = 0 and <I, D> = 0 leave the objective unchanged), so X is not compared
    assert F_star * (1 - 1e-6) <= F <= F_star * (1 + 2e-6)


def test_cycles_at_config_size(B):
    """The 30,000-atom chain (about 1.1 million pairs) with k <= 16: the initial
    PG step and a few cycles, checked by properties that hold at any size
    (monotone BM phase, the reported objective equals the FP64 objective of
    the returned factor, V^T e = 0, rank <= k_max)."""
    n = 30_000
    p, i, j, d, w, lam = _problem(n, 3)
    k_max = 16
    h = _handle(B, p, w, lam, k_max, False, _options(B, bm_epochs=30, lmsvd_imax=20))
    try:
        info = B.bm_edm_init(h)
        assert 1 <= info["rank"] <= k_max
        for _ in range(3):
            V = B.bm_edm_get_factor(h, n).astype(np.float64)
            F0 = E.objective(V, i, j, d, w, lam)
            F1 = B.bm_edm_bm_phase(h, 30)
            assert F1 <= F0 * (1 + 1e-6)
            info = B.bm_edm_prox_step(h)
            assert 1 <= info["rank"] <= k_max
            V = B.bm_edm_get_factor(h, n).astype(np.float64)
            F = E.objective(V, i, j, d, w, lam)
            assert abs(info["F"] - F) <= 1e-5 * abs(F)
            assert np.abs(V.sum(axis=0)).max() <= 1e-3 * np.abs(V).max() * np.sqrt(n)
    finally:
        B.bm_edm_destroy(h)
def test_small_and_degenerate_cases(B):
    # a chain of 6 points with k_max = 1, and lambda large enough that X* = 0
    p, i, j, d, w, lam = _problem(6, 5)
    h = _handle(B, p, w, lam, 1, False)
    try:
        info = B.bm_edm_init(h)
        assert 0 <= info["rank"] <= 1
        res = B.bm_edm_solve(h, max_outer=50, tol=1e-10)
        assert np.isfinite(res["F"])
    finally:
        B.bm_edm_destroy(h)
    big = 1e6
    h = _handle(B, p, w, big, 4, False)
    try:
        info = B.bm_edm_init(h)
        assert info["rank"] == 0
        assert B.bm_edm_get_factor(h, p.n).shape == (p.n, 0)
        assert abs(info["F"] - 0.5 * float(np.sum(w * d ** 4))) <= 1e-5 * 0.5 * float(np.sum(w * d ** 4))
    finally:
        B.bm_edm_destroy(h)
    h = _handle(B, p, w, lam, 4, False)
    try:
        with pytest.raises(B.BMError):
            B.bm_edm_set_options(h, _options(B, lmsvd_p=2))
    finally:
        B.bm_edm_destroy(h)
