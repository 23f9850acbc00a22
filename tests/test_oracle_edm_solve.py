"""Pins of the distance-geometry QSDP oracle (oracle/edm_oracle.py) against
facts independent of it: the variational inequality of a projection onto a
convex set (Lemma "PiX"), dense operators, finite differences, brute-force
line search, the exact operator norm, the dense exact PG step, the definition
of Polak-Ribiere+ CG with exact steps, and the dense convex optimum of the
QSDP."""
import numpy as np
import pytest

from oracle import bm_oracle as O
from oracle import edm_oracle as E
from cg_pin import check_pr_plus
from synth import self_avoiding_chain


def _chain(n, seed):
    p = self_avoiding_chain(n=n, seed=seed)
    i, j, d, w = E.pair_arrays(p.i, p.j, p.d, 1.0)
    return p, i, j, d, w


def test_projection_is_the_euclidean_projection_onto_the_feasible_set():
    rng = np.random.default_rng(0)
    n = 25
    A = rng.standard_normal((n, n))
    G = A + A.T
    P = E.dense_project(G)
    assert np.linalg.eigvalsh(P).min() >= -1e-10
    assert np.abs(P @ np.ones(n)).max() <= 1e-10
    J = np.eye(n) - np.ones((n, n)) / n
    for _ in range(20):
        M = rng.standard_normal((n, rng.integers(1, n)))
        Y = J @ M @ M.T @ J                       # a feasible point
        # <G - P, Y - P> <= 0 characterises the projection onto a convex set
        assert np.sum((G - P) * (Y - P)) <= 1e-9 * (1 + np.abs(G).sum())


def test_laplacian_apply_matches_dense_sum_of_E_ij():
    rng = np.random.default_rng(1)
    n, npairs = 12, 30
    i = rng.integers(0, n, npairs)
    j = (i + rng.integers(1, n, npairs)) % n
    c = rng.standard_normal(npairs)
    U = rng.standard_normal((n, 3))
    L = np.zeros((n, n))
    for a, b, cc in zip(i, j, c):
        e = np.zeros(n)
        e[a], e[b] = 1.0, -1.0
        L += cc * np.outer(e, e)
    assert np.allclose(E.laplacian_apply(n, i, j, c, U), L @ U, atol=1e-12)


def test_gradient_and_line_search_quartic():
    p, i, j, d, w = _chain(40, 11)
    rng = np.random.default_rng(2)
    lam = O.edm_lambda(p.n, d)
    V = E.center(p.X_true @ rng.standard_normal((3, 4)) * 0.5 + 0.1 * rng.standard_normal((p.n, 4)))
    g = E.gradient(V, i, j, d, w, lam)
    h = 1e-6
    for _ in range(5):
        a, b = rng.integers(0, p.n), rng.integers(0, 4)
        Vp, Vm = V.copy(), V.copy()
        Vp[a, b] += h
        Vm[a, b] -= h
        fd = (E.objective(Vp, i, j, d, w, lam) - E.objective(Vm, i, j, d, w, lam)) / (2 * h)
        assert abs(fd - g[a, b]) <= 1e-6 * (1 + abs(g).max())
    D = E.center(rng.standard_normal(V.shape))
    c = E.line_search_coeffs(V, D, i, j, d, w, lam)
    for s in (0.0, 0.3, -0.7, 1.9):
        poly = sum(c[q] * s ** q for q in range(5))
        assert abs(poly - E.objective(V + s * D, i, j, d, w, lam)) <= 1e-9 * (1 + abs(poly))
    V2, F = E.bm_phase(V, i, j, d, w, lam, 6)
    assert all(b <= a * (1 + 1e-12) + 1e-12 for a, b in zip(F, F[1:]))
    assert np.abs(V2.sum(axis=0)).max() <= 1e-9


def test_bm_phase_is_pr_plus_cg_with_exact_steps():
    """The BM phase's iterates (calls of 1 ... 6 epochs from one centred start)
    against the definition of Polak-Ribiere+ CG with an exact line search on
    g(V) = f(V V^T) + lam ||V||^2, by central differences of E.objective and
    brute-force steps (tests/cg_pin.py).  On this chain one step has a
    negative Polak-Ribiere ratio (PR+ restarts there) and others tell the
    Polak-Ribiere ratio from the Fletcher-Reeves one."""
    n = 10
    p, i, j, d, w = _chain(n, 3)
    lam = O.edm_lambda(n, d)
    V0 = E.center(np.random.default_rng(3).standard_normal((n, 2)))
    xs = [V0.ravel()]
    for e in range(1, 7):
        V, _ = E.bm_phase(V0, i, j, d, w, lam, e)
        xs.append(V.ravel())
    restarts, fr_apart = check_pr_plus(xs, lambda v: E.objective(v.reshape(n, 2), i, j, d, w, lam))
    assert restarts >= 1 and fr_apart >= 1


def test_lipschitz_bound_dominates_the_operator_norm():
    p, i, j, d, w = _chain(30, 12)
    n = p.n
    w = np.random.default_rng(3).uniform(0.5, 2.0, i.shape[0])
    # A(X)_p = sqrt(w_p) <E_p, X>: ||A* A|| = lambda_max of the Gram of sqrt(w_p) vec(E_p)
    rows = []
    for a, b, ww in zip(i, j, w):
        e = np.zeros(n)
        e[a], e[b] = 1.0, -1.0
        rows.append(np.sqrt(ww) * np.outer(e, e).ravel())
    M = np.array(rows)
    exact = np.linalg.eigvalsh(M @ M.T).max()
    bound = E.lipschitz(n, i, j, w)
    assert bound >= exact * (1 - 1e-12)
    assert bound <= 4.0 * exact


def test_lipschitz_bound_is_exact_for_disjoint_pairs():
    """Pairs without a common point have orthogonal E_p (<E_p, E_q> = ((e_i - e_j)^T
    (e_k - e_l))^2 = 0), so the Gram of sqrt(w_p) vec(E_p) is diagonal with
    entries ||E_p||_F^2 w_p = 4 w_p: ||A* A|| = 4 max w, which the bound must equal."""
    n = 12
    i = np.arange(0, n, 2)
    j = np.arange(1, n, 2)
    w = np.random.default_rng(5).uniform(0.5, 2.0, i.shape[0])
    assert E.lipschitz(n, i, j, w) == pytest.approx(4.0 * w.max(), rel=1e-14)


def test_shift_makes_the_operator_positive_semidefinite():
    """sigma bounds the negative part of Z = V V^T - alpha L_{w r} - alpha lam J,
    so Z + sigma I is positive semidefinite (dense eigenvalues).  The case is
    one stretched pair: x = (e_0 - e_1)/sqrt(2) gives x^T Z x = D/2 - 2c for
    D = ||v_0 - v_1||^2 and c = alpha (D - d^2), so with d^2 = D/10 the
    smallest eigenvalue is below -1.3 D while sigma = 2c = 1.8 D: half of the
    bound would not do."""
    n = 6
    rng = np.random.default_rng(6)
    V = 0.05 * rng.standard_normal((n, 2))
    V[0], V[1] = [1.0, 0.0], [-1.0, 0.0]
    V = E.center(V)
    Dist = float(np.sum((V[0] - V[1]) ** 2))
    i, j, d, w = E.pair_arrays([0], [1], [np.sqrt(0.1 * Dist)], 1.0)
    Zop = E.z_operator(V, i, j, d, w, 0.0, 1.0)
    Z = Zop.z(np.eye(n))
    ev = np.linalg.eigvalsh(0.5 * (Z + Z.T))
    assert ev.min() <= -1.3 * Dist
    assert ev.min() + Zop.sigma >= -1e-12 * Zop.sigma
    assert ev.min() + 0.5 * Zop.sigma < 0


def test_rank_rule_of_the_qsdp_experiments():
    """Supplement, QSDP implementation details: if every computed eigenvalue is
    positive the next step computes k + floor(n / 20) of them (capped at
    k_max here), otherwise as many as were positive; the new factor keeps the
    positive pairs, V = U_+ diag(sqrt(mu_+))."""
    n, k = 100, 5
    U = np.linalg.qr(np.random.default_rng(7).standard_normal((n, k)))[0]
    V, rank, k_next = E.prox_from_eig(U, np.array([5.0, 4.0, 3.0, 2.0, 1.0]), k, 40, n)
    assert (rank, k_next) == (5, 10)
    assert np.allclose(V, U * np.sqrt([5.0, 4.0, 3.0, 2.0, 1.0]))
    assert E.prox_from_eig(U, np.array([5.0, 4.0, 3.0, 2.0, 1.0]), k, 8, n)[2] == 8
    V, rank, k_next = E.prox_from_eig(U, np.array([3.0, 2.0, 0.0, -1.0, -2.0]), k, 40, n)
    assert (rank, k_next) == (2, 2)
    assert np.allclose(V, U[:, :2] * np.sqrt([3.0, 2.0]))


@pytest.mark.parametrize("n, k0", [(20, 3), (40, 6)])
def test_initial_rank_is_fifteen_percent_of_n(n, k0):
    """Supplement, QSDP implementation details: k_0 = min(100, floor(0.15 n))
    eigenpairs in the initial step."""
    p, i, j, d, w = _chain(n, 14)
    lam = O.edm_lambda(n, d)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    _, info = E.init_step(n, i, j, d, w, lam, alpha, 50, O.Options())
    assert info.mu.shape[0] == k0


def test_solve_cycle_is_bm_phase_then_pg_step_with_alpha_one_over_l():
    """Algorithm 1 on the QSDP (supplement, implementation details): each cycle
    runs the BM phase from W_t, then one inexact PG step with the fixed step
    alpha = 1/L from its result."""
    n = 20
    p, i, j, d, w = _chain(n, 15)
    lam = O.edm_lambda(n, d)
    opt = O.Options()
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    st0, _ = E.init_step(n, i, j, d, w, lam, alpha, 10, opt)
    V, _ = E.bm_phase(st0.V, i, j, d, w, lam, opt.bm_epochs)
    st1, _ = E.prox_step(E.EdmState(V=V, U=st0.U, k_eig=st0.k_eig, t=st0.t), i, j, d, w, lam, alpha, 10, opt)
    _, F, _ = E.solve(n, i, j, d, w, lam, 10, opt, max_outer=1, tol=0.0)
    assert F[1] == E.objective(st1.V, i, j, d, w, lam)


def test_pg_step_equals_dense_exact_projection():
    p, i, j, d, w = _chain(40, 13)
    n = p.n
    lam = O.edm_lambda(n, d)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    rng = np.random.default_rng(4)
    V = E.center(p.X_true @ rng.standard_normal((3, 5)) * 0.7)
    V, _ = E.bm_phase(V, i, j, d, w, lam, 4)
    X = V @ V.T
    Xd = E.dense_project(X - alpha * (E.dense_grad_f(X, i, j, d, w) + lam * np.eye(n)))
    rpos = int(np.sum(np.linalg.eigvalsh(Xd) > 1e-9 * np.abs(Xd).max()))
    opt = O.Options(lmsvd_tol=1e-14, lmsvd_imax=400)
    st = E.EdmState(V=V, U=np.zeros((n, 0)), k_eig=rpos + 3)
    st2, info = E.prox_step(st, i, j, d, w, lam, alpha, 40, opt)
    assert info.rank == rpos
    Xn = st2.V @ st2.V.T
    assert np.linalg.norm(Xn - Xd) <= 1e-7 * np.linalg.norm(Xd)


def test_solve_reaches_the_dense_convex_optimum():
    n = 30
    p, i, j, d, w = _chain(n, 17)
    lam = O.edm_lambda(n, d)
    X_star, F_star = E.dense_solve(n, i, j, d, w, lam)
    st, F, ranks = E.solve(n, i, j, d, w, lam, 30, O.Options(lmsvd_tol=1e-12, lmsvd_imax=200),
                           max_outer=300, tol=1e-14)
    assert abs(F[-1] - F_star) <= 1e-6 * abs(F_star)
    ev = np.linalg.eigvalsh(X_star)
    assert ranks[-1] == int(np.sum(ev > 1e-6 * ev.max()))
    assert np.abs(st.V.sum(axis=0)).max() <= 1e-8


def test_warm_start_fills_from_the_counter_stream_of_the_step():
    """With no previous vectors the warm start of step t is the centred
    Gaussian block of counter stream 2000 + t, orthonormalised."""
    n, k, t = 15, 4, 3
    st = E.EdmState(V=np.zeros((n, 0)), U=np.zeros((n, 0)), k_eig=k, t=t)
    Q = E.warm_start(st, n, k, 0, t)
    G = O.counter_normal(0, 2000 + t, n * k).reshape(k, n).T
    G = G - G.mean(axis=0)
    P = Q @ Q.T
    assert Q.shape == (n, k)
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e-12
    assert np.linalg.norm(G - P @ G) <= 1e-10 * np.linalg.norm(G)


def test_initial_eigenvectors_stay_orthogonal_to_e():
    """Lemma "PiX": X+ = P_S+(J Z J) lives on ker(e^T), and the initial step
    starts from centred Gaussians, so every computed eigenvector is orthogonal
    to e, also when some of the k_0 leading eigenvalues are not positive
    (lambda > 0, the kernel-estimation sign, where e's eigenvalue 0 of Z would
    otherwise compete)."""
    n = 40
    p, i, j, d, w = _chain(n, 16)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    lam = 50.0 * float(np.max(d * d))
    st, info = E.init_step(n, i, j, d, w, lam, alpha, 20, O.Options(lmsvd_tol=1e-12, lmsvd_imax=300))
    assert np.min(info.mu) <= 0.0
    assert np.abs(st.U.T @ np.ones(n)).max() <= 1e-9


def test_large_lambda_gives_the_zero_solution():
    """For lam above the largest eigenvalue of sum w d^2 E_ij the initial Z_{-1}
    = alpha (L_{w d^2} - lam J) is negative semidefinite on ker(e^T), so X_0 = 0,
    and X = 0 is optimal (f's gradient at 0 is -L_{w d^2}, and lam <I, .> beats
    it on the feasible set): rank 0 and F = 1/2 sum w d^4 throughout."""
    import warnings
    n = 12
    p, i, j, d, w = _chain(n, 18)
    Ld = E.laplacian_apply(n, i, j, w * d * d, np.eye(n))
    lam = 1.5 * float(np.linalg.eigvalsh(Ld).max())
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        st, F, ranks = E.solve(n, i, j, d, w, lam, 6, O.Options(), max_outer=5)
    assert st.V.shape[1] == 0 and all(r == 0 for r in ranks)
    assert F[-1] == pytest.approx(0.5 * float(np.sum(w * d ** 4)), rel=1e-14)


def test_dense_reference_gradient_and_optimality():
    """The dense references themselves: dense_grad_f against central
    differences of dense_objective's smooth part (symmetric perturbations
    E_ab + E_ba), and dense_solve's result is a fixed point of the projected
    gradient map X = P_X(X - alpha (grad f(X) + lam I)), which for the convex
    QSDP is its optimality condition (P_X pinned by the variational-inequality
    test above)."""
    n = 30
    p, i, j, d, w = _chain(n, 17)
    lam = O.edm_lambda(n, d)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((n, n))
    X = A @ A.T / n
    G = E.dense_grad_f(X, i, j, d, w)
    h = 1e-6
    for a, b in ((0, 1), (3, 3), (5, 17), (29, 2)):
        D = np.zeros((n, n))
        D[a, b] += 1.0
        D[b, a] += 1.0
        fp = E.dense_objective(X + h * D, i, j, d, w, 0.0)
        fm = E.dense_objective(X - h * D, i, j, d, w, 0.0)
        assert abs((fp - fm) / (2 * h) - float(np.sum(G * D))) <= 1e-6 * (1 + abs(float(np.sum(G * D))))
    X_star, F_star = E.dense_solve(n, i, j, d, w, lam)
    alpha = 1.0 / E.lipschitz(n, i, j, w)
    step = E.dense_project(X_star - alpha * (E.dense_grad_f(X_star, i, j, d, w) + lam * np.eye(n)))
    assert np.linalg.norm(step - X_star) <= 1e-7 * np.linalg.norm(X_star)
    assert F_star == pytest.approx(E.dense_objective(X_star, i, j, d, w, lam), rel=1e-14)
