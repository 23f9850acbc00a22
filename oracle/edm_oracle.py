"""Plain FP64 CPU oracle for BM-Global on the distance-geometry QSDP.

TEST INFRASTRUCTURE ONLY, under the same rules as ``bm_oracle``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm
of ``bench.py`` may import it; the library never does.

Problem (Eq. "QSDP", the molecular-conformation / kernel-estimation form):

    min  f(X) + lam <I, X>,  f(X) = 1/2 sum_{(i,j) in Omega} w_ij (X_ii + X_jj - 2 X_ij - d_ij^2)^2
    s.t. X positive semidefinite, <E, X> = 0  (E = e e^T),

factored as X = V V^T with V^T e = 0 (Eq. "EDM"); <E_ij, V V^T> = ||v_i - v_j||^2.
Algorithm 1 here:

  * BM phase: Polak-Ribiere+ directions on g(V) = f(V V^T) + lam ||V||^2
    (gradient 2 (L_{w r} + lam I) V with L_c = sum_{(i,j)} c_ij E_ij) and the
    exact line search on the quartic g(V + s D); the centring V^T e = 0 is
    kept because every gradient and direction has columns summing to zero.
  * PG step (Eq. "inexactpg" with Psi = lam <I, .> + delta_X): by Lemma
    "PiX" and Eq. "proxsym", X+ = P_S+(J (X~ - alpha grad f(X~) - alpha lam I) J)
    = P_S+(Z), Z = V V^T - alpha L_{w r} - alpha lam J, J = I - e e^T / n.  The
    leading eigenpairs of Z come from the LmSVD iteration (Algorithm 2) on the
    shifted operator Z + sigma J (positive semidefinite, equal to Z + sigma I
    on ker(e^T) and 0 along e, so its leading eigenvectors are those of the
    largest eigenvalues of Z on ker(e^T)); X+ keeps the positive part,
    V+ = U diag(sqrt(mu_+)).

Readings (each also in the design notes):
  * alpha = 1/L with L the Gershgorin bound of ||A* A||: the Gram of the
    E_ij under <.,.> has 4 w_p on the diagonal and sqrt(w_p w_q) where pairs
    p, q share one point, so L = max_p 4 w_p + sqrt(w_p) (S_i + S_j - 2 sqrt(w_p)),
    S_v = sum of sqrt(w) over the pairs at v;
  * sigma = alpha (max_v 2 sum_{pairs at v} w |r| + max(lam, 0)), the
    Gershgorin bound of the negative part of Z;
  * rank rule (Sec. "Implementation details" of the QSDP experiments): k
    eigenpairs are computed; if all are positive the next step computes
    k + floor(n / 20) (capped at k_max), otherwise the number of positive ones;
  * warm start: orth([U_t, V]) completed with counter-generator Gaussian
    columns (stream 2000 + t) projected off e, to the k of the rank rule;
  * initial point: one PG step from X = 0 (the paper runs APG there): Z_{-1} =
    alpha sum w d^2 E_ij - alpha lam J, k_0 = min(100, floor(0.15 n)),
    started from Gaussian columns (stream 1) projected off e.

Parity status: pinned by tests/test_oracle_edm_solve.py (Lemma "PiX" through
projection optimality, the dense exact PG step, the line-search quartic,
monotone BM phase, the BM phase's iterates against the definition of
Polak-Ribiere+ CG with exact steps, the Lipschitz bound exact for disjoint
pairs, Z + sigma I positive semidefinite where half of sigma is not, the
rank rule and initial rank of the QSDP experiments, the cycle order and
alpha = 1/L, and the dense convex optimum of the QSDP).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from oracle import bm_oracle as O

STREAM_EDM_INIT = 1
STREAM_EDM_FILL = 2000


def pair_arrays(i, j, d, w):
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    d = np.asarray(d, dtype=np.float64)
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), i.shape).copy()
    return i, j, d, w


def residual(V, i, j, d):
    """r_ij = <E_ij, V V^T> - d_ij^2 = ||v_i - v_j||^2 - d_ij^2."""
    diff = V[i] - V[j]
    return np.sum(diff * diff, axis=1) - d * d


def objective(V, i, j, d, w, lam):
    """g(V) = f(V V^T) + lam <I, V V^T> (Eq. "EDM")."""
    r = residual(V, i, j, d)
    return 0.5 * float(np.sum(w * r * r)) + lam * float(np.sum(V * V))


def laplacian_apply(n, i, j, c, U):
    """(sum_{(i,j)} c_ij E_ij) U: row i gains c (u_i - u_j), row j loses it."""
    D = c[:, None] * (U[i] - U[j])
    out = np.zeros((n, U.shape[1]))
    np.add.at(out, i, D)
    np.add.at(out, j, -D)
    return out


def gradient(V, i, j, d, w, lam):
    r = residual(V, i, j, d)
    return 2.0 * laplacian_apply(V.shape[0], i, j, w * r, V) + 2.0 * lam * V


def lipschitz(n, i, j, w):
    """Gershgorin bound of ||A* A|| (see the module notes)."""
    sw = np.sqrt(w)
    S = np.zeros(n)
    np.add.at(S, i, sw)
    np.add.at(S, j, sw)
    return float(np.max(4.0 * w + sw * (S[i] + S[j] - 2.0 * sw)))


def center(U):
    return U - U.mean(axis=0, keepdims=True)


# ---------------------------------------------------------------------------
# BM phase
# ---------------------------------------------------------------------------
def line_search_coeffs(V, D, i, j, d, w, lam):
    """g(V + s D) = c0 + c1 s + c2 s^2 + c3 s^3 + c4 s^4: with a = 2 <v_i - v_j,
    D_i - D_j>, b = ||D_i - D_j||^2 the residual moves as r + a s + b s^2."""
    r = residual(V, i, j, d)
    dv = V[i] - V[j]
    dd = D[i] - D[j]
    a = 2.0 * np.sum(dv * dd, axis=1)
    b = np.sum(dd * dd, axis=1)
    c = np.zeros(5)
    c[0] = 0.5 * np.sum(w * r * r) + lam * np.sum(V * V)
    c[1] = np.sum(w * r * a) + 2.0 * lam * np.sum(V * D)
    c[2] = 0.5 * np.sum(w * (a * a + 2.0 * r * b)) + lam * np.sum(D * D)
    c[3] = np.sum(w * a * b)
    c[4] = 0.5 * np.sum(w * b * b)
    return c


def bm_phase(V, i, j, d, w, lam, epochs):
    """Polak-Ribiere+ with the exact quartic line search; returns (V, F list)."""
    F = [objective(V, i, j, d, w, lam)]
    g_prev = D = None
    for _ in range(epochs):
        g = gradient(V, i, j, d, w, lam)
        if g_prev is None:
            D = -g
        else:
            beta = max(0.0, float(np.sum(g * (g - g_prev))) / max(float(np.sum(g_prev * g_prev)), 1e-300))
            D = -g + beta * D
            if float(np.sum(D * g)) >= 0:
                D = -g
        c = line_search_coeffs(V, D, i, j, d, w, lam)
        s = O.quartic_argmin(c)
        if s > 0:
            V = V + s * D
        F.append(objective(V, i, j, d, w, lam))
        g_prev = g
    return V, F


# ---------------------------------------------------------------------------
# PG step
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class ZOperator:
    """Z = V V^T - alpha L_{w r} - alpha lam J and its shift sigma."""
    V: np.ndarray
    c: np.ndarray          # alpha * w * r per pair
    alpha: float
    lam: float
    sigma: float
    i: np.ndarray
    j: np.ndarray

    def z(self, U):
        n = U.shape[0]
        return (self.V @ (self.V.T @ U) - laplacian_apply(n, self.i, self.j, self.c, U)
                - self.alpha * self.lam * center(U))

    def zs(self, U):
        """(Z + sigma J) U: sigma I on ker(e^T), where X+ lives (Lemma "PiX"),
        and 0 along e, so that rounding along e is not amplified (with
        sigma I, e would carry the eigenvalue sigma, above every other one
        once lam > 0 pushes the spectrum on ker(e^T) below zero)."""
        return self.z(U) + self.sigma * center(U)


def z_operator(V, i, j, d, w, lam, alpha):
    n = V.shape[0]
    r = residual(V, i, j, d) if V.shape[1] else -d * d
    c = alpha * w * r
    rowabs = np.zeros(n)
    np.add.at(rowabs, i, np.abs(c))
    np.add.at(rowabs, j, np.abs(c))
    sigma = 2.0 * float(np.max(rowabs)) + alpha * max(lam, 0.0)
    return ZOperator(V, c, alpha, lam, sigma, i, j)


@dataclasses.dataclass
class EdmState:
    V: np.ndarray
    U: np.ndarray           # eigenvectors of the last PG step
    k_eig: int              # eigenpairs the next PG step computes
    t: int = 0


@dataclasses.dataclass
class EdmProxInfo:
    mu: np.ndarray          # computed eigenvalues of Z, descending
    rank: int
    k_eig_next: int
    iters: int


def top_eigpairs(Zop: ZOperator, U0, k, opt: O.Options):
    """Leading k eigenpairs of Z from LmSVD (Algorithm 2) on Z + sigma J."""
    Uh, theta, iters, _ = O.lmsvd(Zop.zs, U0, p=opt.lmsvd_p, tol=opt.lmsvd_tol, imax=opt.lmsvd_imax,
                                  tau=opt.tau, min_iter=opt.lmsvd_min_iter)
    kk = min(k, Uh.shape[1])
    return Uh[:, :kk], theta[:kk] - Zop.sigma, iters


def prox_from_eig(U, mu, k_eig, k_max, n):
    pos = mu > 0
    rank = int(np.sum(pos))
    Vn = U[:, pos] * np.sqrt(mu[pos])
    if rank == len(mu):
        k_next = min(k_max, k_eig + n // 20)
    else:
        k_next = max(1, rank)
    return Vn, rank, k_next


def warm_start(st: EdmState, n, k, seed, t):
    blocks = [b for b in (st.U, st.V) if b.shape[1]]
    M = np.hstack(blocks) if blocks else np.zeros((n, 0))
    Q = np.zeros((n, 0))
    if M.shape[1]:
        Q, _ = O.orth(center(M), max_cols=k)
    if Q.shape[1] < k:
        extra = k - Q.shape[1]
        G = O.counter_normal(seed, STREAM_EDM_FILL + t, n * extra).reshape(extra, n).T
        Q2, _ = O.orth(center(G), F=Q if Q.shape[1] else None)
        Q = np.hstack([Q, Q2])
    return Q[:, :k]


def prox_step(st: EdmState, i, j, d, w, lam, alpha, k_max, opt: O.Options):
    n = st.V.shape[0]
    Zop = z_operator(st.V, i, j, d, w, lam, alpha)
    U0 = warm_start(st, n, st.k_eig, opt.seed, st.t)
    U, mu, iters = top_eigpairs(Zop, U0, st.k_eig, opt)
    Vn, rank, k_next = prox_from_eig(U, mu, st.k_eig, k_max, n)
    return EdmState(V=Vn, U=U, k_eig=k_next, t=st.t + 1), EdmProxInfo(mu, rank, k_next, iters)


def init_step(n, i, j, d, w, lam, alpha, k_max, opt: O.Options):
    """One PG step from X = 0: Z_{-1} = alpha sum w d^2 E_ij - alpha lam J."""
    k0 = max(1, min(100, int(0.15 * n), k_max))
    V0 = np.zeros((n, 0))
    Zop = z_operator(V0, i, j, d, w, lam, alpha)
    G = O.counter_normal(opt.seed, STREAM_EDM_INIT, n * k0).reshape(k0, n).T
    U, mu, iters = top_eigpairs(Zop, center(G), k0, opt)
    Vn, rank, k_next = prox_from_eig(U, mu, k0, k_max, n)
    return EdmState(V=Vn, U=U, k_eig=k_next, t=0), EdmProxInfo(mu, rank, k_next, iters)


def solve(n, i, j, d, w, lam, k_max, opt: O.Options = O.Options(), max_outer=100, tol=1e-10):
    """Algorithm 1 on the QSDP: initial PG step, then cycles of bm_epochs BM
    iterations and one PG step with alpha = 1/L."""
    i, j, d, w = pair_arrays(i, j, d, w)
    alpha = 1.0 / lipschitz(n, i, j, w)
    st, _ = init_step(n, i, j, d, w, lam, alpha, k_max, opt)
    F = [objective(st.V, i, j, d, w, lam)]
    ranks = [st.V.shape[1]]
    for _ in range(max_outer):
        V, _ = bm_phase(st.V, i, j, d, w, lam, opt.bm_epochs)
        st = EdmState(V=V, U=st.U, k_eig=st.k_eig, t=st.t)
        st, info = prox_step(st, i, j, d, w, lam, alpha, k_max, opt)
        F.append(objective(st.V, i, j, d, w, lam))
        ranks.append(info.rank)
        if abs(F[-2] - F[-1]) / (1.0 + abs(F[-2])) < tol:
            break
    return st, F, ranks


# ---------------------------------------------------------------------------
# Dense references (small n only): the exact projection of Lemma "PiX" and
# the convex optimum by dense projected-gradient iterations.
# ---------------------------------------------------------------------------
def dense_project(G):
    """P_X(G) = P_S+(J G J) (Lemma "PiX")."""
    n = G.shape[0]
    J = np.eye(n) - np.ones((n, n)) / n
    S = J @ (0.5 * (G + G.T)) @ J
    lam_, E = np.linalg.eigh(S)
    lp = np.maximum(lam_, 0.0)
    return (E * lp) @ E.T


def dense_grad_f(X, i, j, d, w):
    r = X[i, i] + X[j, j] - 2.0 * X[i, j] - d * d
    n = X.shape[0]
    G = np.zeros((n, n))
    c = w * r
    np.add.at(G, (i, i), c)
    np.add.at(G, (j, j), c)
    np.add.at(G, (i, j), -c)
    np.add.at(G, (j, i), -c)
    return G


def dense_objective(X, i, j, d, w, lam):
    r = X[i, i] + X[j, j] - 2.0 * X[i, j] - d * d
    return 0.5 * float(np.sum(w * r * r)) + lam * float(np.trace(X))


def dense_solve(n, i, j, d, w, lam, iters=200000, tol=1e-9):
    """Accelerated projected gradient (Beck and Teboulle 2009) with adaptive
    restart on objective increase (O'Donoghue and Candes 2015), from X = 0:
    X+ = P_X(Y - alpha (grad f(Y) + lam I)); stops when the step
    ||X+ - X||_F <= tol (1 + ||X||_F)."""
    i, j, d, w = pair_arrays(i, j, d, w)
    alpha = 1.0 / lipschitz(n, i, j, w)
    X = np.zeros((n, n))
    Y = X.copy()
    t = 1.0
    F = dense_objective(X, i, j, d, w, lam)
    for _ in range(iters):
        Xn = dense_project(Y - alpha * (dense_grad_f(Y, i, j, d, w) + lam * np.eye(n)))
        Fn = dense_objective(Xn, i, j, d, w, lam)
        if Fn > F:            # restart the momentum
            Y, t = X.copy(), 1.0
            continue
        step = np.linalg.norm(Xn - X)
        tn = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        Y = Xn + ((t - 1.0) / tn) * (Xn - X)
        X, t, F = Xn, tn, Fn
        if step <= tol * (1.0 + np.linalg.norm(X)):
            break
    return X, F
