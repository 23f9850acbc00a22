"""Plain FP64 CPU oracle for the SpaRSA variant of the inexact PG step
(supplement Sec. "The SpaRSA variant for Matrix Completion").

TEST INFRASTRUCTURE ONLY, under the same rules as ``bm_oracle``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm
of ``bench.py`` may import it; the library never does.

The step size of the PG step at X~_t = W_t H_t^T is chosen per step instead of
fixed:

  * Barzilai-Borwein initial value (Eq. "proxBB"), clipped to
    [alpha_min, alpha_max], from X_t = X~_t and X_{t-1} = X~_{t-1} (the last
    two points where the PG step was taken).  The printed ratio
    <dX, dG> / ||dX||^2 is a curvature (an inverse step length); as a step
    size its reciprocal is used:  alpha_BB = ||dX||_F^2 / <dX, dG>.  For
    f = 1/2 ||P_Omega(X - A)||^2, dG = P_Omega(dX), so <dX, dG> =
    ||r_t - r_{t-1}||^2 (residuals on Omega); <dX, dG> = 0 gives alpha_max.
  * ||dX||_F^2 from the factors (Eq. "trace", with the sign of its last term
    corrected and the factor 2 restored):
    tr(W_t^T W_t H_t^T H_t) + tr(W_{t-1}^T W_{t-1} H_{t-1}^T H_{t-1})
    - 2 tr((W_{t-1}^T W_t)(H_t^T H_{t-1})).
  * Backtracking: the smallest i >= 0 such that alpha = alpha_BB beta^i gives
    an X_{t+1} satisfying Eq. "back" or Eq. "decrease", with Q of
    Eq. "proxgrad":  Q(Y) = <grad f(X~), Y - X~> + ||Y - X~||^2 / (2 alpha)
    + lam (||Y||_* - ||X~||_*).  On Omega, Y - X~ = r(Y) - r(X~), so
    <grad f(X~), Y - X~> = <r~, r(Y) - r~>.  At most max_backtracks
    reductions; if none is accepted the last trial is kept (flag 0).
  * The first PG step (no previous point) starts from opt.alpha, clipped
    to [alpha_min, alpha_max] like every initial value.

Readings (the paper gives no values): alpha_min = 1e-3, alpha_max = 1e3,
beta = 0.5, delta = 0.995 (with L = 1, the fixed step alpha = 1.99 satisfies
Eq. "back" exactly when delta >= alpha / 2), max_backtracks = 30.

Parity status: pinned by tests/test_oracle_sparsa.py (Eq. "trace" and the
nuclear norm against dense evaluations, <dX, dG> against the dense gradient
difference, the full-observation case alpha_BB = 1, the acceptance tests
re-evaluated densely with the flag naming the test that held and the trial
one reduction earlier failing both, alpha_BB from the two points where the
PG steps were taken and the first step's fixed alpha, no backtracking when
alpha_max <= 1/L, and the soft-impute optimum reached by the SpaRSA solve).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from oracle import bm_oracle as O


@dataclasses.dataclass
class BbOptions:
    alpha_min: float = 1e-3
    alpha_max: float = 1e3
    beta: float = 0.5
    delta: float = 0.995
    max_backtracks: int = 30


@dataclasses.dataclass
class BbPoint:
    """X~_{t-1} = W H^T and its residual on Omega (CSR order)."""
    W: np.ndarray
    H: np.ndarray
    r: np.ndarray


@dataclasses.dataclass
class BbInfo:
    alpha_bb: float      # Eq. "proxBB" value (before backtracking)
    alpha: float         # accepted step
    backtracks: int
    accepted_by: int     # 1: Eq. "back", 2: Eq. "decrease" (only), 0: none within max_backtracks


def frob_diff2(W1, H1, W0, H0) -> float:
    """||W1 H1^T - W0 H0^T||_F^2 from k x k Grams (Eq. "trace", corrected)."""
    t11 = float(np.sum((W1.T @ W1) * (H1.T @ H1)))
    t00 = float(np.sum((W0.T @ W0) * (H0.T @ H0)))
    t01 = float(np.sum((W0.T @ W1) * (H0.T @ H1)))
    return t11 + t00 - 2.0 * t01


def nuclear_norm(W, H) -> float:
    """||W H^T||_*: with W = Q_W R_W, the singular values of W H^T are those of
    H R_W^T (an n x k matrix), the square roots of eig(R_W H^T H R_W^T)."""
    if W.shape[1] == 0:
        return 0.0
    _, Rw = np.linalg.qr(W)
    S = Rw @ (H.T @ H) @ Rw.T
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    return float(np.sum(np.sqrt(np.maximum(ev, 0.0))))


def bb_alpha(W, H, r, prev: Optional[BbPoint], o: BbOptions, alpha0: float) -> float:
    if prev is None:
        a = alpha0
    else:
        num = frob_diff2(W, H, prev.W, prev.H)
        dr = r - prev.r
        den = float(dr @ dr)
        a = o.alpha_max if den <= 0 else num / den
    return max(o.alpha_min, min(o.alpha_max, a))


def prox_step_bb(ix: O.Index, st: O.State, lam: float, k_max: int, opt: O.Options, o: BbOptions,
                 prev: Optional[BbPoint]):
    """One PG step with the SpaRSA step rule.  Returns (state, ProxInfo,
    BbInfo, BbPoint of X~_t for the next call)."""
    r = O.residual(ix, st.W, st.H)
    f = 0.5 * float(r @ r)
    nuc = nuclear_norm(st.W, st.H)
    F0 = f + lam * nuc
    a0 = bb_alpha(st.W, st.H, r, prev, o, opt.alpha)
    out = None
    for i in range(o.max_backtracks + 1):
        a = a0 * o.beta ** i
        st1, info = O.prox_step(ix, st, lam, k_max, opt, alpha=a)
        r1 = O.residual(ix, st1.W, st1.H)
        f1 = 0.5 * float(r1 @ r1)
        lin = float(r @ (r1 - r))
        d2 = frob_diff2(st1.W, st1.H, st.W, st.H)
        back = f1 <= f + lin + o.delta / a * d2
        F1 = f1 + lam * float(np.sum(info.sigma))
        Q = lin + d2 / (2.0 * a) + lam * (float(np.sum(info.sigma)) - nuc)
        dec = F1 <= F0 + o.delta * Q
        out = (st1, info, BbInfo(a0, a, i, 1 if back else (2 if dec else 0)))
        if back or dec:
            break
    st1, info, bb = out
    return st1, info, bb, BbPoint(st.W.copy(), st.H.copy(), r)


def solve_bb(ix: O.Index, lam: float, k_init: int, k_max: int, opt: O.Options = O.Options(),
             o: BbOptions = BbOptions(), max_outer: int = 100, tol: float = 1e-10,
             F_target: Optional[float] = None):
    """Algorithm 1 with the SpaRSA PG step: the initial PG step from 0, then
    cycles of bm_epochs BM iterations and pg_steps PG steps."""
    st, info0 = O.init_step(ix, lam, k_init, k_max, opt)
    F_hist = [O.objective(ix, st.W, st.H, lam)]
    bb_hist = []
    prev = None
    for _ in range(max_outer):
        st, _ = O.bm_phase(ix, st, lam, opt.bm_epochs)
        for _ in range(opt.pg_steps):
            st, info, bb, prev = prox_step_bb(ix, st, lam, k_max, opt, o, prev)
            bb_hist.append(bb)
        F = O.objective(ix, st.W, st.H, lam)
        F_hist.append(F)
        if F_target is not None and F <= F_target:
            break
        if abs(F_hist[-2] - F) / (1.0 + abs(F_hist[-2])) < tol:
            break
    return st, F_hist, bb_hist


def dense_check(ix: O.Index, st: O.State, st1: O.State, lam: float, alpha: float, delta: float):
    """Eq. "back" and Eq. "decrease" evaluated with dense matrices (small
    problems only): returns (back holds, decrease holds)."""
    m, n = ix.m, ix.n
    A = np.zeros((m, n))
    mask = np.zeros((m, n), dtype=bool)
    rows = ix.rows_of_entries()
    A[rows, ix.col] = ix.val
    mask[rows, ix.col] = True
    X0 = st.W @ st.H.T
    X1 = st1.W @ st1.H.T
    G = np.where(mask, X0 - A, 0.0)
    f0 = 0.5 * float(np.sum(G * G))
    R1 = np.where(mask, X1 - A, 0.0)
    f1 = 0.5 * float(np.sum(R1 * R1))
    D = X1 - X0
    lin = float(np.sum(G * D))
    d2 = float(np.sum(D * D))
    nuc0 = float(np.sum(np.linalg.svd(X0, compute_uv=False)))
    nuc1 = float(np.sum(np.linalg.svd(X1, compute_uv=False)))
    back = f1 <= f0 + lin + delta / alpha * d2 + 1e-9 * (1 + abs(f0))
    Q = lin + d2 / (2 * alpha) + lam * (nuc1 - nuc0)
    dec = f1 + lam * nuc1 <= f0 + lam * nuc0 + delta * Q + 1e-9 * (1 + abs(f0))
    return back, dec
