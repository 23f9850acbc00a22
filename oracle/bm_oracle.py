"""Plain FP64 CPU oracle for BM-Global on matrix completion.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import it; the library itself never does and shares no code
with it.

Everything here is float64 numpy, written to be read against the paper
(Lee, Liang, Tang & Toh, "Escaping spurious local minima of low-rank matrix
factorization through convex lifting", arXiv 2204.14067).  Library
primitives (sorting, dense/sparse matrix products, ``eigh``, ``roots``)
serve as single steps; there is no blocking or fusion.

Notation (paper): X = W H^T (W: m x k, H: n x k, m <= n after transpose),
Omega the observed set, A the observed values, R = P_Omega(X - A),
Z = X - alpha*R (Eq. "zt"), L(U) = Z Z^T U (Eq. "ZZ"/"ssi").

Readings taken where the paper leaves a choice (each also listed in the
design notes):
  * orth() is the eigen-based construction of Eq. "PUi"/"orth-W", applied
    to column-normalised blocks, dropping Gram eigenvalues <= tau, and
    applied twice (the second pass is the identity in exact arithmetic and
    restores orthogonality lost to rounding);
  * LmSVD (Algorithm 2) keeps the L-images of the stored blocks, so one
    application of L per iteration; it stops when the Ritz values change by
    at most tol * theta_1, and reports s = sqrt(theta) of the last
    Rayleigh-Ritz step;
  * the rank safeguard (Sec. "Ensuring sufficient precision") uses the
    explicit "or" trigger, reads R_t as the previous warm start U^{t-1,0},
    and draws xi_t from the SplitMix64/Box-Muller counter generator below;
  * the BM phase is the builder's own monotone solver: Polak-Ribiere+
    directions with an exact line search on the quartic phi(s) (the paper
    only requires the non-increase condition, Eq. "nonincrease").

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, finite differences, brute force, invariants);
tests/oracle_mutations.py plants plausible mistakes in a copy of this file
and the other oracles and checks that a pin catches each one.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# Counter-based generator for the random vectors the method draws
# (SplitMix64: Steele, Lea & Flood 2014; Box-Muller 1958).
# ---------------------------------------------------------------------------
_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1

STREAM_INIT_SKETCH = 1      # Gaussian U~^{-1,0} of the initial step (Sec. "Initialization")
STREAM_SAFEGUARD = 1000     # + t : xi_t of Eq. "rt"


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def counter_normal(seed: int, stream: int, count: int) -> np.ndarray:
    """count standard normals: key = mix64(seed*gamma + stream);
    u_i = ((mix64(key + i*gamma) >> 11) + 1) * 2^-53, i = 0..2*count-1;
    x_j = sqrt(-2 ln u_{2j}) cos(2 pi u_{2j+1})."""
    key = _mix64(np.array([(seed * _GAMMA + stream) & _M64], dtype=np.uint64))[0]
    ctr = np.arange(2 * count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(key + ctr * np.uint64(_GAMMA))
    u = ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u[0::2])) * np.cos(2.0 * math.pi * u[1::2])


# ---------------------------------------------------------------------------
# Omega: index structures (Sec. 1, definition of P_Omega; m <= n by transpose)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Index:
    m: int                 # internal rows (m <= n)
    n: int
    transposed: bool       # caller's matrix was n x m
    row_ptr: np.ndarray    # int64 [m+1]
    col: np.ndarray        # int32 [nnz], CSR order (row, col ascending)
    val: np.ndarray        # float64 [nnz], CSR order
    col_ptr: np.ndarray    # int64 [n+1]
    row: np.ndarray        # int32 [nnz], CSC order (col, row ascending)
    cval: np.ndarray       # float64 [nnz], CSC order
    csr2csc: np.ndarray    # int64 [nnz]: CSC position of CSR entry e
    csc2csr: np.ndarray    # int64 [nnz]: CSR position of CSC entry q

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def rows_of_entries(self) -> np.ndarray:
        return np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.row_ptr))

    def sparse(self, values: np.ndarray) -> sp.csr_matrix:
        """P_Omega-supported m x n matrix with the given CSR-ordered values."""
        return sp.csr_matrix((values, self.col.astype(np.int64), self.row_ptr), shape=(self.m, self.n))


def build_index(m: int, n: int, rows, cols, vals) -> Index:
    """Canonical CSR (sorted by (row, col)) and CSC (sorted by (col, row)) of Omega.

    Omega is a set (Sec. 1), so duplicate (i, j) pairs are rejected, as are
    out-of-range indices and non-finite values.  If m > n the matrix is
    stored transposed so that m <= n internally (Sec. 1).
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    if m < 1 or n < 1:
        raise ValueError("m and n must be >= 1")
    if rows.shape != cols.shape or rows.shape != vals.shape:
        raise ValueError("rows, cols, vals must have equal length")
    if rows.size and (rows.min() < 0 or rows.max() >= m or cols.min() < 0 or cols.max() >= n):
        raise ValueError("index out of range")
    if not np.all(np.isfinite(vals)):
        raise ValueError("non-finite value")
    transposed = m > n
    if transposed:
        m, n, rows, cols = n, m, cols, rows
    order = np.lexsort((cols, rows))
    r_s, c_s, a_s = rows[order], cols[order], vals[order]
    if r_s.size > 1:
        same = (r_s[1:] == r_s[:-1]) & (c_s[1:] == c_s[:-1])
        if np.any(same):
            raise ValueError("duplicate (row, col) entry")
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(r_s, minlength=m))
    csc2csr = np.lexsort((r_s, c_s))
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum(np.bincount(c_s, minlength=n))
    csr2csc = np.empty_like(csc2csr)
    csr2csc[csc2csr] = np.arange(csc2csr.shape[0])
    return Index(m, n, transposed, row_ptr, c_s.astype(np.int32), a_s, col_ptr,
                 r_s[csc2csr].astype(np.int32), a_s[csc2csr], csr2csc, csc2csr)


def value_codes(ix: Index):
    """One-byte encoding of the observed values (not part of the paper's
    method; it only changes how A is stored): when every a_e is an integer
    with |a_e| < 2^24 and max(a) - min(a) <= 255, a_e = code_e + offset with
    offset = min(a) and code_e in [0, 255].  Returns (offset, CSR codes, CSC
    codes) as uint8 arrays, or None when the values do not qualify."""
    v = ix.val
    if v.size == 0:
        return None
    if not np.all(v == np.rint(v)) or np.abs(v).max() >= 2.0 ** 24:
        return None
    lo, hi = float(v.min()), float(v.max())
    if hi - lo > 255:
        return None
    return lo, (ix.val - lo).astype(np.uint8), (ix.cval - lo).astype(np.uint8)


# ---------------------------------------------------------------------------
# Loss and gradient of (MF) / (BM-nuclear)
# ---------------------------------------------------------------------------
def residual(ix: Index, W: np.ndarray, H: np.ndarray) -> np.ndarray:
    """r_e = <W_i, H_j> - a_e for e = (i, j) in Omega, CSR order (Eq. "mc")."""
    ri = ix.rows_of_entries()
    if W.shape[1] == 0:
        return -ix.val.copy()
    return np.einsum("ek,ek->e", W[ri], H[ix.col]) - ix.val


def loss_grad(ix: Index, W: np.ndarray, H: np.ndarray, lam: float):
    """f = 1/2 ||P_Omega(W H^T - A)||^2, F = f + lam/2 (||W||^2 + ||H||^2) (Eq. "mf"),
    gW = R H + lam W, gH = R^T W + lam H.  Returns (f, F, gW, gH, r)."""
    r = residual(ix, W, H)
    f = 0.5 * float(r @ r)
    F = f + 0.5 * lam * (float(np.sum(W * W)) + float(np.sum(H * H)))
    R = ix.sparse(r)
    gW = R @ H + lam * W
    gH = R.T @ W + lam * H
    return f, F, np.asarray(gW), np.asarray(gH), r


def objective(ix: Index, W: np.ndarray, H: np.ndarray, lam: float) -> float:
    return loss_grad(ix, W, H, lam)[1]


# ---------------------------------------------------------------------------
# Small dense linear algebra
# ---------------------------------------------------------------------------
def eig_desc(S: np.ndarray):
    """Eigenpairs of a symmetric matrix, eigenvalues in descending order."""
    S = 0.5 * (S + S.T)
    w, V = np.linalg.eigh(S)
    return w[::-1].copy(), V[:, ::-1].copy()


def orth(M: np.ndarray, F: Optional[np.ndarray] = None, tau: float = 1e-6,
         LM: Optional[np.ndarray] = None, LF: Optional[np.ndarray] = None,
         max_cols: Optional[int] = None):
    """New orthonormal columns Q2 with ran([F, Q2]) = ran([F, M]) (Eq. "PUi", "orth-W").

    F (optional) has orthonormal columns.  Columns of M are scaled to unit
    norm, projected onto ker(F^T) (Eq. "PUi"); with P^T P = E Lam E^T the
    new columns are P E Lam^{-1/2} (Eq. "orth-W"), keeping eigenvalues > tau
    (at most max_cols of them, largest first).  A second pass repeats the
    projection and scaling.  If LM/LF (images of M/F under a linear map L)
    are given, the same coefficients produce L(Q2).  Returns (Q2, LQ2).
    """
    mrows = M.shape[0]
    s = np.sqrt(np.sum(M * M, axis=0))
    keep = s > 0
    Mh = M[:, keep] / s[keep]
    LMh = LM[:, keep] / s[keep] if LM is not None else None
    for pass_no in range(2):
        if F is not None and F.shape[1] > 0:
            C = F.T @ Mh
            Mh = Mh - F @ C
            if LMh is not None:
                LMh = LMh - LF @ C
        if Mh.shape[1] == 0:
            break
        lam_, E = eig_desc(Mh.T @ Mh)
        good = lam_ > tau
        if pass_no == 0 and max_cols is not None:
            good &= np.arange(lam_.shape[0]) < max_cols
        T = E[:, good] / np.sqrt(lam_[good])
        Mh = Mh @ T
        if LMh is not None:
            LMh = LMh @ T
    if Mh.shape[1] == 0:
        Mh = np.zeros((mrows, 0))
        LMh = np.zeros((mrows, 0)) if LM is not None else None
    return Mh, LMh


# ---------------------------------------------------------------------------
# The operator Z = W H^T - alpha R and L(U) = Z Z^T U (Eq. "zt", "ZZ")
# ---------------------------------------------------------------------------
class ZOperator:
    def __init__(self, ix: Index, W: np.ndarray, H: np.ndarray, r: np.ndarray, alpha: float):
        self.ix, self.W, self.H, self.alpha = ix, W, H, alpha
        self.R = ix.sparse(r)
        self.r = r
        self.n_L = 0

    def zt(self, U: np.ndarray) -> np.ndarray:
        """Z^T U = H (W^T U) - alpha R^T U   (n x q)."""
        return self.H @ (self.W.T @ U) - self.alpha * (self.R.T @ U)

    def z(self, Y: np.ndarray) -> np.ndarray:
        """Z Y = W (H^T Y) - alpha R Y   (m x q)."""
        return self.W @ (self.H.T @ Y) - self.alpha * (self.R @ Y)

    def L(self, U: np.ndarray) -> np.ndarray:
        self.n_L += 1
        return self.z(self.zt(U))

    def frob2(self) -> float:
        """||Z||_F^2 = <W^T W, H^T H> - 2 alpha <P_Omega(W H^T), R> + alpha^2 ||R||^2."""
        x = self.r + self.ix.val
        WtW = self.W.T @ self.W
        HtH = self.H.T @ self.H
        return float(np.sum(WtW * HtH) - 2.0 * self.alpha * (x @ self.r)
                     + self.alpha ** 2 * (self.r @ self.r))


# ---------------------------------------------------------------------------
# LmSVD (Algorithm 2) with L-images of the stored blocks
# ---------------------------------------------------------------------------
def lmsvd(Lop, U0: np.ndarray, p: int = 1, tol: float = 1e-6, imax: int = 50,
          tau: float = 1e-6, min_iter: int = 2):
    """Approximate leading eigenvectors of L = Z Z^T from the warm start U0.

    Iteration i: S = ran(U^{t,i}, ..., U^{t,i-p}) with U^{t,j} = orth(L(U^_{j-1}));
    orthonormal basis by Eq. "PUi"/"orth-W" with the newest block first;
    Rayleigh-Ritz on (Q, L(Q)) gives U^ (top k Ritz vectors, Eq. "lmsvd-opt").
    Stops when max |theta - theta_prev| <= tol*theta_1 (at least min_iter
    Rayleigh-Ritz steps) or after imax.  Returns (U^, theta, iterations, L count).
    """
    B0, _ = orth(U0, tau=tau)
    nL = 1
    blocks = [(B0, Lop(B0))]
    k = B0.shape[1]
    theta_prev = None
    Uh = B0
    theta = np.zeros(0)
    it = 0
    for it in range(1, imax + 1):
        Bn, LBn = blocks[0]
        if len(blocks) > 1:
            Mo = np.hstack([b for b, _ in blocks[1:]])
            LMo = np.hstack([lb for _, lb in blocks[1:]])
            Q2, LQ2 = orth(Mo, F=Bn, LM=LMo, LF=LBn, tau=tau)
            Q = np.hstack([Bn, Q2])
            LQ = np.hstack([LBn, LQ2])
        else:
            Q, LQ = Bn, LBn
        if Q.shape[1] == 0:
            return Q, np.zeros(0), it, nL
        th_all, V = eig_desc(Q.T @ LQ)
        kk = min(k, Q.shape[1])
        Uh = Q @ V[:, :kk]
        LUh = LQ @ V[:, :kk]
        theta = th_all[:kk]
        if (it >= min_iter and theta_prev is not None and theta_prev.shape == theta.shape
                and np.max(np.abs(theta - theta_prev)) <= tol * max(theta[0], 1e-300)):
            break
        if it == imax:
            break
        theta_prev = theta
        Bnew, _ = orth(LUh, tau=tau)
        if Bnew.shape[1] == 0:
            break
        nL += 1
        blocks = [(Bnew, Lop(Bnew))] + blocks[:p]
    return Uh, theta, it, nL


# ---------------------------------------------------------------------------
# Exact SVD of U^T Z, singular value soft-threshold, refactor (Eq. "exactSVD",
# "approxSVD", "truncate"; Alg. 1 W <- U sqrt(Sigma), H <- V sqrt(Sigma))
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class ProxResult:
    W: np.ndarray
    H: np.ndarray
    U: np.ndarray
    V: np.ndarray
    sigma: np.ndarray        # retained, thresholded singular values Sigma_t
    sigma_hat: np.ndarray    # all singular values of U^T Z (descending)
    k_new: int
    cap_hit: bool
    eps: float               # ||Z - Z~||_F (Sec. "Inexact PG", monitoring formula)
    u_trunc: Optional[np.ndarray]


def svt_refactor(Zop: ZOperator, Uh: np.ndarray, thresh: float, k_max: int) -> ProxResult:
    m, n = Zop.W.shape[0], Zop.H.shape[0]
    if Uh.shape[1] == 0:
        e2 = max(Zop.frob2(), 0.0)
        return ProxResult(np.zeros((m, 0)), np.zeros((n, 0)), np.zeros((m, 0)), np.zeros((n, 0)),
                          np.zeros(0), np.zeros(0), 0, False, math.sqrt(e2), None)
    Bt = Zop.zt(Uh)                                  # (U^T Z)^T, n x k_t
    s2, Ut = eig_desc(Bt.T @ Bt)                     # B B^T = U~ diag(s^2) U~^T
    sh = np.sqrt(np.maximum(s2, 0.0))
    sig = sh - thresh
    k_new = int(np.sum(sig > 0))
    cap_hit = k_new > k_max
    k_new = min(k_new, k_max)
    U = Uh @ Ut[:, :k_new]
    V = (Bt @ Ut[:, :k_new]) / sh[:k_new]
    sq = np.sqrt(sig[:k_new])
    e2 = Zop.frob2() - float(np.sum(sh ** 2))
    u_tr = Uh @ Ut[:, k_new] if Uh.shape[1] > k_new else None
    return ProxResult(U * sq, V * sq, U, V, sig[:k_new].copy(), sh, k_new, cap_hit,
                      math.sqrt(max(e2, 0.0)), u_tr)


# ---------------------------------------------------------------------------
# Solver state and one inexact proximal-gradient step with the safeguard
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    alpha: float = 1.99
    lmsvd_p: int = 1
    lmsvd_imax: int = 50
    lmsvd_tol: float = 1e-6
    lmsvd_min_iter: int = 2
    tau: float = 1e-6          # Gram-eigenvalue drop threshold in orth()
    ritz_rel: float = 1e-6     # keep s_j > ritz_rel * s_1 (Algorithm 2, J_s)
    psi0: float = 0.1
    seed: int = 0
    bm_epochs: int = 3
    pg_steps: int = 1


@dataclasses.dataclass
class State:
    W: np.ndarray
    H: np.ndarray
    U_prev: np.ndarray            # U_t: retained left singular vectors of the last prox
    U_prev2: Optional[np.ndarray]  # U_{t-1}
    u: Optional[np.ndarray]       # vector of the largest truncated singular value
    psi: float
    rank_hist: list
    prev_warm_cols: int
    t: int = 0
    bm_changed: bool = False


@dataclasses.dataclass
class ProxInfo:
    k_new: int
    warm_cols: int
    lmsvd_iters: int
    n_L: int
    eps: float
    cap_hit: bool
    sigma: np.ndarray
    sigma_hat: np.ndarray


def warm_start(st: State, k_max: int, opt: Options):
    """U^{t,0} of Eq. "rt0"/"rt0-1" plus the safeguard column of Eq. "rt"."""
    m = st.W.shape[0]
    base = st.U_prev
    second = st.W if (st.bm_changed or st.U_prev2 is None) else st.U_prev2
    cap = k_max + 1
    if base.shape[1] >= cap:
        Uh0 = base[:, :cap]
    else:
        extra, _ = orth(second, F=base if base.shape[1] else None, tau=opt.tau,
                        max_cols=cap - base.shape[1])
        Uh0 = np.hstack([base, extra])
    trig = (st.rank_hist[-1] == st.rank_hist[-2]) or (st.prev_warm_cols <= st.rank_hist[-1] + 1)
    if trig and Uh0.shape[1] < cap:
        g = counter_normal(opt.seed, STREAM_SAFEGUARD + st.t, m)
        if st.u is not None:
            ut = st.u - Uh0 @ (Uh0.T @ st.u)
        else:
            ut = np.zeros(m)
        g = g - Uh0 @ (Uh0.T @ g)
        nut2 = float(ut @ ut)
        if nut2 > 0:
            g = g - ut * (float(ut @ g) / nut2)
        ng = float(np.linalg.norm(g))
        if ng > 0:   # else [U^, u_t] spans R^m: no xi_t orthogonal to it, no column
            g = g / ng
            col = ut + st.psi * g if st.u is not None else g
            extra, _ = orth(col[:, None], F=Uh0 if Uh0.shape[1] else None, tau=opt.tau)
            Uh0 = np.hstack([Uh0, extra])
    return Uh0


def prox_step(ix: Index, st: State, lam: float, k_max: int, opt: Options, alpha=None):
    """One inexact PG step from X~_t = W H^T (Eq. "inexactpg") with LmSVD."""
    alpha = opt.alpha if alpha is None else alpha
    r = residual(ix, st.W, st.H)
    Zop = ZOperator(ix, st.W, st.H, r, alpha)
    U0 = warm_start(st, k_max, opt)
    warm_cols = U0.shape[1]
    if warm_cols > 0:
        Uh, theta, iters, _ = lmsvd(Zop.L, U0, p=opt.lmsvd_p, tol=opt.lmsvd_tol,
                                     imax=opt.lmsvd_imax, tau=opt.tau, min_iter=opt.lmsvd_min_iter)
        s = np.sqrt(np.maximum(theta, 0.0))
        if s.shape[0]:
            Uh = Uh[:, s > opt.ritz_rel * s[0]]
    else:
        Uh, iters = U0, 0
    res = svt_refactor(Zop, Uh, lam * alpha, k_max)
    return _advance(st, res, warm_cols), ProxInfo(res.k_new, warm_cols, iters, Zop.n_L, res.eps,
                                                    res.cap_hit, res.sigma, res.sigma_hat)


def _advance(st: State, res: ProxResult, warm_cols: int) -> State:
    psi = st.psi / 2.0 if res.k_new == warm_cols - 1 else st.psi
    return State(W=res.W, H=res.H, U_prev=res.U, U_prev2=st.U_prev, u=res.u_trunc, psi=psi,
                 rank_hist=st.rank_hist + [res.k_new], prev_warm_cols=warm_cols, t=st.t + 1,
                 bm_changed=False)


# ---------------------------------------------------------------------------
# Initial point: one inexact PG step from X_{-1} = 0 with alpha = 1/L = 1,
# HMT range finder + Nystrom (Sec. "Initialization", Eq. "nys")
# ---------------------------------------------------------------------------
def init_step(ix: Index, lam: float, k_init: int, k_max: int, opt: Options) -> tuple:
    m, n = ix.m, ix.n
    W0 = np.zeros((m, 0))
    H0 = np.zeros((n, 0))
    Zop = ZOperator(ix, W0, H0, -ix.val.copy(), 1.0)    # Z_{-1} = -grad f(0) = P_Omega(A)
    G = counter_normal(opt.seed, STREAM_INIT_SKETCH, m * k_init).reshape(k_init, m).T
    Q, _ = orth(Zop.L(G), tau=opt.tau)                   # Q = orth(A_{-1} U~)
    AQ = Zop.L(Q)
    C = Q.T @ AQ                                         # Q^T A Q
    cw, CE = eig_desc(C)
    cpos = cw > opt.tau * max(cw[0], 1e-300) if cw.shape[0] else cw > 0
    Cpinv = (CE[:, cpos] / cw[cpos]) @ CE[:, cpos].T      # (Q^T A Q)^dagger
    Qh, _ = orth(AQ, tau=opt.tau)                        # A Q = Q^ R^
    Rh = Qh.T @ AQ
    s2, Ut = eig_desc(Rh @ Cpinv @ Rh.T)
    keep = np.sqrt(np.maximum(s2, 0.0)) > opt.ritz_rel * math.sqrt(max(s2[0], 0.0)) if s2.shape[0] else s2 > 0
    Uh = Qh @ Ut[:, keep]
    res = svt_refactor(Zop, Uh, lam * 1.0, k_max)
    st = State(W=res.W, H=res.H, U_prev=res.U, U_prev2=None, u=res.u_trunc, psi=opt.psi0,
               rank_hist=[0, res.k_new], prev_warm_cols=Uh.shape[1], t=0, bm_changed=False)
    return st, ProxInfo(res.k_new, Uh.shape[1], 0, Zop.n_L, res.eps, res.cap_hit, res.sigma, res.sigma_hat)


# ---------------------------------------------------------------------------
# BM phase: monotone solver on (MF) with exact line search
# ---------------------------------------------------------------------------
def line_search_coeffs(ix: Index, W, H, DW, DH, r, lam):
    """Coefficients c0..c4 of phi(s) = F~(W + s DW, H + s DH):
    phi(s) = 1/2 sum_e (r_e + s b_e + s^2 c_e)^2 + lam/2 (||W+sDW||^2 + ||H+sDH||^2),
    b_e = <DW_i, H_j> + <W_i, DH_j>, c_e = <DW_i, DH_j>."""
    ri = ix.rows_of_entries()
    cj = ix.col
    b = np.einsum("ek,ek->e", DW[ri], H[cj]) + np.einsum("ek,ek->e", W[ri], DH[cj])
    c = np.einsum("ek,ek->e", DW[ri], DH[cj])
    c0 = 0.5 * (r @ r) + 0.5 * lam * (np.sum(W * W) + np.sum(H * H))
    c1 = (r @ b) + lam * (np.sum(W * DW) + np.sum(H * DH))
    c2 = 0.5 * (b @ b + 2.0 * (r @ c)) + 0.5 * lam * (np.sum(DW * DW) + np.sum(DH * DH))
    c3 = b @ c
    c4 = 0.5 * (c @ c)
    return np.array([c0, c1, c2, c3, c4], dtype=np.float64)


def quartic_argmin(c: np.ndarray) -> float:
    """argmin_{s >= 0} of c0 + c1 s + c2 s^2 + c3 s^3 + c4 s^4 among 0 and the
    real positive roots of phi'(s) = c1 + 2 c2 s + 3 c3 s^2 + 4 c4 s^3."""
    d = np.array([4 * c[4], 3 * c[3], 2 * c[2], c[1]])
    while d.shape[0] > 1 and d[0] == 0:
        d = d[1:]
    cand = [0.0]
    if d.shape[0] > 1:
        for z in np.roots(d):
            if abs(z.imag) <= 1e-9 * max(1.0, abs(z.real)) and z.real > 0:
                cand.append(float(z.real))
    phi = [np.polyval(c[::-1], s) for s in cand]
    return cand[int(np.argmin(phi))]


def bm_phase(ix: Index, st: State, lam: float, epochs: int):
    """`epochs` iterations of Polak-Ribiere+ nonlinear CG with exact line search.
    Each step satisfies phi(s*) <= phi(0), hence Eq. "nonincrease"."""
    W, H = st.W.copy(), st.H.copy()
    trace = []
    g_prev = None
    DW = DH = None
    moved = False
    for e in range(epochs):
        f, F, gW, gH, r = loss_grad(ix, W, H, lam)
        trace.append(F)
        if W.shape[1] == 0:
            break
        if g_prev is None:
            DW, DH = -gW, -gH
        else:
            num = np.sum(gW * (gW - g_prev[0])) + np.sum(gH * (gH - g_prev[1]))
            den = np.sum(g_prev[0] ** 2) + np.sum(g_prev[1] ** 2)
            beta = max(0.0, num / den) if den > 0 else 0.0
            DW, DH = -gW + beta * DW, -gH + beta * DH
            if np.sum(DW * gW) + np.sum(DH * gH) >= 0:
                DW, DH = -gW, -gH
        c = line_search_coeffs(ix, W, H, DW, DH, r, lam)
        s = quartic_argmin(c)
        if s > 0:
            moved = True
        W = W + s * DW
        H = H + s * DH
        g_prev = (gW, gH)
    st2 = dataclasses.replace(st, W=W, H=H, bm_changed=st.bm_changed or moved)
    return st2, trace


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class SolveInfo:
    F_hist: list
    k_hist: list
    eps_hist: list
    lmsvd_iters: list
    outer: int


def solve(ix: Index, lam: float, k_init: int, k_max: int, opt: Options = Options(),
          max_outer: int = 100, tol: float = 1e-10, F_target: Optional[float] = None,
          state: Optional[State] = None):
    """BM-Global (Algorithm 1): initial PG step from 0, then cycles of
    `bm_epochs` BM iterations and `pg_steps` inexact PG steps; the rank is
    the number of singular values that survive the threshold.  With `state`
    (a State returned by an earlier call) the cycles resume from it instead
    of the initial step."""
    if state is None:
        st, info0 = init_step(ix, lam, k_init, k_max, opt)
        k0, eps0 = info0.k_new, info0.eps
    else:
        st, k0, eps0 = state, state.W.shape[1], float("nan")
    F_hist = [objective(ix, st.W, st.H, lam)]
    k_hist = [k0]
    eps_hist = [eps0]
    its = [0]
    outer = 0
    for outer in range(1, max_outer + 1):
        st, _ = bm_phase(ix, st, lam, opt.bm_epochs)
        for _ in range(opt.pg_steps):
            st, info = prox_step(ix, st, lam, k_max, opt)
            eps_hist.append(info.eps)
            its.append(info.lmsvd_iters)
        F = objective(ix, st.W, st.H, lam)
        F_hist.append(F)
        k_hist.append(st.W.shape[1])
        if F_target is not None and F <= F_target:
            break
        if abs(F_hist[-2] - F) / (1.0 + abs(F_hist[-2])) < tol:
            break
    return st, SolveInfo(F_hist, k_hist, eps_hist, its, outer)


def problem_from_arrays(m, n, rows, cols, vals) -> Index:
    return build_index(m, n, rows, cols, vals)


# ---------------------------------------------------------------------------
# PSD / distance-geometry factorised loss (Eq. "EDM", supplement Sec. "The BM
# formulations for the RKE problem and the molecular conformation problem")
# ---------------------------------------------------------------------------
def edm_loss_grad(V: np.ndarray, i: np.ndarray, j: np.ndarray, d: np.ndarray, w, lam: float):
    """g(V) = 1/2 sum_{(i,j)} w_ij (<E_ij, V V^T> - d_ij^2)^2 + lam ||V||_F^2,
    E_ij = (e_i - e_j)(e_i - e_j)^T, so <E_ij, V V^T> = ||v_i - v_j||^2;
    grad g(V) = 2 (sum w_ij r_ij E_ij + lam I) V.  Returns (g, grad, r)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.broadcast_to(np.asarray(w, dtype=np.float64), (i.shape[0],))
    diff = V[i] - V[j]
    r = np.sum(diff * diff, axis=1) - np.asarray(d, dtype=np.float64) ** 2
    g = 0.5 * float(np.sum(w * r * r)) + lam * float(np.sum(V * V))
    E = sp.coo_matrix((np.concatenate([w * r, w * r, -w * r, -w * r]),
                       (np.concatenate([i, j, i, j]), np.concatenate([i, j, j, i]))),
                      shape=(V.shape[0], V.shape[0])).tocsr()
    grad = 2.0 * (E @ V) + 2.0 * lam * V
    return g, np.asarray(grad), r


def edm_lambda(n: int, d: np.ndarray) -> float:
    """lambda = -10 sqrt(n) / sum d_ij^2 (the molecular-conformation setting)."""
    return -10.0 * math.sqrt(n) / float(np.sum(np.asarray(d, dtype=np.float64) ** 2))
