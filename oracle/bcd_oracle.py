"""Plain FP64 CPU oracle for the column-wise block coordinate descent BM
solver: the form of polyMF-SS the paper adopts for the BM phase of matrix
completion (Sec. "Experiments", matrix completion setting): block coordinate
descent where each block is one column of W and the same column of H,
updated with an exact line search.

TEST INFRASTRUCTURE ONLY, under the same rules as ``bm_oracle``: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm
of ``bench.py`` may import it; the library never does.

One epoch visits the columns c = 0, ..., k-1 in order.  For block c, with the
residual r_e = <W_i, H_j> - a_e on Omega (Eq. "mf"):

  * block gradient  g_w = R h_c + lam w_c,  g_h = R^T w_c + lam h_c;
  * direction       (d_w, d_h) = -(g_w, g_h);
  * exact line search on F(W + s d_w e_c^T, H + s d_h e_c^T): on Omega the
    residual moves as r_e + s b_e + s^2 c_e with b_e = d_w,i h_c,j +
    w_c,i d_h,j and c_e = d_w,i d_h,j, so F is the quartic
        F + s <grad, d> + s^2 (1/2 sum (b^2 + 2 r c) + lam/2 (|d_w|^2 + |d_h|^2))
          + s^3 sum b c + s^4 1/2 sum c^2,
    minimised over s >= 0 by the same rule as the full-gradient BM phase
    (bm_oracle.quartic_argmin);
  * update w_c, h_c and the residual.

The paper describes the solver only to this level; the block gradient
direction with an exact line search is the reading used here.

Parity status: pinned by tests/test_oracle_bcd.py (block gradient against
central finite differences, the line-search quartic against the objective
along the direction, its minimiser against a brute-force grid, F
nonincreasing after every block, full observation reaching the closed-form
optimum of the factored problem, and a sweep rebuilt from central
differences and brute-force steps in column order).
"""
from __future__ import annotations

import numpy as np

from oracle import bm_oracle as O


def block_quartic(ix: O.Index, W, H, lam: float, c: int, r=None):
    """(coefficients c0..c4, d_w, d_h, b, cc) of block c at (W, H)."""
    if r is None:
        r = O.residual(ix, W, H)
    R = ix.sparse(r)
    w, h = W[:, c], H[:, c]
    gw = R @ h + lam * w
    gh = R.T @ w + lam * h
    dw, dh = -gw, -gh
    ri = ix.rows_of_entries()
    cj = ix.col
    b = dw[ri] * h[cj] + w[ri] * dh[cj]
    cc = dw[ri] * dh[cj]
    F = 0.5 * float(r @ r) + 0.5 * lam * (float(np.sum(W * W)) + float(np.sum(H * H)))
    coef = np.array([
        F,
        float(r @ b) + lam * (float(w @ dw) + float(h @ dh)),
        0.5 * float(b @ b + 2.0 * (r @ cc)) + 0.5 * lam * (float(dw @ dw) + float(dh @ dh)),
        float(b @ cc),
        0.5 * float(cc @ cc),
    ])
    return coef, dw, dh, b, cc


def bcd_epoch(ix: O.Index, W, H, lam: float):
    """One sweep over the k column blocks.  Returns (W, H, F after each block)."""
    W, H = W.copy(), H.copy()
    r = O.residual(ix, W, H)
    trace = []
    for c in range(W.shape[1]):
        coef, dw, dh, b, cc = block_quartic(ix, W, H, lam, c, r)
        s = O.quartic_argmin(coef)
        if s > 0:
            W[:, c] += s * dw
            H[:, c] += s * dh
            r = r + s * b + s * s * cc
        trace.append(float(np.polyval(coef[::-1], s)))
    return W, H, trace


def bcd_phase(ix: O.Index, W, H, lam: float, epochs: int):
    """`epochs` sweeps; returns (W, H, F after each sweep)."""
    F = []
    for _ in range(epochs):
        W, H, tr = bcd_epoch(ix, W, H, lam)
        F.append(tr[-1] if tr else O.objective(ix, W, H, lam))
    return W, H, F
