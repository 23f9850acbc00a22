"""Pins of the column-block coordinate descent oracle (oracle/bcd_oracle.py):
the block gradient against central finite differences, the line-search
quartic against the objective along the direction, its minimiser against a
brute-force grid, F nonincreasing block by block, full observation
reaching the closed-form optimum of the factored problem, and a whole sweep
rebuilt from central differences and brute-force steps in column order."""
import numpy as np

from cg_pin import fd_gradient, global_step
from oracle import bcd_oracle as C
from oracle import bm_oracle as O
from synth import planted_uniform


def _small(seed=3, lam=0.5):
    p = planted_uniform(m=30, n=45, rank=3, frac=0.4, noise_sd=0.1, lam=lam, seed=seed)
    return p, O.build_index(p.m, p.n, p.rows, p.cols, p.vals)


def test_block_direction_is_minus_the_block_gradient():
    p, ix = _small()
    rng = np.random.default_rng(0)
    W, H = rng.standard_normal((ix.m, 4)) * 0.5, rng.standard_normal((ix.n, 4)) * 0.5
    coef, dw, dh, _, _ = C.block_quartic(ix, W, H, p.lam, 2)
    eps = 1e-6
    for i in (0, 7, 29):
        Wp, Wm = W.copy(), W.copy()
        Wp[i, 2] += eps
        Wm[i, 2] -= eps
        fd = (O.objective(ix, Wp, H, p.lam) - O.objective(ix, Wm, H, p.lam)) / (2 * eps)
        assert abs(fd + dw[i]) <= 1e-6 * (1 + abs(fd))
    for j in (1, 20, 44):
        Hp, Hm = H.copy(), H.copy()
        Hp[j, 2] += eps
        Hm[j, 2] -= eps
        fd = (O.objective(ix, W, Hp, p.lam) - O.objective(ix, W, Hm, p.lam)) / (2 * eps)
        assert abs(fd + dh[j]) <= 1e-6 * (1 + abs(fd))


def test_quartic_matches_objective_and_bruteforce_minimiser():
    p, ix = _small(seed=5)
    rng = np.random.default_rng(1)
    W, H = rng.standard_normal((ix.m, 3)), rng.standard_normal((ix.n, 3))
    coef, dw, dh, _, _ = C.block_quartic(ix, W, H, p.lam, 1)
    for s in (0.0, 0.01, 0.1, 0.7):
        W2, H2 = W.copy(), H.copy()
        W2[:, 1] += s * dw
        H2[:, 1] += s * dh
        val = np.polyval(coef[::-1], s)
        assert abs(val - O.objective(ix, W2, H2, p.lam)) <= 1e-9 * (1 + abs(val))
    s_star = O.quartic_argmin(coef)
    grid = np.linspace(0.0, max(4 * s_star, 1e-3), 20001)
    vals = np.polyval(coef[::-1], grid)
    assert np.polyval(coef[::-1], s_star) <= vals.min() + 1e-10 * (1 + abs(vals.min()))


def test_objective_nonincreasing_block_by_block():
    p, ix = _small(seed=7)
    rng = np.random.default_rng(2)
    W, H = rng.standard_normal((ix.m, 5)) * 0.3, rng.standard_normal((ix.n, 5)) * 0.3
    F0 = O.objective(ix, W, H, p.lam)
    prev = F0
    for _ in range(4):
        W, H, tr = C.bcd_epoch(ix, W, H, p.lam)
        for f in tr:
            assert f <= prev * (1 + 1e-12) + 1e-12
            prev = f
        assert abs(tr[-1] - O.objective(ix, W, H, p.lam)) <= 1e-9 * abs(tr[-1])


def test_full_observation_reaches_the_closed_form_optimum():
    """Omega = all entries: min over rank-k factors of 1/2 ||W H^T - A||^2 +
    lam/2 (||W||^2 + ||H||^2) equals the nuclear-norm problem's optimum
    sum_{s > lam} (lam s - lam^2 / 2) + sum_{s <= lam} s^2 / 2 when k is at
    least the number of singular values above lam."""
    rng = np.random.default_rng(4)
    m, n = 10, 14
    A = rng.standard_normal((m, n))
    rows, cols = np.divmod(np.arange(m * n), n)
    ix = O.build_index(m, n, rows, cols, A[rows, cols])
    s = np.linalg.svd(A, compute_uv=False)
    lam = 0.5 * (s[2] + s[3])
    F_star = float(np.sum(np.where(s > lam, lam * s - 0.5 * lam ** 2, 0.5 * s ** 2)))
    W, H = rng.standard_normal((ix.m, 3)) * 0.5, rng.standard_normal((ix.n, 3)) * 0.5
    W, H, F = C.bcd_phase(ix, W, H, lam, 3000)
    assert abs(F[-1] - F_star) <= 1e-8 * F_star


def test_sweep_is_exact_block_steps_in_column_order():
    """One sweep rebuilt without the oracle's block machinery: for c = 0, 1,
    ..., k - 1 in turn, the block gradient of column c of W and H by central
    differences of the objective, and the exact step along its negative by a
    brute-force scalar minimisation (tests/cg_pin.py).  Blocks taken in
    another order reach a different point."""
    p = planted_uniform(m=6, n=8, rank=2, frac=0.6, noise_sd=0.1, lam=0.5, seed=9)
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals)
    rng = np.random.default_rng(2)
    W0, H0 = rng.standard_normal((ix.m, 3)) * 0.5, rng.standard_normal((ix.n, 3)) * 0.5
    W, H = W0.copy(), H0.copy()
    for c in range(3):
        def F(v, c=c, W=W, H=H):
            W2, H2 = W.copy(), H.copy()
            W2[:, c], H2[:, c] = v[:ix.m], v[ix.m:]
            return O.objective(ix, W2, H2, p.lam)

        x = np.concatenate([W[:, c], H[:, c]])
        d = -fd_gradient(F, x)
        x = x + global_step(F, x, d) * d
        W, H = W.copy(), H.copy()
        W[:, c], H[:, c] = x[:ix.m], x[ix.m:]
    Wc, Hc, _ = C.bcd_epoch(ix, W0, H0, p.lam)
    scale = np.abs(np.concatenate([W.ravel(), H.ravel()])).max()
    assert np.abs(Wc - W).max() <= 1e-7 * scale and np.abs(Hc - H).max() <= 1e-7 * scale
    Wr, Hr = W0[:, ::-1].copy(), H0[:, ::-1].copy()
    Wr, Hr, _ = C.bcd_epoch(ix, Wr, Hr, p.lam)
    assert np.abs(Wr[:, ::-1] - W).max() > 1e-4 * scale


def test_phase_reports_the_objective_after_each_sweep():
    p, ix = _small(seed=7)
    rng = np.random.default_rng(3)
    W0, H0 = rng.standard_normal((ix.m, 4)) * 0.5, rng.standard_normal((ix.n, 4)) * 0.5
    W, H, F = C.bcd_phase(ix, W0, H0, p.lam, 2)
    W1, H1, _ = C.bcd_phase(ix, W0, H0, p.lam, 1)
    assert len(F) == 2
    assert abs(F[0] - O.objective(ix, W1, H1, p.lam)) <= 1e-12 * F[0]
    assert abs(F[1] - O.objective(ix, W, H, p.lam)) <= 1e-12 * F[1]
