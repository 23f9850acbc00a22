"""Brute-force check of a BM phase's iterates against the definition of
Polak-Ribiere+ nonlinear CG with an exact line search, shared by the pins of
both oracles.

Given the iterates x_0 ... x_E of one BM phase (x_e from a call of e epochs)
and the objective F as a plain function, the gradients come from central
differences of F and the steps from a brute-force scalar minimisation, so
neither the oracle's gradient nor its line-search coefficients nor its
quartic minimiser take part:

  * step 0 is steepest descent: x_1 - x_0 = -s_0 g_0;
  * step e lies in span{-g_e, x_e - x_(e-1)}, with coefficient s_e > 0 on
    -g_e and beta_e = max(0, <g_e, g_e - g_(e-1)> / ||g_(e-1)||^2) on the
    previous direction d_(e-1) = (x_e - x_(e-1)) / s_(e-1);
  * s_e is the global minimiser over s >= 0 of F along d_e.
"""
import numpy as np


def fd_gradient(F, x, h=1e-5):
    """Central differences of F (error h^2 / 6 times its third derivative
    along each coordinate)."""
    g = np.empty_like(x)
    for i in range(x.size):
        e = np.zeros_like(x)
        e[i] = h
        g[i] = (F(x + e) - F(x - e)) / (2 * h)
    return g


def global_step(F, x, d):
    """argmin over s >= 0 of phi(s) = F(x + s d) for an objective of degree 4:
    phi is recovered by interpolation at five points, every critical point
    lies within the Cauchy bound of phi', a dense grid covers that range, and
    the best grid point is refined by bounded Brent on F itself."""
    from scipy.optimize import minimize_scalar
    t = np.arange(5.0)
    poly = np.polyfit(t, [F(x + ti * d) for ti in t], 4)
    dp = np.polyder(poly)
    bound = 1.0 + np.max(np.abs(dp[1:] / dp[0]))
    grid = np.linspace(0.0, bound, 400_001)
    i = int(np.argmin(np.polyval(poly, grid)))
    if i == 0:
        return 0.0
    lo, hi = grid[i - 1], grid[min(i + 1, grid.size - 1)]
    return minimize_scalar(lambda s: F(x + s * d), bounds=(lo, hi), method="bounded",
                           options={"xatol": 1e-13 * bound}).x


def check_pr_plus(xs, F, rtol=1e-6):
    """Assert the properties above for the iterates xs (flat vectors) of F.
    Returns (restarts, fr_apart): the steps whose Polak-Ribiere ratio was
    negative (PR+ restarts there), and those where the Fletcher-Reeves ratio
    ||g_e||^2 / ||g_(e-1)||^2 differs from it by more than 1e-2, so that a
    caller can make sure its case tells the rules apart."""
    gs = [fd_gradient(F, x) for x in xs]
    s_prev = None
    restarts = fr_apart = 0
    for e in range(len(xs) - 1):
        step = xs[e + 1] - xs[e]
        if e == 0:
            s_e = -(step @ gs[0]) / (gs[0] @ gs[0])
            fit = -s_e * gs[0]
        else:
            basis = np.stack([-gs[e], xs[e] - xs[e - 1]], axis=1)
            (s_e, b), *_ = np.linalg.lstsq(basis, step, rcond=None)
            fit = basis @ np.array([s_e, b])
            beta = b * s_prev / s_e
            pr = (gs[e] @ (gs[e] - gs[e - 1])) / (gs[e - 1] @ gs[e - 1])
            fr = (gs[e] @ gs[e]) / (gs[e - 1] @ gs[e - 1])
            assert abs(beta - max(0.0, pr)) <= rtol * (1.0 + abs(pr)), (e, beta, pr)
            restarts += pr < 0
            fr_apart += abs(fr - pr) > 1e-2
        assert np.linalg.norm(step - fit) <= 0.1 * rtol * np.linalg.norm(step), e
        assert s_e > 0, e
        s_num = global_step(F, xs[e], step / s_e)
        assert abs(s_num - s_e) <= rtol * s_e, (e, s_num, s_e)
        s_prev = s_e
    return restarts, fr_apart
