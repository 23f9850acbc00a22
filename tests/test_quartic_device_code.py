"""The device form of the exact line search's step rule (csrc/quartic.cuh:
argmin over s >= 0 of a quartic among 0 and the positive roots of its cubic
derivative, Cardano / trigonometric roots polished by Newton), compiled from
the same source as host C++ and checked on the CPU against a brute-force
minimisation: random quartics, and the branches the closed form has (a
quadratic or linear derivative, a double root, no positive root)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2204_14067_gb300", "csrc", "quartic.cuh")

HARNESS = r"""
#include <cmath>
#include <cstdio>
using std::acos; using std::cbrt; using std::cos; using std::fabs; using std::fmax; using std::fmin;
using std::isfinite; using std::sqrt;
#include "quartic.cuh"
int main() {
  double c[5];
  while (std::scanf("%lf %lf %lf %lf %lf", &c[0], &c[1], &c[2], &c[3], &c[4]) == 5)
    std::printf("%.17g\n", bm::quartic_argmin_d(c));
  return 0;
}
"""


@pytest.fixture(scope="module")
def argmin(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("quartic")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([gxx, "-O2", "-std=c++17", "-D__device__=", f"-I{os.path.dirname(HEADER)}", str(src),
                    "-o", str(exe)], check=True, capture_output=True, timeout=120)

    def run(cs):
        text = "\n".join(" ".join(repr(float(v)) for v in c) for c in cs) + "\n"
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True, timeout=120)
        return np.array([float(x) for x in out.stdout.split()])
    return run


def _phi(c, s):
    return np.polyval(np.asarray(c)[::-1], s)


def _check(c, s):
    """phi(s) is within rounding of the least value over a dense grid of
    [0, R], R past every critical point (Cauchy bound of phi')."""
    c = np.asarray(c, dtype=np.float64)
    d = np.array([4 * c[4], 3 * c[3], 2 * c[2], c[1]])
    nz = np.nonzero(np.abs(d) > 0)[0]
    lead = d[nz[0]] if nz.size else 1.0
    R = 1.0 + (np.max(np.abs(d[nz[0] + 1:] / lead)) if nz.size and nz[0] < 3 else 1.0)
    grid = np.linspace(0.0, R, 200_001)
    best = _phi(c, grid).min()
    assert s >= 0 and np.isfinite(s)
    assert _phi(c, s) <= best + 1e-9 * (1.0 + abs(best)), (c, s, _phi(c, s), best)


def test_random_quartics(argmin):
    rng = np.random.default_rng(3)
    cs = rng.standard_normal((400, 5))
    cs[:, 4] = np.abs(cs[:, 4]) + 1e-3            # bounded below, as every line-search quartic
    for c, s in zip(cs, argmin(cs)):
        _check(c, s)


def test_degenerate_branches(argmin):
    cs = [
        [1.0, -2.0, 1.0, 0.0, 0.0],        # quadratic: minimiser 1
        [1.0, -2.0, 0.5, 1e-20, 0.0],      # cubic term below the quartic threshold: quadratic branch
        [0.0, 3.0, 1.0, 0.0, 0.0],         # increasing from 0: s = 0
        [2.0, -1.0, 0.0, 0.0, 1.0],        # phi' = 4 s^3 - 1: s = 4^(-1/3)
        [0.0, 0.0, -1.0, 0.0, 0.5],        # phi' = 2 s^3 - 2 s: roots 0, 1 (double well)
        [0.0, 0.0, 0.0, 0.0, 1.0],         # s^4: every root at 0
        [5.0, 1.0, 2.0, 3.0, 4.0],         # no positive critical point: s = 0
        [0.0, 1.0, -0.5, -1.0 / 3.0, 0.25],  # phi' = (s - 1)^2 (s + 1): a double root, phi rising: s = 0
        [1.0, -4.0, 6.0, -4.0, 1.0],       # phi = (s - 1)^4: a triple root of phi' (zero discriminant), s = 1
    ]
    s = argmin(cs)
    for c, si in zip(cs, s):
        _check(c, si)
    assert abs(s[0] - 1.0) <= 1e-12 and s[2] == 0.0 and s[6] == 0.0 and s[7] == 0.0
    assert abs(s[3] - 4.0 ** (-1.0 / 3.0)) <= 1e-12 and abs(s[4] - 1.0) <= 1e-12
    assert abs(s[8] - 1.0) <= 1e-4          # a quartic this flat fixes s only to about eps^(1/4)
