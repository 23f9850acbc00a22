"""Resume of the oracle's Algorithm 1 from a returned state: the cycles after
the break are the cycles of an uninterrupted run (bit-identical)."""
import numpy as np

from oracle import bm_oracle as O
from synth import named_config


def test_oracle_resume_is_uninterrupted_run():
    p = named_config("tiny")
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    full, fi = O.solve(ix, p.lam, 8, 64, O.Options(), max_outer=6, tol=0.0)
    half, hi = O.solve(ix, p.lam, 8, 64, O.Options(), max_outer=3, tol=0.0)
    rest, ri = O.solve(ix, p.lam, 8, 64, O.Options(), max_outer=3, tol=0.0, state=half)
    assert np.array_equal(full.W, rest.W) and np.array_equal(full.H, rest.H)
    assert full.t == rest.t and full.rank_hist == rest.rank_hist and full.psi == rest.psi
    assert fi.F_hist[3:] == ri.F_hist
