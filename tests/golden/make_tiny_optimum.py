"""Write tests/golden/tiny_optimum.txt: the FP64 oracle's converged objective
and rank of Algorithm 1 on the 500 x 300 planted problem (lambda = 0.5,
k0 = 8, k_max = 64, default options).  Calls only the oracle."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import bm_oracle as O  # noqa: E402
from synth import named_config  # noqa: E402


def main():
    p = named_config("tiny")
    ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
    st, info = O.solve(ix, p.lam, 8, 64, O.Options(), max_outer=400, tol=1e-14)
    with open(os.path.join(HERE, "tiny_optimum.txt"), "w") as f:
        f.write("# Algorithm 1, FP64 oracle, tiny planted problem (500 x 300, lambda 0.5, k0 8, k_max 64)\n")
        f.write(f"F_star {info.F_hist[-1]!r}\n")
        f.write(f"rank {st.W.shape[1]}\n")
        f.write(f"cycles {info.outer}\n")


if __name__ == "__main__":
    main()
