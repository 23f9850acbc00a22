"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws problem data only (index sets, observed values, random
factors).  It holds none of the method's arithmetic, so both the FP64 oracle
and the CUDA path can consume its output without sharing code.
"""
from .gen import (  # noqa: F401
    Problem,
    planted_uniform,
    zipf_ratings,
    named_config,
    random_factors,
    PairProblem,
    self_avoiding_chain,
    serving_requests,
)
