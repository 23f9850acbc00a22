"""FP64 CPU oracle (test infrastructure only; never imported by the library)."""
from . import bm_oracle  # noqa: F401
