"""The C-ABI library builds, loads and exports every symbol of include/bm.h."""
import ctypes
import os

import pytest

from paper_2204_14067_gb300 import binding


def test_library_exports_every_header_symbol():
    if not os.path.exists(binding.LIB_PATH):
        from paper_2204_14067_gb300 import build
        build.build()
    L = ctypes.CDLL(binding.LIB_PATH)
    names = binding.header_symbols()
    assert "bm_create" in names and "bm_loss_grad" in names and "bm_prox_step" in names
    assert "bm_solve" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # every header symbol has a ctypes signature in the binding
    assert set(names) <= set(binding._SIGS), set(names) - set(binding._SIGS)


def test_default_options_without_gpu():
    o = binding.bm_default_options()
    assert o.alpha == pytest.approx(1.99) and o.bm_epochs == 3 and o.pg_steps == 1
    assert o.psi0 == pytest.approx(0.1) and o.lmsvd_p == 1
