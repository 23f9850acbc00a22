"""GB300-native (sm_103a) BM-Global hot path for nuclear-norm regularised
matrix completion: CUDA kernels behind the C ABI of include/bm.h, with a thin
ctypes binding (paper_2204_14067_gb300.binding)."""
from .binding import (  # noqa: F401
    BMError,
    bm_bm_phase,
    bm_create,
    bm_default_options,
    bm_destroy,
    bm_dims,
    bm_edm_create,
    bm_edm_destroy,
    bm_edm_loss_grad,
    bm_edm_set_factor,
    bm_get_factors,
    bm_get_index,
    bm_init,
    bm_last_error,
    bm_loss_grad,
    bm_loss_grad_csr_noalloc,
    bm_profile_enable,
    bm_profile_read,
    bm_prox_step,
    bm_set_factors,
    bm_set_stream,
    bm_solve,
    header_symbols,
    lib,
)
