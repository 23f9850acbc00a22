// Inexact proximal-gradient step (filled in below the minimal slice).
#include "ctx.cuh"

namespace bm {
struct ProxState {};
void prox_create(bm_ctx& h) { h.ps = new ProxState(); }
void prox_destroy(bm_ctx& h) { delete h.ps; h.ps = nullptr; }
void prox_reset(bm_ctx&) {}
void prox_step_dev(bm_ctx&, double, bm_prox_info*) { throw Error{BM_ERR_INVALID, "bm_prox_step: not built"}; }
void init_step_dev(bm_ctx&, bm_prox_info*) { throw Error{BM_ERR_INVALID, "bm_init: not built"}; }
}  // namespace bm
