// Distance-geometry handle, shared by the loss/gradient pass (edm.cu) and the
// Algorithm 1 solve of the distance-geometry QSDP (edm_solve.cu).
#pragma once
#include "ctx.cuh"

namespace bm {
struct EdmSolveState;   // edm_solve.cu
void edm_solve_destroy(EdmSolveState* s);
// forget the warm start and the rank schedule (a new factor was set)
void edm_solve_reset(EdmSolveState* s);
}  // namespace bm

struct bm_edm_ctx {
  int64_t n = 0, npairs = 0;
  double lambda = 0;
  int k_max = 0, k = 0, ld = 4;
  cudaStream_t stream = nullptr;      // stream the calls run on
  cudaStream_t own_stream = nullptr;  // the handle's own stream
  bm::DevBuf<int64_t> row_ptr;
  bm::DevBuf<int32_t> col;
  bm::DevBuf<float> dsq, w;    // d_ij^2 and w_ij in CSR order (both directions of every pair)
  bm::Segs seg;
  bm::DevBuf<float> V, gV, partial;
  bm::DevBuf<double> fseg, red;
  std::string err;
  // solve state (edm_solve.cu)
  bm_options opt{};            // solver parameters (bm_edm_set_options)
  bm_ctx core;                 // stream and scratch of the dense routines
  bm::EdmSolveState* ss = nullptr;
  ~bm_edm_ctx() { bm::edm_solve_destroy(ss); }
};

namespace bm {
// g(V) of Eq. "EDM" at the current factor; with want_grad the gradient goes
// to h.gV; with r_out the residual r_ij = ||v_i - v_j||^2 - d_ij^2 of every
// directed entry (CSR order).  Returns after a stream synchronisation; with
// sync = false it returns NaN at once and g(V) is left in h.red[0].
double edm_loss_grad_dev(bm_edm_ctx& h, bool want_grad, float* r_out, bool sync = true);
}  // namespace bm
