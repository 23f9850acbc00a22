// Autotuning of the sparse passes' work splits (panel counts).
//
// Each sparse pass gathers rows of one factor-sized block per observed entry.
// When that block is larger than L2, the order in which warps visit the
// segments decides how many gathers miss: with P panels the segments are
// visited panel by panel, so the rows gathered at any moment come from one
// P-th of the block.  The best P depends on the block size, the rank and the
// entry distribution, so it is measured: every pass kind is timed with the
// natural split and with each candidate panel count, and the fastest is kept.
// Results differ between panel counts only in the order of floating-point
// additions (partials are combined per row in entry order).
#include <algorithm>

#include "ctx.cuh"

namespace bm {
namespace {

// Bytes of the block a pass kind gathers from (its working set in L2).
size_t gathered_bytes(const bm_ctx& h, int kind) {
  const Index& ix = h.ix;
  const size_t w = h.bf_active() ? 2 : 4;
  const size_t q = (size_t)round_up4(std::min(h.k_max + 1, h.k + 1));
  switch (kind) {
    case kPassGradCsr: return (size_t)ix.n * h.ld * w;
    case kPassGradCsc: return (size_t)ix.m * h.ld * w;
    case kPassLsCsr: return 2 * (size_t)ix.n * h.ld * w;
    case kPassSpmmCsr: return (size_t)ix.n * q * 4;
    default: return (size_t)ix.m * q * 4;
  }
}

void launch_kind(bm_ctx& h, int kind) {
  if (kind == kPassSpmmCsr || kind == kPassSpmmCsc) tuning_spmm_dev(h, kind == kPassSpmmCsr);
  else tuning_pass_dev(h, kind);
}

// Fastest of three timed launches after one warm-up launch (ms).
float time_kind(bm_ctx& h, int kind, cudaEvent_t e0, cudaEvent_t e1) {
  launch_kind(h, kind);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    BM_CUDA(cudaEventRecord(e0, h.stream));
    launch_kind(h, kind);
    BM_CUDA(cudaEventRecord(e1, h.stream));
    BM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    BM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  return best;
}

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  Events() {
    BM_CUDA(cudaEventCreate(&a));
    BM_CUDA(cudaEventCreate(&b));
  }
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

void autotune_dev(bm_ctx& h, int max_panels, bm_tune_info* info) {
  static_assert(kPassKinds == BM_PASS_KINDS, "pass kinds of the header and the library differ");
  BM_REQUIRE(h.k >= 1, BM_ERR_INVALID, "bm_autotune: no factors yet (call bm_init or bm_set_factors first)");
  BM_REQUIRE(max_panels >= 1 && max_panels <= BM_MAX_PANELS, BM_ERR_INVALID,
             "bm_autotune: max_panels must be in [1, BM_MAX_PANELS]");
  int l2 = 0;
  BM_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h.device));
  // the passes read the residual and the search directions: make both defined
  residual_dev(h);
  BM_CUDA(cudaMemsetAsync(h.DW.get(), 0, (size_t)h.ix.m * h.ld * sizeof(float), h.stream));
  BM_CUDA(cudaMemsetAsync(h.DH.get(), 0, (size_t)h.ix.n * h.ld * sizeof(float), h.stream));
  const bool prof = h.prof.on;
  h.prof.on = false;
  Events ev;
  static const int kCand[] = {2, 3, 4, 6, 8, 12, 16};
  bm_tune_info out{};
  for (int kind = 0; kind < kPassKinds; ++kind) {
    h.ix.panels[kind] = 1;
    const float t1 = time_kind(h, kind, ev.a, ev.b);
    ++out.timed;
    int best = 1;
    float tb = t1;
    if (gathered_bytes(h, kind) * 4 >= (size_t)l2) {
      for (int P : kCand) {
        if (P > max_panels) break;
        ensure_panel_segs(h, pass_is_csr(kind), P);
        h.ix.panels[kind] = P;
        const float t = time_kind(h, kind, ev.a, ev.b);
        ++out.timed;
        if (t < 0.98f * tb) best = P, tb = t;   // keep the simpler split unless clearly faster
      }
    }
    h.ix.panels[kind] = best;
    out.panels[kind] = best;
    out.ms[kind] = tb;
    out.ms_single[kind] = t1;
  }
  h.prof.on = prof;
  h.tuned = true;
  if (info) *info = out;
}

}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_autotune(bm_handle h, int32_t max_panels, bm_tune_info* info) {
  if (!h) return BM_ERR_INVALID;
  return guard_call(h->err, [&] { autotune_dev(*h, max_panels, info); });
}

bm_status bm_set_panels(bm_handle h, const int32_t* panels) {
  if (!h || !panels) return BM_ERR_INVALID;
  return guard_call(h->err, [&] {
    for (int k = 0; k < kPassKinds; ++k)
      BM_REQUIRE(panels[k] >= 1 && panels[k] <= BM_MAX_PANELS, BM_ERR_INVALID,
                 "bm_set_panels: panel counts must be in [1, BM_MAX_PANELS]");
    for (int k = 0; k < kPassKinds; ++k) {
      ensure_panel_segs(*h, pass_is_csr(k), panels[k]);
      h->ix.panels[k] = panels[k];
    }
    h->tuned = true;
  });
}

bm_status bm_get_panels(bm_handle h, int32_t* panels) {
  if (!h || !panels) return BM_ERR_INVALID;
  for (int k = 0; k < kPassKinds; ++k) panels[k] = h->ix.panels[k];
  return BM_OK;
}

}  // extern "C"
