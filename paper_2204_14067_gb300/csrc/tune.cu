// Autotuning of the sparse passes' work splits (panel counts).
//
// Each sparse pass gathers rows of one factor-sized block per observed entry.
// When that block is larger than L2, the order in which warps visit the
// segments decides how many gathers miss: with P panels the segments are
// visited panel by panel, so the rows gathered at any moment come from one
// P-th of the block.  The best P depends on the block size, the rank and the
// entry distribution, so it is measured: every pass kind is timed with the
// natural split and with each candidate panel count, and the fastest is kept.
// The kernel layout (a lane group per segment, or a whole warp per segment)
// is timed the same way, with every panel count.  Results differ between
// panel counts and layouts only in the order of floating-point additions
// (partials are combined per row in entry order).
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

// Gather-only pass: every entry loads its gathered FP32 row (V float4 chunks
// per lane, 8 lanes per entry, 4 entries per warp step) and adds it into
// registers; one value per warp is written so that the loads are not removed.
// No index, value or output traffic beyond the entries' indices: the time is
// what moving the gathered rows alone takes on this GPU.
template <int V>
__global__ void __launch_bounds__(256) k_gather_roof(const int32_t* __restrict__ idx, int64_t nnz,
                                                     const float* __restrict__ X, int ld, int nchunk,
                                                     float* __restrict__ out) {
  const int lane = threadIdx.x & 31, g = lane >> 3, l = lane & 7;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t e0 = warp * 32; e0 < nnz; e0 += nwarps * 32) {
    const int j = e0 + lane < nnz ? __ldg(idx + e0 + lane) : 0;
#pragma unroll 2
    for (int t = 0; t < 8; ++t) {
      const int jj = __shfl_sync(0xffffffffu, j, t * 4 + g);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = l + 8 * v;
        if (c < nchunk) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(X + (int64_t)jj * ld) + c);
          acc.x += x.x;
          acc.y += x.y;
          acc.z += x.z;
          acc.w += x.w;
        }
      }
    }
  }
  acc.x += acc.y + acc.z + acc.w;
#pragma unroll
  for (int mk = 16; mk > 0; mk >>= 1) acc.x += __shfl_xor_sync(0xffffffffu, acc.x, mk);
  if (lane == 0) out[warp] = acc.x;
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
    // start from the automatic layout with one panel; keep a candidate only
    // when it is clearly (2 %) faster than the best so far
    h.ix.layout[kind] = -1;
    h.ix.panels[kind] = 1;
    const int lay0 = pass_ws(h.ix, kind) ? 1 : 0;
    h.ix.layout[kind] = lay0;
    const float t1 = time_kind(h, kind, ev.a, ev.b);
    ++out.timed;
    int best = 1, best_lay = lay0;
    float tb = t1;
    const bool big = gathered_bytes(h, kind) * 4 >= (size_t)l2;
    for (int lay : {lay0, 1 - lay0}) {
      h.ix.layout[kind] = lay;
      for (int P : kCand) {
        if (P == 2 && lay != lay0) {      // the other layout with one panel first
          h.ix.panels[kind] = 1;
          const float t = time_kind(h, kind, ev.a, ev.b);
          ++out.timed;
          if (t < 0.98f * tb) best = 1, best_lay = lay, tb = t;
        }
        if (!big || P > max_panels) break;
        ensure_panel_segs(h, pass_is_csr(kind), P);
        h.ix.panels[kind] = P;
        const float t = time_kind(h, kind, ev.a, ev.b);
        ++out.timed;
        if (t < 0.98f * tb) best = P, best_lay = lay, tb = t;
      }
    }
    h.ix.panels[kind] = best;
    h.ix.layout[kind] = best_lay;
    out.panels[kind] = best;
    out.layout[kind] = best_lay;
    out.ms[kind] = tb;
    out.ms_single[kind] = t1;
  }
  h.prof.on = prof;
  h.tuned = true;
  if (info) *info = out;
}

// Fastest of three timed gather-only passes over the entries of pass kind
// `kind` in index order (ms); *bytes = rows gathered x row bytes.
float gather_roof_dev(bm_ctx& h, int kind, double* bytes) {
  const Index& ix = h.ix;
  const bool csr = pass_is_csr(kind);
  const float* X = csr ? h.H.get() : h.W.get();
  const int32_t* idx = csr ? ix.col.get() : ix.row.get();
  const int nchunk = h.ld / 4;
  const int V = (nchunk + 7) / 8;
  const int grid = num_sms() * 8;
  DevBuf<float> out;
  out.alloc((size_t)grid * 8);
  Events ev;
  float best = 1e30f;
  for (int r = 0; r < 4; ++r) {
    BM_CUDA(cudaEventRecord(ev.a, h.stream));
    switch (V) {
      case 1: k_gather_roof<1><<<grid, 256, 0, h.stream>>>(idx, ix.nnz, X, h.ld, nchunk, out.get()); break;
      case 2: k_gather_roof<2><<<grid, 256, 0, h.stream>>>(idx, ix.nnz, X, h.ld, nchunk, out.get()); break;
      case 3: k_gather_roof<3><<<grid, 256, 0, h.stream>>>(idx, ix.nnz, X, h.ld, nchunk, out.get()); break;
      default: k_gather_roof<4><<<grid, 256, 0, h.stream>>>(idx, ix.nnz, X, h.ld, nchunk, out.get()); break;
    }
    BM_CHECK_LAUNCH();
    BM_CUDA(cudaEventRecord(ev.b, h.stream));
    BM_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    BM_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
    if (r > 0) best = std::min(best, ms);      // the first launch warms up
  }
  *bytes = (double)ix.nnz * (double)nchunk * 16.0;
  return best;
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

bm_status bm_gather_roof(bm_handle h, int32_t kind, double* ms, double* gbs) {
  if (!h) return BM_ERR_INVALID;
  return guard_call(h->err, [&] {
    BM_REQUIRE(kind >= 0 && kind < kPassKinds, BM_ERR_INVALID, "bm_gather_roof: unknown pass kind");
    BM_REQUIRE(h->k >= 1, BM_ERR_INVALID, "bm_gather_roof: no factors yet");
    double bytes = 0;
    const float t = gather_roof_dev(*h, kind, &bytes);
    if (ms) *ms = t;
    if (gbs) *gbs = bytes / (t * 1e-3) / 1e9;
  });
}

bm_status bm_set_layout(bm_handle h, const int32_t* layout) {
  if (!h || !layout) return BM_ERR_INVALID;
  return guard_call(h->err, [&] {
    for (int k = 0; k < kPassKinds; ++k)
      BM_REQUIRE(layout[k] >= -1 && layout[k] <= 1, BM_ERR_INVALID, "bm_set_layout: layouts must be -1, 0 or 1");
    for (int k = 0; k < kPassKinds; ++k) h->ix.layout[k] = layout[k];
  });
}

bm_status bm_get_layout(bm_handle h, int32_t* layout) {
  if (!h || !layout) return BM_ERR_INVALID;
  for (int k = 0; k < kPassKinds; ++k) layout[k] = pass_ws(h->ix, k) ? 1 : 0;
  return BM_OK;
}

}  // extern "C"
