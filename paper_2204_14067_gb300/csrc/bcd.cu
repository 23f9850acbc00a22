// Column-block coordinate descent for the BM phase of matrix completion: the
// form of polyMF-SS the paper adopts (matrix completion experiments): each
// block is one column of W and the same column of H, updated with an exact
// line search.  For block c, with the residual r_e = <W_i, H_j> - a_e on Omega:
//
//   g_w = R h_c + lam w_c,  g_h = R^T w_c + lam h_c,  (d_w, d_h) = -(g_w, g_h);
//   on Omega the residual moves as r + s b + s^2 cc with b_e = d_w,i h_c,j +
//   w_c,i d_h,j and cc_e = d_w,i d_h,j, so the objective along the direction
//   is the quartic  F - s G + s^2 (1/2 sum (b^2 + 2 r cc) + lam/2 G)
//   + s^3 sum b cc + s^4 1/2 sum cc^2,  G = |g_w|^2 + |g_h|^2,
//   minimised over s >= 0 (the full-gradient BM phase's rule); then w_c, h_c
//   and the residual (CSR and CSC order) are updated in place.
//
// Every pass is a warp per row (column) segment of the existing work splits,
// and block c's residual update shares its two passes with block c+1's
// gradient (three passes over Omega per block);
// the column being updated is copied to contiguous vectors first so the
// per-entry gathers read 4 bytes from an L2-resident vector.  Rows spanning
// several segments use the partial slots and a fixed-order fix-up, and the
// reductions are two-stage, so results are deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "dense.cuh"

namespace bm {

struct BcdState {
  DevBuf<float> wc, hc, gw, gh;     // column c of W and H, block gradients (contiguous)
  DevBuf<float> wn, hn, gwn, ghn;   // the same for column c+1 (the fused passes fill them)
  DevBuf<double> segs4;             // line-search sums per CSR segment (4 each)
  DevBuf<double> part, out;         // reduction partials and the 5 scalars read back
};

void bcd_destroy(BcdState* s) { delete s; }

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

int parts_n() { return std::max(1, std::min(1024, 2 * num_sms())); }

int seg_grid(int64_t nseg) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(nseg, 1), 8), (int64_t)num_sms() * 16));
}

struct SegView {
  const int32_t* row;
  const int64_t* beg;
  const int64_t* end;
  const int32_t* slot;
  int64_t nseg;
};

SegView view(const Segs& s) { return SegView{s.row.get(), s.beg.get(), s.end.get(), s.slot.get(), s.nseg}; }

__global__ void k_col_get(const float* __restrict__ X, int ld, int c, int64_t rows, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = X[i * ld + c];
}

__global__ void k_col_axpy(float* __restrict__ X, int ld, int c, int64_t rows, const float* __restrict__ d, float s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    X[i * ld + c] = fmaf(s, d[i], X[i * ld + c]);
}

__global__ void k_col_fixup(const int32_t* __restrict__ mrow, const int32_t* __restrict__ mfirst,
                            const int32_t* __restrict__ mcount, int64_t nmulti, const float* __restrict__ partial,
                            const float* __restrict__ own, float lam, float* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nmulti; q += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int u = 0; u < mcount[q]; ++u) acc += partial[mfirst[q] + u];
    const int i = mrow[q];
    out[i] = fmaf(lam, own[i], acc);
  }
}

// per CSR segment: (sum b^2 + 2 r cc, sum b cc, sum cc^2) with d = -g
__global__ void __launch_bounds__(kThreads) k_col_ls(SegView sg, const int32_t* __restrict__ col,
                                                    const float* __restrict__ r, const float* __restrict__ wc,
                                                    const float* __restrict__ hc, const float* __restrict__ gw,
                                                    const float* __restrict__ gh, double* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < sg.nseg; s += nwarps) {
    const int i = sg.row[s];
    const int64_t beg = sg.beg[s], end = sg.end[s];
    const float dwi = -gw[i], wi = wc[i];
    float s2 = 0.f, s3 = 0.f, s4 = 0.f;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int j = __ldg(col + e);
      const float dhj = -__ldg(gh + j), hj = __ldg(hc + j), re = __ldg(r + e);
      const float b = fmaf(dwi, hj, wi * dhj), cc = dwi * dhj;
      s2 = fmaf(b, b, fmaf(2.f * re, cc, s2));
      s3 = fmaf(b, cc, s3);
      s4 = fmaf(cc, cc, s4);
    }
    double d2 = s2, d3 = s3, d4 = s4;
    for (int o = 16; o > 0; o >>= 1) {
      d2 += __shfl_xor_sync(kFull, d2, o);
      d3 += __shfl_xor_sync(kFull, d3, o);
      d4 += __shfl_xor_sync(kFull, d4, o);
    }
    if (lane == 0) {
      sums[4 * s + 0] = d2;
      sums[4 * s + 1] = d3;
      sums[4 * s + 2] = d4;
      sums[4 * s + 3] = 0.0;
    }
  }
}

// r_e += s b_e + s^2 cc_e over the segments of one order: the segment's own
// index is `own_is_row ? i : j`, the entry index gives the other
__global__ void __launch_bounds__(kThreads) k_col_update(SegView sg, const int32_t* __restrict__ idx, bool own_is_row,
                                                        float* __restrict__ r, const float* __restrict__ wc,
                                                        const float* __restrict__ hc, const float* __restrict__ gw,
                                                        const float* __restrict__ gh, float step) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float s2 = step * step;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < sg.nseg; s += nwarps) {
    const int o = sg.row[s];
    const int64_t beg = sg.beg[s], end = sg.end[s];
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int x = __ldg(idx + e);
      const int i = own_is_row ? o : x, j = own_is_row ? x : o;
      const float dwi = -gw[i], dhj = -gh[j];
      const float b = fmaf(dwi, hc[j], wc[i] * dhj), cc = dwi * dhj;
      r[e] = fmaf(step, b, fmaf(s2, cc, r[e]));
    }
  }
}

// The residual update of block c fused with the block gradient of block c+1
// over the same segments: r_e += step b_e + step^2 cc_e (block c's vectors;
// skipped when update is false), then out_o = sum_e r_e x[idx_e] + lam own_o
// (block c+1's vectors), with the partial slots of the plain column SpMV.
// The arithmetic per entry is that of k_col_update followed by a plain column SpMV.
struct FusedCols {
  const float *wc, *hc, *gw, *gh;   // block c (update)
  float step;
  bool update;
  const float *x, *own;             // block c+1: gathered vector and owned vector
};
__global__ void __launch_bounds__(kThreads) k_col_update_spmv(SegView sg, const int32_t* __restrict__ idx,
                                                             bool own_is_row, float* __restrict__ r, FusedCols f,
                                                             float lam, float* __restrict__ out,
                                                             float* __restrict__ partial) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float s2 = f.step * f.step;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < sg.nseg; s += nwarps) {
    const int o = sg.row[s];
    const int64_t beg = sg.beg[s], end = sg.end[s];
    float acc = 0.f;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int xi = __ldg(idx + e);
      float re = r[e];
      if (f.update) {
        const int i = own_is_row ? o : xi, j = own_is_row ? xi : o;
        const float dwi = -f.gw[i], dhj = -f.gh[j];
        const float b = fmaf(dwi, f.hc[j], f.wc[i] * dhj), cc = dwi * dhj;
        re = fmaf(f.step, b, fmaf(s2, cc, re));
        r[e] = re;
      }
      acc = fmaf(re, __ldg(f.x + xi), acc);
    }
    for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(kFull, acc, w);
    if (lane == 0) {
      const int slot = sg.slot[s];
      if (slot < 0)
        out[o] = fmaf(lam, f.own[o], acc);
      else
        partial[slot] = acc;
    }
  }
}

// part[3 b + q], q: |gw|^2, |gh|^2 contributions, then the 4 line-search sums
__global__ void __launch_bounds__(kThreads) k_norm2_part(const float* __restrict__ a, int64_t na,
                                                        const float* __restrict__ b, int64_t nb,
                                                        double* __restrict__ part) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t0; i < na; i += st) acc += (double)a[i] * a[i];
  for (int64_t i = t0; i < nb; i += st) acc += (double)b[i] * b[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out[q] (q < w) = sum over rows of part[w * row + q], fixed order, one block
__global__ void __launch_bounds__(kThreads) k_rows_sum(const double* __restrict__ part, int64_t rows, int w,
                                                      double* __restrict__ out) {
  __shared__ double sh[4][kThreads];
  double acc[4] = {0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x)
    for (int q = 0; q < w; ++q) acc[q] += part[w * i + q];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < w) out[threadIdx.x] = sh[threadIdx.x][0];
}

BcdState& state(bm_ctx& h) {
  if (!h.bcd) h.bcd = new BcdState();
  BcdState& s = *h.bcd;
  const Index& ix = h.ix;
  s.wc.alloc(ix.m);
  s.hc.alloc(ix.n);
  s.gw.alloc(ix.m);
  s.gh.alloc(ix.n);
  s.wn.alloc(ix.m);
  s.hn.alloc(ix.n);
  s.gwn.alloc(ix.m);
  s.ghn.alloc(ix.n);
  s.segs4.alloc(4 * (size_t)std::max<int64_t>(ix.rs.nseg, 1));
  s.part.alloc(4 * (size_t)parts_n() + 8);
  s.out.alloc(8);
  return s;
}

int grid1(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), 256), (int64_t)num_sms() * 8));
}

// residual update of the block in `cur` (if update) + block gradient into `out`
void col_update_spmv(bm_ctx& h, const Segs& sg, const int32_t* idx, bool own_is_row, float* r, const FusedCols& f,
                     float* out) {
  BM_REQUIRE((int64_t)h.sc.partial.n >= sg.nslots, BM_ERR_INVALID, "column solver: partial buffer too small");
  if (sg.nseg)
    BM_LAUNCH(h, "bcd_update_spmv", k_col_update_spmv<<<seg_grid(sg.nseg), kThreads, 0, h.stream>>>(
                                        view(sg), idx, own_is_row, r, f, (float)h.lambda, out, h.sc.partial.get()));
  if (sg.nmulti)
    BM_LAUNCH(h, "bcd_fixup", k_col_fixup<<<grid1(sg.nmulti), 256, 0, h.stream>>>(
                                  sg.mrow.get(), sg.mfirst.get(), sg.mcount.get(), sg.nmulti, h.sc.partial.get(), f.own,
                                  (float)h.lambda, out));
}

}  // namespace

// `epochs` sweeps over the k column blocks.  Returns F at entry; *F_out = F
// after the last block (read off the last quartic).
double bcd_phase_dev(bm_ctx& h, int epochs, double* F_out) {
  const Index& ix = h.ix;
  double f = residual_dev(h);
  const int64_t mW = ix.m * (int64_t)h.ld, nH = ix.n * (int64_t)h.ld;
  double F = f + 0.5 * h.lambda * (dot_dev(h, h.W.get(), h.W.get(), mW) + dot_dev(h, h.H.get(), h.H.get(), nH));
  const double F_entry = F;
  if (epochs <= 0 || h.k == 0 || ix.nnz == 0) {
    if (F_out) *F_out = F;
    return F_entry;
  }
  BcdState& s = state(h);
  const int parts = parts_n();
  // Per block: the block gradient (for the first block its own two passes;
  // afterwards fused with the previous block's residual update), the
  // line-search sums, one read-back of five scalars, the column updates.
  float *wc = s.wc.get(), *hc = s.hc.get(), *gw = s.gw.get(), *gh = s.gh.get();
  float *wn = s.wn.get(), *hn = s.hn.get(), *gwn = s.gwn.get(), *ghn = s.ghn.get();
  float prev_step = 0.f;
  const int total = epochs * h.k;
  for (int b = 0; b < total; ++b) {
    const int c = b % h.k;
    BM_LAUNCH(h, "bcd_col", k_col_get<<<grid1(ix.m), 256, 0, h.stream>>>(h.W.get(), h.ld, c, ix.m, wn));
    BM_LAUNCH(h, "bcd_col", k_col_get<<<grid1(ix.n), 256, 0, h.stream>>>(h.H.get(), h.ld, c, ix.n, hn));
    // block gradients g_w = R h_c + lam w_c (rows), g_h = R^T w_c + lam h_c (columns), after
    // the previous block's residual update in the same passes
    FusedCols fr{wc, hc, gw, gh, prev_step, b > 0 && prev_step > 0.f, hn, wn};
    FusedCols fc{wc, hc, gw, gh, prev_step, b > 0 && prev_step > 0.f, wn, hn};
    col_update_spmv(h, ix.rs, ix.col.get(), true, h.r_csr.get(), fr, gwn);
    col_update_spmv(h, ix.cs, ix.row.get(), false, h.r_csc.get(), fc, ghn);
    std::swap(wc, wn);
    std::swap(hc, hn);
    std::swap(gw, gwn);
    std::swap(gh, ghn);
    // G = |g_w|^2 + |g_h|^2 and the line-search sums
    BM_LAUNCH(h, "bcd_norm", k_norm2_part<<<parts, kThreads, 0, h.stream>>>(gw, ix.m, gh, ix.n, s.part.get()));
    BM_LAUNCH(h, "bcd_norm", k_rows_sum<<<1, kThreads, 0, h.stream>>>(s.part.get(), parts, 1, s.out.get()));
    BM_LAUNCH(h, "bcd_ls", k_col_ls<<<seg_grid(ix.rs.nseg), kThreads, 0, h.stream>>>(
                               view(ix.rs), ix.col.get(), h.r_csr.get(), wc, hc, gw, gh, s.segs4.get()));
    BM_LAUNCH(h, "bcd_ls", k_rows_sum<<<1, kThreads, 0, h.stream>>>(s.segs4.get(), ix.rs.nseg, 4, s.out.get() + 1));
    double o[5];
    BM_CUDA(cudaMemcpyAsync(o, s.out.get(), 5 * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
    const double G = o[0];
    double q[5] = {F, -G, 0.5 * o[1] + 0.5 * h.lambda * G, o[2], 0.5 * o[3]};
    BM_REQUIRE(std::isfinite(G) && std::isfinite(q[2]), BM_ERR_NUMERIC, "column solver: non-finite sums");
    const double st = quartic_argmin_ext(q);
    prev_step = st > 0 ? (float)st : 0.f;
    if (st > 0) {
      const float sf = (float)st;
      BM_LAUNCH(h, "bcd_axpy", k_col_axpy<<<grid1(ix.m), 256, 0, h.stream>>>(h.W.get(), h.ld, c, ix.m, gw, -sf));
      BM_LAUNCH(h, "bcd_axpy", k_col_axpy<<<grid1(ix.n), 256, 0, h.stream>>>(h.H.get(), h.ld, c, ix.n, gh, -sf));
      F = (((q[4] * st + q[3]) * st + q[2]) * st + q[1]) * st + q[0];
      h.bm_changed = true;
      h.bf_dirty = true;
    }
  }
  // the last block's residual update (the residual stays consistent with W, H)
  if (prev_step > 0.f) {
    BM_LAUNCH(h, "bcd_update", k_col_update<<<seg_grid(ix.rs.nseg), kThreads, 0, h.stream>>>(
                                   view(ix.rs), ix.col.get(), true, h.r_csr.get(), wc, hc, gw, gh, prev_step));
    BM_LAUNCH(h, "bcd_update", k_col_update<<<seg_grid(ix.cs.nseg), kThreads, 0, h.stream>>>(
                                   view(ix.cs), ix.row.get(), false, h.r_csc.get(), wc, hc, gw, gh, prev_step));
  }
  BM_CUDA(cudaStreamSynchronize(h.stream));
  if (F_out) *F_out = F;
  return F_entry;
}

}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_bcd_phase(bm_handle h, int32_t epochs, double* F) {
  if (!h) return BM_ERR_INVALID;
  return guard_call(h->err, [&] {
    BM_REQUIRE(epochs >= 0, BM_ERR_INVALID, "bm_bcd_phase: epochs must be >= 0");
    bcd_phase_dev(*h, epochs, F);
  });
}

}  // extern "C"
