// Sparse loss and gradient of (MF): SDDMM residual + the two SpMMs, the
// exact line-search coefficients of the BM phase, and dense FP64-reduced
// helpers.  One warp owns one segment of a row (CSR pass) or a column (CSC
// pass); four lanes share one observed entry, each lane holding V float4
// chunks of the k-vector, so a warp advances eight entries at a time.
#include <algorithm>

#include "ctx.cuh"
#include "pipe.cuh"
#include <cuda_bf16.h>

namespace bm {
namespace {

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
__device__ __forceinline__ void axpy4(float4& acc, float s, float4 x) {
  acc.x = fmaf(s, x.x, acc.x);
  acc.y = fmaf(s, x.y, acc.y);
  acc.z = fmaf(s, x.z, acc.z);
  acc.w = fmaf(s, x.w, acc.w);
}

// Rows split over several segments: out_i = sum of partials (segment order) + lam own_i
__global__ void k_fixup(const int32_t* __restrict__ mrow, const int32_t* __restrict__ mfirst,
                        const int32_t* __restrict__ mcount, int64_t nmulti, const float* __restrict__ partial,
                        const float* __restrict__ own, int ld, float lam, float* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nmulti * ld;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / ld;
    const int c = (int)(t - q * ld);
    const int i = mrow[q];
    const int64_t f = mfirst[q];
    const int cnt = mcount[q];
    // four running sums over the partials in segment order (u mod 4), added
    // in a fixed order: deterministic, and four loads in flight
    const float* pp = partial + f * ld + c;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int u = 0;
    for (; u + 3 < cnt; u += 4) {
      s0 += pp[(int64_t)u * ld];
      s1 += pp[(int64_t)(u + 1) * ld];
      s2 += pp[(int64_t)(u + 2) * ld];
      s3 += pp[(int64_t)(u + 3) * ld];
    }
    for (; u < cnt; ++u) s0 += pp[(int64_t)u * ld];
    const int64_t o = (int64_t)i * ld + c;
    out[o] = fmaf(lam, own[o], (s0 + s1) + (s2 + s3));
  }
}

// Deterministic single-block sum of doubles: out[0] = sum x[0..n)
__global__ void k_sum_double(const double* __restrict__ x, int64_t n, int stride, int comp,
                             double* __restrict__ out) {
  __shared__ double sh[1024];
  // two running sums per thread (loads in flight), added in a fixed order
  double s = 0.0, t = 0.0;
  const int64_t b = blockDim.x;
  int64_t i = threadIdx.x;
  for (; i + b < n; i += 2 * b) {
    s += x[i * stride + comp];
    t += x[(i + b) * stride + comp];
  }
  if (i < n) s += x[i * stride + comp];
  sh[threadIdx.x] = s + t;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

constexpr int kDotBlocks = 304;
constexpr int kDotThreads = 256;

// Block partials of sum x_i y_i (float4 loads, compensated FP32 per thread)
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const float* __restrict__ x,
                                                             const float* __restrict__ y, int64_t n4,
                                                             double* __restrict__ part) {
  __shared__ double sh[kDotThreads];
  float s = 0.f, comp = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a = reinterpret_cast<const float4*>(x)[i];
    const float4 b = reinterpret_cast<const float4*>(y)[i];
    const float p = dot4(a, b);
    const float yk = p - comp;
    const float t = s + yk;
    comp = (t - s) - yk;
    s = t;
  }
  sh[threadIdx.x] = (double)s - (double)comp;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ x, float a, int64_t n4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 v = reinterpret_cast<float4*>(y)[i];
    axpy4(v, a, reinterpret_cast<const float4*>(x)[i]);
    reinterpret_cast<float4*>(y)[i] = v;
  }
}

__global__ void k_xpby(float* __restrict__ y, const float* __restrict__ x, float b, int64_t n4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 xv = reinterpret_cast<const float4*>(x)[i];
    float4 v = reinterpret_cast<float4*>(y)[i];
    v.x = fmaf(b, v.x, -xv.x);
    v.y = fmaf(b, v.y, -xv.y);
    v.z = fmaf(b, v.z, -xv.z);
    v.w = fmaf(b, v.w, -xv.w);
    reinterpret_cast<float4*>(y)[i] = v;
  }
}


void run_pass(bm_ctx& h, bool csr, bool store_r, double* fseg, float* partial = nullptr) {
  const Index& ix = h.ix;
  const Segs& sg = pass_segs(ix, csr ? kPassGradCsr : kPassGradCsc);
  PipeArgs a{};
  a.seg_row = sg.row.get();
  a.seg_beg = sg.beg.get();
  a.seg_end = sg.end.get();
  a.seg_slot = sg.slot.get();
  a.nseg = sg.nseg;
  a.idx = csr ? ix.col.get() : ix.row.get();
  a.scal = csr ? ix.val.get() : ix.cval.get();
  a.scal8 = ix.codec ? (csr ? ix.val8.get() : ix.cval8.get()) : nullptr;
  a.scal_off = ix.code_off;
  a.o0 = csr ? h.W.get() : h.H.get();
  a.g0 = csr ? h.H.get() : h.W.get();
  a.ld = h.ld;
  a.nchunk = h.ld / 4;
  a.lam = (float)h.lambda;
  a.out = csr ? h.gW.get() : h.gH.get();
  a.ld_out = h.ld;
  a.partial = partial ? partial : h.sc.partial.get();
  a.ld_part = h.ld;
  a.fseg = fseg;
  a.r_out = (store_r && csr) ? h.r_csr.get() : nullptr;
  const bool bf = h.bf_active();
  if (bf) {
    ensure_bf16(h);
    a.g0b = csr ? h.Hb.get() : h.Wb.get();
    a.ldb = h.ldb;
  }
  BM_LAUNCH(h, csr ? (bf ? "grad_csr_bf16" : "grad_csr") : (bf ? "grad_csc_bf16" : "grad_csc"),
            launch_pipe<0>(a, h.stream, bf, pass_ws(ix, csr ? kPassGradCsr : kPassGradCsc)));
  if (sg.nmulti) {
    const int64_t work = sg.nmulti * h.ld;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), num_sms() * 8));
    BM_LAUNCH(h, csr ? "grad_fixup" : "grad_fixup_csc",
              k_fixup<<<grid, 256, 0, h.stream>>>(sg.mrow.get(), sg.mfirst.get(), sg.mcount.get(), sg.nmulti,
                                                  a.partial, a.o0, h.ld, a.lam, a.out));
  }
}

}  // namespace

void side_fork(bm_ctx& h) {
  if (!h.fork_ev) BM_CUDA(cudaEventCreateWithFlags(&h.fork_ev, cudaEventDisableTiming));
  if (!h.join_ev) BM_CUDA(cudaEventCreateWithFlags(&h.join_ev, cudaEventDisableTiming));
  if (!h.side_stream) BM_CUDA(cudaStreamCreateWithFlags(&h.side_stream, cudaStreamNonBlocking));
  BM_CUDA(cudaEventRecord(h.fork_ev, h.stream));
  BM_CUDA(cudaStreamWaitEvent(h.side_stream, h.fork_ev, 0));
}

// A failure here leaves the error pending in the context: the next call on
// the handle's stream (the result read-back) reports it.
void side_join(bm_ctx& h) noexcept {
  if (!h.side_stream) return;
  if (cudaEventRecord(h.join_ev, h.side_stream) == cudaSuccess) cudaStreamWaitEvent(h.stream, h.join_ev, 0);
}

// sum x_i y_i into out (device) on stream st, without waiting; part: kDotBlocks doubles
void dot_async(cudaStream_t st, const float* x, const float* y, int64_t count, double* part, double* out) {
  k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(x, y, count / 4, part);
  BM_CHECK_LAUNCH();
  k_sum_double<<<1, 1024, 0, st>>>(part, kDotBlocks, 1, 0, out);
  BM_CHECK_LAUNCH();
}

double dot_dev(bm_ctx& h, const float* x, const float* y, int64_t count) {
  double* part = h.sc.red.get();
  double* out = h.sc.scal.get();
  const int64_t n4 = count / 4;
  k_dot_partial<<<kDotBlocks, kDotThreads, 0, h.stream>>>(x, y, n4, part);
  BM_CHECK_LAUNCH();
  k_sum_double<<<1, 1024, 0, h.stream>>>(part, kDotBlocks, 1, 0, out);
  BM_CHECK_LAUNCH();
  double r;
  BM_CUDA(cudaMemcpyAsync(&r, out, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  return r;
}

void axpy_dev(bm_ctx& h, float* y, const float* x, float a, int64_t count) {
  const int64_t n4 = count / 4;
  if (!n4) return;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n4, 256), num_sms() * 8));
  k_axpy<<<grid, 256, 0, h.stream>>>(y, x, a, n4);
  BM_CHECK_LAUNCH();
}

void xpby_dev(bm_ctx& h, float* y, const float* x, float b, int64_t count) {
  const int64_t n4 = count / 4;
  if (!n4) return;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n4, 256), num_sms() * 8));
  k_xpby<<<grid, 256, 0, h.stream>>>(y, x, b, n4);
  BM_CHECK_LAUNCH();
}

LossOut loss_grad_dev(bm_ctx& h, bool want_grad, bool store_r) {
  const Index& ix = h.ix;
  LossOut o{0, 0, 0};
  double* fseg = h.sc.fseg.get();
  double* sc = h.sc.scal.get();
  // ||W||^2 and ||H||^2 on the side stream, overlapping the passes (they only
  // read W and H); one read-back of the three sums at the end
  ensure_bf16(h);   // the BF16 copies both passes may gather, before the fork
  if (want_grad) {
    const Segs& sc2 = pass_segs(ix, kPassGradCsc);
    h.sc.partial2.alloc((size_t)std::max<int64_t>(1, sc2.nslots) * h.ld);
  }
  {
    SideScope fork(h);
    {
      OnSideStream side(h);
      dot_async(h.stream, h.W.get(), h.W.get(), ix.m * h.ld, h.sc.red.get(), sc + 12);
      dot_async(h.stream, h.H.get(), h.H.get(), ix.n * h.ld, h.sc.red.get() + kDotBlocks, sc + 13);
      // the column pass beside the row pass (they share only read-only
      // inputs; its split rows use their own partial buffer): the passes'
      // tails overlap
      if (want_grad) run_pass(h, false, false, nullptr, h.sc.partial2.get());
    }
    run_pass(h, true, store_r, fseg);
    k_sum_double<<<1, 1024, 0, h.stream>>>(fseg, pass_segs(ix, kPassGradCsr).nseg, 1, 0, sc + 1);
    BM_CHECK_LAUNCH();
  }   // the handle's stream waits for the side stream here
  double v[13];
  BM_CUDA(cudaMemcpyAsync(v, sc + 1, sizeof(v), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  o.f = v[0];
  o.nW2 = v[11];
  o.nH2 = v[12];
  return o;
}

__global__ void k_to_bf16(const float* __restrict__ src, int64_t rows, int ld, uint16_t* __restrict__ dst, int ldb) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * ldb;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ldb;
    const int c = (int)(t - r * ldb);
    const float x = c < ld ? src[r * ld + c] : 0.f;
    dst[t] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
  }
}

__global__ void k_permute(const float* __restrict__ src, const int32_t* __restrict__ map, float* __restrict__ dst,
                          int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = __ldg(src + __ldg(map + q));
}

void to_bf16_dev(bm_ctx& h, const float* src, int64_t rows, int ld, uint16_t* dst, int ldb) {
  if (rows == 0) return;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows * ldb, 256), (int64_t)num_sms() * 16));
  BM_LAUNCH(h, "to_bf16", k_to_bf16<<<grid, 256, 0, h.stream>>>(src, rows, ld, dst, ldb));
}

void ensure_bf16(bm_ctx& h) {
  if (!h.bf_active() || !h.bf_dirty) return;
  h.ldb = ((h.ld + 7) / 8) * 8;
  to_bf16_dev(h, h.W.get(), h.ix.m, h.ld, h.Wb.get(), h.ldb);
  to_bf16_dev(h, h.H.get(), h.ix.n, h.ld, h.Hb.get(), h.ldb);
  h.bf_dirty = false;
}

double residual_dev(bm_ctx& h) {
  const Index& ix = h.ix;
  double* fseg = h.sc.fseg.get();
  run_pass(h, true, true, fseg);
  k_sum_double<<<1, 1024, 0, h.stream>>>(fseg, pass_segs(ix, kPassGradCsr).nseg, 1, 0, h.sc.scal.get() + 1);
  BM_CHECK_LAUNCH();
  if (ix.nnz) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix.nnz, 256), (int64_t)num_sms() * 16));
    BM_LAUNCH(h, "permute_r", k_permute<<<grid, 256, 0, h.stream>>>(h.r_csr.get(), ix.csc2csr.get(), h.r_csc.get(),
                                                                   ix.nnz));
  }
  double f = 0;
  BM_CUDA(cudaMemcpyAsync(&f, h.sc.scal.get() + 1, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  return f;
}

namespace {
// The line-search pass: per-segment sums of r b, b^2 + 2 r c, b c, c^2.
// Returns the segment count of the split it used.
int64_t ls_pass(bm_ctx& h) {
  const Index& ix = h.ix;
  const Segs& sg = pass_segs(ix, kPassLsCsr);
  PipeArgs a{};
  a.seg_row = sg.row.get();
  a.seg_beg = sg.beg.get();
  a.seg_end = sg.end.get();
  a.seg_slot = sg.slot.get();
  a.nseg = sg.nseg;
  a.idx = ix.col.get();
  a.scal = h.r_csr.get();
  a.o0 = h.W.get();
  a.o1 = h.DW.get();
  a.g0 = h.H.get();
  a.g1 = h.DH.get();
  a.ld = h.ld;
  a.nchunk = h.ld / 4;
  a.fseg = h.sc.fseg.get();
  const bool bf = h.bf_active();
  if (bf) {
    ensure_bf16(h);
    to_bf16_dev(h, h.DH.get(), ix.n, h.ld, h.DHb.get(), h.ldb);
    a.g0b = h.Hb.get();
    a.g1b = h.DHb.get();
    a.ldb = h.ldb;
  }
  BM_LAUNCH(h, bf ? "linesearch_csr_bf16" : "linesearch_csr", launch_pipe<2>(a, h.stream, bf, pass_ws(ix, kPassLsCsr)));
  return sg.nseg;
}
}  // namespace

void tuning_pass_dev(bm_ctx& h, int kind) {
  if (kind == kPassGradCsr) run_pass(h, true, false, h.sc.fseg.get());
  else if (kind == kPassGradCsc) run_pass(h, false, false, nullptr);
  else if (kind == kPassLsCsr) ls_pass(h);
}

void line_search_coeffs_dev(bm_ctx& h, double c[5]) {
  const Index& ix = h.ix;
  const int64_t nseg = ls_pass(h);
  for (int q = 0; q < 4; ++q) {
    k_sum_double<<<1, 1024, 0, h.stream>>>(h.sc.fseg.get(), nseg, 4, q, h.sc.scal.get() + 2 + q);
    BM_CHECK_LAUNCH();
  }
  double sums[4];
  BM_CUDA(cudaMemcpyAsync(sums, h.sc.scal.get() + 2, sizeof(sums), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  const double lam = h.lambda;
  const int64_t mW = ix.m * h.ld, nH = ix.n * h.ld;
  // phi'(0) = <grad F, D> from the gradient already in memory (h.gW, h.gH):
  // equal to sum r b + lam (<W,DW> + <H,DH>) but free of its cancellation
  const double GD = dot_dev(h, h.gW.get(), h.DW.get(), mW) + dot_dev(h, h.gH.get(), h.DH.get(), nH);
  const double DD = dot_dev(h, h.DW.get(), h.DW.get(), mW) + dot_dev(h, h.DH.get(), h.DH.get(), nH);
  c[1] = GD;
  c[2] = 0.5 * sums[1] + 0.5 * lam * DD;
  c[3] = sums[2];
  c[4] = 0.5 * sums[3];
}

}  // namespace bm
