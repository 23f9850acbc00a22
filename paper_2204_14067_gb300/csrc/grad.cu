// Sparse loss and gradient of (MF): SDDMM residual + the two SpMMs, the
// exact line-search coefficients of the BM phase, and dense FP64-reduced
// helpers.  One warp owns one segment of a row (CSR pass) or a column (CSC
// pass); four lanes share one observed entry, each lane holding V float4
// chunks of the k-vector, so a warp advances eight entries at a time.
#include <algorithm>

#include "ctx.cuh"

namespace bm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPassThreads = 256;

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
__device__ __forceinline__ void axpy4(float4& acc, float s, float4 x) {
  acc.x = fmaf(s, x.x, acc.x);
  acc.y = fmaf(s, x.y, acc.y);
  acc.z = fmaf(s, x.z, acc.z);
  acc.w = fmaf(s, x.w, acc.w);
}
__device__ __forceinline__ float4 shfl_xor4(float4 v, int m) {
  v.x += __shfl_xor_sync(kFull, v.x, m);
  v.y += __shfl_xor_sync(kFull, v.y, m);
  v.z += __shfl_xor_sync(kFull, v.z, m);
  v.w += __shfl_xor_sync(kFull, v.w, m);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

struct PassArgs {
  const int32_t* seg_row;
  const int64_t* seg_beg;
  const int64_t* seg_end;
  const int32_t* seg_slot;
  int64_t nseg;
  const int32_t* idx;   // index of the gathered row for each entry (pass order)
  const float* aval;    // observed value A_e (pass order)
  const float* own;     // rows owned by the pass (W for CSR, H for CSC)
  const float* oth;     // gathered rows
  int ld, nchunk;       // leading dimension, ld / 4
  float lam;
  float* out;           // gradient rows
  float* partial;       // partial sums of multi-segment rows
  double* fseg;         // per-segment 1/2 sum r^2 (nullable)
  float* r_out;         // residual in pass order (nullable)
};

// r_e = <own_i, oth_j> - a_e;  out_i = sum_e r_e oth_j + lam own_i
template <int V>
__global__ void __launch_bounds__(kPassThreads) k_grad_pass(PassArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nseg; s += nwarps) {
    const int i = a.seg_row[s];
    const int64_t beg = a.seg_beg[s], end = a.seg_end[s];
    const float* ownrow = a.own + (int64_t)i * a.ld;
    float4 w[V], acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = l + 4 * v;
      w[v] = c < a.nchunk ? ldg4(ownrow + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
      acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float fs = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < end;
      const int j = valid ? __ldg(a.idx + e) : 0;
      const float av = valid ? __ldg(a.aval + e) : 0.f;
#pragma unroll 2
      for (int t = 0; t < 4; ++t) {
        const int src = t * 8 + g;
        const int jj = __shfl_sync(kFull, j, src);
        const float aa = __shfl_sync(kFull, av, src);
        const bool ok = e0 + src < end;
        const float* orow = a.oth + (int64_t)jj * a.ld;
        float4 hv[V];
        float d = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + 4 * v;
          hv[v] = c < a.nchunk ? ldg4(orow + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
          d += dot4(w[v], hv[v]);
        }
        d += __shfl_xor_sync(kFull, d, 1);
        d += __shfl_xor_sync(kFull, d, 2);
        const float r = ok ? d - aa : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) axpy4(acc[v], r, hv[v]);
        if (l == 0) {
          fs = fmaf(r, r, fs);
          if (a.r_out && ok) a.r_out[e0 + src] = r;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      acc[v] = shfl_xor4(acc[v], 4);
      acc[v] = shfl_xor4(acc[v], 8);
      acc[v] = shfl_xor4(acc[v], 16);
    }
    fs = warp_sum(fs);
    if (g == 0) {
      const int slot = a.seg_slot[s];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = l + 4 * v;
        if (c < a.nchunk) {
          if (slot < 0) {
            float4 o = acc[v];
            axpy4(o, a.lam, w[v]);
            *reinterpret_cast<float4*>(a.out + (int64_t)i * a.ld + 4 * c) = o;
          } else {
            *reinterpret_cast<float4*>(a.partial + (int64_t)slot * a.ld + 4 * c) = acc[v];
          }
        }
      }
    }
    if (a.fseg && lane == 0) a.fseg[s] = 0.5 * (double)fs;
  }
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
    float s = 0.f;
    for (int u = 0; u < mcount[q]; ++u) s += partial[(f + u) * ld + c];
    const int64_t o = (int64_t)i * ld + c;
    out[o] = fmaf(lam, own[o], s);
  }
}

// Deterministic single-block sum of doubles: out[0] = sum x[0..n)
__global__ void k_sum_double(const double* __restrict__ x, int64_t n, int stride, int comp,
                             double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i * stride + comp];
  sh[threadIdx.x] = s;
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

// ---------------------------------------------------------------- line search
struct LsArgs {
  const int32_t* seg_row;
  const int64_t* seg_beg;
  const int64_t* seg_end;
  int64_t nseg;
  const int32_t* idx;
  const float* r;        // residual in CSR order
  const float* W;
  const float* DW;
  const float* H;
  const float* DH;
  int ld, nchunk;
  double* part;          // [nseg * 4]: sum r b, sum (b^2 + 2 r c), sum b c, sum c^2
};

// b_e = <DW_i, H_j> + <W_i, DH_j>,  c_e = <DW_i, DH_j>
template <int V>
__global__ void __launch_bounds__(kPassThreads) k_ls_pass(LsArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nseg; s += nwarps) {
    const int i = a.seg_row[s];
    const int64_t beg = a.seg_beg[s], end = a.seg_end[s];
    float4 w[V], dw[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = l + 4 * v;
      const bool in = c < a.nchunk;
      w[v] = in ? ldg4(a.W + (int64_t)i * a.ld + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
      dw[v] = in ? ldg4(a.DW + (int64_t)i * a.ld + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float s_rb = 0.f, s_bb = 0.f, s_bc = 0.f, s_cc = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < end;
      const int j = valid ? __ldg(a.idx + e) : 0;
      const float rv = valid ? __ldg(a.r + e) : 0.f;
#pragma unroll 2
      for (int t = 0; t < 4; ++t) {
        const int src = t * 8 + g;
        const int jj = __shfl_sync(kFull, j, src);
        const float rr = __shfl_sync(kFull, rv, src);
        const bool ok = e0 + src < end;
        float b = 0.f, c = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int cc = l + 4 * v;
          const bool in = cc < a.nchunk;
          const float4 h = in ? ldg4(a.H + (int64_t)jj * a.ld + 4 * cc) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 dh = in ? ldg4(a.DH + (int64_t)jj * a.ld + 4 * cc) : make_float4(0.f, 0.f, 0.f, 0.f);
          b += dot4(dw[v], h) + dot4(w[v], dh);
          c += dot4(dw[v], dh);
        }
        b += __shfl_xor_sync(kFull, b, 1);
        b += __shfl_xor_sync(kFull, b, 2);
        c += __shfl_xor_sync(kFull, c, 1);
        c += __shfl_xor_sync(kFull, c, 2);
        if (ok && l == 0) {
          s_rb = fmaf(rr, b, s_rb);
          s_bb = fmaf(b, b, fmaf(2.f * rr, c, s_bb));
          s_bc = fmaf(b, c, s_bc);
          s_cc = fmaf(c, c, s_cc);
        }
      }
    }
    s_rb = warp_sum(s_rb);
    s_bb = warp_sum(s_bb);
    s_bc = warp_sum(s_bc);
    s_cc = warp_sum(s_cc);
    if (lane == 0) {
      a.part[s * 4 + 0] = s_rb;
      a.part[s * 4 + 1] = s_bb;
      a.part[s * 4 + 2] = s_bc;
      a.part[s * 4 + 3] = s_cc;
    }
  }
}

int pass_grid(int64_t nseg) {
  const int64_t warps_per_block = kPassThreads / 32;
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nseg, warps_per_block), (int64_t)num_sms() * 16));
}

template <int V>
void launch_grad(const PassArgs& a, cudaStream_t st) {
  k_grad_pass<V><<<pass_grid(a.nseg), kPassThreads, 0, st>>>(a);
}

void launch_grad_v(int V, const PassArgs& a, cudaStream_t st) {
  switch (V) {
    case 1: launch_grad<1>(a, st); break;
    case 2: launch_grad<2>(a, st); break;
    case 3: launch_grad<3>(a, st); break;
    case 4: launch_grad<4>(a, st); break;
    case 5: launch_grad<5>(a, st); break;
    case 6: launch_grad<6>(a, st); break;
    case 7: launch_grad<7>(a, st); break;
    case 8: launch_grad<8>(a, st); break;
    default: throw Error{BM_ERR_INVALID, "rank above 128 is not supported"};
  }
}

template <int V>
void launch_ls(const LsArgs& a, cudaStream_t st) {
  k_ls_pass<V><<<pass_grid(a.nseg), kPassThreads, 0, st>>>(a);
}

void launch_ls_v(int V, const LsArgs& a, cudaStream_t st) {
  switch (V) {
    case 1: launch_ls<1>(a, st); break;
    case 2: launch_ls<2>(a, st); break;
    case 3: launch_ls<3>(a, st); break;
    case 4: launch_ls<4>(a, st); break;
    case 5: launch_ls<5>(a, st); break;
    case 6: launch_ls<6>(a, st); break;
    case 7: launch_ls<7>(a, st); break;
    case 8: launch_ls<8>(a, st); break;
    default: throw Error{BM_ERR_INVALID, "rank above 128 is not supported"};
  }
}

int chunks_per_lane(int ld) { return std::max(1, (int)ceil_div(ld / 4, 4)); }

void run_pass(bm_ctx& h, bool csr, bool want_grad, bool store_r, double* fseg) {
  const Index& ix = h.ix;
  const Segs& sg = csr ? ix.rs : ix.cs;
  PassArgs a;
  a.seg_row = sg.row.get();
  a.seg_beg = sg.beg.get();
  a.seg_end = sg.end.get();
  a.seg_slot = sg.slot.get();
  a.nseg = sg.nseg;
  a.idx = csr ? ix.col.get() : ix.row.get();
  a.aval = csr ? ix.val.get() : ix.cval.get();
  a.own = csr ? h.W.get() : h.H.get();
  a.oth = csr ? h.H.get() : h.W.get();
  a.ld = h.ld;
  a.nchunk = h.ld / 4;
  a.lam = (float)h.lambda;
  a.out = csr ? h.gW.get() : h.gH.get();
  a.partial = h.sc.partial.get();
  a.fseg = fseg;
  a.r_out = store_r ? (csr ? h.r_csr.get() : h.r_csc.get()) : nullptr;
  (void)want_grad;
  BM_LAUNCH(h, csr ? "grad_csr" : "grad_csc", launch_grad_v(chunks_per_lane(h.ld), a, h.stream));
  if (sg.nmulti) {
    const int64_t work = sg.nmulti * h.ld;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), num_sms() * 8));
    BM_LAUNCH(h, "grad_fixup",
              k_fixup<<<grid, 256, 0, h.stream>>>(sg.mrow.get(), sg.mfirst.get(), sg.mcount.get(), sg.nmulti,
                                                  h.sc.partial.get(), a.own, h.ld, a.lam, a.out));
  }
}

}  // namespace

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
  run_pass(h, true, want_grad, store_r, fseg);
  k_sum_double<<<1, 1024, 0, h.stream>>>(fseg, ix.rs.nseg, 1, 0, h.sc.scal.get() + 1);
  BM_CHECK_LAUNCH();
  if (want_grad || store_r) run_pass(h, false, want_grad, store_r, nullptr);
  BM_CUDA(cudaMemcpyAsync(&o.f, h.sc.scal.get() + 1, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  o.nW2 = dot_dev(h, h.W.get(), h.W.get(), ix.m * h.ld);
  o.nH2 = dot_dev(h, h.H.get(), h.H.get(), ix.n * h.ld);
  return o;
}

void line_search_coeffs_dev(bm_ctx& h, double c[5]) {
  const Index& ix = h.ix;
  LsArgs a;
  a.seg_row = ix.rs.row.get();
  a.seg_beg = ix.rs.beg.get();
  a.seg_end = ix.rs.end.get();
  a.nseg = ix.rs.nseg;
  a.idx = ix.col.get();
  a.r = h.r_csr.get();
  a.W = h.W.get();
  a.DW = h.DW.get();
  a.H = h.H.get();
  a.DH = h.DH.get();
  a.ld = h.ld;
  a.nchunk = h.ld / 4;
  a.part = h.sc.fseg.get();
  BM_LAUNCH(h, "linesearch_csr", launch_ls_v(chunks_per_lane(h.ld), a, h.stream));
  for (int q = 0; q < 4; ++q) {
    k_sum_double<<<1, 1024, 0, h.stream>>>(a.part, ix.rs.nseg, 4, q, h.sc.scal.get() + 2 + q);
    BM_CHECK_LAUNCH();
  }
  double sums[4];
  BM_CUDA(cudaMemcpyAsync(sums, h.sc.scal.get() + 2, sizeof(sums), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  const double lam = h.lambda;
  const int64_t mW = ix.m * h.ld, nH = ix.n * h.ld;
  const double WDW = dot_dev(h, h.W.get(), h.DW.get(), mW) + dot_dev(h, h.H.get(), h.DH.get(), nH);
  const double DD = dot_dev(h, h.DW.get(), h.DW.get(), mW) + dot_dev(h, h.DH.get(), h.DH.get(), nH);
  c[1] = sums[0] + lam * WDW;
  c[2] = 0.5 * sums[1] + 0.5 * lam * DD;
  c[3] = sums[2];
  c[4] = 0.5 * sums[3];
}

}  // namespace bm
