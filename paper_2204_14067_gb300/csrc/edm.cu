// Distance-geometry factorised loss of Eq. "EDM" (supplement, BM formulation
// of the kernel-estimation and molecular-conformation problems):
//   g(V) = 1/2 sum_{(i,j) in Omega} w_ij (||v_i - v_j||^2 - d_ij^2)^2 + lambda ||V||_F^2
//   grad g(V) = 2 (sum w_ij r_ij E_ij + lambda I) V,  E_ij = (e_i - e_j)(e_i - e_j)^T.
// Omega is stored as a symmetric CSR (both directions of every pair), so row i
// of the gradient, 2 sum_j w_ij r_ij (v_i - v_j) + 2 lambda v_i, needs no atomics.
#include <algorithm>
#include <cmath>

#include "edm.cuh"


namespace bm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
thread_local std::string g_edm_error;

__global__ void k_edm_validate(const int32_t* __restrict__ i, const int32_t* __restrict__ j,
                               const float* __restrict__ d, const float* __restrict__ w, int64_t P, int64_t n,
                               int* __restrict__ flags) {
  int bad_idx = 0, bad_val = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = i[p], b = j[p];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b) bad_idx = 1;
    if (!isfinite(d[p]) || d[p] < 0.f || (w && !isfinite(w[p]))) bad_val = 1;
  }
  if (__any_sync(kFull, bad_idx) && (threadIdx.x & 31) == 0) atomicOr(flags, 1);
  if (__any_sync(kFull, bad_val) && (threadIdx.x & 31) == 0) atomicOr(flags + 1, 1);
}

// directed entries: 2p -> (i, j), 2p+1 -> (j, i); value = pair id
__global__ void k_edm_keys(const int32_t* __restrict__ i, const int32_t* __restrict__ j, int64_t P, uint64_t n,
                           uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = (uint64_t)i[p], b = (uint64_t)j[p];
    keys[2 * p] = a * n + b;
    keys[2 * p + 1] = b * n + a;
    vals[2 * p] = (uint32_t)p;
    vals[2 * p + 1] = (uint32_t)p;
  }
}

__global__ void k_edm_finalize(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sv, int64_t E,
                               uint64_t n, const float* __restrict__ d, const float* __restrict__ w,
                               int32_t* __restrict__ col, float* __restrict__ dsq, float* __restrict__ wo,
                               int* __restrict__ flags) {
  int dup = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = sk[e];
    col[e] = (int32_t)(key % n);
    const uint32_t p = sv[e];
    const float dv = d[p];
    dsq[e] = dv * dv;
    wo[e] = w ? w[p] : 1.f;
    if (e > 0 && sk[e - 1] == key) dup = 1;
  }
  if (__any_sync(kFull, dup) && (threadIdx.x & 31) == 0) atomicOr(flags + 2, 1);
}

struct EdmArgs {
  const int32_t* seg_row;
  const int64_t* seg_beg;
  const int64_t* seg_end;
  const int32_t* seg_slot;
  int64_t nseg;
  const int32_t* col;
  const float* dsq;
  const float* w;
  const float* V;
  int ld, nchunk;
  float lam;
  float* out;
  float* partial;
  double* fseg;
  float* r_out;     // nullable: residual per directed entry
};

// Four lanes per directed entry, V float4 chunks per lane.
template <int VC>
__global__ void __launch_bounds__(256) k_edm_pass(EdmArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nseg; s += nwarps) {
    const int i = a.seg_row[s];
    const int64_t beg = a.seg_beg[s], end = a.seg_end[s];
    float4 vi[VC], acc[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
      const int c = l + 4 * v;
      vi[v] = c < a.nchunk ? __ldg(reinterpret_cast<const float4*>(a.V + (int64_t)i * a.ld) + c)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float fs = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < end;
      const int j = valid ? __ldg(a.col + e) : 0;
      const float dq = valid ? __ldg(a.dsq + e) : 0.f;
      const float wv = valid ? __ldg(a.w + e) : 0.f;
#pragma unroll 2
      for (int t = 0; t < 4; ++t) {
        const int src = t * 8 + g;
        const int jj = __shfl_sync(kFull, j, src);
        const float dd = __shfl_sync(kFull, dq, src);
        const float ww = __shfl_sync(kFull, wv, src);
        const bool ok = e0 + src < end;
        float4 df[VC];
        float sq = 0.f;
#pragma unroll
        for (int v = 0; v < VC; ++v) {
          const int c = l + 4 * v;
          const float4 vj = c < a.nchunk ? __ldg(reinterpret_cast<const float4*>(a.V + (int64_t)jj * a.ld) + c)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
          df[v] = make_float4(vi[v].x - vj.x, vi[v].y - vj.y, vi[v].z - vj.z, vi[v].w - vj.w);
          sq = fmaf(df[v].x, df[v].x, fmaf(df[v].y, df[v].y, fmaf(df[v].z, df[v].z, fmaf(df[v].w, df[v].w, sq))));
        }
        sq += __shfl_xor_sync(kFull, sq, 1);
        sq += __shfl_xor_sync(kFull, sq, 2);
        const float r = ok ? sq - dd : 0.f;
        const float cw = 2.f * ww * r;
#pragma unroll
        for (int v = 0; v < VC; ++v) {
          acc[v].x = fmaf(cw, df[v].x, acc[v].x);
          acc[v].y = fmaf(cw, df[v].y, acc[v].y);
          acc[v].z = fmaf(cw, df[v].z, acc[v].z);
          acc[v].w = fmaf(cw, df[v].w, acc[v].w);
        }
        if (l == 0) {
          fs = fmaf(0.25f * ww * r, r, fs);  // each pair appears twice
          if (a.r_out && ok) a.r_out[e0 + src] = r;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VC; ++v) {
#pragma unroll
      for (int m = 4; m < 32; m <<= 1) {
        acc[v].x += __shfl_xor_sync(kFull, acc[v].x, m);
        acc[v].y += __shfl_xor_sync(kFull, acc[v].y, m);
        acc[v].z += __shfl_xor_sync(kFull, acc[v].z, m);
        acc[v].w += __shfl_xor_sync(kFull, acc[v].w, m);
      }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) fs += __shfl_xor_sync(kFull, fs, m);
    if (g == 0) {
      const int slot = a.seg_slot[s];
#pragma unroll
      for (int v = 0; v < VC; ++v) {
        const int c = l + 4 * v;
        if (c >= a.nchunk) continue;
        float4 o = acc[v];
        if (slot < 0) {
          o.x = fmaf(2.f * a.lam, vi[v].x, o.x);
          o.y = fmaf(2.f * a.lam, vi[v].y, o.y);
          o.z = fmaf(2.f * a.lam, vi[v].z, o.z);
          o.w = fmaf(2.f * a.lam, vi[v].w, o.w);
          reinterpret_cast<float4*>(a.out + (int64_t)i * a.ld)[c] = o;
        } else {
          reinterpret_cast<float4*>(a.partial + (int64_t)slot * a.ld)[c] = o;
        }
      }
    }
    if (lane == 0) a.fseg[s] = (double)fs;
  }
}

__global__ void k_edm_fixup(const int32_t* __restrict__ mrow, const int32_t* __restrict__ mfirst,
                            const int32_t* __restrict__ mcount, int64_t nmulti, const float* __restrict__ partial,
                            const float* __restrict__ V, int ld, float lam, float* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nmulti * ld;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / ld;
    const int c = (int)(t - q * ld);
    float s = 0.f;
    for (int u = 0; u < mcount[q]; ++u) s += partial[((int64_t)mfirst[q] + u) * ld + c];
    const int64_t o = (int64_t)mrow[q] * ld + c;
    out[o] = fmaf(2.f * lam, V[o], s);
  }
}

// g = sum of segment partials + lam ||V||^2, in two deterministic stages:
// block b sums a fixed strided share into part[b], then one block adds the
// parts in order.
constexpr int kTotalThreads = 256;
__global__ void __launch_bounds__(kTotalThreads) k_edm_total_part(const double* __restrict__ fseg, int64_t nseg,
                                                                 const float* __restrict__ V, int64_t nv, double lam,
                                                                 double* __restrict__ part) {
  __shared__ double sh[kTotalThreads];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  for (int64_t i = t0; i < nseg; i += stride) s += fseg[i];
  float q = 0.f;   // FP32 partial of ||V||^2 over this thread's few entries
  for (int64_t i = t0; i < nv; i += stride) q = fmaf(V[i], V[i], q);
  s += lam * (double)q;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kTotalThreads) k_edm_total_final(const double* __restrict__ part, int nparts,
                                                                  double* __restrict__ out) {
  __shared__ double sh[kTotalThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

int total_parts() { return std::max(1, std::min(1024, 2 * num_sms())); }

template <int VC>
void launch_edm(const EdmArgs& a, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(a.nseg, 8), (int64_t)num_sms() * 16));
  k_edm_pass<VC><<<grid, 256, 0, st>>>(a);
}

template <class Fn>
bm_status edm_guarded(bm_edm_ctx* h, Fn&& fn) {
  try {
    fn();
    return BM_OK;
  } catch (const Error& e) {
    (h ? h->err : g_edm_error) = e.msg;
    return e.code;
  } catch (...) {
    (h ? h->err : g_edm_error) = "unexpected exception";
    return BM_ERR_CUDA;
  }
}

template <typename T>
const T* edm_to_device(const T* src, int64_t count, DevBuf<T>& tmp, cudaStream_t st) {
  if (!src || count == 0 || is_device_ptr(src)) return src;
  tmp.alloc(count);
  BM_CUDA(cudaMemcpyAsync(tmp.get(), src, count * sizeof(T), cudaMemcpyHostToDevice, st));
  return tmp.get();
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_edm_create(int64_t n, int64_t npairs, const int32_t* i, const int32_t* j, const float* d,
                        const float* w, double lambda, int32_t k_max, bm_edm_handle* out) {
  if (!out) return BM_ERR_INVALID;
  *out = nullptr;
  bm_edm_ctx* h = nullptr;
  bm_status st = edm_guarded(nullptr, [&] {
    BM_REQUIRE(n >= 2 && n < (1LL << 31), BM_ERR_INVALID, "bm_edm_create: n must be in [2, 2^31)");
    BM_REQUIRE(npairs >= 0 && 2 * npairs < (1LL << 31), BM_ERR_INVALID, "bm_edm_create: too many pairs");
    BM_REQUIRE(npairs == 0 || (i && j && d), BM_ERR_INVALID, "bm_edm_create: NULL pair array");
    BM_REQUIRE(std::isfinite(lambda), BM_ERR_INVALID, "bm_edm_create: lambda must be finite");
    BM_REQUIRE(k_max >= 1 && k_max <= 128 && k_max <= n, BM_ERR_INVALID, "bm_edm_create: k_max out of range");
    h = new bm_edm_ctx();
    h->n = n;
    h->npairs = npairs;
    h->lambda = lambda;
    h->k_max = k_max;
    BM_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    cudaStream_t s = h->stream;
    DevBuf<int32_t> ti, tj;
    DevBuf<float> td, tw;
    const int32_t* id = edm_to_device(i, npairs, ti, s);
    const int32_t* jd = edm_to_device(j, npairs, tj, s);
    const float* dd = edm_to_device(d, npairs, td, s);
    const float* wd = edm_to_device(w, npairs, tw, s);
    DevBuf<int> flags;
    flags.alloc(4);
    BM_CUDA(cudaMemsetAsync(flags.get(), 0, 4 * sizeof(int), s));
    const int64_t E = 2 * npairs;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(npairs, 1), 256), 4096));
    if (npairs) {
      k_edm_validate<<<grid, 256, 0, s>>>(id, jd, dd, wd, npairs, n, flags.get());
      BM_CHECK_LAUNCH();
    }
    int hf[4];
    BM_CUDA(cudaMemcpyAsync(hf, flags.get(), sizeof(hf), cudaMemcpyDeviceToHost, s));
    BM_CUDA(cudaStreamSynchronize(s));
    BM_REQUIRE(!hf[0], BM_ERR_INVALID, "bm_edm_create: pair index out of range or i == j");
    BM_REQUIRE(!hf[1], BM_ERR_INVALID, "bm_edm_create: distances must be finite and >= 0, weights finite");
    h->row_ptr.alloc(n + 1);
    h->col.alloc(std::max<int64_t>(E, 1));
    h->dsq.alloc(std::max<int64_t>(E, 1));
    h->w.alloc(std::max<int64_t>(E, 1));
    {
      DevBuf<uint64_t> k0, k1;
      DevBuf<uint32_t> v0, v1;
      k0.alloc(E); k1.alloc(E); v0.alloc(E); v1.alloc(E);
      if (npairs) {
        k_edm_keys<<<grid, 256, 0, s>>>(id, jd, npairs, (uint64_t)n, k0.get(), v0.get());
        BM_CHECK_LAUNCH();
      }
      sort_pairs_ext(k0, v0, k1, v1, E, key_bits_ext((uint64_t)n * (uint64_t)n), s);
      lower_bounds_ext(k0.get(), E, (uint64_t)n, n, h->row_ptr.get(), s);
      if (E) {
        k_edm_finalize<<<grid, 256, 0, s>>>(k0.get(), v0.get(), E, (uint64_t)n, dd, wd, h->col.get(), h->dsq.get(),
                                            h->w.get(), flags.get());
        BM_CHECK_LAUNCH();
      }
      BM_CUDA(cudaMemcpyAsync(hf, flags.get(), sizeof(hf), cudaMemcpyDeviceToHost, s));
      BM_CUDA(cudaStreamSynchronize(s));
      BM_REQUIRE(!hf[2], BM_ERR_INVALID, "bm_edm_create: a pair appears twice");
    }
    build_segs_ext(h->seg, h->row_ptr, n, s);
    const int ldmax = round_up4(k_max);
    h->V.alloc((size_t)n * ldmax);
    h->gV.alloc((size_t)n * ldmax);
    h->partial.alloc((size_t)std::max<int64_t>(1, h->seg.nslots) * ldmax);
    h->fseg.alloc(std::max<int64_t>(1, h->seg.nseg));
    h->red.alloc(total_parts() + 1);
    BM_CUDA(cudaMemsetAsync(h->V.get(), 0, (size_t)n * ldmax * sizeof(float), s));
    // the dense routines of the solve run on the handle's stream with this scratch
    bm_default_options(&h->opt);
    h->core.stream = h->stream;
    BM_CUDA(cudaGetDevice(&h->core.device));
    h->core.sc.red.alloc(4096);
    h->core.sc.scal.alloc(64);
    BM_CUDA(cudaStreamSynchronize(s));
  });
  if (st != BM_OK) {
    if (h) bm_edm_destroy(h);
    return st;
  }
  *out = h;
  return BM_OK;
}

void bm_edm_destroy(bm_edm_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaStream_t s = h->own_stream;
  delete h;
  if (s) cudaStreamDestroy(s);
}

bm_status bm_edm_set_stream(bm_edm_handle h, void* stream) {
  if (!h) return BM_ERR_INVALID;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->err = "bm_edm_set_stream: synchronising the previous stream failed";
    return BM_ERR_CUDA;
  }
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  return BM_OK;
}

const char* bm_edm_last_error(bm_edm_handle h) { return h ? h->err.c_str() : g_edm_error.c_str(); }

bm_status bm_edm_set_factor(bm_edm_handle h, int32_t k, const float* V) {
  if (!h) return BM_ERR_INVALID;
  return edm_guarded(h, [&] {
    BM_REQUIRE(k >= 1 && k <= h->k_max, BM_ERR_INVALID, "bm_edm_set_factor: k must be in [1, k_max]");
    BM_REQUIRE(V, BM_ERR_INVALID, "bm_edm_set_factor: NULL factor");
    h->k = k;
    h->ld = round_up4(k);
    bm::edm_solve_reset(h->ss);
    BM_CUDA(cudaMemsetAsync(h->V.get(), 0, (size_t)h->n * h->ld * sizeof(float), h->stream));
    BM_CUDA(cudaMemcpy2DAsync(h->V.get(), h->ld * sizeof(float), V, k * sizeof(float), k * sizeof(float), h->n,
                              is_device_ptr(V) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
}

bm_status bm_edm_loss_grad(bm_edm_handle h, double* g, float* gV) {
  if (!h) return BM_ERR_INVALID;
  return edm_guarded(h, [&] {
    BM_REQUIRE(h->k >= 1, BM_ERR_INVALID, "bm_edm_loss_grad: set a factor first");
    const double gv = edm_loss_grad_dev(*h, gV != nullptr, nullptr);
    if (gV) {
      BM_CUDA(cudaMemcpy2DAsync(gV, h->k * sizeof(float), h->gV.get(), h->ld * sizeof(float), h->k * sizeof(float),
                                h->n, is_device_ptr(gV) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
      BM_CUDA(cudaStreamSynchronize(h->stream));
    }
    if (g) *g = gv;
  });
}

}  // extern "C"

namespace bm {

double edm_loss_grad_dev(bm_edm_ctx& hh, bool want_grad, float* r_out, bool sync) {
  bm_edm_ctx* h = &hh;
  EdmArgs a;
  a.seg_row = h->seg.row.get();
  a.seg_beg = h->seg.beg.get();
  a.seg_end = h->seg.end.get();
  a.seg_slot = h->seg.slot.get();
  a.nseg = h->seg.nseg;
  a.col = h->col.get();
  a.dsq = h->dsq.get();
  a.w = h->w.get();
  a.V = h->V.get();
  a.ld = h->ld;
  a.nchunk = h->ld / 4;
  a.lam = (float)h->lambda;
  a.out = h->gV.get();
  a.partial = h->partial.get();
  a.fseg = h->fseg.get();
  a.r_out = r_out;
  const int VC = std::max(1, (a.nchunk + 3) / 4);
  bm_ctx& cx = h->core;
  cx.stream = h->stream;
  if (cx.prof.on) cx.prof.begin("edm_pass", h->stream);
  switch (VC) {
    case 1: launch_edm<1>(a, h->stream); break;
    case 2: launch_edm<2>(a, h->stream); break;
    case 3: launch_edm<3>(a, h->stream); break;
    case 4: launch_edm<4>(a, h->stream); break;
    case 5: launch_edm<5>(a, h->stream); break;
    case 6: launch_edm<6>(a, h->stream); break;
    case 7: launch_edm<7>(a, h->stream); break;
    case 8: launch_edm<8>(a, h->stream); break;
    default: throw Error{BM_ERR_INVALID, "distance-geometry pass: k above 128"};
  }
  BM_CHECK_LAUNCH();
  if (cx.prof.on) cx.prof.end(h->stream);
  if (h->seg.nmulti) {
    const int64_t work = h->seg.nmulti * h->ld;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), num_sms() * 8));
    BM_LAUNCH(cx, "edm_fixup",
              k_edm_fixup<<<grid, 256, 0, h->stream>>>(h->seg.mrow.get(), h->seg.mfirst.get(), h->seg.mcount.get(),
                                                       h->seg.nmulti, h->partial.get(), h->V.get(), h->ld, a.lam,
                                                       a.out));
  }
  (void)want_grad;
  const int parts = total_parts();
  BM_REQUIRE((int64_t)h->red.n >= parts + 1, BM_ERR_INVALID, "distance-geometry pass: reduction buffer too small");
  BM_LAUNCH(cx, "edm_total",
            k_edm_total_part<<<parts, kTotalThreads, 0, h->stream>>>(h->fseg.get(), h->seg.nseg, h->V.get(),
                                                                      h->n * (int64_t)h->ld, h->lambda,
                                                                      h->red.get() + 1));
  BM_LAUNCH(cx, "edm_total",
            k_edm_total_final<<<1, kTotalThreads, 0, h->stream>>>(h->red.get() + 1, parts, h->red.get()));
  if (!sync) return std::nan("");
  double gv = 0;
  BM_CUDA(cudaMemcpyAsync(&gv, h->red.get(), sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  BM_CUDA(cudaStreamSynchronize(h->stream));
  BM_REQUIRE(std::isfinite(gv), BM_ERR_NUMERIC, "distance-geometry loss is not finite");
  return gv;
}

}  // namespace bm
