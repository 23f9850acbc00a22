// Allocation-free variant of the CSR loss/gradient pass.
//
// Some callers cannot allocate device memory at the point where they need a
// gradient: code running inside another framework's memory pool that forbids
// foreign cudaMalloc calls, allocation-free real-time loops, or callers that
// hold only pointers handed to them by someone else.  This entry point takes
// the CSR arrays, the factors and the outputs from the caller and keeps its
// only scratch (one loss partial per row) in a fixed-size array in the
// library's own device memory, so it calls no allocator at all.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "ctx.cuh"

namespace bm {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxDevices = 64;

// Per-row loss partials.  Every call overwrites rows [0, m) before reading
// them, so nothing has to be cleared between calls.  Every GPU that loads the
// library holds this array (2 MiB) until the process exits.
static __device__ __align__(256) double g_noalloc_rowf[BM_NOALLOC_MAX_ROWS];

// The array's device address, looked up once per device (host code must not
// use the symbol itself as an address).
double* g_rowf_addr[kMaxDevices] = {nullptr};
std::mutex g_rowf_mu;
thread_local std::string g_noalloc_error;

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// One warp per row (grid-stride), four lanes per entry, V float4 chunks per lane.
template <int V>
__global__ void __launch_bounds__(256) k_grad_rows_noalloc(int64_t m, const int64_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col,
                                                           const float* __restrict__ val, const float* __restrict__ W,
                                                           const float* __restrict__ H, int ld, float lam,
                                                           float* __restrict__ gW, double* __restrict__ rowf) {
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int nchunk = ld / 4;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nwarps) {
    const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
    float4 w[V], acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = l + 4 * v;
      w[v] = c < nchunk ? ldg4(W + i * ld + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
      acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float fs = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < end;
      const int j = valid ? __ldg(col + e) : 0;
      const float av = valid ? __ldg(val + e) : 0.f;
#pragma unroll 2
      for (int t = 0; t < 4; ++t) {
        const int src = t * 8 + g;
        const int jj = __shfl_sync(kFull, j, src);
        const float aa = __shfl_sync(kFull, av, src);
        const bool ok = e0 + src < end;
        float4 hv[V];
        float d = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + 4 * v;
          hv[v] = c < nchunk ? ldg4(H + (int64_t)jj * ld + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
          d = fmaf(w[v].x, hv[v].x, fmaf(w[v].y, hv[v].y, fmaf(w[v].z, hv[v].z, fmaf(w[v].w, hv[v].w, d))));
        }
        d += __shfl_xor_sync(kFull, d, 1);
        d += __shfl_xor_sync(kFull, d, 2);
        const float r = ok ? d - aa : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          acc[v].x = fmaf(r, hv[v].x, acc[v].x);
          acc[v].y = fmaf(r, hv[v].y, acc[v].y);
          acc[v].z = fmaf(r, hv[v].z, acc[v].z);
          acc[v].w = fmaf(r, hv[v].w, acc[v].w);
        }
        if (l == 0) fs = fmaf(r, r, fs);
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
#pragma unroll
      for (int mk = 4; mk < 32; mk <<= 1) {
        acc[v].x += __shfl_xor_sync(kFull, acc[v].x, mk);
        acc[v].y += __shfl_xor_sync(kFull, acc[v].y, mk);
        acc[v].z += __shfl_xor_sync(kFull, acc[v].z, mk);
        acc[v].w += __shfl_xor_sync(kFull, acc[v].w, mk);
      }
    }
#pragma unroll
    for (int mk = 16; mk > 0; mk >>= 1) fs += __shfl_xor_sync(kFull, fs, mk);
    if (g == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = l + 4 * v;
        if (c < nchunk) {
          float4 o = acc[v];
          o.x = fmaf(lam, w[v].x, o.x);
          o.y = fmaf(lam, w[v].y, o.y);
          o.z = fmaf(lam, w[v].z, o.z);
          o.w = fmaf(lam, w[v].w, o.w);
          *reinterpret_cast<float4*>(gW + i * ld + 4 * c) = o;
        }
      }
    }
    if (lane == 0) rowf[i] = 0.5 * (double)fs;
  }
}

// f = sum of the per-row partials in row order (one block, fixed order).
__global__ void k_sum_rows_noalloc(const double* __restrict__ rowf, int64_t m, double* __restrict__ f) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += rowf[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *f = sh[0];
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <int V>
void launch_rows(int64_t m, const int64_t* rp, const int32_t* col, const float* val, const float* W, const float* H,
                 int ld, float lam, float* gW, double* rowf, cudaStream_t st) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 8), (int64_t)sms * 16));
  k_grad_rows_noalloc<V><<<grid, 256, 0, st>>>(m, rp, col, val, W, H, ld, lam, gW, rowf);
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

const char* bm_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

bm_status bm_loss_grad_csr_noalloc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                   const float* val, const float* W, const float* H, int32_t k, int32_t ld,
                                   double lambda, float* gW, double* f, void* stream) {
  auto fail = [](bm_status s, const char* msg) {
    g_noalloc_error = msg;
    return s;
  };
  if (m < 1 || n < 1) return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: m and n must be >= 1");
  if (m > BM_NOALLOC_MAX_ROWS)
    return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: m exceeds BM_NOALLOC_MAX_ROWS (262144 rows)");
  if (k < 1 || k > 128 || ld < k || (ld & 3) || ld > 128)
    return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: need 1 <= k <= 128 and k <= ld <= 128, ld % 4 == 0");
  // lambda is used in FP32: a finite double above FLT_MAX would become inf
  if (!std::isfinite(lambda) || !std::isfinite((float)lambda))
    return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: lambda must be finite in FP32");
  const void* ptrs[] = {row_ptr, col, val, W, H, gW, f};
  for (const void* p : ptrs)
    if (!p || !on_device(p))
      return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: every array must be a device pointer");
  // the factor rows are read and the gradient rows written as float4
  if (((uintptr_t)W | (uintptr_t)H | (uintptr_t)gW) & 15)
    return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: W, H and gW must be 16-byte aligned");
  if (((uintptr_t)row_ptr | (uintptr_t)f) & 7 || ((uintptr_t)col | (uintptr_t)val) & 3)
    return fail(BM_ERR_INVALID, "bm_loss_grad_csr_noalloc: misaligned row_ptr, col, val or f");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(BM_ERR_CUDA, "bm_loss_grad_csr_noalloc: no current device");
  }
  double* rowf = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_rowf_mu);
    if (!g_rowf_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_rowf);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BM_ERR_CUDA, "bm_loss_grad_csr_noalloc: cudaGetSymbolAddress failed");
      }
      g_rowf_addr[dev] = static_cast<double*>(p);
    }
    rowf = g_rowf_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float lam = (float)lambda;
  const int V = std::max(1, (ld / 4 + 3) / 4);
  switch (V) {
    case 1: launch_rows<1>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    case 2: launch_rows<2>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    case 3: launch_rows<3>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    case 4: launch_rows<4>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    case 5: launch_rows<5>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    case 6: launch_rows<6>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    case 7: launch_rows<7>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
    default: launch_rows<8>(m, row_ptr, col, val, W, H, ld, lam, gW, rowf, st); break;
  }
  k_sum_rows_noalloc<<<1, 1024, 0, st>>>(rowf, m, f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(BM_ERR_CUDA, cudaGetErrorString(e));
  return BM_OK;
}

}  // extern "C"
