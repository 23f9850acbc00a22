// Grams C = A^T B of tall FP32 blocks on the 5th-generation tensor cores.
//
// The PG step's dense k-wide products (W^T U, H^T Y, the Rayleigh-Ritz
// matrix (Z^T Q)^T (Z^T Q)) reduce over the long dimension L (up to the
// 480,189 rows of the recommendation-scale H).  Each FP32 operand value is
// split into three bfloat16 slices, x1 = RN(x), x2 = RN(x - x1),
// x3 = RN(x - x1 - x2) (the differences are exact in FP32, and x1 + x2 + x3
// reproduces x to about 2^-32 relative), and the six
// slice products whose weight is at least 2^-16 of the leading one
// (x1 y1, x1 y2, x2 y1, x1 y3, x3 y1, x2 y2) are accumulated by tcgen05.mma
// (kind::f16, BF16 inputs, FP32 accumulator in tensor memory).  A product
// thus carries about 2^-24 relative error, as an FP32 product does.  The
// leading product x1 y1 and the five small ones accumulate in separate
// tensor-memory accumulators where they fit (the tensor core's FP32
// accumulation rounds each step against the accumulator's magnitude).  Each
// block accumulates its slab of rows in tensor memory and writes its slab
// sum; the slab sums are added in a fixed order in FP64 (k_gram_reduce).
//
// Data path per block (one block per SM, 256 threads):
//   rows [r, r + 32) of A and B  --cp.async-->  FP32 staging ring (3 to 8
//   tiles, as shared memory allows)
//   --CUDA cores-->  bfloat16 slice tiles in the MN-major core-matrix layout
//   (8 K-rows x 16 bytes per core matrix; K-adjacent core matrices 128 B
//   apart, M/N-adjacent 512 B apart; two slice buffers)  --one thread-->
//   tcgen05.mma per (M tile, slice pair), tcgen05.commit to an mbarrier per
//   slice buffer  --epilogue-->  tcgen05.ld of the accumulators, slab sums.
// Every mbarrier wait has an iteration limit; on expiry the block records
// an error status, poisons its slab sum with NaN and still frees its
// tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "dense.cuh"
#include "pipe.cuh"

namespace bm {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 32;            // rows per staged tile: two BF16 MMA K-steps of 16
constexpr int kTcMaxStages = 8;        // deepest FP32 staging ring (tiles in flight + 1)
constexpr int kTcMaxCols = 256;        // widest A or B block
constexpr long long kTcSpinLimit = 1ll << 26;   // mbarrier polls (with 64 ns sleeps: about 4 s)
constexpr int kTcLbo = 128;            // bytes between K-adjacent core matrices
constexpr int kTcSbo = 512;            // bytes between M/N-adjacent core matrices (4 K-blocks of 8 rows)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start address, leading
// byte offset (between core matrices adjacent along K), stride byte offset
// (adjacent along M or N), descriptor version 1 (bits 46-48).  The staged
// slice tiles keep K-adjacent core matrices 128 B apart and M/N-adjacent ones
// 512 B apart (a 32-row tile holds four K-blocks of 8 rows).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((kTcLbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kTcSbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), BF16 A
// and B (bits 7-9, 10-12), both MN-major (bits 15, 16: the reduction runs
// over the rows of the row-major blocks), N / 8 (bits 17-22), M / 16 (24-28).
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, at most kTcSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; !mbar_test(bar, parity); ++it) {
    if (it > kTcSpinLimit) return false;
    __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive accumulator columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// bfloat16 rounding (to nearest even) of x, returned as the FP32 value and
// its 16-bit pattern.
__device__ __forceinline__ float bf16_round(float x, uint32_t& bits) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  bits = (uint32_t)__bfloat16_as_ushort(b);
  return __bfloat162float(b);
}

// Block of the tensor-core Gram: slab [blockIdx.x * slab, ...) of the rows.
// a, b <= 256 columns; ap = 128 * (number of M tiles), np = N of the MMA
// (b rounded up to 16); sym: B is A (one staged operand serves both).
template <int NST>
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const float* __restrict__ A, int lda, int a,
                                                         const float* __restrict__ B, int ldb, int b, int64_t L,
                                                         int64_t slab, int sym, int ap, int np, int tmem_cols,
                                                         float2* __restrict__ part, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base_slot;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a4 = (a + 3) >> 2, b4 = sym ? 0 : (b + 3) >> 2;
  const int stage_floats = kTcRows * 4 * (a4 + b4);
  float* stage = reinterpret_cast<float*>(smem);                                  // NST FP32 tiles
  unsigned char* slices = smem + (((size_t)NST * stage_floats * 4 + 1023) & ~(size_t)1023);
  const int sliceA = ap * 64, sliceB = sym ? 0 : np * 64;                          // bytes per slice tile
  const int buf_bytes = 3 * (sliceA + sliceB);                                    // one slice buffer
  const int nmt = ap / 128;
  const bool split = 2 * nmt * np <= tmem_cols;   // room for a second accumulator per M tile
  const int64_t r0 = (int64_t)blockIdx.x * slab;
  const int64_t r1 = min(L, r0 + slab);
  const int ntile = (int)((r1 - r0 + kTcRows - 1) / kTcRows);

  // zero both slice buffers once: groups past the last column stay zero
  for (int i = tid; i < 2 * buf_bytes / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(slices)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    failed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;

  auto load_tile = [&](int t) {
    float* dst = stage + (t % NST) * stage_floats;
    const int64_t rb = r0 + (int64_t)t * kTcRows;
    const int per_row = a4 + b4;
    for (int idx = tid; idx < kTcRows * per_row; idx += kTcThreads) {
      const int r = idx / per_row, c = idx - r * per_row;
      const bool ok = rb + r < r1;
      const float* src = c < a4 ? A + (ok ? (rb + r) * lda : 0) + 4 * c : B + (ok ? (rb + r) * ldb : 0) + 4 * (c - a4);
      cp_async16(dst + 4 * idx, src, ok);
    }
  };
  // prologue: tiles 0 .. NST - 2 in flight
#pragma unroll
  for (int t = 0; t < NST - 1; ++t) {
    if (t < ntile) load_tile(t);
    cp_async_commit();
  }

  const uint32_t idesc = tc_idesc(128, np);
  for (int t = 0; t < ntile; ++t) {
    const int sb = t & 1;
    cp_async_wait<NST - 2>();      // tile t has landed
    __syncthreads();
    // the MMAs of tile t - 2 read this slice buffer: wait for them
    if (t >= 2 && !failed && !mbar_wait(smem_u32(&bars[sb]), (uint32_t)(((t >> 1) - 1) & 1))) failed = 1;
    // cut the FP32 tile into three bfloat16 slice tiles (MN-major core matrices)
    const float* src = stage + (t % NST) * stage_floats;
    unsigned char* buf = slices + sb * buf_bytes;
    const int ga = (a + 7) >> 3, gb = sym ? 0 : (b + 7) >> 3;
    for (int it = tid; it < kTcRows * (ga + gb); it += kTcThreads) {
      const int k = it / (ga + gb), g = it - k * (ga + gb);
      const bool isA = g < ga;
      const int gg = isA ? g : g - ga;
      const int ncol = isA ? a : b;
      const float* row = src + k * 4 * (a4 + b4) + (isA ? 0 : 4 * a4);
      float xv[8];
      if (8 * gg + 8 <= ncol) {
        const float4 u0 = *reinterpret_cast<const float4*>(row + 8 * gg);
        const float4 u1 = *reinterpret_cast<const float4*>(row + 8 * gg + 4);
        xv[0] = u0.x; xv[1] = u0.y; xv[2] = u0.z; xv[3] = u0.w;
        xv[4] = u1.x; xv[5] = u1.y; xv[6] = u1.z; xv[7] = u1.w;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) xv[q] = 8 * gg + q < ncol ? row[8 * gg + q] : 0.f;
      }
      uint32_t w1[4], w2[4], w3[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t lo1, hi1, lo2, hi2, lo3, hi3;
        const float s10 = bf16_round(xv[2 * q], lo1), s11 = bf16_round(xv[2 * q + 1], hi1);
        const float r0v = xv[2 * q] - s10, r1v = xv[2 * q + 1] - s11;
        const float s20 = bf16_round(r0v, lo2), s21 = bf16_round(r1v, hi2);
        bf16_round(r0v - s20, lo3);
        bf16_round(r1v - s21, hi3);
        w1[q] = lo1 | (hi1 << 16);
        w2[q] = lo2 | (hi2 << 16);
        w3[q] = lo3 | (hi3 << 16);
      }
      const int off = gg * kTcSbo + (k >> 3) * kTcLbo + (k & 7) * 16;
      unsigned char* base = buf + (isA ? 0 : 3 * sliceA);
      const int stride = isA ? sliceA : sliceB;
      *reinterpret_cast<uint4*>(base + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
      *reinterpret_cast<uint4*>(base + stride + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      *reinterpret_cast<uint4*>(base + 2 * stride + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
    }
    proxy_fence();
    __syncthreads();
    if (tid == 0 && !failed) {
      tc_fence_after();
      const uint32_t abase = smem_u32(buf);
      const uint32_t bbase = sym ? abase : abase + 3 * sliceA;
      const int bstride = sym ? sliceA : sliceB;
      // slice pairs (i, j) with weight >= 2^-16: 11, 12, 21, 13, 31, 22
      const int pi[6] = {0, 0, 1, 0, 2, 1}, pj[6] = {0, 1, 0, 2, 0, 1};
      // the leading product x1 y1 goes to accumulator 0 of the M tile, the five
      // small ones (weights 2^-8 .. 2^-16) to accumulator 1 when there is room:
      // each accumulation rounds against the size of its own accumulator
      for (int mt = 0; mt < nmt; ++mt) {
        for (int ks = 0; ks < kTcRows / 16; ++ks) {          // K-steps of 16 rows: two K-blocks each
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const uint64_t da = tc_desc(abase + pi[q] * sliceA + mt * 16 * kTcSbo + ks * 2 * kTcLbo);
            const uint64_t db = tc_desc(bbase + pj[q] * bstride + ks * 2 * kTcLbo);
            const bool second = split && q > 0;
            const uint32_t d = tmem + (uint32_t)(mt * np + (second ? nmt * np : 0));
            const bool first_use = t == 0 && ks == 0 && (q == 0 || (split && q == 1));
            tc_mma(d, da, db, idesc, first_use ? 0u : 1u);
          }
        }
      }
      tc_commit(smem_u32(&bars[sb]));
    }
    // prefetch tile t + NST - 1 into the stage read in the previous iteration
    if (t + NST - 1 < ntile) load_tile(t + NST - 1);
    cp_async_commit();
  }
  cp_async_wait<0>();
  // all MMAs done: the last commit covers every earlier one
  __syncthreads();
  if (ntile > 0 && !failed && !mbar_wait(smem_u32(&bars[(ntile - 1) & 1]), (uint32_t)(((ntile - 1) >> 1) & 1)))
    failed = 1;
  __syncthreads();
  tc_fence_after();
  // epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows of C), half the columns
  const int quad = warp & 3, half = warp >> 2;
  const int bad = failed;
  float2* out = part + (int64_t)blockIdx.x * a * b;
  for (int mt = 0; mt < nmt; ++mt) {
    const int m = mt * 128 + quad * 32 + lane;
    for (int c0 = half * 8; c0 < np; c0 += 16) {
      float v[8];
      if (ntile > 0) {
        tc_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(mt * np + c0), v);
        if (split) {
          float v2[8];
          tc_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(nmt * np + mt * np + c0), v2);
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] += v2[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = 0.f;
      }
      if (m < a) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + q < b) out[(int64_t)m * b + c0 + q] = make_float2(bad ? NAN : v[q], 0.f);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  if (tid == 0 && bad) atomicExch(status, 1);
}

}  // namespace

// Tensor-core form of gram_dev for plain Grams (see the file comment).
// Returns false (nothing launched) when the shape or layout does not fit it:
// a or b above 256, row strides or base pointers not 16-byte aligned.
bool gram_tc_dev(bm_ctx& h, DenseWork& w, const Tall& A, const Tall& B, double* C, const char* tag) {
  const int a = A.cols, b = B.cols;
  const int sym = (A.p == B.p && A.ld == B.ld && a == b) ? 1 : 0;
  if (a < 1 || b < 1 || a > kTcMaxCols || b > kTcMaxCols) return false;
  if ((A.ld & 3) || (B.ld & 3) || ((uintptr_t)A.p & 15) || ((uintptr_t)B.p & 15)) return false;
  const int64_t L = A.rows;
  const int nmt = (a + 127) / 128;
  const int ap = 128 * nmt;
  const int np = sym ? ((a + 15) / 16) * 16 : ((b + 15) / 16) * 16;
  // one FP32 accumulator per M tile, a second one for the small slice
  // products when 2 * nmt * np columns fit the 512 of tensor memory
  const int need = 2 * nmt * np <= 512 ? 2 * nmt * np : nmt * np;
  int cols = 32;
  while (cols < need) cols <<= 1;
  if (cols > 512) return false;
  const int a4 = (a + 3) / 4, b4 = sym ? 0 : (b + 3) / 4;
  const size_t tile_bytes = (size_t)kTcRows * 4 * (a4 + b4) * 4;
  const size_t slice_bytes = (size_t)2 * 3 * (ap * 64 + (sym ? 0 : np * 64));
  // as many staging tiles in flight as 200 KB of shared memory allow (3 .. 8)
  int nst = kTcMaxStages;
  while (nst > 3 && ((nst * tile_bytes + 1023) & ~(size_t)1023) + slice_bytes + 1024 > 200 * 1024) --nst;
  nst = nst >= 8 ? 8 : (nst >= 6 ? 6 : (nst >= 4 ? 4 : 3));
  const size_t smem = ((nst * tile_bytes + 1023) & ~(size_t)1023) + slice_bytes + 1024;
  if (smem > 220 * 1024) return false;
  int64_t gx = std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 256), (int64_t)num_sms()));
  const int64_t slab = ceil_div(ceil_div(L, gx), kTcRows) * kTcRows;
  gx = std::max<int64_t>(1, ceil_div(L, slab));
  w.gram_part.alloc((size_t)gx * a * b);
  if (!w.tc_status.get()) {
    w.tc_status.alloc(1);
    BM_CUDA(cudaMemsetAsync(w.tc_status.get(), 0, sizeof(int), h.stream));
  }
  float2* part = reinterpret_cast<float2*>(w.gram_part.get());
#define BM_TC_LAUNCH(N)                                                                                       \
  allow_max_smem((const void*)k_gram_tc<N>);                                                                  \
  BM_LAUNCH(h, tag, k_gram_tc<N><<<(unsigned)gx, kTcThreads, smem, h.stream>>>(A.p, A.ld, a, B.p, B.ld, b, L,   \
                                                                               slab, sym, ap, np, cols, part,  \
                                                                               w.tc_status.get()));
  switch (nst) {
    case 8: BM_TC_LAUNCH(8) break;
    case 6: BM_TC_LAUNCH(6) break;
    case 4: BM_TC_LAUNCH(4) break;
    default: BM_TC_LAUNCH(3) break;
  }
#undef BM_TC_LAUNCH
  gram_reduce_dev(h, part, (int)gx, a, b, sym, C);
  return true;
}

}  // namespace bm

using namespace bm;

namespace {
thread_local std::string g_dense_error;
}

extern "C" {

const char* bm_dense_last_error(void) { return g_dense_error.c_str(); }

bm_status bm_dense_gram(const float* A, int64_t L, int32_t a, int32_t lda, const float* B, int32_t b, int32_t ldb,
                        double* C, int32_t mode, void* stream) {
  bm_ctx cx;
  // scratch kept between calls, one set per host thread
  thread_local DenseWork w;
  thread_local DevBuf<double> chunk;
  return guard_call(g_dense_error, [&] {
    BM_REQUIRE(L >= 0 && a >= 1 && b >= 1 && lda >= a && ldb >= b && lda % 4 == 0 && ldb % 4 == 0, BM_ERR_INVALID,
               "bm_dense_gram: need L >= 0, 1 <= a <= lda, 1 <= b <= ldb, lda and ldb multiples of 4");
    BM_REQUIRE(mode >= 0 && mode <= 2, BM_ERR_INVALID, "bm_dense_gram: mode must be 0, 1 or 2");
    BM_REQUIRE(A && B && C && is_device_ptr(A) && is_device_ptr(B) && is_device_ptr(C), BM_ERR_INVALID,
               "bm_dense_gram: A, B and C must be device pointers");
    BM_REQUIRE(!((uintptr_t)A & 15) && !((uintptr_t)B & 15), BM_ERR_INVALID,
               "bm_dense_gram: A and B must be 16-byte aligned");
    BM_CUDA(cudaGetDevice(&cx.device));
    cx.stream = (cudaStream_t)stream;
    const Tall TA{const_cast<float*>(A), L, a, lda};
    const Tall TB{const_cast<float*>(B), L, b, ldb};
    if (mode == 2) {
      BM_REQUIRE(a <= 256 && b <= 256, BM_ERR_INVALID, "bm_dense_gram: mode 2 needs a, b <= 256");
      if (w.tc_status.get()) BM_CUDA(cudaMemsetAsync(w.tc_status.get(), 0, sizeof(int), cx.stream));
      if (L == 0) {
        BM_CUDA(cudaMemsetAsync(C, 0, (size_t)a * b * sizeof(double), cx.stream));
      } else if (!gram_tc_dev(cx, w, TA, TB, C, "dense_gram_tc")) {
        // too wide for one block's shared memory: column chunks of B
        chunk.alloc((size_t)a * 64);
        for (int c0 = 0; c0 < b; c0 += 64) {
          const int cb = std::min(64, b - c0);
          const Tall TBc{const_cast<float*>(B) + c0, L, cb, ldb};
          BM_REQUIRE(gram_tc_dev(cx, w, TA, TBc, chunk.get(), "dense_gram_tc"), BM_ERR_INVALID,
                     "bm_dense_gram: shape not supported by the tensor-core Gram");
          BM_CUDA(cudaMemcpy2DAsync(C + c0, (size_t)b * sizeof(double), chunk.get(), (size_t)cb * sizeof(double),
                                    (size_t)cb * sizeof(double), (size_t)a, cudaMemcpyDeviceToDevice, cx.stream));
        }
      }
      int st = 0;
      if (w.tc_status.get())
        BM_CUDA(cudaMemcpyAsync(&st, w.tc_status.get(), sizeof(int), cudaMemcpyDeviceToHost, cx.stream));
      BM_CUDA(cudaStreamSynchronize(cx.stream));
      BM_REQUIRE(st == 0, BM_ERR_NUMERIC, "bm_dense_gram: a tensor-core barrier wait ran out of time");
    } else {
      cx.opt.tensor_grams = 0;
      gram_dev(cx, w, TA, TB, C, mode == 1, "dense_gram");
      BM_CUDA(cudaStreamSynchronize(cx.stream));
    }
  });
}

bm_status bm_sym_eig(const double* S, int32_t n, double* evals, double* evecs, int32_t mode, void* stream) {
  bm_ctx cx;
  thread_local DenseWork w;
  return guard_call(g_dense_error, [&] {
    BM_REQUIRE(n >= 1 && n <= 256, BM_ERR_INVALID, "bm_sym_eig: need 1 <= n <= 256");
    BM_REQUIRE(mode >= 0 && mode <= 2, BM_ERR_INVALID, "bm_sym_eig: mode must be 0, 1 or 2");
    BM_REQUIRE(S && evals && evecs && is_device_ptr(S) && is_device_ptr(evals) && is_device_ptr(evecs),
               BM_ERR_INVALID, "bm_sym_eig: S, evals and evecs must be device pointers");
    BM_CUDA(cudaGetDevice(&cx.device));
    cx.stream = (cudaStream_t)stream;
    sym_eig_dev(cx, w, S, n, evals, evecs, mode == 0 ? kEigFast : (mode == 1 ? kEigRelative : kEigDouble));
    BM_CUDA(cudaStreamSynchronize(cx.stream));
  });
}

}  // extern "C"
