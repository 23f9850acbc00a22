// Thin dense blocks (Grams, thin products), the q-wide residual SpMM, the
// one-CTA symmetric eigensolver and small helpers of the proximal step.
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "dense.cuh"
#include "pipe.cuh"

namespace bm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float comp(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// ---------------------------------------------------------------- Gram C = A^T B
// Each thread owns an 8 x 4 micro-tile of C (8 columns of A by 4 of B); a
// block walks a slab of rows in tiles of kGramRows rows, double-buffered in
// shared memory by cp.async.  Sums are unevaluated FP32 pairs (hi + lo), so
// no FP64 arithmetic runs in the loop (FP64 is slow on this part): plain
// Grams sum a tile in FP32 and add it to the pair by an error-free two-sum;
// compensated Grams apply the error-free product and two-sum to every term
// (Ogita-Rump-Oishi Dot2).  Slab partials leave as FP32 pairs.
constexpr int kGramRows = 32;
constexpr int kGramMaxThreads = 512;
// slab blocks per SM of the row split: the compensated Grams' dependent
// two-sum chains want more resident warps (measured: 10 blocks per SM
// 0.75 -> 0.62 ms for the 480,189 x 64 symmetric Gram), the plain ones fewer
constexpr int kGramBlocksPerSmPlain = 3;
constexpr int kGramBlocksPerSmComp = 10;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ float comp8(const float4& u, const float4& v, int i) {
  return i < 4 ? comp(u, i) : comp(v, i - 4);
}

template <bool COMP>
__global__ void __launch_bounds__(kGramMaxThreads) k_gram(const float* __restrict__ A, int lda, int a,
                                                          const float* __restrict__ B, int ldb, int b, int64_t L,
                                                          int64_t slab, int sym, float2* __restrict__ part) {
  extern __shared__ float4 sm4[];
  const int ng = (a + 7) >> 3, na = 2 * ng, a4 = (a + 3) >> 2, nb = (b + 3) >> 2;
  const int stage = kGramRows * (na + nb);
  const int mt = blockIdx.y * blockDim.x + threadIdx.x;
  int ti = 0, tj = 0;
  bool active;
  if (sym) {
    // symmetric Grams (A = B): only micro-tiles that reach the diagonal or
    // above are enumerated, column block by column block
    int rem = mt;
    active = false;
    for (int c = 0; c < nb; ++c) {
      const int cnt = min(ng, (4 * c + 3) / 8 + 1);
      if (rem < cnt) {
        ti = rem;
        tj = c;
        active = true;
        break;
      }
      rem -= cnt;
    }
  } else {
    active = mt < ng * nb;
    ti = active ? mt / nb : 0;
    tj = active ? mt % nb : 0;
  }
  float hi[32], lo[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) hi[q] = 0.f, lo[q] = 0.f;
  const int64_t r0 = (int64_t)blockIdx.x * slab;
  const int64_t r1 = min(L, r0 + slab);
  const int ntile = (int)((r1 - r0 + kGramRows - 1) / kGramRows);
  auto load = [&](int t) {
    float4* As = sm4 + (t & 1) * stage;
    float4* Bs = As + kGramRows * na;
    const int64_t rb = r0 + (int64_t)t * kGramRows;
    const int nr = (int)min((int64_t)kGramRows, r1 - rb);
    for (int idx = threadIdx.x; idx < nr * na; idx += blockDim.x) {
      const int r = idx / na, c = idx - r * na;
      if (c < a4) cp_async16(reinterpret_cast<float*>(As + idx), A + (rb + r) * lda + 4 * c, true);
      else As[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int idx = threadIdx.x; idx < nr * nb; idx += blockDim.x) {
      const int r = idx / nb, c = idx - r * nb;
      cp_async16(reinterpret_cast<float*>(Bs + idx), B + (rb + r) * ldb + 4 * c, true);
    }
  };
  if (ntile > 0) load(0);
  cp_async_commit();
  for (int t = 0; t < ntile; ++t) {
    if (t + 1 < ntile) load(t + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float4* As = sm4 + (t & 1) * stage;
    const float4* Bs = As + kGramRows * na;
    const int nr = (int)min((int64_t)kGramRows, r1 - (r0 + (int64_t)t * kGramRows));
    if (active) {
      if (COMP) {
        for (int r = 0; r < nr; ++r) {
          const float4 u = As[r * na + 2 * ti], v = As[r * na + 2 * ti + 1], bv = Bs[r * nb + tj];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float x = comp8(u, v, p), y = comp(bv, q);
              const float pr = __fmul_rn(x, y);
              const float pe = fmaf(x, y, -pr);
              float s, e;
              two_sum(hi[p * 4 + q], pr, s, e);
              hi[p * 4 + q] = s;
              lo[p * 4 + q] = __fadd_rn(lo[p * 4 + q], __fadd_rn(e, pe));
            }
          }
        }
      } else {
        float s[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) s[q] = 0.f;
        for (int r = 0; r < nr; ++r) {
          const float4 u = As[r * na + 2 * ti], v = As[r * na + 2 * ti + 1], bv = Bs[r * nb + tj];
#pragma unroll
          for (int p = 0; p < 8; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) s[p * 4 + q] = fmaf(comp8(u, v, p), comp(bv, q), s[p * 4 + q]);
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          float t2, e;
          two_sum(hi[q], s[q], t2, e);
          hi[q] = t2;
          lo[q] = __fadd_rn(lo[q], e);
        }
      }
    }
    __syncthreads();
  }
  if (active) {
    float2* out = part + (int64_t)blockIdx.x * a * b;
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 8 * ti + p, j = 4 * tj + q;
        if (i < a && j < b) out[i * b + j] = make_float2(hi[p * 4 + q], lo[p * 4 + q]);
      }
  }
}

// C[e] = sum over slabs of the FP32-pair partials, in slab order: warp w of a
// block adds slabs w, w + 8, ... of 32 consecutive entries, then the eight
// warp sums are added in warp order.  Symmetric Grams read entry (j, i) for i > j.
__global__ void __launch_bounds__(256) k_gram_reduce(const float2* __restrict__ part, int slabs, int a, int b,
                                                     int sym, double* __restrict__ C) {
  __shared__ float2 red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ab = a * b;
  const int e = blockIdx.x * 32 + lane;
  int src = e;
  if (e < ab && sym) {
    const int i = e / b, j = e - (e / b) * b;
    if (i > j) src = j * b + i;
  }
  float hi = 0.f, lo = 0.f;
  if (e < ab) {
    for (int g = warp; g < slabs; g += 8) {
      const float2 p = part[(int64_t)g * ab + src];
      float s, err;
      two_sum(hi, p.x, s, err);
      hi = s;
      lo = __fadd_rn(lo, __fadd_rn(err, p.y));
    }
  }
  red[warp][lane] = make_float2(hi, lo);
  __syncthreads();
  if (warp == 0 && e < ab) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += (double)red[w][lane].x + (double)red[w][lane].y;
    C[e] = s;
  }
}

// ---------------------------------------------------------------- Y = beta Y + gamma A C
// A persistent block walks row tiles of R = 8 * groups rows.  C (a x b) stays
// in shared memory for the whole launch; each A tile is staged transposed
// (column t of the tile is R contiguous floats), so a thread owning 8 rows x 4
// columns of Y issues two 16-byte loads of A and one of C per 32 FMAs.
constexpr int kGemmThreads = 256;

__global__ void __launch_bounds__(kGemmThreads, 3) k_gemm(const float* __restrict__ A, int lda, int a,
                                                          const float* __restrict__ C, int ldc, int b,
                                                          float* __restrict__ Y, int ldy, int64_t L, float beta,
                                                          float gamma, int groups) {
  extern __shared__ float4 gsm[];
  const int nb4 = (b + 3) >> 2, a4 = (a + 3) >> 2;
  const int R = 8 * groups;
  float4* Cs = gsm;                                              // a x nb4
  float* At = reinterpret_cast<float*>(gsm + (size_t)a * nb4);   // (4 a4) x R, transposed tile
  for (int idx = threadIdx.x; idx < a * nb4; idx += blockDim.x) {
    const int t = idx / nb4, c = idx - t * nb4;
    float4 v;
    v.x = 4 * c + 0 < b ? C[t * ldc + 4 * c + 0] : 0.f;
    v.y = 4 * c + 1 < b ? C[t * ldc + 4 * c + 1] : 0.f;
    v.z = 4 * c + 2 < b ? C[t * ldc + 4 * c + 2] : 0.f;
    v.w = 4 * c + 3 < b ? C[t * ldc + 4 * c + 3] : 0.f;
    Cs[idx] = v;
  }
  const int g = threadIdx.x / nb4, cj = threadIdx.x - g * nb4;
  const bool owner = g < groups;
  for (int64_t r0 = (int64_t)blockIdx.x * R; r0 < L; r0 += (int64_t)gridDim.x * R) {
    __syncthreads();
    // rows vary fastest so that the transposed stores hit consecutive banks
    for (int idx = threadIdx.x; idx < R * a4; idx += blockDim.x) {
      const int c = idx / R, r = idx - c * R;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r0 + r < L) v = ldg4(A + (r0 + r) * lda + 4 * c);
      At[(4 * c + 0) * R + r] = v.x;
      At[(4 * c + 1) * R + r] = v.y;
      At[(4 * c + 2) * R + r] = v.z;
      At[(4 * c + 3) * R + r] = v.w;
    }
    __syncthreads();
    if (owner) {
      float4 acc[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
      const float* ap = At + 8 * g;
      for (int t = 0; t < a; ++t) {
        const float4 x0 = *reinterpret_cast<const float4*>(ap + t * R);
        const float4 x1 = *reinterpret_cast<const float4*>(ap + t * R + 4);
        const float4 cv = Cs[t * nb4 + cj];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const float x = comp8(x0, x1, p);
          acc[p].x = fmaf(x, cv.x, acc[p].x);
          acc[p].y = fmaf(x, cv.y, acc[p].y);
          acc[p].z = fmaf(x, cv.z, acc[p].z);
          acc[p].w = fmaf(x, cv.w, acc[p].w);
        }
      }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const int64_t row = r0 + 8 * g + p;
        if (row < L) {
          float4* yp = reinterpret_cast<float4*>(Y + row * ldy + 4 * cj);
          float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
          if (beta != 0.f) y = *yp;
          y.x = fmaf(gamma, acc[p].x, beta * y.x);
          y.y = fmaf(gamma, acc[p].y, beta * y.y);
          y.z = fmaf(gamma, acc[p].z, beta * y.z);
          y.w = fmaf(gamma, acc[p].w, beta * y.w);
          *yp = y;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- q-wide SpMM of the residual
__global__ void k_spmm_fixup(const int32_t* __restrict__ mrow, const int32_t* __restrict__ mfirst,
                             const int32_t* __restrict__ mcount, int64_t nmulti, const float* __restrict__ partial,
                             int ldp, int cols, float gamma, float* __restrict__ out, int ldo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nmulti * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / cols;
    const int c = (int)(t - q * cols);
    const int64_t f = mfirst[q];
    float s = 0.f;
    for (int u = 0; u < mcount[q]; ++u) s += partial[(f + u) * ldp + c];
    float* o = out + (int64_t)mrow[q] * ldo + c;
    *o = fmaf(gamma, s, *o);
  }
}

// ---------------------------------------------------------------- symmetric eigensolver
constexpr int kEigMax = 256;
constexpr int kEigThreads = 512;

template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Householder reduction to tridiagonal form (Golub & Van Loan, Sec. 8.3.1),
// accumulation of Q, then the implicit-shift QL iteration on the tridiagonal
// matrix.  The products of the reduction and the accumulation run four
// threads to a row.  In the QL phase warp 0 finds the unreduced block and
// lane 0 computes the rotations of one sweep (their chain is sequential),
// while the other warps apply the previous sweep's rotations to the rows of
// Z^T: the vector work of sweep s overlaps the rotation chain of sweep s + 1.
// Eigenvalues leave sorted descending.
template <typename T>
__global__ void __launch_bounds__(kEigThreads) k_sym_eig(const double* __restrict__ S, int n,
                                                          double* __restrict__ evals, double* __restrict__ evecs,
                                                          T* gA, T* gZ, int a_smem, int z_smem,
                                                          int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char eig_raw[];
  __shared__ T d[kEigMax], e[kEigMax], vv[kEigMax], pp[kEigMax], bet[kEigMax];
  __shared__ T rc[2][kEigMax], rs[2][kEigMax];
  __shared__ int rm[2], rcnt[2];
  __shared__ T red[32];
  __shared__ int sh_state, sh_done;
  __shared__ T sh_anorm;
  T* A = a_smem ? reinterpret_cast<T*>(eig_raw) : gA;
  T* Z = z_smem ? reinterpret_cast<T*>(eig_raw) + (a_smem ? (size_t)n * n : 0) : gZ;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const T eps = sizeof(T) == 8 ? (T)DBL_EPSILON : (T)FLT_EPSILON;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    A[idx] = (T)(0.5 * (S[i * n + j] + S[j * n + i]));
  }
  __syncthreads();
  // ---- tridiagonalisation (Golub & Van Loan, Sec. 8.3.1)
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    T x = tid < L ? A[(k + 1 + tid) * n + k] : (T)0;
    const T ss = block_sum<T>(x * x, red);
    const T x0 = A[(k + 1) * n + k];
    const T alpha = ss > 0 ? (x0 > 0 ? -sqrt(ss) : sqrt(ss)) : (T)0;
    const T v0 = x0 - alpha;
    const T vtv = ss - x0 * x0 + v0 * v0;
    const T beta = vtv > 0 ? (T)2 / vtv : (T)0;
    __syncthreads();
    if (tid < L) {
      const T v = tid == 0 ? v0 : x;
      vv[tid] = v;
      A[(k + 1 + tid) * n + k] = v;
    }
    if (tid == 0) {
      bet[k] = beta;
      d[k] = A[k * n + k];
      e[k] = alpha;
    }
    __syncthreads();
    if (beta != (T)0) {
      // p = beta A22 v: four threads per row of the (symmetric) trailing
      // block, each summing every fourth column; v^T p summed on the way
      T vp = 0;
      for (int r0 = 0; r0 < L; r0 += nt >> 2) {   // uniform trip count: every lane joins the shuffles
        const int r = r0 + (tid >> 2);
        T acc = 0;
        if (r < L) {
          const T* Ar = A + (k + 1 + r) * n + (k + 1);
          for (int c = tid & 3; c < L; c += 4) acc += Ar[c] * vv[c];
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc *= beta;
        if (r < L && (tid & 3) == 0) {
          pp[r] = acc;
          vp += vv[r] * acc;
        }
      }
      const T Kc = (T)0.5 * beta * block_sum<T>(vp, red);
      // A22 -= v p'^T + p' v^T with p' = p - Kc v
      for (int r = tid >> 2; r < L; r += nt >> 2) {
        const T vr = vv[r], pr = pp[r] - Kc * vr;
        T* Ar = A + (k + 1 + r) * n + (k + 1);
        for (int c = tid & 3; c < L; c += 4) Ar[c] -= vr * (pp[c] - Kc * vv[c]) + pr * vv[c];
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(n - 2) * n + (n - 2)];
      e[n - 2] = A[(n - 1) * n + (n - 2)];
    }
    d[n - 1] = A[(n - 1) * n + (n - 1)];
    e[n - 1] = 0;
  }
  __syncthreads();
  // ---- Q = H_0 ... H_{n-3} as Z^T (row i = column i of Q), a warp per row
  for (int idx = tid; idx < n * n; idx += nt) Z[idx] = (idx / n == idx % n) ? (T)1 : (T)0;
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const int L = n - k - 1;
    if (tid < L) vv[tid] = A[(k + 1 + tid) * n + k];
    __syncthreads();
    const T beta = bet[k];
    if (beta != (T)0) {
      // four threads per row of Z^T, each on every fourth column
      for (int j0 = k + 1; j0 < n; j0 += nt >> 2) {   // uniform trip count: every lane joins the shuffles
        const int j = j0 + (tid >> 2);
        T* Zj = Z + j * n + k + 1;
        T t = 0;
        if (j < n)
          for (int c = tid & 3; c < L; c += 4) t += Zj[c] * vv[c];
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t *= beta;
        if (j < n)
          for (int c = tid & 3; c < L; c += 4) Zj[c] -= t * vv[c];
      }
    }
    __syncthreads();
  }
  // ---- implicit QL on T / ||T||
  if (tid == 0) {
    sh_state = 0;
    sh_done = 0;
    rcnt[0] = rcnt[1] = 0;
    T an = 0;
    for (int i = 0; i < n; ++i) an = fmax(an, fabs(d[i]) + fabs(e[i]) + (i ? fabs(e[i - 1]) : (T)0));
    sh_anorm = an;
    const T inv = an > 0 ? (T)1 / an : (T)1;
    for (int i = 0; i < n; ++i) d[i] *= inv, e[i] *= inv;
  }
  __syncthreads();
  const T scale = sh_anorm > 0 ? sh_anorm : (T)1;
  int l = 0, iter = 0;   // warp 0's position
  int buf = 0;
  while (true) {
    if (warp == 0) {
      int cnt = 0, mm = 0;
      while (l < n) {
        int m = n - 1;
        for (int base = l; base < n - 1; base += 32) {
          const int q = base + lane;
          bool small = false;
          if (q < n - 1) {
            const T em = fabs(e[q]);
            small = em <= eps * (fabs(d[q]) + fabs(d[q + 1])) || em <= eps;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, small);
          if (bal) {
            m = base + __ffs(bal) - 1;
            break;
          }
        }
        if (m == l) {
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > 60) {
          if (lane == 0) sh_state = 1;
          ++l;
          iter = 0;
          continue;
        }
        if (lane == 0) {
          T g = (d[l + 1] - d[l]) / ((T)2 * e[l]);
          T r = sqrt(g * g + (T)1);
          g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
          T s = 1, c = 1, p = 0;
          bool early = false;
          T ei = e[m - 1], di = d[m - 1], dn = d[m];
          T* cs = rc[buf];
          T* sn = rs[buf];
          for (int i = m - 1; i >= l; --i) {
            const T ei_next = i > l ? e[i - 1] : (T)0, di_next = i > l ? d[i - 1] : (T)0;
            const T f = s * ei, b = c * ei;
            const T t2 = fma(f, f, g * g);
            if (!(t2 > (T)(sizeof(T) == 8 ? 1e-200 : 1e-30))) {
              e[i + 1] = (T)0;
              d[i + 1] = dn - p;
              e[m] = 0;
              early = true;
              break;
            }
            if constexpr (sizeof(T) == 4) {
              // 1/sqrt(t2) estimate y0 and one Newton step h = (3 - t2 y0^2) / 2,
              // applied to the three products after they are formed
              const T y0 = rsqrtf(t2);
              const T h = fmaf(-0.5f * t2, y0 * y0, 1.5f);
              r = (t2 * y0) * h;
              s = (f * y0) * h;
              c = (g * y0) * h;
            } else {
              const T y = rsqrt(t2);
              r = t2 * y;
              s = f * y;
              c = g * y;
            }
            e[i + 1] = r;
            g = dn - p;
            r = fma(di - g, s, (T)2 * b * c);
            p = s * r;
            d[i + 1] = g + p;
            g = fma(c, r, -b);
            cs[cnt] = c;
            sn[cnt] = s;
            ++cnt;
            ei = ei_next;
            dn = di;
            di = di_next;
          }
          if (!early) {
            d[l] -= p;
            e[l] = g;
            e[m] = 0;
          }
        }
        cnt = __shfl_sync(0xffffffffu, cnt, 0);
        __syncwarp();
        mm = m;
        break;
      }
      if (lane == 0) {
        rm[buf] = mm;
        rcnt[buf] = cnt;
        sh_done = (cnt == 0);
      }
    } else {
      // apply the sweep warp 0 produced in the previous round
      const int cnt = rcnt[buf ^ 1], m = rm[buf ^ 1];
      const T* cs = rc[buf ^ 1];
      const T* sn = rs[buf ^ 1];
      for (int q = tid - 32; q < n; q += nt - 32) {
        if (cnt == 0) break;
        T zf = Z[m * n + q];
        for (int t = 0; t < cnt; ++t) {
          const int i = m - 1 - t;
          const T zi = Z[i * n + q];
          Z[(i + 1) * n + q] = sn[t] * zi + cs[t] * zf;
          zf = cs[t] * zi - sn[t] * zf;
        }
        Z[(m - cnt) * n + q] = zf;
      }
    }
    __syncthreads();
    const bool done = sh_done;
    buf ^= 1;
    // every thread has read sh_done and the counts before warp 0 writes the next round
    __syncthreads();
    if (done) break;
  }
  for (int i = tid; i < n; i += nt) d[i] *= scale;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const T di = d[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T dj = d[j];
      rank += (dj > di) || (dj == di && j < i);
    }
    evals[rank] = (double)di;
    if (!isfinite((double)di)) atomicOr(status, 2);
    for (int q = 0; q < n; ++q) evecs[q * n + rank] = (double)Z[i * n + q];
  }
  if (tid == 0 && sh_state) atomicOr(status, 1);
}


// One-CTA FP32 symmetric eigensolver with one divide-and-conquer level on the
// tridiagonal matrix: T = diag(T1, T2) + beta v v^T (Cuppen), the two halves
// by implicit QL at the same time (warps 0 and 1 generate the rotations, the
// other warps apply them), then the rank-one merge: deflation of negligible
// components and close poles, the secular equation by bisection from the
// nearer pole, the eigenvector components recomputed from the computed roots
// (Gu & Eisenstat, SIAM J. Matrix Anal. Appl. 16 (1995)), and the merged
// vectors as one product.
constexpr int kDcMin = 24;
constexpr int kDcMax = 150;   // A and Z (n rows of dc_ld(n) floats each) in shared memory

// Row stride of A and Z: at least n + 1, and 4 modulo 32, so that the eight
// rows a warp reads four consecutive columns of (four threads to a row) fall
// in 32 different shared-memory banks.
__host__ __device__ constexpr int dc_ld(int n) { return ((n + 1 + 27) / 32) * 32 + 4; }

__device__ __forceinline__ void ql_sweep_chain(float* d, float* e, int l, int m, float* cs, float* sn, int& cnt) {
  float g = (d[l + 1] - d[l]) / (2.f * e[l]);
  float r = sqrtf(g * g + 1.f);
  g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
  float s = 1, c = 1, p = 0;
  bool early = false;
  float ei = e[m - 1], di = d[m - 1], dn = d[m];
  cnt = 0;
  for (int i = m - 1; i >= l; --i) {
    const float ei_next = i > l ? e[i - 1] : 0.f, di_next = i > l ? d[i - 1] : 0.f;
    const float f = s * ei, b = c * ei;
    const float t2 = fmaf(f, f, g * g);
    if (!(t2 > 1e-30f)) {
      e[i + 1] = 0.f;
      d[i + 1] = dn - p;
      e[m] = 0.f;
      early = true;
      break;
    }
    const float y0 = rsqrtf(t2);
    const float h = fmaf(-0.5f * t2, y0 * y0, 1.5f);
    r = (t2 * y0) * h;
    s = (f * y0) * h;
    c = (g * y0) * h;
    e[i + 1] = r;
    g = dn - p;
    r = fmaf(di - g, s, 2.f * b * c);
    p = s * r;
    d[i + 1] = g + p;
    g = fmaf(c, r, -b);
    cs[cnt] = c;
    sn[cnt] = s;
    ++cnt;
    ei = ei_next;
    dn = di;
    di = di_next;
  }
  if (!early) {
    d[l] -= p;
    e[l] = g;
    e[m] = 0.f;
  }
}

__global__ void __launch_bounds__(kEigThreads) k_sym_eig_dc(const double* __restrict__ S, int n,
                                                            double* __restrict__ evals, double* __restrict__ evecs,
                                                            float* __restrict__ gW, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char eig_raw[];
  __shared__ float d[kEigMax], e[kEigMax], vv[kEigMax], pp[kEigMax], bet[kEigMax];
  __shared__ float rc[2][2][kEigMax], rs[2][2][kEigMax];
  __shared__ int rm[2][2], rcnt[2][2];
  __shared__ float red[32];
  __shared__ int sh_state, sh_done[2], sh_K, sh_nrot;
  __shared__ float sh_anorm, sh_beta;
  // merge: sorted poles and components, roots, recomputed components
  __shared__ float ds[kDcMax], zs[kDcMax], dk[kDcMax], zk[kDcMax], tau[kDcMax], zhat[kDcMax], lam[kDcMax];
  __shared__ int perm[kDcMax], kidx[kDcMax], org[kDcMax], kslot[kDcMax];
  __shared__ int rot_a[kDcMax], rot_b[kDcMax];
  __shared__ float rot_c[kDcMax], rot_s[kDcMax];
  const int lda = dc_ld(n), ldz = lda;
  float* A = reinterpret_cast<float*>(eig_raw);
  float* Z = A + (size_t)n * lda;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const float eps = FLT_EPSILON;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    A[i * lda + j] = (float)(0.5 * (S[i * n + j] + S[j * n + i]));
  }
  __syncthreads();
  // ---- tridiagonalisation (Golub & Van Loan, Sec. 8.3.1), four threads to a row
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    float x = tid < L ? A[(k + 1 + tid) * lda + k] : 0.f;
    const float ss = block_sum<float>(x * x, red);
    const float x0 = A[(k + 1) * lda + k];
    const float alpha = ss > 0 ? (x0 > 0 ? -sqrtf(ss) : sqrtf(ss)) : 0.f;
    const float v0 = x0 - alpha;
    const float vtv = ss - x0 * x0 + v0 * v0;
    const float beta = vtv > 0 ? 2.f / vtv : 0.f;
    __syncthreads();
    if (tid < L) {
      const float v = tid == 0 ? v0 : x;
      vv[tid] = v;
      A[(k + 1 + tid) * lda + k] = v;
    }
    if (tid == 0) {
      bet[k] = beta;
      d[k] = A[k * lda + k];
      e[k] = alpha;
    }
    __syncthreads();
    if (beta != 0.f) {
      float vp = 0;
      for (int r0 = 0; r0 < L; r0 += nt >> 2) {   // uniform trip count: every lane joins the shuffles
        const int r = r0 + (tid >> 2);
        float acc = 0;
        if (r < L) {
          const float* Ar = A + (k + 1 + r) * lda + (k + 1);
          float a1 = 0.f, a2 = 0.f, a3 = 0.f;
          int c = tid & 3;
          for (; c + 12 < L; c += 16) {
            acc = fmaf(Ar[c], vv[c], acc);
            a1 = fmaf(Ar[c + 4], vv[c + 4], a1);
            a2 = fmaf(Ar[c + 8], vv[c + 8], a2);
            a3 = fmaf(Ar[c + 12], vv[c + 12], a3);
          }
          for (; c < L; c += 4) acc = fmaf(Ar[c], vv[c], acc);
          acc += (a1 + a2) + a3;
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc *= beta;
        if (r < L && (tid & 3) == 0) {
          pp[r] = acc;
          vp += vv[r] * acc;
        }
      }
      const float Kc = 0.5f * beta * block_sum<float>(vp, red);
      for (int r = tid >> 2; r < L; r += nt >> 2) {
        const float vr = vv[r], pr = pp[r] - Kc * vr;
        float* Ar = A + (k + 1 + r) * lda + (k + 1);
#pragma unroll 4
        for (int c = tid & 3; c < L; c += 4) Ar[c] -= vr * (pp[c] - Kc * vv[c]) + pr * vv[c];
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    d[n - 2] = A[(n - 2) * lda + (n - 2)];
    e[n - 2] = A[(n - 1) * lda + (n - 2)];
    d[n - 1] = A[(n - 1) * lda + (n - 1)];
    e[n - 1] = 0;
  }
  __syncthreads();
  // ---- Q = H_0 ... H_{n-3} as Z^T (row i = column i of Q; row stride n + 1)
  for (int idx = tid; idx < n * ldz; idx += nt) {
    const int i = idx / ldz, j = idx - i * ldz;
    Z[idx] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const int L = n - k - 1;
    if (tid < L) vv[tid] = A[(k + 1 + tid) * lda + k];
    __syncthreads();
    const float beta = bet[k];
    if (beta != 0.f) {
      for (int j0 = k + 1; j0 < n; j0 += nt >> 2) {
        const int j = j0 + (tid >> 2);
        float* Zj = Z + j * ldz + k + 1;
        float t = 0;
        if (j < n) {
          float t1 = 0.f, t2 = 0.f, t3 = 0.f;
          int c = tid & 3;
          for (; c + 12 < L; c += 16) {
            t = fmaf(Zj[c], vv[c], t);
            t1 = fmaf(Zj[c + 4], vv[c + 4], t1);
            t2 = fmaf(Zj[c + 8], vv[c + 8], t2);
            t3 = fmaf(Zj[c + 12], vv[c + 12], t3);
          }
          for (; c < L; c += 4) t = fmaf(Zj[c], vv[c], t);
          t += (t1 + t2) + t3;
        }
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t *= beta;
        if (j < n) {
#pragma unroll 4
          for (int c = tid & 3; c < L; c += 4) Zj[c] -= t * vv[c];
        }
      }
    }
    __syncthreads();
  }
  // ---- scale T to ||T|| <= 1, split T = diag(T1, T2) + beta v v^T, v = e_{s-1} + e_s
  const int s_split = n / 2;
  if (tid == 0) {
    sh_state = 0;
    sh_done[0] = sh_done[1] = 0;
    rcnt[0][0] = rcnt[0][1] = rcnt[1][0] = rcnt[1][1] = 0;
    float an = 0;
    for (int i = 0; i < n; ++i) an = fmaxf(an, fabsf(d[i]) + fabsf(e[i]) + (i ? fabsf(e[i - 1]) : 0.f));
    sh_anorm = an;
    const float inv = an > 0 ? 1.f / an : 1.f;
    for (int i = 0; i < n; ++i) d[i] *= inv, e[i] *= inv;
    const float b = e[s_split - 1];
    sh_beta = b;
    d[s_split - 1] -= b;
    d[s_split] -= b;
    e[s_split - 1] = 0.f;
  }
  // column n of Z carries v through the rotations of the halves: afterwards it
  // holds z = diag(Q1, Q2)^T v
  for (int i = tid; i < n; i += nt) Z[i * ldz + n] = (i == s_split - 1 || i == s_split) ? 1.f : 0.f;
  __syncthreads();
  const float scale = sh_anorm > 0 ? sh_anorm : 1.f;
  // ---- implicit QL on both halves: warp p generates the sweeps of half p
  {
    int l = warp == 1 ? s_split : 0, iter = 0;
    const int bhi = warp == 1 ? n - 1 : s_split - 1;
    int buf = 0;
    while (true) {
      if (warp < 2) {
        int cnt = 0, mm = 0;
        while (l <= bhi) {
          int m = bhi;
          for (int base = l; base < bhi; base += 32) {
            const int q = base + lane;
            bool small = false;
            if (q < bhi) {
              const float em = fabsf(e[q]);
              small = em <= eps * (fabsf(d[q]) + fabsf(d[q + 1])) || em <= eps;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, small);
            if (bal) {
              m = base + __ffs(bal) - 1;
              break;
            }
          }
          if (m == l) {
            ++l;
            iter = 0;
            continue;
          }
          if (++iter > 60) {
            if (lane == 0) sh_state = 1;
            ++l;
            iter = 0;
            continue;
          }
          if (lane == 0) ql_sweep_chain(d, e, l, m, rc[warp][buf], rs[warp][buf], cnt);
          cnt = __shfl_sync(0xffffffffu, cnt, 0);
          __syncwarp();
          mm = m;
          break;
        }
        if (lane == 0) {
          rm[warp][buf] = mm;
          rcnt[warp][buf] = cnt;
          sh_done[warp] = cnt == 0;
        }
      } else {
        // apply the sweeps of the previous round to the columns of Z^T (and column n)
        const int ncol = n + 1;
        for (int idx = tid - 64; idx < 2 * ncol; idx += nt - 64) {
          const int p = idx >= ncol ? 1 : 0, q = idx - p * ncol;
          const int cnt = rcnt[p][buf ^ 1], m = rm[p][buf ^ 1];
          if (cnt == 0) continue;
          const float* cs = rc[p][buf ^ 1];
          const float* sn = rs[p][buf ^ 1];
          float zf = Z[m * ldz + q];
#pragma unroll 4
          for (int t = 0; t < cnt; ++t) {
            const int i = m - 1 - t;
            const float zi = Z[i * ldz + q];
            Z[(i + 1) * ldz + q] = sn[t] * zi + cs[t] * zf;
            zf = cs[t] * zi - sn[t] * zf;
          }
          Z[(m - cnt) * ldz + q] = zf;
        }
      }
      __syncthreads();
      const bool done = sh_done[0] && sh_done[1];
      buf ^= 1;
      __syncthreads();
      if (done) break;
    }
  }
  // ---- rank-one merge: eigenvalues of D + rho z z^T (D = d, z = Z[.][n] / sqrt 2,
  // rho = 2 beta); for beta < 0 the problem -D + |rho| z z^T is solved and negated
  const float beta0 = sh_beta;
  if (beta0 != 0.f) {
    const bool neg = beta0 < 0.f;
    const float rho = 2.f * fabsf(beta0);
    const float rs2 = 0.70710678118654752f;
    for (int i = tid; i < n; i += nt) {
      const float di = neg ? -d[i] : d[i];
      int rank = 0;
      for (int j = 0; j < n; ++j) {
        const float dj = neg ? -d[j] : d[j];
        rank += (dj < di) || (dj == di && j < i);
      }
      perm[rank] = i;
      ds[rank] = di;
      zs[rank] = Z[i * ldz + n] * rs2;
    }
    __syncthreads();
    if (tid == 0) {
      // deflation (LAPACK DLAED2's rules): a negligible component leaves d_r as an
      // eigenvalue; two close poles are rotated so that one component vanishes
      float dmax = 0, zmax = 0;
      for (int r = 0; r < n; ++r) dmax = fmaxf(dmax, fabsf(ds[r])), zmax = fmaxf(zmax, fabsf(zs[r]));
      const float tol = 8.f * eps * fmaxf(dmax, rho * zmax);
      int K = 0, nrot = 0, prev = -1;
      for (int r = 0; r < n; ++r) {
        if (rho * fabsf(zs[r]) <= tol) continue;
        if (prev >= 0) {
          const float zp = zs[prev], zr = zs[r];
          const float t = hypotf(zp, zr);
          const float c = zr / t, sg = -zp / t;
          const float off = (ds[r] - ds[prev]) * c * sg;
          if (fabsf(off) <= tol) {
            // rotate (prev, r): z_prev -> 0, z_r -> t; prev leaves as deflated
            zs[r] = t;
            zs[prev] = 0.f;
            const float dp = ds[prev], dr = ds[r];
            ds[prev] = dp * c * c + dr * sg * sg;
            ds[r] = dp * sg * sg + dr * c * c;
            rot_a[nrot] = perm[prev];
            rot_b[nrot] = perm[r];
            rot_c[nrot] = c;
            rot_s[nrot] = sg;
            ++nrot;
            --K;   // prev was counted
            prev = r;
            kidx[K++] = r;
            continue;
          }
        }
        prev = r;
        kidx[K++] = r;
      }
      sh_K = K;
      sh_nrot = nrot;
    }
    __syncthreads();
    const int K = sh_K, nrot = sh_nrot;
    // the deflating rotations act on the vectors (rows of Z^T), in order
    if (warp == 0) {
      for (int t = 0; t < nrot; ++t) {
        const int a = rot_a[t], b = rot_b[t];
        const float c = rot_c[t], sg = rot_s[t];
        for (int q = lane; q < n; q += 32) {
          const float xa = Z[a * ldz + q], xb = Z[b * ldz + q];
          Z[a * ldz + q] = c * xa + sg * xb;
          Z[b * ldz + q] = c * xb - sg * xa;
        }
        __syncwarp();
      }
    }
    for (int j = tid; j < K; j += nt) {
      dk[j] = ds[kidx[j]];
      zk[j] = zs[kidx[j]];
    }
    __syncthreads();
    // secular equation f(x) = 1 + rho sum_i zk_i^2 / (dk_i - x) = 0, one root per
    // interval (dk_j, dk_j+1), the last in (dk_K-1, dk_K-1 + rho |zk|^2); each
    // root is found as an offset tau from the nearer pole dk_org by Newton's
    // method on f inside a bracket that every step narrows (bisection where a
    // Newton step would leave it); two threads per root split the sums
    float zz = 0.f;
    for (int i = 0; i < K; ++i) zz += zk[i] * zk[i];
    for (int j0 = 0; j0 < K; j0 += nt >> 1) {   // uniform trip count: both threads of a pair join the shuffles
      const int j = j0 + (tid >> 1), h = tid & 1;
      const bool act = j < K;
      const bool inner = act && j < K - 1;
      const float w = inner ? dk[j + 1] - dk[j] : 0.f;
      float fmid = 0.f;
      if (inner)
        for (int i = h; i < K; i += 2) fmid += zk[i] * zk[i] / ((dk[i] - dk[j]) - 0.5f * w);
      fmid += __shfl_xor_sync(0xffffffffu, fmid, 1);
      int o = 0;
      float lo = 0.f, hi = 0.f;
      if (inner) {
        if (1.f + rho * fmid >= 0.f) {
          o = j;
          hi = 0.5f * w;
        } else {
          o = j + 1;
          lo = -0.5f * w;
        }
      } else if (act) {
        o = K - 1;
        hi = rho * zz * 1.0001f;
      }
      const float dorg = act ? dk[o] : 0.f;
      float t = 0.5f * (lo + hi);
      for (int it = 0; it < 40; ++it) {
        float f = 0.f, fp = 0.f;
        if (act)
          for (int i = h; i < K; i += 2) {
            const float rcp = __fdividef(1.f, (dk[i] - dorg) - t);
            const float zr = zk[i] * rcp;
            f = fmaf(zk[i], zr, f);
            fp = fmaf(zr, zr, fp);
          }
        f += __shfl_xor_sync(0xffffffffu, f, 1);
        fp += __shfl_xor_sync(0xffffffffu, fp, 1);
        bool stop = true;
        if (act) {
          const float F = fmaf(rho, f, 1.f);
          if (F < 0.f) lo = t;
          else hi = t;
          float tn = t - F / (rho * fp);
          if (!(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
          stop = fabsf(tn - t) <= 2.f * eps * fmaxf(fabsf(t), fabsf(tn)) || hi - lo <= 2.f * eps * fmaxf(fabsf(lo), fabsf(hi));
          t = tn;
        }
        if (__all_sync(0xffffffffu, stop)) break;
      }
      if (act && h == 0) {
        org[j] = o;
        tau[j] = t;
        lam[j] = dorg + t;
      }
    }
    __syncthreads();
    for (int i = tid; i < K; i += nt) {
      float prod = ((dk[org[K - 1]] - dk[i]) + tau[K - 1]) / rho;
      for (int k = 0; k < i; ++k) prod *= __fdividef((dk[org[k]] - dk[i]) + tau[k], dk[k] - dk[i]);
      for (int k = i; k < K - 1; ++k) prod *= __fdividef((dk[org[k]] - dk[i]) + tau[k], dk[k + 1] - dk[i]);
      zhat[i] = copysignf(sqrtf(fmaxf(prod, 0.f)), zk[i]);
    }
    __syncthreads();
    // merged vectors: u_j(i) = zhat_i / (dk_i - lam_j), normalised, as row j of
    // W (shared memory, in A's place)
    float* W = A;
    for (int j = tid; j < K; j += nt) {
      const float dorg = dk[org[j]], tj = tau[j];
      float nrm = 0.f;
      for (int i = 0; i < K; ++i) {
        const float u = __fdividef(zhat[i], (dk[i] - dorg) - tj);
        W[j * K + i] = u;
        nrm = fmaf(u, u, nrm);
      }
      const float inv = rsqrtf(nrm);
      for (int i = 0; i < K; ++i) W[j * K + i] *= inv;
    }
    for (int i = tid; i < K; i += nt) kslot[i] = perm[kidx[i]];
    __syncthreads();
    // new rows j = sum_i u_j(i) row(slot_i), four rows j per thread, through
    // global scratch (Z is read until every product is formed)
    const int nb = (K + 3) / 4;
    for (int o = tid; o < nb * n; o += nt) {
      const int jb = o / n, q = o - jb * n, j0 = 4 * jb;
      const int j1 = min(j0 + 1, K - 1), j2 = min(j0 + 2, K - 1), j3 = min(j0 + 3, K - 1);
      float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 4
      for (int i = 0; i < K; ++i) {
        const float z = Z[kslot[i] * ldz + q];
        a0 = fmaf(W[j0 * K + i], z, a0);
        a1 = fmaf(W[j1 * K + i], z, a1);
        a2 = fmaf(W[j2 * K + i], z, a2);
        a3 = fmaf(W[j3 * K + i], z, a3);
      }
      gW[(size_t)j0 * n + q] = a0;
      if (j0 + 1 < K) gW[(size_t)(j0 + 1) * n + q] = a1;
      if (j0 + 2 < K) gW[(size_t)(j0 + 2) * n + q] = a2;
      if (j0 + 3 < K) gW[(size_t)(j0 + 3) * n + q] = a3;
    }
    __syncthreads();
    for (int o = tid; o < K * n; o += nt) {
      const int j = o / n, q = o - j * n;
      Z[kslot[j] * ldz + q] = gW[o];
    }
    // eigenvalues back in the original order of the rows
    for (int r = tid; r < n; r += nt) d[perm[r]] = neg ? -ds[r] : ds[r];
    __syncthreads();
    for (int j = tid; j < K; j += nt) d[perm[kidx[j]]] = neg ? -lam[j] : lam[j];
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) d[i] *= scale;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const float di = d[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float dj = d[j];
      rank += (dj > di) || (dj == di && j < i);
    }
    evals[rank] = (double)di;
    if (!isfinite((double)di)) atomicOr(status, 2);
    for (int q = 0; q < n; ++q) evecs[q * n + rank] = (double)Z[i * ldz + q];
  }
  if (tid == 0 && sh_state) atomicOr(status, 1);
}


// ---------------------------------------------------------------- parallel Jacobi (FP32)
// Two-sided cyclic Jacobi with the round-robin ordering: in each round the
// n/2 disjoint pairs (p, q) are rotated at once (rotation angles from the
// 2x2 blocks, Golub & Van Loan Sec. 8.5), rows then columns of A and columns
// of V updated in parallel.  Sweeps stop when every off-diagonal entry is
// below eps * sqrt(|a_pp a_qq|) or, for null blocks, eps * max|diag|.
constexpr int kJacMax = 160;
// FP32 relative rotation threshold of the refinement sweeps: a few units of
// FP32 rounding above it, so that the sweeps terminate (a threshold at the
// rounding level itself keeps rotating on rounding noise).
constexpr float kJacRelTol = 2e-6f;
constexpr int kJacThreads = 512;

__device__ __forceinline__ void rr_pair(int r, int k, int np, int& p, int& q) {
  // players 0..np-1, player np-1 fixed, others rotate (np even)
  if (k == 0) {
    p = np - 1;
    q = r;
  } else {
    p = (r + k) % (np - 1);
    q = (r - k + (np - 1)) % (np - 1);
  }
}

template <typename T>
__global__ void __launch_bounds__(kJacThreads) k_jacobi_eig(const double* __restrict__ S, int n, int max_sweeps,
                                                          T tol, double* __restrict__ evals, double* __restrict__ evecs,
                                                          int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char jac_raw[];
  T* jac_sm = reinterpret_cast<T*>(jac_raw);
  const int np = n + (n & 1);           // padded size (even)
  T* A = jac_sm;                        // np x np
  T* V = jac_sm + np * np;              // np x np, column j = vector j
  __shared__ T cs_[kJacMax / 2], sn_[kJacMax / 2];
  __shared__ int pp_[kJacMax / 2], qq_[kJacMax / 2];
  __shared__ int sh_rot;
  __shared__ T sh_floor;
  const T eps = tol;   // rotate while |a_pq| > tol * sqrt(|a_pp a_qq|)
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < np * np; idx += nt) {
    const int i = idx / np, j = idx - i * np;
    A[idx] = (i < n && j < n) ? (T)(0.5 * (S[i * n + j] + S[j * n + i])) : (T)0;
    V[idx] = i == j ? (T)1 : (T)0;
  }
  __syncthreads();
  if (tid == 0) {
    T fro = 0;
    for (int idx = 0; idx < np * np; ++idx) fro += A[idx] * A[idx];
    sh_floor = eps * (T)1e-3 * sqrt(fro);   // absolute floor for (near) null 2x2 blocks
  }
  __syncthreads();
  const int half = np / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) sh_rot = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      if (tid < half) {
        int p, q;
        rr_pair(r, tid, np, p, q);
        if (p > q) { const int t = p; p = q; q = t; }
        const T apq = A[p * np + q], app = A[p * np + p], aqq = A[q * np + q];
        T c = 1, s = 0;
        const T thr = fmax(eps * sqrt(fabs(app * aqq)), sh_floor);
        if (fabs(apq) > thr && apq != (T)0) {
          const T th = (aqq - app) / ((T)2 * apq);
          const T t = (th >= (T)0 ? (T)1 : (T)-1) / (fabs(th) + sqrt(th * th + (T)1));
          c = (T)1 / sqrt(t * t + (T)1);
          s = t * c;
          sh_rot = 1;
        }
        cs_[tid] = c;
        sn_[tid] = s;
        pp_[tid] = p;
        qq_[tid] = q;
      }
      // a round in which no pair rotates leaves A and V as they are
      if (!__syncthreads_or(tid < half && sn_[tid] != (T)0)) continue;
      // rows p, q of A: a warp per pair, lanes along the row
      const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
      for (int k = warp; k < half; k += nwarp) {
        const T c = cs_[k], s = sn_[k];
        if (s == (T)0) continue;
        const int p = pp_[k], q = qq_[k];
        for (int col = lane; col < np; col += 32) {
          const T ap = A[p * np + col], aq = A[q * np + col];
          A[p * np + col] = c * ap - s * aq;
          A[q * np + col] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns p, q of A and V: a warp per pair, lanes down the column
      for (int k = warp; k < half; k += nwarp) {
        const T c = cs_[k], s = sn_[k];
        if (s == (T)0) continue;
        const int p = pp_[k], q = qq_[k];
        for (int row = lane; row < np; row += 32) {
          const T ap = A[row * np + p], aq = A[row * np + q];
          A[row * np + p] = c * ap - s * aq;
          A[row * np + q] = s * ap + c * aq;
          const T vp = V[row * np + p], vq = V[row * np + q];
          V[row * np + p] = c * vp - s * vq;
          V[row * np + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
    // read the flag everywhere before thread 0 resets it for the next sweep
    const int rot = sh_rot;
    __syncthreads();
    if (!rot) break;
  }
  // sort the first n diagonal entries descending (the padding index stays out)
  for (int i = tid; i < n; i += nt) {
    const T di = A[i * np + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T dj = A[j * np + j];
      rank += (dj > di) || (dj == di && j < i);
    }
    evals[rank] = (double)di;
    if (!isfinite((double)di)) atomicOr(status, 2);
    for (int q = 0; q < n; ++q) evecs[q * n + rank] = (double)V[q * np + i];
  }
  if (tid == 0 && sweep >= max_sweeps) atomicOr(status, 4);
}

// C = A^T B (FP64, n x n row-major), one thread per entry
__global__ void k_small_mm_tn(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C, int n) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += A[k * n + i] * B[k * n + j];
    C[idx] = acc;
  }
}


// ---------------------------------------------------------------- Cholesky QR step
// T = R^{-1} with R^T R = S (upper Cholesky factor), S symmetric positive
// definite (the Gram of an almost orthonormal block).  One block, FP32.  The
// right-looking factorisation updates the upper triangle of the Schur
// complement, A_rc -= A_jr A_jc / A_jj (four threads to a row, one barrier
// per column), and scales the rows by 1 / sqrt(A_jj) at the end; the inverse
// is formed column by column (one thread per column, back substitution) in
// shared memory when it fits, else in T.
__host__ __device__ constexpr int chol_ld(int n) { return ((n + 27) / 32) * 32 + 4; }

__global__ void __launch_bounds__(512) k_chol_inv(const double* __restrict__ S, int n, float* __restrict__ T, int ldt,
                                                int* __restrict__ status, double* __restrict__ inv_fro2, int x_smem) {
  extern __shared__ __align__(16) float ch_sm[];
  const int lda = chol_ld(n);
  float* A = ch_sm;                       // n x lda, upper triangle becomes R
  float* X = x_smem ? A + (size_t)n * lda : T;
  const int ldx = x_smem ? lda : ldt;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    A[i * lda + j] = (float)(0.5 * (S[i * n + j] + S[j * n + i]));
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const float a = A[j * lda + j];
    if (tid == 0 && !(a > 0.f)) atomicOr(status, 8);
    const float inv = a > 0.f ? 1.f / a : 0.f;
    const float* Aj = A + j * lda;
    for (int r = j + 1 + (tid >> 2); r < n; r += nt >> 2) {
      const float f = Aj[r] * inv;
      float* Ar = A + r * lda;
#pragma unroll 4
      for (int c = r + (tid & 3); c < n; c += 4) Ar[c] = fmaf(-f, Aj[c], Ar[c]);
    }
    __syncthreads();
  }
  for (int j = tid; j < n; j += nt) {
    const float a = A[j * lda + j];
    const float rs = a > 0.f ? rsqrtf(a) : 1.f;
    for (int c = j + 1; c < n; ++c) A[j * lda + c] *= rs;
    A[j * lda + j] = a > 0.f ? a * rs : 1.f;
  }
  __syncthreads();
  // X = R^{-1}: column c solves R x = e_c by back substitution; ||R^{-1}||_F^2
  // is summed on the way
  double sq = 0.0;
  for (int c = tid; c < n; c += nt) {
    for (int i = n - 1; i > c; --i) X[i * ldx + c] = 0.f;
    for (int i = c; i >= 0; --i) {
      const float* Ri = A + i * lda;
      float a0 = (i == c) ? 1.f : 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int k = i + 1;
      for (; k + 3 <= c; k += 4) {
        a0 = fmaf(-Ri[k], X[k * ldx + c], a0);
        a1 = fmaf(-Ri[k + 1], X[(k + 1) * ldx + c], a1);
        a2 = fmaf(-Ri[k + 2], X[(k + 2) * ldx + c], a2);
        a3 = fmaf(-Ri[k + 3], X[(k + 3) * ldx + c], a3);
      }
      for (; k <= c; ++k) a0 = fmaf(-Ri[k], X[k * ldx + c], a0);
      const float x = ((a0 + a1) + (a2 + a3)) / Ri[i];
      X[i * ldx + c] = x;
      sq += (double)x * (double)x;
    }
  }
  if (inv_fro2) {
    __shared__ double red[16];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
    if ((tid & 31) == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) t += red[w];
      *inv_fro2 = t;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * ldt; idx += nt) {
    const int i = idx / ldt, c = idx - i * ldt;
    if (c >= n) T[idx] = 0.f;
    else if (x_smem) T[idx] = X[i * ldx + c];
  }
}

__global__ void k_select_scale(const double* __restrict__ E, int n, int rows, const int* __restrict__ cols,
                               const double* __restrict__ scale, int ncols, float* __restrict__ T, int ldt) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * ldt; idx += gridDim.x * blockDim.x) {
    const int r = idx / ldt, c = idx - r * ldt;
    T[idx] = c < ncols ? (float)(E[r * n + cols[c]] * scale[c]) : 0.f;
  }
}

__global__ void k_to_f32(const double* __restrict__ S, int rows, int cols, int lds, float* __restrict__ T, int ldt) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * ldt; idx += gridDim.x * blockDim.x) {
    const int r = idx / ldt, c = idx - r * ldt;
    T[idx] = c < cols ? (float)S[r * lds + c] : 0.f;
  }
}

// One Newton-Schulz step towards the orthogonal factor of V (Higham, "Functions
// of Matrices", Sec. 8.3): out = V (3 I - M) / 2 with M = V^T V; an
// orthogonality error d of V leaves about (3/2) d^2 (FP64, n x n row-major).
__global__ void k_newton_schulz(const double* __restrict__ V, const double* __restrict__ M, double* __restrict__ out,
                                int n) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += V[i * n + k] * M[k * n + j];
    out[idx] = 1.5 * V[idx] - 0.5 * acc;
  }
}

__global__ void k_small_mm(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C,
                           int r, int s, int t, int transB) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < r * t; idx += gridDim.x * blockDim.x) {
    const int i = idx / t, j = idx - i * t;
    double acc = 0.0;
    for (int k = 0; k < s; ++k) acc += A[i * s + k] * (transB ? B[j * s + k] : B[k * t + j]);
    C[idx] = acc;
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// SplitMix64 counter generator: key = mix(seed*gamma + stream),
// u_i = ((mix(key + i*gamma) >> 11) + 1) 2^-53, x_j = sqrt(-2 ln u_2j) cos(2 pi u_2j+1)
__global__ void k_counter_normal(uint64_t seed, uint64_t stream, uint64_t offset, int64_t count,
                                 float* __restrict__ X, int ld, int col) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  const uint64_t key = mix64(seed * G + stream);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t j = offset + (uint64_t)i;
    const uint64_t z1 = mix64(key + (2 * j) * G), z2 = mix64(key + (2 * j + 1) * G);
    const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = ((double)(z2 >> 11) + 1.0) * 0x1.0p-53;
    X[i * ld + col] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
  }
}

__global__ void k_negate(const float* __restrict__ a, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = -a[i];
}

__global__ void k_res_sums(const float* __restrict__ r, const float* __restrict__ a, int64_t n,
                           double* __restrict__ part) {
  __shared__ double s1[256], s2[256];
  double x = 0.0, y = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double rv = r[i];
    x += rv * rv;
    y += rv * (double)a[i];
  }
  s1[threadIdx.x] = x;
  s2[threadIdx.x] = y;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s1[threadIdx.x] += s1[threadIdx.x + o], s2[threadIdx.x] += s2[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[2 * blockIdx.x] = s1[0], part[2 * blockIdx.x + 1] = s2[0];
}

__global__ void k_sum_pairs(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < nb; ++i) a += part[2 * i], b += part[2 * i + 1];
    out[0] = a;
    out[1] = b;
  }
}

__global__ void k_copy_cols(const float* __restrict__ src, int lds, int s0, float* __restrict__ dst, int ldd,
                            int d0, int c, int64_t rows) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < rows * c;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / c;
    const int j = (int)(idx - r * c);
    dst[r * ldd + d0 + j] = src[r * lds + s0 + j];
  }
}

int grid1(int64_t work, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, threads), (int64_t)num_sms() * 8));
}

}  // namespace

void gram_dev(bm_ctx& h, DenseWork& w, const Tall& A, const Tall& B, double* C, bool compensated, const char* tag) {
  BM_REQUIRE(A.rows == B.rows, BM_ERR_INVALID, "gram: row mismatch");
  const int a = A.cols, b = B.cols;
  if (a == 0 || b == 0) return;
  const int64_t L = A.rows;
  if (L == 0) {
    BM_CUDA(cudaMemsetAsync(C, 0, (size_t)a * b * sizeof(double), h.stream));
    return;
  }
  const int sym = (A.p == B.p && A.ld == B.ld && a == b) ? 1 : 0;
  // symmetric plain Grams (the Rayleigh-Ritz matrix) on the tensor cores when
  // the handle allows it and the shape fits: measured 0.43 -> 0.26 ms at the
  // recommendation-scale size; the thin non-symmetric products (W^T U, H^T Y)
  // run faster on the FP32 pipes (0.18 against 0.31 ms: staging and slicing
  // two operands dominate at these widths) and stay there
  if (!compensated && sym && h.opt.tensor_grams == 1 && gram_tc_dev(h, w, A, B, C, tag)) return;
  const int ng = (a + 7) / 8, nb = (b + 3) / 4;
  int tiles = ng * nb;
  if (sym) {   // the kernel enumerates only the micro-tiles on or above the diagonal
    tiles = 0;
    for (int c = 0; c < nb; ++c) tiles += std::min(ng, (4 * c + 3) / 8 + 1);
  }
  // short blocks (few rows): each thread's chain is (slab rows) x (its 32
  // products), so the micro-tiles spread over more, smaller blocks and the
  // slabs shrink to one 32-row tile
  const bool short_rows = L <= 16 * kGramRows * 64;
  const int per_block = short_rows ? 128 : kGramMaxThreads;
  const int gy = (tiles + per_block - 1) / per_block;
  const int threads = (int)(ceil_div(ceil_div(tiles, gy), 32) * 32);
  int64_t gx = std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, short_rows ? kGramRows : 64),
                                                      std::max<int64_t>(1, (int64_t)(compensated ? kGramBlocksPerSmComp : kGramBlocksPerSmPlain) * num_sms() / gy)));
  const int64_t slab = ceil_div(ceil_div(L, gx), kGramRows) * kGramRows;
  gx = ceil_div(L, slab);
  static_assert(sizeof(double) == sizeof(float2), "FP32-pair partials share the FP64 scratch");
  w.gram_part.alloc((size_t)gx * a * b);
  const size_t smem = (size_t)2 * kGramRows * (2 * ng + nb) * sizeof(float4);
  BM_REQUIRE(smem <= 200 * 1024, BM_ERR_INVALID, "gram: block too wide");
  float2* part = reinterpret_cast<float2*>(w.gram_part.get());
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (compensated) {
    allow_max_smem((const void*)k_gram<true>);
    BM_LAUNCH(h, tag, k_gram<true><<<grid, threads, smem, h.stream>>>(A.p, A.ld, a, B.p, B.ld, b, L, slab, sym, part));
  } else {
    allow_max_smem((const void*)k_gram<false>);
    BM_LAUNCH(h, tag, k_gram<false><<<grid, threads, smem, h.stream>>>(A.p, A.ld, a, B.p, B.ld, b, L, slab, sym, part));
  }
  gram_reduce_dev(h, part, (int)gx, a, b, sym, C);
}

void gram_reduce_dev(bm_ctx& h, const float2* part, int slabs, int a, int b, int sym, double* C) {
  BM_LAUNCH(h, "gram_reduce", k_gram_reduce<<<(unsigned)ceil_div((int64_t)a * b, 32), 256, 0, h.stream>>>(
                                  part, slabs, a, b, sym, C));
}

void gemm_dev(bm_ctx& h, const Tall& A, const float* C, int ldc, const Tall& Y, float beta, float gamma,
              const char* tag) {
  const int a = A.cols, b = Y.cols;
  if (b == 0 || A.rows == 0) return;
  if (a == 0) {
    if (beta == 0.f) zero_dev(h, Y);
    return;
  }
  const int nb4 = (b + 3) / 4, a4 = (a + 3) / 4;
  BM_REQUIRE(nb4 <= kGemmThreads, BM_ERR_INVALID, "gemm: too many columns");
  const int groups = std::max(1, std::min(32, kGemmThreads / nb4));
  const int R = 8 * groups;
  const size_t smem = (size_t)a * nb4 * sizeof(float4) + (size_t)4 * a4 * R * sizeof(float);
  BM_REQUIRE(smem <= 200 * 1024, BM_ERR_INVALID, "gemm: block too large");
  allow_max_smem((const void*)k_gemm);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(A.rows, R), (int64_t)num_sms() * 3));
  BM_LAUNCH(h, tag, k_gemm<<<grid, kGemmThreads, smem, h.stream>>>(A.p, A.ld, a, C, ldc, b, Y.p, Y.ld, A.rows,
                                                                   beta, gamma, groups));
}

// ---------------------------------------------------------------- shared SpMM launches
// Longest time a product waits for the other participants' products before
// the products that have arrived are launched without them.
constexpr int kCombineWaitUs = 100;

struct SpmmCombiner {
  struct Req {
    bm_ctx* h;
    bool csr;
    const float* vals;
    Tall X, Out;
    float gamma;
  };
  std::mutex mu;
  std::condition_variable cv;
  int live = 0;
  uint64_t gen = 0;
  std::vector<Req> pending;
  std::map<bm_ctx*, cudaEvent_t> ready;   // per participant: its stream's work so far
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  DevBuf<PipeArgs> args_d;
  DevBuf<int64_t> prefix_d;
  int cap = 0;                             // slices the device tables hold
  bm_status fail = BM_OK;   // sticky until spmm_combiner_begin: a failed launch fails every later product
  std::string fail_msg;
  int64_t launches = 0;   // batched SpMM launches
  int64_t products = 0;   // products handed in

  // Launch every pending product (called with mu held, by the last arrival or
  // by a product that waited long enough).  After a failed launch nothing is
  // launched again in this batched step: a participant woken late then reads
  // the failure, never a later generation's success, as its own.
  void launch_all() {
    if (fail == BM_OK) {
      try {
        launch_pending();
      } catch (const Error& e) {
        fail = e.code;
        fail_msg = e.msg;
      } catch (...) {
        fail = BM_ERR_CUDA;
        fail_msg = "spmm combiner: launch failed";
      }
    }
    pending.clear();
    ++gen;
    cv.notify_all();
  }

  // Batched launches of the pending products on the combiner's stream (throws).
  void launch_pending() {
    for (const Req& r : pending) BM_CUDA(cudaStreamWaitEvent(st, ready.at(r.h), 0));
    struct Slice {
      const Req* r;
      PipeArgs a;
      bool ws;
      int cols;
      const Segs* sg;
    };
    std::vector<Slice> sl;
    for (const Req& r : pending) {
      const Index& ix = r.h->ix;
      const int kind = r.csr ? kPassSpmmCsr : kPassSpmmCsc;
      const Segs& sg = pass_segs(ix, kind);
      for (int c0 = 0; c0 < r.X.cols; c0 += kSpmmCols) {
        const int cols = std::min(kSpmmCols, r.X.cols - c0);
        PipeArgs a{};
        a.seg_row = sg.row.get();
        a.seg_beg = sg.beg.get();
        a.seg_end = sg.end.get();
        a.seg_slot = sg.slot.get();
        a.nseg = sg.nseg;
        a.idx = r.csr ? ix.col.get() : ix.row.get();
        a.scal = r.vals;
        a.g0 = r.X.p + c0;
        a.ld = r.X.ld;
        a.nchunk = (cols + 3) / 4;
        a.gamma = r.gamma;
        a.out = r.Out.p + c0;
        a.ld_out = r.Out.ld;
        a.partial = r.h->sc.partial.get();
        a.ld_part = 4 * a.nchunk;
        BM_REQUIRE((int64_t)std::max<int64_t>(1, sg.nslots) * a.ld_part <= (int64_t)r.h->sc.partial.n,
                   BM_ERR_INVALID, "spmm: partial buffer too small");
        sl.push_back({&r, a, pass_ws(ix, kind), cols, &sg});
      }
    }
    // one launch per (orientation, row width, layout)
    std::stable_sort(sl.begin(), sl.end(), [](const Slice& x, const Slice& y) {
      return std::make_tuple(x.r->csr, x.a.nchunk, x.ws) < std::make_tuple(y.r->csr, y.a.nchunk, y.ws);
    });
    if ((int)sl.size() > cap) throw Error{BM_ERR_INVALID, "spmm combiner: more products than the tables hold"};
    std::vector<PipeArgs> A;
    std::vector<int64_t> P;
    size_t off = 0, poff = 0;
    for (size_t g0 = 0; g0 < sl.size();) {
      size_t g1 = g0 + 1;
      while (g1 < sl.size() && sl[g1].r->csr == sl[g0].r->csr && sl[g1].a.nchunk == sl[g0].a.nchunk &&
             sl[g1].ws == sl[g0].ws)
        ++g1;
      A.clear();
      P.assign(1, 0);
      for (size_t i = g0; i < g1; ++i) {
        A.push_back(sl[i].a);
        P.push_back(P.back() + sl[i].a.nseg);
      }
      // pageable sources: the copies are staged before the calls return
      BM_CUDA(cudaMemcpyAsync(args_d.get() + off, A.data(), A.size() * sizeof(PipeArgs), cudaMemcpyHostToDevice,
                              st));
      BM_CUDA(cudaMemcpyAsync(prefix_d.get() + poff, P.data(), P.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                              st));
      launch_direct_batch<1>(args_d.get() + off, prefix_d.get() + poff, (int)A.size(), P.back(),
                             sl[g0].a.nchunk, false, sl[g0].ws, st);
      BM_CHECK_LAUNCH();
      ++launches;
      off += A.size();
      poff += P.size();
      g0 = g1;
    }
    for (const Slice& x : sl) {
      const Segs& sg = *x.sg;
      if (!sg.nmulti) continue;
      k_spmm_fixup<<<grid1(sg.nmulti * x.cols), 256, 0, st>>>(sg.mrow.get(), sg.mfirst.get(), sg.mcount.get(),
                                                               sg.nmulti, x.a.partial, x.a.ld_part, x.cols,
                                                               x.a.gamma, x.a.out, x.a.ld_out);
      BM_CHECK_LAUNCH();
    }
    BM_CUDA(cudaEventRecord(done, st));
  }
};

SpmmCombiner* spmm_combiner_create(int participants_max) {
  auto c = std::make_unique<SpmmCombiner>();
  BM_CUDA(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
  BM_CUDA(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
  // at most two column slices per product (q <= 2 kSpmmCols)
  c->cap = 2 * std::max(1, participants_max);
  c->args_d.alloc((size_t)c->cap);
  c->prefix_d.alloc((size_t)2 * c->cap);
  return c.release();
}

void spmm_combiner_destroy(SpmmCombiner* c) {
  if (!c) return;
  if (c->st) {
    cudaStreamSynchronize(c->st);
    cudaStreamDestroy(c->st);
  }
  if (c->done) cudaEventDestroy(c->done);
  for (auto& kv : c->ready) cudaEventDestroy(kv.second);
  delete c;
}

void spmm_combiner_begin(SpmmCombiner* c, int participants) {
  std::lock_guard<std::mutex> lk(c->mu);
  c->live = participants;
  c->pending.clear();
  c->fail = BM_OK;
  c->fail_msg.clear();
}

void spmm_combiner_leave(SpmmCombiner* c) {
  std::lock_guard<std::mutex> lk(c->mu);
  --c->live;
  if (c->live > 0 && (int)c->pending.size() == c->live) c->launch_all();
}

int64_t spmm_combiner_launches(const SpmmCombiner* c) { return c ? c->launches : 0; }
int64_t spmm_combiner_products(const SpmmCombiner* c) { return c ? c->products : 0; }

namespace {
void spmm_combined(bm_ctx& h, bool csr, const float* vals, const Tall& X, const Tall& Out, float gamma) {
  SpmmCombiner& c = *h.comb;
  std::unique_lock<std::mutex> lk(c.mu);
  auto it = c.ready.find(&h);
  if (it == c.ready.end()) {
    cudaEvent_t ev = nullptr;
    BM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    it = c.ready.emplace(&h, ev).first;
  }
  BM_CUDA(cudaEventRecord(it->second, h.stream));
  c.pending.push_back({&h, csr, vals, X, Out, gamma});
  ++c.products;
  const uint64_t g = c.gen;
  if ((int)c.pending.size() == c.live) {
    c.launch_all();
  } else if (!c.cv.wait_for(lk, std::chrono::microseconds(kCombineWaitUs), [&] { return c.gen != g; })) {
    // waited long enough for the others: launch what has arrived
    c.launch_all();
  }
  if (c.fail != BM_OK) throw Error{c.fail, c.fail_msg};
  // A later generation may already have re-recorded `done` (one launched by a
  // product that waited long enough); that record follows this generation's
  // launches on the combiner's stream, so waiting for it covers them too.
  BM_CUDA(cudaStreamWaitEvent(h.stream, c.done, 0));
}
}  // namespace

void spmm_dev(bm_ctx& h, bool csr, const float* vals, const Tall& X, const Tall& Out, float gamma) {
  if (X.cols == 0) return;
  if (h.comb) {
    spmm_combined(h, csr, vals, X, Out, gamma);
    return;
  }
  const Index& ix = h.ix;
  const Segs& sg = pass_segs(ix, csr ? kPassSpmmCsr : kPassSpmmCsc);
  if (X.cols == 0) return;
  // one launch per slice of at most kSpmmCols columns (the kernel's widest row)
  for (int c0 = 0; c0 < X.cols; c0 += kSpmmCols) {
    const int cols = std::min(kSpmmCols, X.cols - c0);
    PipeArgs a{};
    a.seg_row = sg.row.get();
    a.seg_beg = sg.beg.get();
    a.seg_end = sg.end.get();
    a.seg_slot = sg.slot.get();
    a.nseg = sg.nseg;
    a.idx = csr ? ix.col.get() : ix.row.get();
    a.scal = vals;
    a.g0 = X.p + c0;
    a.ld = X.ld;
    a.nchunk = (cols + 3) / 4;
    a.gamma = gamma;
    a.out = Out.p + c0;
    a.ld_out = Out.ld;
    a.partial = h.sc.partial.get();
    a.ld_part = 4 * a.nchunk;
    BM_REQUIRE((int64_t)std::max<int64_t>(1, sg.nslots) * a.ld_part <= (int64_t)h.sc.partial.n, BM_ERR_INVALID,
               "spmm: partial buffer too small");
    // The residual products of the PG step gather FP32 rows: BF16 operands
    // leave LmSVD short of its stop tolerance (the factor gathers of the BM
    // phase are the ones that use BF16).
    BM_LAUNCH(h, csr ? "spmm_csr" : "spmm_csc",
              launch_pipe<1>(a, h.stream, false, pass_ws(ix, csr ? kPassSpmmCsr : kPassSpmmCsc)));
    if (sg.nmulti) {
      BM_LAUNCH(h, "spmm_fixup",
                k_spmm_fixup<<<grid1(sg.nmulti * cols), 256, 0, h.stream>>>(
                    sg.mrow.get(), sg.mfirst.get(), sg.mcount.get(), sg.nmulti, a.partial, a.ld_part, cols, gamma,
                    a.out, Out.ld));
    }
  }
}

void sym_eig_dev(bm_ctx& h, DenseWork& w, const double* S, int n, double* evals, double* evecs, EigMode mode) {
  BM_REQUIRE(n >= 1 && n <= kEigMax, BM_ERR_INVALID, "eigensolver: size out of range");
  const int npd = n + (n & 1);
  const bool jac64 = mode == kEigDouble && (size_t)2 * npd * npd * sizeof(double) <= 200 * 1024;
  const bool jac32 = mode == kEigRelative && npd <= kJacMax;
  if (jac64 || jac32) {
    // FP32 QL for approximate vectors V0, one FP64 Newton-Schulz step to an
    // orthogonal V (so that S' below is a similarity transform of S, not a
    // congruence whose eigenvalues would carry the FP32 orthogonality error of
    // V0 as a relative error), S' = V^T S V in FP64, Jacobi sweeps on the
    // almost diagonal S' (FP64 or FP32), vectors V * V'
    w.scratch.alloc((size_t)4 * n * n);
    double* V0 = w.scratch.get();
    double* T1 = V0 + (size_t)n * n;
    double* S2 = T1 + (size_t)n * n;
    double* V = S2 + (size_t)n * n;
    sym_eig_dev(h, w, S, n, evals, V0, kEigFast);
    // one output per thread, 64-thread blocks: n^2 outputs spread over many SMs
    // (FP64 issues slowly on this part)
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)n * n, 64), (int64_t)num_sms() * 16));
    BM_LAUNCH(h, "eig_rotate", k_small_mm_tn<<<g, 64, 0, h.stream>>>(V0, V0, S2, n));
    BM_LAUNCH(h, "eig_rotate", k_newton_schulz<<<g, 64, 0, h.stream>>>(V0, S2, V, n));
    BM_LAUNCH(h, "eig_rotate", k_small_mm<<<g, 64, 0, h.stream>>>(S, V, T1, n, n, n, 0));
    BM_LAUNCH(h, "eig_rotate", k_small_mm_tn<<<g, 64, 0, h.stream>>>(V, T1, S2, n));
    w.status.alloc(1);
    BM_CUDA(cudaMemsetAsync(w.status.get(), 0, sizeof(int), h.stream));
    if (jac64) {
      const size_t smem = (size_t)2 * npd * npd * sizeof(double);
      allow_max_smem((const void*)k_jacobi_eig<double>);
      BM_LAUNCH(h, "jacobi_eig_f64",
                k_jacobi_eig<double><<<1, kJacThreads, smem, h.stream>>>(S2, n, 20, 4e-15, evals, T1, w.status.get()));
    } else {
      const size_t smem = (size_t)2 * npd * npd * sizeof(float);
      allow_max_smem((const void*)k_jacobi_eig<float>);
      BM_LAUNCH(h, "jacobi_eig_rel",
                k_jacobi_eig<float><<<1, kJacThreads, smem, h.stream>>>(S2, n, 20, kJacRelTol, evals, T1, w.status.get()));
    }
    BM_LAUNCH(h, "eig_rotate", k_small_mm<<<g, 64, 0, h.stream>>>(V, T1, evecs, n, n, n, 0));
    int st = 0;
    BM_CUDA(cudaMemcpyAsync(&st, w.status.get(), sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
    BM_REQUIRE(!(st & 2), BM_ERR_NUMERIC, "eigensolver: non-finite eigenvalue");
    return;
  }
  const bool dbl = mode != kEigFast;
  if (!dbl && n >= kDcMin && n <= kDcMax) {
    // one divide-and-conquer level (k_sym_eig_dc); its merge writes through
    // global scratch of n x n floats
    w.status.alloc(1);
    BM_CUDA(cudaMemsetAsync(w.status.get(), 0, sizeof(int), h.stream));
    DevBuf<double>& gbuf = h.sc.eig_glob;
    gbuf.alloc(2 * (size_t)kEigMax * kEigMax);
    allow_max_smem((const void*)k_sym_eig_dc);
    const size_t smem = (size_t)2 * n * dc_ld(n) * sizeof(float);
    BM_LAUNCH(h, "sym_eig_f32", k_sym_eig_dc<<<1, kEigThreads, smem, h.stream>>>(
                                    S, n, evals, evecs, reinterpret_cast<float*>(gbuf.get()), w.status.get()));
    int st = 0;
    BM_CUDA(cudaMemcpyAsync(&st, w.status.get(), sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
    BM_REQUIRE(st == 0, BM_ERR_NUMERIC, st & 2 ? "eigensolver: non-finite eigenvalue" : "eigensolver: QL did not converge");
    return;
  }
  const size_t es = dbl ? 8 : 4;
  const size_t nn = (size_t)n * n * es;
  const size_t cap = 200 * 1024;
  int a_sm = 0, z_sm = 0;
  if (2 * nn <= cap) a_sm = z_sm = 1;
  else if (nn <= cap) a_sm = 1;
  w.status.alloc(1);
  BM_CUDA(cudaMemsetAsync(w.status.get(), 0, sizeof(int), h.stream));
  DevBuf<double>& gbuf = h.sc.eig_glob;  // global storage when shared memory is too small
  if (!(a_sm && z_sm)) gbuf.alloc(2 * (size_t)kEigMax * kEigMax);
  const size_t smem = (a_sm + z_sm) * nn;
  if (dbl) {
    allow_max_smem((const void*)k_sym_eig<double>);
    double* gA = gbuf.get();
    double* gZ = gbuf.get() ? gbuf.get() + (size_t)kEigMax * kEigMax : nullptr;
    BM_LAUNCH(h, "sym_eig_f64", k_sym_eig<double><<<1, kEigThreads, smem, h.stream>>>(
                                    S, n, evals, evecs, gA, gZ, a_sm, z_sm, w.status.get()));
  } else {
    allow_max_smem((const void*)k_sym_eig<float>);
    float* gA = reinterpret_cast<float*>(gbuf.get());
    float* gZ = gA ? gA + (size_t)kEigMax * kEigMax : nullptr;
    BM_LAUNCH(h, "sym_eig_f32", k_sym_eig<float><<<1, kEigThreads, smem, h.stream>>>(
                                    S, n, evals, evecs, gA, gZ, a_sm, z_sm, w.status.get()));
  }
  int st = 0;
  BM_CUDA(cudaMemcpyAsync(&st, w.status.get(), sizeof(int), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  BM_REQUIRE(st == 0, BM_ERR_NUMERIC, st & 2 ? "eigensolver: non-finite eigenvalue" : "eigensolver: QL did not converge");
}

namespace {
// Returns the status word (0: R^{-1} in T) and, with fro2, ||R^{-1}||_F^2.
int chol_inv_run(bm_ctx& h, DenseWork& w, const double* S, int n, float* T, int ldt, double* fro2) {
  BM_REQUIRE(n >= 1 && n <= 200, BM_ERR_INVALID, "cholesky: size out of range");
  const size_t one = (size_t)n * chol_ld(n) * sizeof(float);
  const int x_smem = 2 * one <= 200 * 1024 ? 1 : 0;   // R^{-1} in shared memory beside R when it fits
  const size_t smem = (1 + x_smem) * one;
  w.status.alloc(1);
  w.scratch.alloc(1);
  BM_CUDA(cudaMemsetAsync(w.status.get(), 0, sizeof(int), h.stream));
  allow_max_smem((const void*)k_chol_inv);
  BM_LAUNCH(h, "chol_inv", k_chol_inv<<<1, 512, smem, h.stream>>>(S, n, T, ldt, w.status.get(),
                                                                  fro2 ? w.scratch.get() : nullptr, x_smem));
  int st = 0;
  BM_CUDA(cudaMemcpyAsync(&st, w.status.get(), sizeof(int), cudaMemcpyDeviceToHost, h.stream));
  if (fro2) BM_CUDA(cudaMemcpyAsync(fro2, w.scratch.get(), sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  return st;
}
}  // namespace

void chol_inv_dev(bm_ctx& h, DenseWork& w, const double* S, int n, float* T, int ldt) {
  const int st = chol_inv_run(h, w, S, n, T, ldt, nullptr);
  BM_REQUIRE(st == 0, BM_ERR_NUMERIC, "cholesky: Gram matrix not positive definite");
}

bool chol_inv_try_dev(bm_ctx& h, DenseWork& w, const double* S, int n, float* T, int ldt, double* inv_fro2) {
  double f = 0.0;
  const int st = chol_inv_run(h, w, S, n, T, ldt, &f);
  if (st != 0 || !std::isfinite(f)) return false;
  *inv_fro2 = f;
  return true;
}

void select_scale_dev(bm_ctx& h, const double* E, int n, int rows, const int* cols_h, const double* scale_h,
                      int cols, float* T, int ldt) {
  DevBuf<int>& dcols = h.sc.sel_cols;
  DevBuf<double>& dscale = h.sc.sel_scale;
  dcols.alloc(std::max(cols, 1));
  dscale.alloc(std::max(cols, 1));
  if (cols) {
    BM_CUDA(cudaMemcpyAsync(dcols.get(), cols_h, cols * sizeof(int), cudaMemcpyHostToDevice, h.stream));
    BM_CUDA(cudaMemcpyAsync(dscale.get(), scale_h, cols * sizeof(double), cudaMemcpyHostToDevice, h.stream));
  }
  BM_LAUNCH(h, "small", k_select_scale<<<grid1(rows * ldt), 256, 0, h.stream>>>(E, n, rows, dcols.get(), dscale.get(),
                                                                              cols, T, ldt));
  BM_CUDA(cudaStreamSynchronize(h.stream));  // host arrays may go out of scope
}

void small_to_f32_dev(bm_ctx& h, const double* S, int rows, int cols, int lds, float* T, int ldt) {
  if (rows == 0) return;
  BM_LAUNCH(h, "small", k_to_f32<<<grid1(rows * ldt), 256, 0, h.stream>>>(S, rows, cols, lds, T, ldt));
}

void small_mm_dev(bm_ctx& h, const double* A, const double* B, double* C, int r, int s, int t, bool transB) {
  if (r == 0 || t == 0) return;
  BM_LAUNCH(h, "small", k_small_mm<<<grid1(r * t), 256, 0, h.stream>>>(A, B, C, r, s, t, transB ? 1 : 0));
}

void counter_normal_dev(bm_ctx& h, uint64_t seed, uint64_t stream, int64_t count, const Tall& X, int col) {
  // offset: column c of a sketch uses counters [c*count, (c+1)*count)
  BM_LAUNCH(h, "rng", k_counter_normal<<<grid1(count), 256, 0, h.stream>>>(seed, stream, (uint64_t)col * count,
                                                                          count, X.p, X.ld, col));
}

void negate_values_dev(bm_ctx& h, const float* a, float* out, int64_t count) {
  if (!count) return;
  BM_LAUNCH(h, "negate", k_negate<<<grid1(count), 256, 0, h.stream>>>(a, out, count));
}

void residual_sums_dev(bm_ctx& h, const float* r, const float* a, int64_t nnz, double out[2]) {
  const int nb = 304;
  double* part = h.sc.red.get();
  if (nnz == 0) {
    out[0] = out[1] = 0;
    return;
  }
  BM_LAUNCH(h, "res_sums", k_res_sums<<<nb, 256, 0, h.stream>>>(r, a, nnz, part));
  BM_LAUNCH(h, "res_sums", k_sum_pairs<<<1, 32, 0, h.stream>>>(part, nb, h.sc.scal.get() + 8));
  BM_CUDA(cudaMemcpyAsync(out, h.sc.scal.get() + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
}

void copy_cols_dev(bm_ctx& h, const Tall& src, int s0, const Tall& dst, int d0, int c) {
  if (c == 0 || src.rows == 0) return;
  BM_LAUNCH(h, "copy_cols", k_copy_cols<<<grid1(src.rows * c), 256, 0, h.stream>>>(src.p, src.ld, s0, dst.p, dst.ld,
                                                                                  d0, c, src.rows));
}

void zero_dev(bm_ctx& h, const Tall& X) {
  if (X.rows == 0) return;
  BM_CUDA(cudaMemsetAsync(X.p, 0, (size_t)X.rows * X.ld * sizeof(float), h.stream));
}

}  // namespace bm
