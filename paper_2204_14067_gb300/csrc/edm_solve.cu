// Algorithm 1 on the distance-geometry QSDP (Eq. "QSDP" with the factored
// problem Eq. "EDM"):
//
//   min  1/2 sum_{(i,j)} w_ij (X_ii + X_jj - 2 X_ij - d_ij^2)^2 + lambda <I, X>
//   s.t. X positive semidefinite, <E, X> = 0,      X = V V^T, V^T e = 0.
//
// BM phase: Polak-Ribiere+ directions on g(V) with the exact line search on
// the quartic g(V + s D) (every gradient and direction keeps V^T e = 0).
// PG step: by Lemma "PiX" and Eq. "proxsym", X+ = P_S+(Z) with
// Z = V V^T - alpha L_{w r} - alpha lambda J (J = I - e e^T / n,
// L_c = sum c_ij E_ij); the leading eigenpairs of Z come from LmSVD
// (Algorithm 2) on Z + sigma J, positive semidefinite and equal to Z + sigma I on ker(e^T); X+ keeps
// the positive eigenvalues, V+ = U diag(sqrt(mu_+)).  alpha = 1/L with the
// Gershgorin bound of ||A* A||; sigma the Gershgorin bound of the negative
// part of Z; the rank rule of the paper's QSDP experiments; the initial point
// is one PG step from X = 0.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "dense.cuh"
#include "edm.cuh"
#include "quartic.cuh"

namespace bm {

struct EdmSolveState {
  int qcap = 0;     // columns of one LmSVD block (k_max + 1)
  int ldq2 = 4;     // row stride of the n-side blocks (2 qcap, rounded up)
  DenseWork dw;
  DevBuf<float> blk[13];
  DevBuf<float> c;         // alpha w r per directed entry
  DevBuf<float> D, gp;     // BM direction, previous gradient (n x ld)
  DevBuf<double> G, E, ev, colsum;
  DevBuf<double> rowbuf, segsums, sums4;   // per-row bounds, line-search partials
  DevBuf<double> dotpart, scal;            // dot-product partials; 8 scalars read back per sync
  DevBuf<double> ctl;                      // BM-phase control scalars (device-resident)
  // the BM phase's iterations as one CUDA graph, re-captured when the row
  // stride, the iteration count or the stream changes
  cudaGraphExec_t bm_graph = nullptr;
  int graph_ld = -1, graph_epochs = -1;
  cudaStream_t graph_stream = nullptr;
  ~EdmSolveState() {
    if (bm_graph) cudaGraphExecDestroy(bm_graph);
  }
  DevBuf<float> Ts;
  double alpha = 0, sigma = 0;
  int ku = 0;              // columns of U_t in blk[kUp]
  int k_eig = 0;           // eigenpairs the next PG step computes
  int t = 0;
  bool initialized = false;
};

void edm_solve_destroy(EdmSolveState* s) { delete s; }

void edm_solve_reset(EdmSolveState* s) {
  if (!s) return;
  s->ku = 0;
  s->k_eig = 0;
  s->t = 0;
  s->initialized = false;
}

namespace {

enum { kB0 = 0, kB1, kB2, kQ, kZQ, kU, kZU, kX1, kX2, kX3, kX4, kW, kUp };
constexpr uint64_t kStreamEdmInit = 1;
constexpr uint64_t kStreamEdmFill = 2000;
constexpr unsigned kFullMask = 0xffffffffu;

// ---------------------------------------------------------------- kernels
struct PairArgs {
  const int32_t* seg_row;
  const int64_t* seg_beg;
  const int64_t* seg_end;
  const int32_t* seg_slot;
  int64_t nseg;
  const int32_t* col;
  const float* coef;       // per directed entry
  const float* U;          // gathered / owned block
  const float* D;          // second block (line search)
  const float* dsq;
  const float* w;
  int ld, nchunk;
  float gamma;
  float* out;
  int ld_out;
  float* partial;
  double* sums;            // line search: 4 per segment
};

// out_i += gamma * sum_{e in row i} coef_e (u_i - u_j); rows over several
// segments write partial rows, combined in entry order by the fix-up.
template <int VC>
__global__ void __launch_bounds__(256) k_pair_lap(PairArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nseg; s += nwarps) {
    const int i = a.seg_row[s];
    const int64_t beg = a.seg_beg[s], end = a.seg_end[s];
    float4 ui[VC], acc[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
      const int c = l + 4 * v;
      ui[v] = c < a.nchunk ? __ldg(reinterpret_cast<const float4*>(a.U + (int64_t)i * a.ld) + c)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < end;
      const int j = valid ? __ldg(a.col + e) : 0;
      const float cf = valid ? __ldg(a.coef + e) : 0.f;
#pragma unroll 2
      for (int t = 0; t < 4; ++t) {
        const int src = t * 8 + g;
        const int jj = __shfl_sync(kFullMask, j, src);
        const float cc = __shfl_sync(kFullMask, cf, src);
#pragma unroll
        for (int v = 0; v < VC; ++v) {
          const int c = l + 4 * v;
          if (c < a.nchunk) {
            const float4 uj = __ldg(reinterpret_cast<const float4*>(a.U + (int64_t)jj * a.ld) + c);
            acc[v].x = fmaf(cc, ui[v].x - uj.x, acc[v].x);
            acc[v].y = fmaf(cc, ui[v].y - uj.y, acc[v].y);
            acc[v].z = fmaf(cc, ui[v].z - uj.z, acc[v].z);
            acc[v].w = fmaf(cc, ui[v].w - uj.w, acc[v].w);
          }
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VC; ++v) {
#pragma unroll
      for (int m = 4; m < 32; m <<= 1) {
        acc[v].x += __shfl_xor_sync(kFullMask, acc[v].x, m);
        acc[v].y += __shfl_xor_sync(kFullMask, acc[v].y, m);
        acc[v].z += __shfl_xor_sync(kFullMask, acc[v].z, m);
        acc[v].w += __shfl_xor_sync(kFullMask, acc[v].w, m);
      }
    }
    if (g == 0) {
      const int slot = a.seg_slot[s];
#pragma unroll
      for (int v = 0; v < VC; ++v) {
        const int c = l + 4 * v;
        if (c >= a.nchunk) continue;
        if (slot < 0) {
          float4* op = reinterpret_cast<float4*>(a.out + (int64_t)i * a.ld_out) + c;
          float4 o = *op;
          o.x = fmaf(a.gamma, acc[v].x, o.x);
          o.y = fmaf(a.gamma, acc[v].y, o.y);
          o.z = fmaf(a.gamma, acc[v].z, o.z);
          o.w = fmaf(a.gamma, acc[v].w, o.w);
          *op = o;
        } else {
          reinterpret_cast<float4*>(a.partial + (int64_t)slot * 4 * a.nchunk)[c] = acc[v];
        }
      }
    }
  }
}

__global__ void k_pair_lap_fixup(const int32_t* __restrict__ mrow, const int32_t* __restrict__ mfirst,
                                 const int32_t* __restrict__ mcount, int64_t nmulti, const float* __restrict__ partial,
                                 int ldp, int cols, float gamma, float* __restrict__ out, int ldo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nmulti * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t / cols;
    const int c = (int)(t - q * cols);
    float s = 0.f;
    for (int u = 0; u < mcount[q]; ++u) s += partial[((int64_t)mfirst[q] + u) * ldp + c];
    float* o = out + (int64_t)mrow[q] * ldo + c;
    *o = fmaf(gamma, s, *o);
  }
}

// Line-search sums per segment over directed entries (each pair twice):
// a = 2 <v_i - v_j, d_i - d_j>, b = ||d_i - d_j||^2, r = ||v_i - v_j||^2 - d^2;
// sums[4s..4s+3] = (sum w r a, sum w (a^2 + 2 r b), sum w a b, sum w b^2).
template <int VC>
__global__ void __launch_bounds__(256) k_pair_ls(PairArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nseg; s += nwarps) {
    const int i = a.seg_row[s];
    const int64_t beg = a.seg_beg[s], end = a.seg_end[s];
    float4 vi[VC], di[VC];
#pragma unroll
    for (int v = 0; v < VC; ++v) {
      const int c = l + 4 * v;
      const bool in = c < a.nchunk;
      vi[v] = in ? __ldg(reinterpret_cast<const float4*>(a.U + (int64_t)i * a.ld) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      di[v] = in ? __ldg(reinterpret_cast<const float4*>(a.D + (int64_t)i * a.ld) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < end;
      const int j = valid ? __ldg(a.col + e) : 0;
      const float dq = valid ? __ldg(a.dsq + e) : 0.f;
      const float wv = valid ? __ldg(a.w + e) : 0.f;
#pragma unroll 2
      for (int t = 0; t < 4; ++t) {
        const int src = t * 8 + g;
        const int jj = __shfl_sync(kFullMask, j, src);
        const float dd = __shfl_sync(kFullMask, dq, src);
        const float ww = __shfl_sync(kFullMask, wv, src);
        const bool ok = e0 + src < end;
        float sq = 0.f, av = 0.f, bv = 0.f;
#pragma unroll
        for (int v = 0; v < VC; ++v) {
          const int c = l + 4 * v;
          if (c < a.nchunk) {
            const float4 vj = __ldg(reinterpret_cast<const float4*>(a.U + (int64_t)jj * a.ld) + c);
            const float4 dj = __ldg(reinterpret_cast<const float4*>(a.D + (int64_t)jj * a.ld) + c);
            const float4 x = make_float4(vi[v].x - vj.x, vi[v].y - vj.y, vi[v].z - vj.z, vi[v].w - vj.w);
            const float4 y = make_float4(di[v].x - dj.x, di[v].y - dj.y, di[v].z - dj.z, di[v].w - dj.w);
            sq = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, sq))));
            av = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, av))));
            bv = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, bv))));
          }
        }
#pragma unroll
        for (int m = 1; m < 4; m <<= 1) {
          sq += __shfl_xor_sync(kFullMask, sq, m);
          av += __shfl_xor_sync(kFullMask, av, m);
          bv += __shfl_xor_sync(kFullMask, bv, m);
        }
        if (ok && l == 0) {
          const float r = sq - dd, A = 2.f * av;
          s1 = fmaf(ww * r, A, s1);
          s2 = fmaf(ww, fmaf(A, A, 2.f * r * bv), s2);
          s3 = fmaf(ww * A, bv, s3);
          s4 = fmaf(ww * bv, bv, s4);
        }
      }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      s1 += __shfl_xor_sync(kFullMask, s1, m);
      s2 += __shfl_xor_sync(kFullMask, s2, m);
      s3 += __shfl_xor_sync(kFullMask, s3, m);
      s4 += __shfl_xor_sync(kFullMask, s4, m);
    }
    if (lane == 0) {
      a.sums[4 * s + 0] = s1;
      a.sums[4 * s + 1] = s2;
      a.sums[4 * s + 2] = s3;
      a.sums[4 * s + 3] = s4;
    }
  }
}

// out[q] = sum over segments of sums[4 s + q], two deterministic stages:
// block b adds a fixed strided share into part[4 b + q], one block adds the parts.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_sum4_part(const double* __restrict__ sums, int64_t nseg,
                                                          double* __restrict__ part) {
  __shared__ double sh[4][kSumThreads];
  double acc[4] = {0, 0, 0, 0};
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x)
    for (int q = 0; q < 4; ++q) acc[q] += sums[4 * s + q];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// part[2 b + q] = sum over a fixed strided share of x_q . y_q (q = 0, 1; float4 chunks)
__global__ void __launch_bounds__(kSumThreads) k_dots2_part(const float4* __restrict__ x0,
                                                           const float4* __restrict__ y0,
                                                           const float4* __restrict__ x1,
                                                           const float4* __restrict__ y1, int64_t n4,
                                                           double* __restrict__ part) {
  __shared__ double sh[2][kSumThreads];
  float a0 = 0.f, a1 = 0.f;   // a thread sums only a few chunks; FP64 across threads
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 u = x0[i], v = y0[i], p = x1[i], q = y1[i];
    a0 = fmaf(u.x, v.x, fmaf(u.y, v.y, fmaf(u.z, v.z, fmaf(u.w, v.w, a0))));
    a1 = fmaf(p.x, q.x, fmaf(p.y, q.y, fmaf(p.z, q.z, fmaf(p.w, q.w, a1))));
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) part[2 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kSumThreads) k_dots2_final(const double* __restrict__ part, int parts,
                                                            double* __restrict__ out) {
  __shared__ double sh[2][kSumThreads];
  double a0 = 0.0, a1 = 0.0;
  for (int i = threadIdx.x; i < parts; i += blockDim.x) {
    a0 += part[2 * i];
    a1 += part[2 * i + 1];
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) out[threadIdx.x] = sh[threadIdx.x][0];
}

// BM-phase control scalars, kept on the device (slots of EdmSolveState::ctl)
enum { kCF = 0, kCBeta, kCGGPrev, kCFirst, kCStep, kCFLast, kCGG, kCGP, kCDoG, kCGD, kCDD, kCS1, kCS2, kCS3,
       kCS4, kCBad, kCtlSlots };

__global__ void k_edm_ctrl_init(double* __restrict__ ctl) {
  for (int i = threadIdx.x; i < kCtlSlots; i += blockDim.x) ctl[i] = i == kCFirst ? 1.0 : 0.0;
}

// F of the current factor, and beta of Polak-Ribiere+ with the restart rule:
// beta = 0 when <-g + beta D_prev, g> >= 0 (not a descent direction)
__global__ void k_edm_ctrl_dir(double* __restrict__ ctl, const double* __restrict__ F) {
  const double f = F[0], gg = ctl[kCGG], gp = ctl[kCGP], dog = ctl[kCDoG];
  double beta = 0.0;
  if (ctl[kCFirst] == 0.0 && ctl[kCGGPrev] > 0) {
    beta = fmax(0.0, (gg - gp) / ctl[kCGGPrev]);
    if (beta > 0 && -gg + beta * dog >= 0) beta = 0.0;
  }
  if (!isfinite(f)) ctl[kCBad] = 1.0;
  ctl[kCF] = f;
  ctl[kCBeta] = beta;
  ctl[kCGGPrev] = gg;
  ctl[kCFirst] = 0.0;
}

// step = argmin over s >= 0 of g(V + s D) (each pair twice among the directed entries)
__global__ void k_edm_ctrl_step(double* __restrict__ ctl, double lam) {
  double c[5];
  c[0] = ctl[kCF];
  c[1] = ctl[kCGD];
  c[2] = 0.25 * ctl[kCS2] + lam * ctl[kCDD];
  c[3] = 0.5 * ctl[kCS3];
  c[4] = 0.25 * ctl[kCS4];
  const double st = quartic_argmin_d(c);
  ctl[kCStep] = st;
  ctl[kCFLast] = st > 0 ? poly4d(c, st) : c[0];
  if (!isfinite(ctl[kCFLast])) ctl[kCBad] = 1.0;
}

// D = -g + beta D (D not read when beta = 0: it may hold no direction yet)
__global__ void k_edm_dir(float4* __restrict__ D, const float4* __restrict__ g, int64_t n4,
                          const double* __restrict__ ctl) {
  const float beta = (float)ctl[kCBeta];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 gv = g[i];
    float4 v = beta != 0.f ? D[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    v.x = fmaf(beta, v.x, -gv.x);
    v.y = fmaf(beta, v.y, -gv.y);
    v.z = fmaf(beta, v.z, -gv.z);
    v.w = fmaf(beta, v.w, -gv.w);
    D[i] = v;
  }
}

// V += step D; g_prev = g
__global__ void k_edm_update(float4* __restrict__ V, const float4* __restrict__ D, const float4* __restrict__ g,
                             float4* __restrict__ gp, int64_t n4, const double* __restrict__ ctl) {
  const float st = (float)ctl[kCStep];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    if (st > 0.f) {
      const float4 d = D[i];
      float4 x = V[i];
      x.x = fmaf(st, d.x, x.x);
      x.y = fmaf(st, d.y, x.y);
      x.z = fmaf(st, d.z, x.z);
      x.w = fmaf(st, d.w, x.w);
      V[i] = x;
    }
    gp[i] = g[i];
  }
}

// coef_e = alpha w_e r_e (r_e of the directed entry; r_e = -d_e^2 when V = 0)
__global__ void k_pair_coef(const float* __restrict__ r, const float* __restrict__ dsq, const float* __restrict__ w,
                            int64_t E, float alpha, float* __restrict__ coef) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
    coef[e] = alpha * w[e] * (r ? r[e] : -dsq[e]);
}

// |coef| row sums (Gershgorin) and sqrt(w) row sums (Lipschitz bound)
__global__ void k_row_abs(const int64_t* __restrict__ row_ptr, const float* __restrict__ v, int64_t n, int sqrt_mode,
                          double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += sqrt_mode ? sqrt((double)v[e]) : fabs((double)v[e]);
    out[i] = s;
  }
}

// column sums of a block (one block per column, fixed order)
__global__ void k_col_sums(const float* __restrict__ U, int64_t n, int ld, double* __restrict__ out) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += U[i * ld + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// out(:, c) = a_out * out(:, c) + a * U(:, c) + b * colsum(c) / n
// (out may be U itself: no __restrict__ on either)
__global__ void k_cols_combine(float* out, int ldo, const float* U, int ldu, int64_t n,
                               int cols, float a_out, float a, const double* __restrict__ colsum, double b_over_n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * cols; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols;
    const int c = (int)(t - i * cols);
    const float mean_term = colsum ? (float)(b_over_n * colsum[c]) : 0.f;
    out[i * ldo + c] = fmaf(a_out, out[i * ldo + c], fmaf(a, U[i * ldu + c], mean_term));
  }
}

int sum_parts() { return std::max(1, std::min(1024, 2 * num_sms())); }

int grid_n(int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(work, 1), 256), (int64_t)num_sms() * 16));
}

// ---------------------------------------------------------------- helpers
bm_ctx& core(bm_edm_ctx& h) {
  h.core.stream = h.stream;
  return h.core;
}
Tall nb(bm_edm_ctx& h, int which, int cols) { return Tall{h.ss->blk[which].get(), h.n, cols, h.ss->ldq2}; }
Tall Vv(bm_edm_ctx& h) { return Tall{h.V.get(), h.n, h.k, h.ld}; }

std::vector<double> d2h(bm_edm_ctx& h, const double* d, size_t n) {
  std::vector<double> v(n);
  if (n) {
    BM_CUDA(cudaMemcpyAsync(v.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
  }
  return v;
}

// column means removed: U -= 1 mean(U)^T (keeps blocks in ker(e^T) against rounding drift)
void center_block(bm_edm_ctx& h, const Tall& U) {
  if (U.cols == 0) return;
  EdmSolveState& s = *h.ss;
  BM_LAUNCH(core(h), "edm_colsum", k_col_sums<<<U.cols, 256, 0, h.stream>>>(U.p, U.rows, U.ld, s.colsum.get()));
  BM_LAUNCH(core(h), "edm_center", k_cols_combine<<<grid_n(U.rows * U.cols), 256, 0, h.stream>>>(
                                       U.p, U.ld, U.p, U.ld, U.rows, U.cols, 0.f, 1.f, s.colsum.get(),
                                       -1.0 / (double)U.rows));
}

// out += gamma * L_coef U  (U, out n-side blocks, at most 128 columns per launch)
void pair_lap(bm_edm_ctx& h, const Tall& U, const Tall& out, float gamma) {
  EdmSolveState& s = *h.ss;
  for (int c0 = 0; c0 < U.cols; c0 += 128) {
    const int cols = std::min(128, U.cols - c0);
    PairArgs a{};
    a.seg_row = h.seg.row.get();
    a.seg_beg = h.seg.beg.get();
    a.seg_end = h.seg.end.get();
    a.seg_slot = h.seg.slot.get();
    a.nseg = h.seg.nseg;
    a.col = h.col.get();
    a.coef = s.c.get();
    a.U = U.p + c0;
    a.ld = U.ld;
    a.nchunk = (cols + 3) / 4;
    a.gamma = gamma;
    a.out = out.p + c0;
    a.ld_out = out.ld;
    a.partial = h.partial.get();
    BM_REQUIRE((int64_t)std::max<int64_t>(1, h.seg.nslots) * 4 * a.nchunk <= (int64_t)h.partial.n, BM_ERR_INVALID,
               "distance-geometry SpMM: partial buffer too small");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(a.nseg, 8), (int64_t)num_sms() * 16));
    const int VC = (a.nchunk + 3) / 4;
    switch (VC) {
      case 1: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<1><<<grid, 256, 0, h.stream>>>(a)); break;
      case 2: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<2><<<grid, 256, 0, h.stream>>>(a)); break;
      case 3: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<3><<<grid, 256, 0, h.stream>>>(a)); break;
      case 4: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<4><<<grid, 256, 0, h.stream>>>(a)); break;
      case 5: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<5><<<grid, 256, 0, h.stream>>>(a)); break;
      case 6: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<6><<<grid, 256, 0, h.stream>>>(a)); break;
      case 7: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<7><<<grid, 256, 0, h.stream>>>(a)); break;
      default: BM_LAUNCH(core(h), "edm_lap", k_pair_lap<8><<<grid, 256, 0, h.stream>>>(a)); break;
    }
    if (h.seg.nmulti) {
      BM_LAUNCH(core(h), "edm_lap_fixup",
                k_pair_lap_fixup<<<grid_n(h.seg.nmulti * cols), 256, 0, h.stream>>>(
                    h.seg.mrow.get(), h.seg.mfirst.get(), h.seg.mcount.get(), h.seg.nmulti, h.partial.get(),
                    4 * a.nchunk, cols, gamma, out.p + c0, out.ld));
    }
  }
}

// out = (Z + sigma J) U = V (V^T U) - L_c U + (sigma - alpha lam) J U.  On ker(e^T), where every
// LmSVD block lies, this is Z + sigma I; on e it is 0 rather than sigma, so the rounding error
// along e that each product leaves is damped instead of growing into the leading Ritz vectors.
void zs_apply(bm_edm_ctx& h, const Tall& U, const Tall& out) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  if (h.k > 0) {
    gram_dev(cx, s.dw, Vv(h), U, s.G.get(), false, "edm_gram_VtU");
    small_to_f32_dev(cx, s.G.get(), h.k, U.cols, U.cols, s.Ts.get(), s.ldq2);
    gemm_dev(cx, Vv(h), s.Ts.get(), s.ldq2, out, 0.f, 1.f, "edm_gemm_V");
  } else {
    zero_dev(cx, out);
  }
  pair_lap(h, U, out, -1.f);
  const double sh = s.sigma - s.alpha * h.lambda;
  BM_LAUNCH(cx, "edm_colsum", k_col_sums<<<U.cols, 256, 0, h.stream>>>(U.p, U.rows, U.ld, s.colsum.get()));
  BM_LAUNCH(cx, "edm_shift", k_cols_combine<<<grid_n(U.rows * U.cols), 256, 0, h.stream>>>(
                                 out.p, out.ld, U.p, U.ld, U.rows, U.cols, 1.f, (float)sh, s.colsum.get(),
                                 -sh / (double)U.rows));
}

// Orthonormal new columns for ran([F, M]) (Eq. "PUi"/"orth-W"), two passes,
// written to blk[out] at column out_col; returns the count.  M and F must not
// be the work blocks X1..X4.
int edm_orth(bm_edm_ctx& h, const Tall& M, const Tall* F, double tau, int max_cols, int out, int out_col) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  const int c = M.cols;
  if (c == 0) return 0;
  gram_dev(cx, s.dw, M, M, s.G.get(), true, "edm_gram_orth");
  std::vector<double> G0 = d2h(h, s.G.get(), (size_t)c * c);
  std::vector<int> sel;
  std::vector<double> sc;
  for (int j = 0; j < c; ++j) {
    const double dg = G0[(size_t)j * c + j];
    if (dg > 0 && std::isfinite(dg)) sel.push_back(j), sc.push_back(1.0 / std::sqrt(dg));
  }
  int c1 = (int)sel.size();
  if (c1 == 0) return 0;
  {
    std::vector<double> I((size_t)c * c, 0.0);
    for (int j = 0; j < c; ++j) I[(size_t)j * c + j] = 1.0;
    BM_CUDA(cudaMemcpyAsync(s.E.get(), I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, h.stream));
    select_scale_dev(cx, s.E.get(), c, c, sel.data(), sc.data(), c1, s.Ts.get(), s.ldq2);
  }
  int a = kX1, b = kX2;
  gemm_dev(cx, M, s.Ts.get(), s.ldq2, nb(h, a, c1), 0.f, 1.f, "edm_gemm_orth");
  const bool useF = F && F->cols > 0;
  for (int pass = 0; pass < 2; ++pass) {
    Tall Mh = nb(h, a, c1);
    if (useF) {
      gram_dev(cx, s.dw, *F, Mh, s.G.get(), true, "edm_gram_orth");
      small_to_f32_dev(cx, s.G.get(), F->cols, c1, c1, s.Ts.get(), s.ldq2);
      gemm_dev(cx, *F, s.Ts.get(), s.ldq2, Mh, 1.f, -1.f, "edm_gemm_orth");
    }
    gram_dev(cx, s.dw, Mh, Mh, s.G.get(), true, "edm_gram_orth");
    int c2 = c1;
    bool chol = false;
    if (pass == 0 && (max_cols < 0 || max_cols >= c1)) {
      double f = 0.0;
      chol = chol_inv_try_dev(cx, s.dw, s.G.get(), c1, s.Ts.get(), s.ldq2, &f) && f > 0 &&
             1.0 / f >= std::max(1e-2, 10.0 * tau);
    }
    if (chol) {
      // Ts = R^{-1}
    } else if (pass == 0) {
      sym_eig_dev(cx, s.dw, s.G.get(), c1, s.ev.get(), s.E.get(), kEigFast);
      std::vector<double> lam = d2h(h, s.ev.get(), c1);
      std::vector<int> keep;
      std::vector<double> sv;
      for (int j = 0; j < c1; ++j) {
        if (!(lam[j] > tau)) break;
        if (max_cols >= 0 && j >= max_cols) break;
        keep.push_back(j);
        sv.push_back(1.0 / std::sqrt(lam[j]));
      }
      c2 = (int)keep.size();
      if (c2 == 0) return 0;
      select_scale_dev(cx, s.E.get(), c1, c1, keep.data(), sv.data(), c2, s.Ts.get(), s.ldq2);
    } else {
      chol_inv_dev(cx, s.dw, s.G.get(), c1, s.Ts.get(), s.ldq2);
    }
    gemm_dev(cx, Mh, s.Ts.get(), s.ldq2, nb(h, b, c2), 0.f, 1.f, "edm_gemm_orth");
    std::swap(a, b);
    c1 = c2;
  }
  copy_cols_dev(cx, nb(h, a, c1), 0, nb(h, out, out_col + c1), out_col, c1);
  return c1;
}

struct EigOut {
  int cols = 0;
  int iters = 0;
  std::vector<double> mu;   // eigenvalues of Z (theta - sigma), descending
};

// LmSVD (Algorithm 2) on Z + sigma J (= Z + sigma I on ker(e^T)) from the warm start blk[kW] (c0 columns):
// Ritz vectors in blk[kU], at most kmax of them.
EigOut edm_lmsvd(bm_edm_ctx& h, int c0, int kmax) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  const bm_options& o = h.opt;
  EigOut r;
  int B[3] = {kB0, kB1, kB2};
  int kc[3] = {0, 0, 0};
  const int k0 = edm_orth(h, nb(h, kW, c0), nullptr, o.tau, -1, B[0], 0);
  if (k0 == 0) return r;
  kc[0] = k0;
  int nbk = 1;
  const int k = std::min(k0, kmax);
  std::vector<double> theta_prev;
  for (int it = 1; it <= o.lmsvd_imax; ++it) {
    r.iters = it;
    int q = kc[0];
    Tall Q = nb(h, B[0], kc[0]);
    if (nbk > 1) {
      copy_cols_dev(cx, nb(h, B[0], kc[0]), 0, nb(h, kQ, kc[0]), 0, kc[0]);
      Tall F = nb(h, B[0], kc[0]);
      const int c2 = edm_orth(h, nb(h, B[1], kc[1]), &F, o.tau, -1, kQ, kc[0]);
      q = kc[0] + c2;
      Q = nb(h, kQ, q);
    }
    const Tall ZQ = nb(h, kZQ, q);
    zs_apply(h, Q, ZQ);
    gram_dev(cx, s.dw, Q, ZQ, s.G.get(), true, "edm_gram_rr");      // Q^T (Z + sigma J) Q
    sym_eig_dev(cx, s.dw, s.G.get(), q, s.ev.get(), s.E.get(), kEigRelative);
    std::vector<double> th = d2h(h, s.ev.get(), q);
    const int kk = std::min(k, q);
    std::vector<int> sel(kk);
    std::vector<double> one(kk, 1.0);
    for (int j = 0; j < kk; ++j) sel[j] = j;
    select_scale_dev(cx, s.E.get(), q, q, sel.data(), one.data(), kk, s.Ts.get(), s.ldq2);
    gemm_dev(cx, Q, s.Ts.get(), s.ldq2, nb(h, kU, kk), 0.f, 1.f, "edm_gemm_rr");
    gemm_dev(cx, ZQ, s.Ts.get(), s.ldq2, nb(h, kZU, kk), 0.f, 1.f, "edm_gemm_rr");
    th.resize(kk);
    r.cols = kk;
    r.mu.assign(th.begin(), th.end());
    bool conv = false;
    if (it >= o.lmsvd_min_iter && theta_prev.size() == th.size() && kk > 0) {
      double md = 0;
      for (int j = 0; j < kk; ++j) md = std::max(md, std::fabs(th[j] - theta_prev[j]));
      conv = md <= o.lmsvd_tol * std::max(th[0], 1e-300);
    }
    if (conv || it == o.lmsvd_imax) break;
    theta_prev = th;
    const int fb = B[2];
    const int cn = edm_orth(h, nb(h, kZU, kk), nullptr, o.tau, -1, fb, 0);
    if (cn == 0) break;
    B[2] = B[1];
    B[1] = B[0];
    kc[1] = kc[0];
    B[0] = fb;
    kc[0] = cn;
    nbk = std::min(nbk + 1, o.lmsvd_p + 1);
  }
  for (auto& m : r.mu) m -= s.sigma;
  return r;
}

// coefficients alpha w r of the current factor (r = -d^2 when V = 0) and the shift sigma
void prepare_z(bm_edm_ctx& h) {
  EdmSolveState& s = *h.ss;
  const int64_t E = 2 * h.npairs;
  const float* r = nullptr;
  if (h.k > 0) {
    edm_loss_grad_dev(h, false, s.c.get());   // residual per directed entry, into c
    r = s.c.get();
  }
  if (E) {
    BM_LAUNCH(core(h), "edm_coef", k_pair_coef<<<grid_n(E), 256, 0, h.stream>>>(r, h.dsq.get(), h.w.get(), E,
                                                                                 (float)s.alpha, s.c.get()));
  }
  BM_LAUNCH(core(h), "edm_rowabs", k_row_abs<<<grid_n(h.n), 256, 0, h.stream>>>(h.row_ptr.get(), s.c.get(), h.n, 0,
                                                                                 s.rowbuf.get()));
  std::vector<double> rs = d2h(h, s.rowbuf.get(), (size_t)h.n);
  double mx = 0.0;
  for (double v : rs) mx = std::max(mx, v);
  s.sigma = 2.0 * mx + s.alpha * std::max(h.lambda, 0.0);
}

// V = U diag(sqrt(mu_+)) over the positive mu; rank rule for the next step
int refactor(bm_edm_ctx& h, const EigOut& eg, int k_eig) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  int rank = 0;
  while (rank < eg.cols && eg.mu[rank] > 0) ++rank;
  rank = std::min(rank, h.k_max);
  h.k = rank;
  h.ld = std::max(4, round_up4(rank));
  BM_CUDA(cudaMemsetAsync(h.V.get(), 0, (size_t)h.n * h.ld * sizeof(float), h.stream));
  if (rank > 0) {
    std::vector<double> I((size_t)eg.cols * eg.cols, 0.0);
    for (int j = 0; j < eg.cols; ++j) I[(size_t)j * eg.cols + j] = 1.0;
    BM_CUDA(cudaMemcpyAsync(s.E.get(), I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, h.stream));
    std::vector<int> sel(rank);
    std::vector<double> sq(rank);
    for (int j = 0; j < rank; ++j) sel[j] = j, sq[j] = std::sqrt(eg.mu[j]);
    select_scale_dev(cx, s.E.get(), eg.cols, eg.cols, sel.data(), sq.data(), rank, s.Ts.get(), s.ldq2);
    gemm_dev(cx, nb(h, kU, eg.cols), s.Ts.get(), s.ldq2, Vv(h), 0.f, 1.f, "edm_gemm_Vnew");
    center_block(h, Vv(h));   // V^T e = 0 against rounding
  }
  // U_t for the next warm start
  copy_cols_dev(cx, nb(h, kU, eg.cols), 0, nb(h, kUp, eg.cols), 0, eg.cols);
  s.ku = eg.cols;
  const bool all_pos = rank == eg.cols;
  return all_pos ? std::min(h.k_max, k_eig + (int)(h.n / 20)) : std::max(1, rank);
}

void ensure_state(bm_edm_ctx& h) {
  if (h.ss) return;
  EdmSolveState* s = new EdmSolveState();
  h.ss = s;
  s->qcap = h.k_max + 1;
  s->ldq2 = round_up4(2 * s->qcap);
  for (auto& b : s->blk) b.alloc((size_t)h.n * s->ldq2);
  s->D.alloc((size_t)h.n * round_up4(h.k_max));
  s->gp.alloc((size_t)h.n * round_up4(h.k_max));
  const size_t q2 = (size_t)2 * s->qcap;
  s->G.alloc(q2 * q2);
  s->E.alloc(q2 * q2);
  s->ev.alloc(q2);
  s->colsum.alloc(q2);
  s->Ts.alloc(q2 * s->ldq2);
  s->c.alloc(std::max<int64_t>(2 * h.npairs, 1));
  s->rowbuf.alloc(std::max<int64_t>(h.n, 1));
  s->segsums.alloc(4 * std::max<int64_t>(1, h.seg.nseg));
  s->sums4.alloc(4 * (sum_parts() + 1));
  s->dotpart.alloc(2 * (size_t)sum_parts());
  s->scal.alloc(8);
  s->ctl.alloc(32);
  // SpMM partial rows up to 128 columns
  const int64_t need = std::max<int64_t>(1, h.seg.nslots) * 128;
  if ((int64_t)h.partial.n < need) {
    h.partial.release();
    h.partial.alloc(need);
  }
  // Lipschitz bound of ||A* A|| (Gershgorin): max_p 4 w_p + sqrt(w_p) (S_i + S_j - 2 sqrt(w_p))
  BM_LAUNCH(core(h), "edm_sqrtw", k_row_abs<<<grid_n(h.n), 256, 0, h.stream>>>(h.row_ptr.get(), h.w.get(), h.n, 1,
                                                                                s->rowbuf.get()));
  std::vector<double> S = d2h(h, s->rowbuf.get(), (size_t)h.n);
  std::vector<int64_t> rp(h.n + 1);
  std::vector<int32_t> col(std::max<int64_t>(2 * h.npairs, 1));
  std::vector<float> w(std::max<int64_t>(2 * h.npairs, 1));
  BM_CUDA(cudaMemcpyAsync(rp.data(), h.row_ptr.get(), (h.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, h.stream));
  if (h.npairs) {
    BM_CUDA(cudaMemcpyAsync(col.data(), h.col.get(), 2 * h.npairs * sizeof(int32_t), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaMemcpyAsync(w.data(), h.w.get(), 2 * h.npairs * sizeof(float), cudaMemcpyDeviceToHost, h.stream));
  }
  BM_CUDA(cudaStreamSynchronize(h.stream));
  double L = 0.0;
  for (int64_t i = 0; i < h.n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const double sw = std::sqrt((double)w[e]);
      L = std::max(L, 4.0 * w[e] + sw * (S[i] + S[col[e]] - 2.0 * sw));
    }
  s->alpha = L > 0 ? 1.0 / L : 1.0;
}

// warm start: orth([U_t, V]) up to k columns, completed with Gaussian columns
int warm_start(bm_edm_ctx& h, int k, uint64_t stream) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  int c = 0;
  const int mcols = s.ku + h.k;
  if (mcols > 0) {
    Tall M = nb(h, kZQ, mcols);
    copy_cols_dev(cx, nb(h, kUp, s.ku), 0, M, 0, s.ku);
    copy_cols_dev(cx, Vv(h), 0, M, s.ku, h.k);
    center_block(h, M);
    c = edm_orth(h, M, nullptr, h.opt.tau, k, kW, 0);
  }
  if (c < k) {
    const int extra = k - c;
    Tall Gm = nb(h, kZU, extra);
    zero_dev(cx, Gm);
    for (int e = 0; e < extra; ++e) counter_normal_dev(cx, h.opt.seed, stream, h.n, Gm, e);
    center_block(h, Gm);
    Tall F = nb(h, kW, c);
    c += edm_orth(h, Gm, c > 0 ? &F : nullptr, h.opt.tau, -1, kW, c);
  }
  return c;
}

struct EdmStepOut {
  int rank, computed, iters, k_next;
  double F;
};

EdmStepOut prox_step(bm_edm_ctx& h) {
  EdmSolveState& s = *h.ss;
  prepare_z(h);
  const int c0 = warm_start(h, s.k_eig, kStreamEdmFill + (uint64_t)s.t);
  EigOut eg = edm_lmsvd(h, c0, s.k_eig);
  const int k_next = refactor(h, eg, s.k_eig);
  EdmStepOut o{h.k, eg.cols, eg.iters, k_next, 0.0};
  s.k_eig = k_next;
  s.t += 1;
  o.F = edm_loss_grad_dev(h, false, nullptr);
  return o;
}

EdmStepOut init_step(bm_edm_ctx& h) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  h.k = 0;
  h.ld = 4;
  s.ku = 0;
  s.t = 0;
  prepare_z(h);
  const int k0 = std::max(1, std::min({100, (int)(0.15 * (double)h.n), h.k_max}));
  Tall Gm = nb(h, kW, k0);
  zero_dev(cx, Gm);
  for (int e = 0; e < k0; ++e) counter_normal_dev(cx, h.opt.seed, kStreamEdmInit, h.n, Gm, e);
  center_block(h, Gm);
  EigOut eg = edm_lmsvd(h, k0, k0);
  const int k_next = refactor(h, eg, k0);
  s.k_eig = k_next;
  s.initialized = true;
  EdmStepOut o{h.k, eg.cols, eg.iters, k_next, 0.0};
  o.F = edm_loss_grad_dev(h, false, nullptr);
  return o;
}

// launch (x0 . y0, x1 . y1) over the n x ld factor layout into out[0..1] (device); no synchronisation
void dots2(bm_edm_ctx& h, const float* x0, const float* y0, const float* x1, const float* y1, double* out) {
  EdmSolveState& s = *h.ss;
  const int parts = sum_parts();
  const int64_t n4 = h.n * (int64_t)h.ld / 4;
  BM_LAUNCH(core(h), "edm_dots", k_dots2_part<<<parts, kSumThreads, 0, h.stream>>>(
                                     reinterpret_cast<const float4*>(x0), reinterpret_cast<const float4*>(y0),
                                     reinterpret_cast<const float4*>(x1), reinterpret_cast<const float4*>(y1), n4,
                                     s.dotpart.get()));
  BM_LAUNCH(core(h), "edm_dots", k_dots2_final<<<1, kSumThreads, 0, h.stream>>>(s.dotpart.get(), parts, out));
}

// Polak-Ribiere+ with the exact quartic line search; returns F after the last iteration
// Launch the BM phase's `epochs` iterations: every decision (beta, restart,
// step) is taken on the device, so they run back to back without host round
// trips (and can be captured as one graph).
void bm_phase_launch(bm_edm_ctx& h, int epochs) {
  EdmSolveState& s = *h.ss;
  bm_ctx& cx = core(h);
  const int64_t cnt = h.n * (int64_t)h.ld, n4 = cnt / 4;
  double* ctl = s.ctl.get();
  BM_LAUNCH(cx, "edm_ctrl", k_edm_ctrl_init<<<1, 32, 0, h.stream>>>(ctl));
  PairArgs a{};
  a.seg_row = h.seg.row.get();
  a.seg_beg = h.seg.beg.get();
  a.seg_end = h.seg.end.get();
  a.seg_slot = h.seg.slot.get();
  a.nseg = h.seg.nseg;
  a.col = h.col.get();
  a.U = h.V.get();
  a.D = s.D.get();
  a.dsq = h.dsq.get();
  a.w = h.w.get();
  a.ld = h.ld;
  a.nchunk = h.ld / 4;
  a.sums = s.segsums.get();
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(a.nseg, 8), (int64_t)num_sms() * 16));
  const int parts = sum_parts();
  float4* V4 = reinterpret_cast<float4*>(h.V.get());
  float4* D4 = reinterpret_cast<float4*>(s.D.get());
  float4* g4 = reinterpret_cast<float4*>(h.gV.get());
  float4* gp4 = reinterpret_cast<float4*>(s.gp.get());
  for (int e = 0; e < epochs; ++e) {
    edm_loss_grad_dev(h, true, nullptr, false);                      // g(V) into h.red[0], gradient
    dots2(h, h.gV.get(), h.gV.get(), h.gV.get(), e > 0 ? s.gp.get() : h.gV.get(), ctl + kCGG);
    if (e > 0) dots2(h, s.D.get(), h.gV.get(), s.D.get(), s.D.get(), ctl + kCDoG);
    BM_LAUNCH(cx, "edm_ctrl", k_edm_ctrl_dir<<<1, 1, 0, h.stream>>>(ctl, h.red.get()));
    BM_LAUNCH(cx, "edm_dir", k_edm_dir<<<grid_n(n4), 256, 0, h.stream>>>(D4, g4, n4, ctl));
    switch ((a.nchunk + 3) / 4) {
      case 1: BM_LAUNCH(cx, "edm_ls", k_pair_ls<1><<<grid, 256, 0, h.stream>>>(a)); break;
      case 2: BM_LAUNCH(cx, "edm_ls", k_pair_ls<2><<<grid, 256, 0, h.stream>>>(a)); break;
      case 3: BM_LAUNCH(cx, "edm_ls", k_pair_ls<3><<<grid, 256, 0, h.stream>>>(a)); break;
      case 4: BM_LAUNCH(cx, "edm_ls", k_pair_ls<4><<<grid, 256, 0, h.stream>>>(a)); break;
      case 5: BM_LAUNCH(cx, "edm_ls", k_pair_ls<5><<<grid, 256, 0, h.stream>>>(a)); break;
      case 6: BM_LAUNCH(cx, "edm_ls", k_pair_ls<6><<<grid, 256, 0, h.stream>>>(a)); break;
      case 7: BM_LAUNCH(cx, "edm_ls", k_pair_ls<7><<<grid, 256, 0, h.stream>>>(a)); break;
      default: BM_LAUNCH(cx, "edm_ls", k_pair_ls<8><<<grid, 256, 0, h.stream>>>(a)); break;
    }
    // block partials, then one pass of the same kernel over them (fixed order)
    BM_LAUNCH(cx, "edm_sum4", k_sum4_part<<<parts, kSumThreads, 0, h.stream>>>(s.segsums.get(), a.nseg,
                                                                                 s.sums4.get() + 4));
    BM_LAUNCH(cx, "edm_sum4", k_sum4_part<<<1, kSumThreads, 0, h.stream>>>(s.sums4.get() + 4, parts, ctl + kCS1));
    dots2(h, h.gV.get(), s.D.get(), s.D.get(), s.D.get(), ctl + kCGD);   // <g, D>, <D, D>
    BM_LAUNCH(cx, "edm_ctrl", k_edm_ctrl_step<<<1, 1, 0, h.stream>>>(ctl, h.lambda));
    BM_LAUNCH(cx, "edm_update", k_edm_update<<<grid_n(n4), 256, 0, h.stream>>>(V4, D4, g4, gp4, n4, ctl));
  }
}

// Polak-Ribiere+ with the exact quartic line search; returns F after the last iteration
double bm_phase(bm_edm_ctx& h, int epochs) {
  EdmSolveState& s = *h.ss;
  if (h.k == 0 || epochs <= 0) return edm_loss_grad_dev(h, false, nullptr);
  bool launched = false;
  if (!core(h).prof.on) {   // timed runs record events around each launch: no graph then
    if (s.bm_graph && (s.graph_ld != h.ld || s.graph_epochs != epochs || s.graph_stream != h.stream)) {
      cudaGraphExecDestroy(s.bm_graph);
      s.bm_graph = nullptr;
    }
    if (!s.bm_graph) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        bool ok = true;
        try {
          bm_phase_launch(h, epochs);
        } catch (...) {
          ok = false;
        }
        const cudaError_t ce = cudaStreamEndCapture(h.stream, &g);
        ok = ok && ce == cudaSuccess && g;
        if (ok && cudaGraphInstantiate(&s.bm_graph, g, 0) == cudaSuccess) {
          s.graph_ld = h.ld;
          s.graph_epochs = epochs;
          s.graph_stream = h.stream;
        } else {
          s.bm_graph = nullptr;
        }
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();   // a failed capture falls back to direct launches
    }
    if (s.bm_graph) {
      BM_CUDA(cudaGraphLaunch(s.bm_graph, h.stream));
      launched = true;
    }
  }
  if (!launched) bm_phase_launch(h, epochs);
  double out[kCtlSlots];
  BM_CUDA(cudaMemcpyAsync(out, s.ctl.get(), sizeof(out), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  BM_REQUIRE(out[kCBad] == 0.0 && std::isfinite(out[kCFLast]), BM_ERR_NUMERIC,
             "distance-geometry BM phase: objective is not finite");
  return out[kCFLast];
}

template <class Fn>
bm_status edm_call(bm_edm_ctx* h, Fn&& fn) {
  return guard_call(h->err, std::forward<Fn>(fn));
}

}  // namespace
}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_edm_set_options(bm_edm_handle h, const bm_options* o) {
  if (!h || !o) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    BM_REQUIRE(o->bm_epochs >= 0 && o->lmsvd_p >= 0 && o->lmsvd_p <= 1 && o->lmsvd_imax >= 1 && o->lmsvd_min_iter >= 1 &&
                   std::isfinite(o->lmsvd_tol) && o->tau > 0,
               BM_ERR_INVALID, "bm_edm_set_options: invalid options");
    h->opt = *o;
  });
}

bm_status bm_edm_profile_enable(bm_edm_handle h, int32_t enable) {
  if (!h) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    BM_CUDA(cudaStreamSynchronize(h->stream));
    h->core.prof.marks.clear();
    h->core.prof.used = 0;
    h->core.prof.on = enable != 0;
  });
}

bm_status bm_edm_profile_read(bm_edm_handle h, int32_t cap, char* names, int64_t* launches, double* total_ms,
                              int32_t* count) {
  if (!h) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    BM_CUDA(cudaStreamSynchronize(h->stream));
    profile_report(h->core.prof, cap, names, launches, total_ms, count);
  });
}

bm_status bm_edm_get_factor(bm_edm_handle h, int32_t* k, float* V) {
  if (!h) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    if (k) *k = h->k;
    if (V && h->k > 0) {
      BM_CUDA(cudaMemcpy2DAsync(V, h->k * sizeof(float), h->V.get(), h->ld * sizeof(float), h->k * sizeof(float),
                                h->n, is_device_ptr(V) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
      BM_CUDA(cudaStreamSynchronize(h->stream));
    }
  });
}

bm_status bm_edm_bm_phase(bm_edm_handle h, int32_t epochs, double* F) {
  if (!h) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    BM_REQUIRE(epochs >= 0, BM_ERR_INVALID, "bm_edm_bm_phase: epochs must be >= 0");
    ensure_state(*h);
    const double f = bm_phase(*h, epochs);
    BM_REQUIRE(std::isfinite(f), BM_ERR_NUMERIC, "bm_edm_bm_phase: objective is not finite");
    if (F) *F = f;
  });
}

bm_status bm_edm_prox_step(bm_edm_handle h, bm_prox_info* info) {
  if (!h) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    ensure_state(*h);
    EdmSolveState& s = *h->ss;
    if (!s.initialized) {
      s.k_eig = std::max(1, std::min(h->k_max, h->k + 1));
      s.initialized = true;
    }
    const EdmStepOut o = prox_step(*h);
    if (info) {
      *info = bm_prox_info{};
      info->k_new = o.rank;
      info->warm_cols = o.computed;
      info->lmsvd_iters = o.iters;
      info->n_L = o.k_next;
      info->cap_hit = o.rank == o.computed ? 1 : 0;
      info->eps = s.sigma;
      info->F = o.F;
    }
  });
}

bm_status bm_edm_init(bm_edm_handle h, bm_prox_info* info) {
  if (!h) return BM_ERR_INVALID;
  return edm_call(h, [&] {
    ensure_state(*h);
    const EdmStepOut o = init_step(*h);
    if (info) {
      *info = bm_prox_info{};
      info->k_new = o.rank;
      info->warm_cols = o.computed;
      info->lmsvd_iters = o.iters;
      info->n_L = o.k_next;
      info->cap_hit = o.rank == o.computed ? 1 : 0;
      info->eps = h->ss->sigma;
      info->F = o.F;
    }
  });
}

bm_status bm_edm_solve(bm_edm_handle h, const bm_solve_opts* o, bm_solve_info* info) {
  if (!h) return BM_ERR_INVALID;
  bool converged = false;
  const bm_status st = edm_call(h, [&] {
    bm_solve_opts so{100, 0, 1e-10, 0.0, 0.0};
    if (o) so = *o;
    BM_REQUIRE(so.max_outer >= 0, BM_ERR_INVALID, "bm_edm_solve: max_outer must be >= 0");
    ensure_state(*h);
    const auto t0 = std::chrono::steady_clock::now();
    if (h->k == 0) {
      init_step(*h);
    } else if (!h->ss->initialized) {   // factor set by the caller
      h->ss->k_eig = std::max(1, std::min(h->k_max, h->k + 1));
      h->ss->initialized = true;
    }
    double F_prev = edm_loss_grad_dev(*h, false, nullptr), F = F_prev;
    int outer = 0;
    for (outer = 1; outer <= so.max_outer; ++outer) {
      bm_phase(*h, h->opt.bm_epochs);
      const EdmStepOut s = prox_step(*h);
      F = s.F;
      BM_REQUIRE(std::isfinite(F), BM_ERR_NUMERIC, "bm_edm_solve: objective is not finite");
      if (so.F_target != 0.0 && F <= so.F_target) { converged = true; break; }
      if (std::fabs(F_prev - F) / (1.0 + std::fabs(F_prev)) < so.tol) { converged = true; break; }
      F_prev = F;
      if (so.time_limit_s > 0 &&
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > so.time_limit_s)
        break;
    }
    if (info) {
      info->outer = std::min(outer, so.max_outer);
      info->k = h->k;
      info->converged = converged ? 1 : 0;
      info->F = F;
      info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  });
  if (st == BM_OK && !converged) {
    h->err = "bm_edm_solve: stopped on max_outer or time_limit_s";
    return BM_ERR_NOT_CONVERGED;
  }
  return st;
}

}  // extern "C"
