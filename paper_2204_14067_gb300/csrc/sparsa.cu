// The SpaRSA step rule for the inexact PG step (supplement Sec. "The SpaRSA
// variant for Matrix Completion"): a Barzilai-Borwein initial step
// (Eq. "proxBB") from the last two points where the PG step was taken, then
// backtracking alpha <- beta alpha until the step satisfies Eq. "back" or
// Eq. "decrease".
//
//   alpha_BB = clip(||dX||_F^2 / <dX, dG>, alpha_min, alpha_max): the printed
//     ratio <dX, dG> / ||dX||^2 is a curvature (inverse step length), so its
//     reciprocal is the step size; for f = 1/2 ||P_Omega(X - A)||^2,
//     dG = P_Omega(dX) and <dX, dG> = ||r_t - r_{t-1}||^2 over Omega.
//   ||X1 - X0||_F^2 from k x k Grams (Eq. "trace" with the sign of its last
//     term corrected): tr(W1'W1 H1'H1) + tr(W0'W0 H0'H0) - 2 tr((W0'W1)(H1'H0)).
//   Eq. "back":     f(X+) <= f(X~) + <r~, r+ - r~> + (delta / alpha) ||X+ - X~||^2
//   Eq. "decrease": F(X+) <= F(X~) + delta Q, Q = <r~, r+ - r~> + ||X+ - X~||^2 / (2 alpha)
//                   + lambda (||X+||_* - ||X~||_*)
//   (on Omega, X+ - X~ = r+ - r~, so <grad f(X~), X+ - X~> = <r~, r+ - r~>).
// A rejected trial restores X~ and the PG-step state (warm start, safeguard)
// exactly, so every trial starts from the same point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "dense.cuh"

namespace bm {

struct BbState {
  bm_bb_options opt{};
  bool have_prev = false;
  int kp = 0, ldp = 4;
  DevBuf<float> Wp, Hp, rp;     // X~_{t-1} (m x ldp, n x ldp) and its residual (CSR order)
  DevBuf<float> Ws, Hs, rt;     // X~_t kept for backtracking, and r~ = r(X~_t)
  DevBuf<double> G1, G2, E, ev, S, T, D;
  DevBuf<double> part;          // reduction partials
  DenseWork dw;
};

void bb_destroy(BbState* s) { delete s; }

void bb_reset(bm_ctx& h) {
  if (h.bb) h.bb->have_prev = false;
}

namespace {

constexpr int kRedThreads = 256;

int red_parts() { return std::max(1, std::min(1024, 2 * num_sms())); }

// part[2 b + 0] = sum (a - b)^2, part[2 b + 1] = sum b (a - b) over a fixed strided share
__global__ void __launch_bounds__(kRedThreads) k_diff_sums(const float* __restrict__ a, const float* __restrict__ b,
                                                          int64_t n, double* __restrict__ part) {
  __shared__ double s0[kRedThreads], s1[kRedThreads];
  double x0 = 0.0, x1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i], d = (double)a[i] - bi;
    x0 += d * d;
    x1 += bi * d;
  }
  s0[threadIdx.x] = x0;
  s1[threadIdx.x] = x1;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}

// out[0..1] = column sums of part (rows of 2), fixed order, one block
__global__ void __launch_bounds__(kRedThreads) k_pair_total(const double* __restrict__ part, int rows,
                                                           double* __restrict__ out) {
  __shared__ double s0[kRedThreads], s1[kRedThreads];
  double x0 = 0.0, x1 = 0.0;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    x0 += part[2 * i];
    x1 += part[2 * i + 1];
  }
  s0[threadIdx.x] = x0;
  s1[threadIdx.x] = x1;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

// D (n x n) = diag(d) * S * diag(d)
__global__ void k_scale_sym(const double* __restrict__ S, const double* __restrict__ d, int n, double* __restrict__ D) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    const int i = t / n, j = t - (t / n) * n;
    D[t] = d[i] * S[t] * d[j];
  }
}

// (sum (a - b)^2, sum b (a - b)) over n entries
void diff_sums(bm_ctx& h, BbState& s, const float* a, const float* b, int64_t n, double out[2]) {
  out[0] = out[1] = 0.0;
  if (n == 0) return;
  const int parts = red_parts();
  BM_LAUNCH(h, "bb_sums", k_diff_sums<<<parts, kRedThreads, 0, h.stream>>>(a, b, n, s.part.get()));
  BM_LAUNCH(h, "bb_sums", k_pair_total<<<1, kRedThreads, 0, h.stream>>>(s.part.get(), parts, s.part.get() + 2 * parts));
  BM_CUDA(cudaMemcpyAsync(out, s.part.get() + 2 * parts, 2 * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
}

// sum_ij A_ij B_ij of two a x b FP64 device matrices (a k x k trace term)
double elem_dot(bm_ctx& h, const double* A, const double* B, size_t count) {
  std::vector<double> x(count), y(count);
  if (count) {
    BM_CUDA(cudaMemcpyAsync(x.data(), A, count * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaMemcpyAsync(y.data(), B, count * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
  }
  double t = 0.0;
  for (size_t i = 0; i < count; ++i) t += x[i] * y[i];
  return t;
}

// ||W1 H1^T - W0 H0^T||_F^2 (Eq. "trace", corrected)
double frob_diff2(bm_ctx& h, BbState& s, const Tall& W1, const Tall& H1, const Tall& W0, const Tall& H0) {
  auto tr = [&](const Tall& Wa, const Tall& Wb, const Tall& Ha, const Tall& Hb) {
    if (Wa.cols == 0 || Wb.cols == 0) return 0.0;
    gram_dev(h, s.dw, Wa, Wb, s.G1.get(), true, "bb_gram");
    gram_dev(h, s.dw, Ha, Hb, s.G2.get(), true, "bb_gram");
    return elem_dot(h, s.G1.get(), s.G2.get(), (size_t)Wa.cols * Wb.cols);
  };
  return tr(W1, W1, H1, H1) + tr(W0, W0, H0, H0) - 2.0 * tr(W0, W1, H0, H1);
}

// ||W H^T||_*: with W^T W = E diag(w) E^T, the singular values of W H^T are
// the square roots of eig(diag(sqrt w) E^T (H^T H) E diag(sqrt w)).
double nuclear_norm(bm_ctx& h, BbState& s, const Tall& W, const Tall& H) {
  const int k = W.cols;
  if (k == 0) return 0.0;
  gram_dev(h, s.dw, W, W, s.G1.get(), true, "bb_gram");
  gram_dev(h, s.dw, H, H, s.G2.get(), true, "bb_gram");
  sym_eig_dev(h, s.dw, s.G1.get(), k, s.ev.get(), s.E.get(), kEigRelative);
  std::vector<double> w(k);
  BM_CUDA(cudaMemcpyAsync(w.data(), s.ev.get(), k * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  std::vector<double> sq(k), I((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) sq[i] = std::sqrt(std::max(w[i], 0.0)), I[(size_t)i * k + i] = 1.0;
  // T = E^T (as I * E^T), S = G2 * E, D = T * S = E^T G2 E
  BM_CUDA(cudaMemcpyAsync(s.D.get(), I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, h.stream));
  small_mm_dev(h, s.D.get(), s.E.get(), s.T.get(), k, k, k, true);
  small_mm_dev(h, s.G2.get(), s.E.get(), s.S.get(), k, k, k, false);
  small_mm_dev(h, s.T.get(), s.S.get(), s.D.get(), k, k, k, false);
  BM_CUDA(cudaMemcpyAsync(s.ev.get(), sq.data(), k * sizeof(double), cudaMemcpyHostToDevice, h.stream));
  BM_LAUNCH(h, "bb_scale", k_scale_sym<<<std::max(1, std::min(64, (k * k + 255) / 256)), 256, 0, h.stream>>>(
                               s.D.get(), s.ev.get(), k, s.S.get()));
  sym_eig_dev(h, s.dw, s.S.get(), k, s.ev.get(), s.E.get(), kEigRelative);
  BM_CUDA(cudaMemcpyAsync(w.data(), s.ev.get(), k * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  double nuc = 0.0;
  for (int i = 0; i < k; ++i) nuc += std::sqrt(std::max(w[i], 0.0));
  return nuc;
}

BbState& bb_state(bm_ctx& h) {
  if (!h.bb) {
    h.bb = new BbState();
    bm_bb_default_options(&h.bb->opt);
  }
  BbState& s = *h.bb;
  const size_t m = (size_t)h.ix.m, n = (size_t)h.ix.n, nnz = (size_t)std::max<int64_t>(h.ix.nnz, 1);
  const size_t ldm = (size_t)h.ldmax;
  s.Wp.alloc(m * ldm);
  s.Hp.alloc(n * ldm);
  s.Ws.alloc(m * ldm);
  s.Hs.alloc(n * ldm);
  s.rp.alloc(nnz);
  s.rt.alloc(nnz);
  const size_t q = (size_t)h.k_max + 1;
  s.G1.alloc(q * q);
  s.G2.alloc(q * q);
  s.E.alloc(q * q);
  s.S.alloc(q * q);
  s.T.alloc(q * q);
  s.D.alloc(q * q);
  s.ev.alloc(q);
  s.part.alloc(2 * (size_t)red_parts() + 2);
  return s;
}

Tall tallW(bm_ctx& h, float* p, int k, int ld) { return Tall{p, h.ix.m, k, ld}; }
Tall tallH(bm_ctx& h, float* p, int k, int ld) { return Tall{p, h.ix.n, k, ld}; }

void copy_factors(bm_ctx& h, float* dW, float* dH, const float* sW, const float* sH, int ld) {
  BM_CUDA(cudaMemcpyAsync(dW, sW, (size_t)h.ix.m * ld * sizeof(float), cudaMemcpyDeviceToDevice, h.stream));
  BM_CUDA(cudaMemcpyAsync(dH, sH, (size_t)h.ix.n * ld * sizeof(float), cudaMemcpyDeviceToDevice, h.stream));
}

}  // namespace

void prox_step_bb_dev(bm_ctx& h, bm_prox_info* info, bm_bb_info* bbi) {
  BbState& s = bb_state(h);
  const bm_bb_options& o = s.opt;
  const int64_t nnz = h.ix.nnz;
  // X~_t: residual, f, nuclear norm; kept for backtracking
  const double f0 = residual_dev(h);
  if (nnz) BM_CUDA(cudaMemcpyAsync(s.rt.get(), h.r_csr.get(), nnz * sizeof(float), cudaMemcpyDeviceToDevice, h.stream));
  const int k0 = h.k, ld0 = h.ld;
  const bool changed0 = h.bm_changed;
  copy_factors(h, s.Ws.get(), s.Hs.get(), h.W.get(), h.H.get(), ld0);
  const Tall W0 = tallW(h, s.Ws.get(), k0, ld0), H0 = tallH(h, s.Hs.get(), k0, ld0);
  const double nuc0 = nuclear_norm(h, s, W0, H0);
  const double F0 = f0 + h.lambda * nuc0;
  std::vector<uint8_t> snap(prox_state_bytes(h));
  prox_state_save(h, snap.data());
  // Eq. "proxBB"
  double a0 = h.opt.alpha;
  if (s.have_prev) {
    const double num = frob_diff2(h, s, W0, H0, tallW(h, s.Wp.get(), s.kp, s.ldp), tallH(h, s.Hp.get(), s.kp, s.ldp));
    double sums[2];
    diff_sums(h, s, s.rt.get(), s.rp.get(), nnz, sums);
    a0 = sums[0] > 0 ? num / sums[0] : o.alpha_max;
  }
  a0 = std::max(o.alpha_min, std::min(o.alpha_max, a0));
  bm_prox_info pi{};
  bm_bb_info bb{a0, a0, 0, 0};
  double F1 = 0.0;
  for (int i = 0; i <= o.max_backtracks; ++i) {
    const double a = a0 * std::pow(o.beta, i);
    if (i > 0) {   // back to X~_t and its PG-step state
      h.k = k0;
      h.ld = ld0;
      copy_factors(h, h.W.get(), h.H.get(), s.Ws.get(), s.Hs.get(), ld0);
      h.bf_dirty = true;
      h.bm_changed = changed0;
      prox_state_load(h, snap.data(), snap.size());
    }
    prox_step_dev(h, a, &pi, false);
    const double f1 = residual_dev(h);
    double sums[2];
    diff_sums(h, s, h.r_csr.get(), s.rt.get(), nnz, sums);   // sums[1] = <r~, r+ - r~>
    const double lin = sums[1];
    const Tall W1 = tallW(h, h.W.get(), h.k, h.ld), H1 = tallH(h, h.H.get(), h.k, h.ld);
    const double d2 = frob_diff2(h, s, W1, H1, W0, H0);
    // balanced factors after the refactor: ||X+||_* = sum Sigma = ||W+||_F^2
    const double nuc1 = h.k > 0 ? dot_dev(h, h.W.get(), h.W.get(), h.ix.m * (int64_t)h.ld) : 0.0;
    F1 = f1 + h.lambda * nuc1;
    const bool back = f1 <= f0 + lin + o.delta / a * d2;
    const double Q = lin + d2 / (2.0 * a) + h.lambda * (nuc1 - nuc0);
    const bool dec = F1 <= F0 + o.delta * Q;
    bb.alpha = a;
    bb.backtracks = i;
    bb.accepted_by = back ? 1 : (dec ? 2 : 0);
    if (back || dec) break;
  }
  // X~_t becomes the previous point of the next step
  std::swap(s.Wp.p, s.Ws.p);
  std::swap(s.Wp.n, s.Ws.n);
  std::swap(s.Hp.p, s.Hs.p);
  std::swap(s.Hp.n, s.Hs.n);
  std::swap(s.rp.p, s.rt.p);
  std::swap(s.rp.n, s.rt.n);
  s.kp = k0;
  s.ldp = ld0;
  s.have_prev = true;
  if (info) {
    *info = pi;
    info->F = F1;
  }
  if (bbi) *bbi = bb;
}

}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_bb_default_options(bm_bb_options* o) {
  if (!o) return BM_ERR_INVALID;
  o->alpha_min = 1e-3;
  o->alpha_max = 1e3;
  o->beta = 0.5;
  o->delta = 0.995;
  o->max_backtracks = 30;
  o->pad_ = 0;
  return BM_OK;
}

bm_status bm_set_bb_options(bm_handle h, const bm_bb_options* o) {
  if (!h || !o) return BM_ERR_INVALID;
  return guard_call(h->err, [&] {
    BM_REQUIRE(o->alpha_min > 0 && o->alpha_max >= o->alpha_min && std::isfinite(o->alpha_max) && o->beta > 0 &&
                   o->beta < 1 && o->delta > 0 && o->delta < 1 && o->max_backtracks >= 0,
               BM_ERR_INVALID, "bm_set_bb_options: need 0 < alpha_min <= alpha_max, beta and delta in (0, 1)");
    bb_state(*h).opt = *o;
  });
}

bm_status bm_prox_step_bb(bm_handle h, bm_prox_info* info, bm_bb_info* bb) {
  if (!h) return BM_ERR_INVALID;
  return guard_call(h->err, [&] {
    BM_REQUIRE(h->k >= 0, BM_ERR_INVALID, "bm_prox_step_bb: no factors");
    prox_step_bb_dev(*h, info, bb);
  });
}

}  // extern "C"
