// Inexact proximal-gradient step (Eq. "inexactpg") and the initial point
// (Sec. "Initialization").  Host code orchestrates device kernels; only
// eigenvalues, column counts and scalars come back to the host to take the
// control decisions (ranks, stopping, drops).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dense.cuh"

namespace bm {

void set_rank_ext(bm_ctx& h, int k);
double objective_ext(bm_ctx& h);
LossOut loss_grad_dev(bm_ctx& h, bool want_grad, bool store_r);

constexpr uint64_t kStreamInitSketch = 1;
constexpr uint64_t kStreamSafeguard = 1000;

struct ProxState {
  int qcap = 0;   // max columns of an L application (k_max + 1, >= k_init)
  int ldq = 4;    // ld of n-side blocks
  int ldq2 = 4;   // ld of m-side blocks (up to 2 qcap columns)
  DenseWork dw;
  DevBuf<float> mbuf[17];   // m-side blocks
  DevBuf<float> Y, Bt;      // n-side blocks (ld ldq): L-application scratch, Z^T U^
  DevBuf<float> YQ;         // Z^T Q of the Rayleigh-Ritz basis (ld ldq2)
  DevBuf<double> G, E, ev, S1, S2;
  DevBuf<float> Ts;
  // safeguard / warm-start state
  bool initialized = false;   // U_prev valid
  int iUprev = 0, iUprev2 = 1, iu = 2;  // U_t, U_{t-1}, truncated vector u
  int ku = 0, ku2 = -1;
  bool have_u = false;
  double psi = 0.1;
  int rank_prev = 0, rank_cur = 0;
  int prev_warm = 0;
  int t = 0;
};

namespace {

// Smallest Gram eigenvalue bound for which orth() takes the Cholesky basis.
constexpr double kOrthCholCert = 1e-2;

enum { kUprevA = 0, kUprevB = 1, kUvec = 2, kU = 3, kB0 = 4, kLB0 = 5, kB1 = 6, kLB1 = 7, kB2 = 8, kLB2 = 9,
       kQ = 10, kLQ = 11, kX1 = 12, kX2 = 13, kX3 = 14, kX4 = 15, kUw = 16 };

Tall mview(bm_ctx& h, int which, int cols) {
  ProxState& ps = *h.ps;
  return Tall{ps.mbuf[which].get(), h.ix.m, cols, ps.ldq2};
}
Tall nview(bm_ctx& h, DevBuf<float>& b, int cols) { return Tall{b.get(), h.ix.n, cols, h.ps->ldq}; }
Tall Wview(bm_ctx& h) { return Tall{h.W.get(), h.ix.m, h.k, h.ld}; }
Tall Hview(bm_ctx& h) { return Tall{h.H.get(), h.ix.n, h.k, h.ld}; }

std::vector<double> to_host(bm_ctx& h, const double* d, size_t n) {
  std::vector<double> v(n);
  if (n) {
    BM_CUDA(cudaMemcpyAsync(v.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
  }
  return v;
}

std::vector<double> diag_to_host(bm_ctx& h, const double* G, int n) {
  std::vector<double> v(n);
  if (n) {
    BM_CUDA(cudaMemcpy2DAsync(v.data(), sizeof(double), G, (n + 1) * sizeof(double), sizeof(double), n,
                              cudaMemcpyDeviceToHost, h.stream));
    BM_CUDA(cudaStreamSynchronize(h.stream));
  }
  return v;
}

// Ts (rows x cols FP32, ld = ldq2) from FP64 E columns `sel` scaled by `scale`.
void make_transform(bm_ctx& h, const double* E, int n, int rows, const std::vector<int>& sel,
                    const std::vector<double>& scale) {
  select_scale_dev(h, E, n, rows, sel.data(), scale.data(), (int)sel.size(), h.ps->Ts.get(), h.ps->ldq2);
}

// Y = Z^T X = H (W^T X) - alpha R^T X
void apply_zt(bm_ctx& h, const Tall& X, const Tall& Y, double alpha) {
  ProxState& ps = *h.ps;
  if (h.k > 0) {
    gram_dev(h, ps.dw, Wview(h), X, ps.G.get(), false, "gram_WtU");
    small_to_f32_dev(h, ps.G.get(), h.k, X.cols, X.cols, ps.Ts.get(), ps.ldq2);
    gemm_dev(h, Hview(h), ps.Ts.get(), ps.ldq2, Y, 0.f, 1.f, "gemm_H");
  } else {
    zero_dev(h, Y);
  }
  spmm_dev(h, false, h.r_csc.get(), X, Y, (float)-alpha);
}

// out = Z Y = W (H^T Y) - alpha R Y  (Eq. "ZZ", the product with Z)
void apply_z(bm_ctx& h, const Tall& Y, const Tall& out, double alpha) {
  ProxState& ps = *h.ps;
  if (h.k > 0) {
    gram_dev(h, ps.dw, Hview(h), Y, ps.G.get(), false, "gram_HtY");
    small_to_f32_dev(h, ps.G.get(), h.k, Y.cols, Y.cols, ps.Ts.get(), ps.ldq2);
    gemm_dev(h, Wview(h), ps.Ts.get(), ps.ldq2, out, 0.f, 1.f, "gemm_W");
  } else {
    zero_dev(h, out);
  }
  spmm_dev(h, true, h.r_csr.get(), Y, out, (float)-alpha);
}

// out = Z Z^T X  (L of Eq. "ssi")
void apply_L(bm_ctx& h, const Tall& X, const Tall& out, double alpha) {
  ProxState& ps = *h.ps;
  Tall Y = nview(h, ps.Y, X.cols);
  apply_zt(h, X, Y, alpha);
  apply_z(h, Y, out, alpha);
}

// Orthonormal new columns for ran([F, M]) by Eq. "PUi"/"orth-W" (two passes).
// M, LM, F, LF must not be the work blocks X1..X4.  Returns the column count;
// the result is copied into out / lout (if given).
int orth_dev(bm_ctx& h, const Tall& M, const Tall* F, const Tall* LM, const Tall* LF, double tau, int max_cols,
             int out_idx, int out_col, int lout_idx) {
  ProxState& ps = *h.ps;
  const int c = M.cols;
  if (c == 0) return 0;
  gram_dev(h, ps.dw, M, M, ps.G.get(), true, "gram_orth");
  std::vector<double> dg = diag_to_host(h, ps.G.get(), c);
  std::vector<int> sel;
  std::vector<double> sc;
  for (int j = 0; j < c; ++j)
    if (dg[j] > 0 && std::isfinite(dg[j])) sel.push_back(j), sc.push_back(1.0 / std::sqrt(dg[j]));
  int c1 = (int)sel.size();
  if (c1 == 0) return 0;
  // Mh = M[:, sel] diag(1/s): transform = identity columns scaled
  {
    std::vector<double> I((size_t)c * c, 0.0);
    for (int j = 0; j < c; ++j) I[(size_t)j * c + j] = 1.0;
    BM_CUDA(cudaMemcpyAsync(ps.S1.get(), I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, h.stream));
    make_transform(h, ps.S1.get(), c, c, sel, sc);
  }
  int a = kX1, la = kX2, b = kX3, lb = kX4;
  gemm_dev(h, M, ps.Ts.get(), ps.ldq2, mview(h, a, c1), 0.f, 1.f, "gemm_orth");
  if (LM) gemm_dev(h, *LM, ps.Ts.get(), ps.ldq2, mview(h, la, c1), 0.f, 1.f, "gemm_orth");
  const bool useF = F && F->cols > 0;
  for (int pass = 0; pass < 2; ++pass) {
    Tall Mh = mview(h, a, c1);
    if (useF) {
      gram_dev(h, ps.dw, *F, Mh, ps.G.get(), true, "gram_orth");
      small_to_f32_dev(h, ps.G.get(), F->cols, c1, c1, ps.Ts.get(), ps.ldq2);
      gemm_dev(h, *F, ps.Ts.get(), ps.ldq2, Mh, 1.f, -1.f, "gemm_orth");
      if (LM) gemm_dev(h, *LF, ps.Ts.get(), ps.ldq2, mview(h, la, c1), 1.f, -1.f, "gemm_orth");
    }
    gram_dev(h, ps.dw, Mh, Mh, ps.G.get(), true, "gram_orth");
    int c2 = c1;
    bool chol_basis = false;
    if (pass == 0 && (max_cols < 0 || max_cols >= c1)) {
      // Eq. "orth-W" keeps every direction when no Gram eigenvalue is <= tau.
      // A Cholesky factor P^T P = R^T R certifies that: lambda_min >= 1 /
      // ||R^{-1}||_F^2.  Then P R^{-1} is an orthonormal basis of the same
      // span, found without the eigensolver (the certificate also bounds the
      // condition number so that the FP32 second pass restores orthogonality).
      double f = 0.0;
      chol_basis = chol_inv_try_dev(h, ps.dw, ps.G.get(), c1, ps.Ts.get(), ps.ldq2, &f) && f > 0 &&
                   1.0 / f >= std::max(kOrthCholCert, 10.0 * tau);
    }
    if (chol_basis) {
      // Ts = R^{-1}, all c1 columns kept
    } else if (pass == 0) {
      // Eq. "orth-W": eigen-decomposition of P^T P, drop eigenvalues <= tau, scale by Lambda^{-1/2}
      sym_eig_dev(h, ps.dw, ps.G.get(), c1, ps.ev.get(), ps.E.get(), kEigFast);
      std::vector<double> lam = to_host(h, ps.ev.get(), c1);
      std::vector<int> keep;
      std::vector<double> s;
      for (int j = 0; j < c1; ++j) {
        if (!(lam[j] > tau)) break;
        if (max_cols >= 0 && j >= max_cols) break;
        keep.push_back(j);
        s.push_back(1.0 / std::sqrt(lam[j]));
      }
      c2 = (int)keep.size();
      if (c2 == 0) return 0;
      make_transform(h, ps.E.get(), c1, c1, keep, s);
    } else {
      // re-orthogonalisation of an almost orthonormal block: Cholesky QR, Q = P R^{-1}
      chol_inv_dev(h, ps.dw, ps.G.get(), c1, ps.Ts.get(), ps.ldq2);
    }
    gemm_dev(h, Mh, ps.Ts.get(), ps.ldq2, mview(h, b, c2), 0.f, 1.f, "gemm_orth");
    if (LM) gemm_dev(h, mview(h, la, c1), ps.Ts.get(), ps.ldq2, mview(h, lb, c2), 0.f, 1.f, "gemm_orth");
    std::swap(a, b);
    std::swap(la, lb);
    c1 = c2;
  }
  copy_cols_dev(h, mview(h, a, c1), 0, mview(h, out_idx, out_col + c1), out_col, c1);
  if (LM && lout_idx >= 0) copy_cols_dev(h, mview(h, la, c1), 0, mview(h, lout_idx, out_col + c1), out_col, c1);
  return c1;
}

double dot_cols(bm_ctx& h, const Tall& x, const Tall& y) {  // single-column blocks (ld 4-padded)
  ProxState& ps = *h.ps;
  gram_dev(h, ps.dw, x, y, ps.G.get(), true, "gram_vec");
  return to_host(h, ps.G.get(), 1)[0];
}

// y = a*x + b*y for single-column blocks, via the thin product
void vec_axpby(bm_ctx& h, const Tall& x, double a, const Tall& y, double b) {
  ProxState& ps = *h.ps;
  float one[4] = {(float)a, 0.f, 0.f, 0.f};
  BM_CUDA(cudaMemcpyAsync(ps.Ts.get(), one, sizeof(one), cudaMemcpyHostToDevice, h.stream));
  gemm_dev(h, x, ps.Ts.get(), 4, y, (float)b, 1.f, "vec");
  BM_CUDA(cudaStreamSynchronize(h.stream));
}

// y -= B (B^T y) for a single column y and a block B
void project_out(bm_ctx& h, const Tall& B, const Tall& y) {
  ProxState& ps = *h.ps;
  if (B.cols == 0) return;
  gram_dev(h, ps.dw, B, y, ps.G.get(), true, "gram_vec");
  small_to_f32_dev(h, ps.G.get(), B.cols, 1, 1, ps.Ts.get(), ps.ldq2);
  gemm_dev(h, B, ps.Ts.get(), ps.ldq2, y, 1.f, -1.f, "vec");
}

struct LmsvdOut {
  int cols;
  int iters;
  int nL;
  std::vector<double> theta;
};

// LmSVD (Algorithm 2) from the warm start in block kUw (c0 columns).  Result:
// the Ritz vectors U^ in kU and their images Z^T U^ in ps.Bt.
//
// The subspace is the paper's: Q = [B_0, orth(B_1 | B_0)] with B_0 =
// orth(L(U^)) the newest block and B_1 the previous one (memory p = 1).  The
// Rayleigh-Ritz matrix Q^T L Q is formed as (Z^T Q)^T (Z^T Q) and L(U^) as
// Z (Z^T U^): in FP32 the product L = Z Z^T carries errors of order
// eps * sigma_1^2 into every column, which would swamp the small singular
// values near the threshold lambda * alpha, while products with Z and Z^T
// alone err by eps * sigma_1 * (size of the column).  The small eigenproblem
// runs in the relative-accuracy mode for the same reason.  Each iteration
// costs one product with Z^T (the basis Q) and one with Z (the Ritz vectors),
// as one application of L would.
LmsvdOut lmsvd_dev(bm_ctx& h, int c0, double alpha) {
  ProxState& ps = *h.ps;
  const bm_options& o = h.opt;
  const int64_t n = h.ix.n;
  LmsvdOut r{0, 0, 0, {}};
  int B[3] = {kB0, kB1, kB2};
  int kc[3] = {0, 0, 0};
  const int k0 = orth_dev(h, mview(h, kUw, c0), nullptr, nullptr, nullptr, o.tau, -1, B[0], 0, -1);
  if (k0 == 0) return r;
  kc[0] = k0;
  int nb = 1;
  const int k = k0;
  std::vector<double> theta_prev;
  for (int it = 1; it <= o.lmsvd_imax; ++it) {
    r.iters = it;
    int q = kc[0];
    Tall Q = mview(h, B[0], kc[0]);
    if (nb > 1) {
      copy_cols_dev(h, mview(h, B[0], kc[0]), 0, mview(h, kQ, kc[0]), 0, kc[0]);
      Tall F = mview(h, B[0], kc[0]);
      const int c2 = orth_dev(h, mview(h, B[1], kc[1]), &F, nullptr, nullptr, o.tau, -1, kQ, kc[0], -1);
      q = kc[0] + c2;
      Q = mview(h, kQ, q);
    }
    const Tall YQ{ps.YQ.get(), n, q, ps.ldq2};
    apply_zt(h, Q, YQ, alpha);                                           // Z^T Q
    r.nL += 1;
    gram_dev(h, ps.dw, YQ, YQ, ps.G.get(), false, "gram_rr");           // Q^T L Q
    sym_eig_dev(h, ps.dw, ps.G.get(), q, ps.ev.get(), ps.E.get(), kEigRelative);
    std::vector<double> th = to_host(h, ps.ev.get(), q);
    const int kk = std::min(k, q);
    std::vector<int> sel(kk);
    std::vector<double> one(kk, 1.0);
    for (int j = 0; j < kk; ++j) sel[j] = j;
    make_transform(h, ps.E.get(), q, q, sel, one);
    gemm_dev(h, Q, ps.Ts.get(), ps.ldq2, mview(h, kU, kk), 0.f, 1.f, "gemm_rr");      // U^
    gemm_dev(h, YQ, ps.Ts.get(), ps.ldq2, nview(h, ps.Bt, kk), 0.f, 1.f, "gemm_rr_y");  // Z^T U^
    th.resize(kk);
    r.cols = kk;
    r.theta = th;
    bool conv = false;
    if (it >= o.lmsvd_min_iter && theta_prev.size() == th.size() && kk > 0) {
      double md = 0;
      for (int j = 0; j < kk; ++j) md = std::max(md, std::fabs(th[j] - theta_prev[j]));
      conv = md <= o.lmsvd_tol * std::max(th[0], 1e-300);
    }
    if (conv || it == o.lmsvd_imax) break;
    theta_prev = th;
    // next block U^{t,i+1} = orth(L(U^)), L(U^) = Z (Z^T U^)
    apply_z(h, nview(h, ps.Bt, kk), mview(h, kLB0, kk), alpha);
    const int fb = B[2];
    const int cn = orth_dev(h, mview(h, kLB0, kk), nullptr, nullptr, nullptr, o.tau, -1, fb, 0, -1);
    if (cn == 0) break;
    // rotate: new block first, keep p older ones
    B[2] = B[1];
    B[1] = B[0];
    kc[1] = kc[0];
    B[0] = fb;
    kc[0] = cn;
    nb = std::min(nb + 1, o.lmsvd_p + 1);
  }
  return r;
}

struct SvtOut {
  int k_new;
  bool cap_hit;
  double eps;
  std::vector<double> sigma_hat;
  double sum_sigma;
};

// Exact SVD of U^T Z, soft-threshold, refactor.  U^ in kU (kf columns).
SvtOut svt_refactor_dev(bm_ctx& h, int kf, double thresh, double alpha, double frob2, bool bt_ready) {
  ProxState& ps = *h.ps;
  SvtOut out{0, false, 0.0, {}, 0.0};
  const Index& ix = h.ix;
  if (kf == 0) {
    set_rank_ext(h, 0);
    BM_CUDA(cudaMemsetAsync(h.W.get(), 0, ix.m * 4 * sizeof(float), h.stream));
    BM_CUDA(cudaMemsetAsync(h.H.get(), 0, ix.n * 4 * sizeof(float), h.stream));
    out.eps = std::sqrt(std::max(frob2, 0.0));
    ps.ku2 = ps.initialized ? ps.ku : -1;
    std::swap(ps.iUprev, ps.iUprev2);
    ps.ku = 0;
    ps.have_u = false;
    return out;
  }
  Tall Uh = mview(h, kU, kf);
  Tall Bt = nview(h, ps.Bt, kf);
  if (!bt_ready) apply_zt(h, Uh, Bt, alpha);                    // (U^T Z)^T
  gram_dev(h, ps.dw, Bt, Bt, ps.G.get(), true, "gram_BBt");     // B B^T
  sym_eig_dev(h, ps.dw, ps.G.get(), kf, ps.ev.get(), ps.E.get(), kEigRelative);
  std::vector<double> s2 = to_host(h, ps.ev.get(), kf);
  std::vector<double> sh(kf);
  double sum_s2 = 0;
  for (int j = 0; j < kf; ++j) sh[j] = std::sqrt(std::max(s2[j], 0.0)), sum_s2 += sh[j] * sh[j];
  int k_new = 0;
  while (k_new < kf && sh[k_new] - thresh > 0) ++k_new;
  out.cap_hit = k_new > h.k_max;
  k_new = std::min(k_new, h.k_max);
  out.k_new = k_new;
  out.sigma_hat = sh;
  out.eps = std::sqrt(std::max(frob2 - sum_s2, 0.0));
  std::vector<int> sel(k_new);
  std::vector<double> cw(k_new), ch(k_new), one(k_new, 1.0);
  for (int j = 0; j < k_new; ++j) {
    sel[j] = j;
    const double sg = sh[j] - thresh;
    out.sum_sigma += sg;
    cw[j] = std::sqrt(sg);
    ch[j] = std::sqrt(sg) / sh[j];
  }
  // new U_t (unscaled) goes to the spare U_prev buffer; the old one becomes U_{t-1}
  const int newU = ps.iUprev2;
  if (k_new > 0) {
    make_transform(h, ps.E.get(), kf, kf, sel, one);
    gemm_dev(h, Uh, ps.Ts.get(), ps.ldq2, mview(h, newU, k_new), 0.f, 1.f, "gemm_U");
  }
  if (kf > k_new) {  // vector of the largest truncated value (Sec. "Ensuring sufficient precision")
    std::vector<int> s1{k_new};
    std::vector<double> o1{1.0};
    make_transform(h, ps.E.get(), kf, kf, s1, o1);
    zero_dev(h, Tall{ps.mbuf[ps.iu].get(), ix.m, 1, 4});
    gemm_dev(h, Uh, ps.Ts.get(), ps.ldq2, Tall{ps.mbuf[ps.iu].get(), ix.m, 1, 4}, 0.f, 1.f, "gemm_U");
    ps.have_u = true;
  } else {
    ps.have_u = false;
  }
  // W = U^ U~ diag(sqrt(Sigma)),  H = B^T U~ diag(sqrt(Sigma) / sigma_hat)
  set_rank_ext(h, k_new);
  if (k_new > 0) {
    make_transform(h, ps.E.get(), kf, kf, sel, cw);
    gemm_dev(h, Uh, ps.Ts.get(), ps.ldq2, Wview(h), 0.f, 1.f, "gemm_W_new");
    make_transform(h, ps.E.get(), kf, kf, sel, ch);
    gemm_dev(h, Bt, ps.Ts.get(), ps.ldq2, Hview(h), 0.f, 1.f, "gemm_H_new");
  } else {
    BM_CUDA(cudaMemsetAsync(h.W.get(), 0, ix.m * 4 * sizeof(float), h.stream));
    BM_CUDA(cudaMemsetAsync(h.H.get(), 0, ix.n * 4 * sizeof(float), h.stream));
  }
  ps.ku2 = ps.initialized ? ps.ku : -1;
  std::swap(ps.iUprev, ps.iUprev2);
  ps.ku = k_new;
  return out;
}

// ||Z||_F^2 = <W^T W, H^T H> - 2 alpha <P_Omega(W H^T), R> + alpha^2 ||R||^2
double frob2_dev(bm_ctx& h, double alpha) {
  ProxState& ps = *h.ps;
  double rs[2];
  residual_sums_dev(h, h.r_csr.get(), h.ix.val.get(), h.ix.nnz, rs);  // sum r^2, sum r a
  double tr = 0;
  if (h.k > 0) {
    gram_dev(h, ps.dw, Wview(h), Wview(h), ps.S1.get(), true, "gram_WtW");
    gram_dev(h, ps.dw, Hview(h), Hview(h), ps.S2.get(), true, "gram_HtH");
    std::vector<double> a = to_host(h, ps.S1.get(), (size_t)h.k * h.k);
    std::vector<double> b = to_host(h, ps.S2.get(), (size_t)h.k * h.k);
    for (size_t i = 0; i < a.size(); ++i) tr += a[i] * b[i];
  }
  const double xr = rs[0] + rs[1];  // sum (r + a) r
  return tr - 2.0 * alpha * xr + alpha * alpha * rs[0];
}

void fill_info(bm_prox_info* info, const SvtOut& s, int warm, const LmsvdOut& l, double F) {
  if (!info) return;
  info->k_new = s.k_new;
  info->warm_cols = warm;
  info->lmsvd_iters = l.iters;
  info->n_L = l.nL;
  info->cap_hit = s.cap_hit ? 1 : 0;
  info->pad_ = 0;
  info->eps = s.eps;
  info->F = F;
}

}  // namespace

void prox_create(bm_ctx& h) {
  h.ps = new ProxState();
  ProxState& ps = *h.ps;
  ps.qcap = std::max(h.k_max + 1, h.opt.k_init);
  ps.ldq = round_up4(ps.qcap);
  ps.ldq2 = round_up4(2 * ps.qcap);
  for (auto& b : ps.mbuf) b.alloc((size_t)h.ix.m * ps.ldq2);
  ps.Y.alloc((size_t)h.ix.n * ps.ldq);
  ps.YQ.alloc((size_t)h.ix.n * ps.ldq2);

  ps.Bt.alloc((size_t)h.ix.n * ps.ldq);
  const size_t q2 = (size_t)2 * ps.qcap;
  ps.G.alloc(q2 * q2);
  ps.E.alloc(q2 * q2);
  ps.ev.alloc(q2);
  ps.S1.alloc(q2 * q2);
  ps.S2.alloc(q2 * q2);
  ps.Ts.alloc(q2 * ps.ldq2);
  // SpMM partials: slot rows as wide as the widest slice of a Z^T product
  ensure_pass_scratch(h, std::min(ps.ldq2, kSpmmCols));
  ps.psi = h.opt.psi0;
}

void prox_destroy(bm_ctx& h) {
  delete h.ps;
  h.ps = nullptr;
}

// After bm_set_factors: U_t := orth(W) so the next step warm-starts from the
// new factors (no U_{t-1}, no truncated vector).
void prox_reset(bm_ctx& h) {
  ProxState& ps = *h.ps;
  ps.initialized = false;
  ps.have_u = false;
  ps.ku = 0;
  ps.ku2 = -1;
  ps.psi = h.opt.psi0;
  ps.rank_prev = h.k;
  ps.rank_cur = h.k;
  ps.prev_warm = h.k + 1;
  ps.t = 0;
  bb_reset(h);
}

void prox_step_dev(bm_ctx& h, double alpha, bm_prox_info* info, bool eval_F) {
  ProxState& ps = *h.ps;
  const bm_options& o = h.opt;
  const int m = (int)h.ix.m;
  (void)m;
  // R at X~ in both orders
  residual_dev(h);
  const double frob2 = frob2_dev(h, alpha);
  if (!ps.initialized) {
    // U_t := orth(W) (factors set by the caller)
    ps.ku = h.k > 0 ? orth_dev(h, Wview(h), nullptr, nullptr, nullptr, 1e-12, -1, ps.iUprev, 0, -1) : 0;
    ps.ku2 = -1;
    ps.initialized = true;
    h.bm_changed = true;
  }
  // ---- warm start U^{t,0} (Eq. "rt0"/"rt0-1") in kUw
  const int cap = h.k_max + 1;
  int c = std::min(ps.ku, cap);
  copy_cols_dev(h, mview(h, ps.iUprev, c), 0, mview(h, kUw, c), 0, c);
  if (c < cap) {
    const bool use_W = h.bm_changed || ps.ku2 < 0;
    Tall second = use_W ? Wview(h) : mview(h, ps.iUprev2, ps.ku2);
    if (second.cols > 0) {
      // the second block must not live in X1..X4; W and U_prev buffers do not
      Tall F = mview(h, kUw, c);
      c += orth_dev(h, second, c > 0 ? &F : nullptr, nullptr, nullptr, o.tau, cap - c, kUw, c, -1);
    }
  }
  // ---- safeguard column (Eq. "rt")
  const bool trig = (ps.rank_cur == ps.rank_prev) || (ps.prev_warm <= ps.rank_cur + 1);
  if (trig && c < cap) {
    Tall Uw = mview(h, kUw, c);
    Tall g{ps.mbuf[kB2].get(), h.ix.m, 1, 4};
    Tall ut{ps.mbuf[kLB2].get(), h.ix.m, 1, 4};
    zero_dev(h, g);
    zero_dev(h, ut);
    counter_normal_dev(h, o.seed, kStreamSafeguard + ps.t, h.ix.m, g, 0);
    if (ps.have_u) {
      copy_cols_dev(h, Tall{ps.mbuf[ps.iu].get(), h.ix.m, 1, 4}, 0, ut, 0, 1);
      project_out(h, Uw, ut);
    }
    project_out(h, Uw, g);
    const double nut2 = dot_cols(h, ut, ut);
    if (nut2 > 0) {
      const double ug = dot_cols(h, ut, g);
      vec_axpby(h, ut, -ug / nut2, g, 1.0);
    }
    const double ng = std::sqrt(std::max(dot_cols(h, g, g), 0.0));
    if (ng > 0) {
      if (ps.have_u) {
        vec_axpby(h, g, ps.psi / ng, ut, 1.0);   // col = u_t + psi * g / ||g||
      } else {
        vec_axpby(h, g, 1.0 / ng, ut, 0.0);      // col = g / ||g||
      }
      Tall F = mview(h, kUw, c);
      c += orth_dev(h, ut, c > 0 ? &F : nullptr, nullptr, nullptr, o.tau, -1, kUw, c, -1);
    }
  }
  const int warm = c;
  // ---- LmSVD and the Ritz filter of Algorithm 2
  LmsvdOut l{0, 0, 0, {}};
  int kf = 0;
  if (warm > 0) {
    l = lmsvd_dev(h, warm, alpha);
    if (!l.theta.empty()) {
      const double s1 = std::sqrt(std::max(l.theta[0], 0.0));
      while (kf < l.cols && std::sqrt(std::max(l.theta[kf], 0.0)) > o.ritz_rel * s1) ++kf;
    }
  }
  SvtOut s = svt_refactor_dev(h, kf, h.lambda * alpha, alpha, frob2, kf > 0);
  // ---- safeguard bookkeeping
  if (s.k_new == warm - 1) ps.psi *= 0.5;
  ps.rank_prev = ps.rank_cur;
  ps.rank_cur = s.k_new;
  ps.prev_warm = warm;
  ps.t += 1;
  h.bm_changed = false;
  const double F = (info && eval_F) ? objective_ext(h) : 0.0;
  fill_info(info, s, warm, l, F);
}

void init_step_dev(bm_ctx& h, bm_prox_info* info) {
  ProxState& ps = *h.ps;
  const bm_options& o = h.opt;
  const Index& ix = h.ix;
  set_rank_ext(h, 0);
  BM_CUDA(cudaMemsetAsync(h.W.get(), 0, ix.m * 4 * sizeof(float), h.stream));
  BM_CUDA(cudaMemsetAsync(h.H.get(), 0, ix.n * 4 * sizeof(float), h.stream));
  // Z_{-1} = -grad f(0) = P_Omega(A): residual R = -A, alpha = 1
  negate_values_dev(h, ix.val.get(), h.r_csr.get(), ix.nnz);
  negate_values_dev(h, ix.cval.get(), h.r_csc.get(), ix.nnz);
  const double alpha = 1.0;
  const int k0 = o.k_init;
  Tall G = mview(h, kB2, k0);
  zero_dev(h, G);
  for (int cc = 0; cc < k0; ++cc) counter_normal_dev(h, o.seed, kStreamInitSketch, ix.m, G, cc);
  apply_L(h, G, mview(h, kLB2, k0), alpha);                                        // A_{-1} U~
  const int cq = orth_dev(h, mview(h, kLB2, k0), nullptr, nullptr, nullptr, o.tau, -1, kB0, 0, -1);  // Q
  LmsvdOut l{0, 0, 2, {}};
  int kf = 0;
  if (cq > 0) {
    apply_L(h, mview(h, kB0, cq), mview(h, kLB0, cq), alpha);                      // A Q
    l.nL = 3;
    gram_dev(h, ps.dw, mview(h, kB0, cq), mview(h, kLB0, cq), ps.S1.get(), true, "gram_rr");  // Q^T A Q
    sym_eig_dev(h, ps.dw, ps.S1.get(), cq, ps.ev.get(), ps.E.get(), kEigRelative);
    std::vector<double> cw = to_host(h, ps.ev.get(), cq);
    std::vector<double> E = to_host(h, ps.E.get(), (size_t)cq * cq);
    // (Q^T A Q)^dagger by the eigen-pseudo-inverse (cutoff tau * largest), formed on the host (cq x cq)
    std::vector<double> P((size_t)cq * cq, 0.0);
    for (int j = 0; j < cq; ++j) {
      if (!(cw[j] > o.tau * std::max(cw[0], 1e-300))) continue;
      for (int a = 0; a < cq; ++a)
        for (int b = 0; b < cq; ++b) P[(size_t)a * cq + b] += E[(size_t)a * cq + j] * E[(size_t)b * cq + j] / cw[j];
    }
    BM_CUDA(cudaMemcpyAsync(ps.S2.get(), P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice, h.stream));
    const int cqh = orth_dev(h, mview(h, kLB0, cq), nullptr, nullptr, nullptr, o.tau, -1, kB1, 0, -1);  // Q^
    if (cqh > 0) {
      gram_dev(h, ps.dw, mview(h, kB1, cqh), mview(h, kLB0, cq), ps.S1.get(), true, "gram_rr");  // R^ = Q^^T A Q
      // M = R^ P R^^T  (cqh x cqh)
      small_mm_dev(h, ps.S1.get(), ps.S2.get(), ps.E.get(), cqh, cq, cq, false);
      small_mm_dev(h, ps.E.get(), ps.S1.get(), ps.G.get(), cqh, cq, cqh, true);
      sym_eig_dev(h, ps.dw, ps.G.get(), cqh, ps.ev.get(), ps.E.get(), kEigRelative);
      std::vector<double> s2 = to_host(h, ps.ev.get(), cqh);
      const double s1 = std::sqrt(std::max(s2[0], 0.0));
      std::vector<int> sel;
      std::vector<double> one;
      for (int j = 0; j < cqh; ++j)
        if (std::sqrt(std::max(s2[j], 0.0)) > o.ritz_rel * s1) sel.push_back(j), one.push_back(1.0);
      kf = (int)sel.size();
      if (kf > 0) {
        make_transform(h, ps.E.get(), cqh, cqh, sel, one);
        gemm_dev(h, mview(h, kB1, cqh), ps.Ts.get(), ps.ldq2, mview(h, kU, kf), 0.f, 1.f, "gemm_rr");
      }
    }
  }
  const double frob2 = frob2_dev(h, alpha);
  ps.initialized = true;
  ps.ku = 0;
  ps.ku2 = -1;
  SvtOut s = svt_refactor_dev(h, kf, h.lambda * alpha, alpha, frob2, false);
  ps.ku2 = -1;
  ps.psi = o.psi0;
  ps.rank_prev = 0;
  ps.rank_cur = s.k_new;
  ps.prev_warm = kf;
  ps.t = 0;
  h.bm_changed = false;
  const double F = info ? objective_ext(h) : 0.0;
  fill_info(info, s, kf, l, F);
}

}  // namespace bm

namespace bm {

void tuning_spmm_dev(bm_ctx& h, bool csr) {
  ProxState& ps = *h.ps;
  const int q = std::max(1, std::min(ps.qcap, h.k + 1));
  const Tall mside = mview(h, kX1, q);
  const Tall nside = nview(h, ps.Y, q);
  if (csr) spmm_dev(h, true, h.r_csr.get(), nside, mside, -1.f);
  else spmm_dev(h, false, h.r_csc.get(), mside, nside, -1.f);
}

}  // namespace bm

namespace bm {

// Serialised PG-step state: the scalars of the warm start and safeguard
// (Eq. "rt0", "rt0-1", "rt": ranks, psi_t, t) followed by U_t (m x ku),
// U_{t-1} (m x ku2) and the truncated vector u (m, if present), FP32, rows
// packed without padding.
struct ProxSnap {
  int32_t initialized, ku, ku2, have_u, rank_prev, rank_cur, prev_warm, t;
  double psi;
};

size_t prox_state_bytes(const bm_ctx& h) {
  const ProxState& ps = *h.ps;
  const size_t m = (size_t)h.ix.m;
  return sizeof(ProxSnap) + m * sizeof(float) * ((size_t)ps.ku + (size_t)std::max(ps.ku2, 0) + (ps.have_u ? 1 : 0));
}

namespace {
void pack_cols(bm_ctx& h, uint8_t*& p, const float* src, int ld, int cols) {
  if (cols <= 0 || h.ix.m == 0) return;
  BM_CUDA(cudaMemcpy2DAsync(p, cols * sizeof(float), src, ld * sizeof(float), cols * sizeof(float), h.ix.m,
                            cudaMemcpyDeviceToHost, h.stream));
  p += (size_t)h.ix.m * cols * sizeof(float);
}
void unpack_cols(bm_ctx& h, const uint8_t*& p, float* dst, int ld, int cols) {
  if (cols <= 0 || h.ix.m == 0) return;
  BM_CUDA(cudaMemcpy2DAsync(dst, ld * sizeof(float), p, cols * sizeof(float), cols * sizeof(float), h.ix.m,
                            cudaMemcpyHostToDevice, h.stream));
  p += (size_t)h.ix.m * cols * sizeof(float);
}
}  // namespace

void prox_state_save(bm_ctx& h, uint8_t* out) {
  ProxState& ps = *h.ps;
  ProxSnap s{ps.initialized ? 1 : 0, ps.ku, ps.ku2, ps.have_u ? 1 : 0, ps.rank_prev, ps.rank_cur, ps.prev_warm, ps.t,
             ps.psi};
  std::memcpy(out, &s, sizeof(s));
  uint8_t* p = out + sizeof(s);
  pack_cols(h, p, ps.mbuf[ps.iUprev].get(), ps.ldq2, ps.ku);
  pack_cols(h, p, ps.mbuf[ps.iUprev2].get(), ps.ldq2, std::max(ps.ku2, 0));
  if (ps.have_u) pack_cols(h, p, ps.mbuf[ps.iu].get(), 4, 1);
  BM_CUDA(cudaStreamSynchronize(h.stream));
}

void prox_state_load(bm_ctx& h, const uint8_t* in, size_t len) {
  ProxState& ps = *h.ps;
  BM_REQUIRE(len >= sizeof(ProxSnap), BM_ERR_INVALID, "bm_set_state: truncated PG state");
  ProxSnap s;
  std::memcpy(&s, in, sizeof(s));
  const int cap = 2 * ps.qcap;
  BM_REQUIRE(s.ku >= 0 && s.ku <= cap && s.ku2 >= -1 && s.ku2 <= cap && s.prev_warm >= 0 && s.t >= 0 &&
                 std::isfinite(s.psi),
             BM_ERR_INVALID, "bm_set_state: invalid PG state");
  const size_t m = (size_t)h.ix.m;
  const size_t need =
      sizeof(ProxSnap) + m * sizeof(float) * ((size_t)s.ku + (size_t)std::max(s.ku2, 0) + (s.have_u ? 1 : 0));
  BM_REQUIRE(len == need, BM_ERR_INVALID, "bm_set_state: PG state size mismatch");
  ps.initialized = s.initialized != 0;
  ps.ku = s.ku;
  ps.ku2 = s.ku2;
  ps.have_u = s.have_u != 0;
  ps.rank_prev = s.rank_prev;
  ps.rank_cur = s.rank_cur;
  ps.prev_warm = s.prev_warm;
  ps.t = s.t;
  ps.psi = s.psi;
  ps.iUprev = kUprevA;
  ps.iUprev2 = kUprevB;
  ps.iu = kUvec;
  const uint8_t* p = in + sizeof(ProxSnap);
  unpack_cols(h, p, ps.mbuf[ps.iUprev].get(), ps.ldq2, ps.ku);
  unpack_cols(h, p, ps.mbuf[ps.iUprev2].get(), ps.ldq2, std::max(ps.ku2, 0));
  if (ps.have_u) {
    BM_CUDA(cudaMemsetAsync(ps.mbuf[ps.iu].get(), 0, m * 4 * sizeof(float), h.stream));
    unpack_cols(h, p, ps.mbuf[ps.iu].get(), 4, 1);
  }
  BM_CUDA(cudaStreamSynchronize(h.stream));
}

}  // namespace bm
