// Batched BM phase over many solves (one handle each).
//
// Every sparse pass of an epoch (loss/gradient CSR and CSC, exact line
// search) runs as one launch over the concatenated segment lists of all
// problems with the same row width; the dense reductions, the Polak-Ribiere+
// direction, the quartic line search and the update run as batched kernels
// with one thread (or one block slice) per problem, reading their scalars from
// device memory.  An epoch therefore needs no host round trip, is captured
// once into a CUDA graph and replayed for every epoch while the problems'
// ranks and the buffers the graph captured stay the same.
#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <cuda_bf16.h>

#include "dense.cuh"
#include "pipe.cuh"
#include "quartic.cuh"

namespace bm {
void ensure_bf16(bm_ctx& h);
}

namespace {
using namespace bm;

constexpr int kSlabs = 64;     // partial-sum slabs per problem
constexpr int kScal = 16;      // device scalars per problem
enum { S_F = 0, S_FENTRY, S_FIRST, S_BETA, S_GGPREV, S_STEP, S_FLAST, S_F_F, S_LS0, S_LS1, S_LS2, S_LS3 };
enum { P_NW = 0, P_GG, P_GP, P_DOG, P_GD, P_DD };  // partial-sum columns

struct DenseP {
  float *W, *H, *gW, *gH, *DW, *DH, *gWp, *gHp;
  int64_t mW, nH;          // floats on the W side (m*ld) and H side (n*ld)
  double lam;
  const double* fseg_csr;  // per-segment 1/2 sum r^2 of the CSR pass
  int64_t nseg_csr;
  const double* fseg_ls;   // per-segment line-search sums (4 each)
  int64_t nseg_ls;
  uint16_t *Wb, *Hb, *DHb; // BF16 copies (nullable)
  int ld, ldb;
};

struct FixP {
  const int32_t *mrow, *mfirst, *mcount;
  int64_t nmulti;
  const float* partial;
  const float* own;
  int ld;
  float lam;
  float* out;
};

__device__ __forceinline__ int find_problem(const int64_t* prefix, int count, int64_t x) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_fix_batch(const FixP* __restrict__ fp, const int64_t* __restrict__ prefix, int count) {
  const int64_t total = prefix[count];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int p = find_problem(prefix, count, t);
    const FixP& f = fp[p];
    const int64_t u = t - prefix[p];
    const int64_t q = u / f.ld;
    const int c = (int)(u - q * f.ld);
    float s = 0.f;
    for (int k = 0; k < f.mcount[q]; ++k) s += f.partial[((int64_t)f.mfirst[q] + k) * f.ld + c];
    const int64_t o = (int64_t)f.mrow[q] * f.ld + c;
    f.out[o] = fmaf(f.lam, f.own[o], s);
  }
}

// Slab partials of the dense dot products of one problem (blockIdx.y).
// phase 0: |W|^2+|H|^2, |g|^2, <g, g_prev>, <D, g>;  phase 1: <g, D>, |D|^2
__global__ void __launch_bounds__(256) k_dots_batch(const DenseP* __restrict__ dp, int phase,
                                                     double* __restrict__ part) {
  __shared__ double sh[4][256];
  const DenseP& d = dp[blockIdx.y];
  const int64_t n4 = (d.mW + d.nH) / 4, mW4 = d.mW / 4;
  const int64_t per = (n4 + kSlabs - 1) / kSlabs;
  const int64_t b0 = blockIdx.x * per, b1 = min(n4, b0 + per);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const bool w = i < mW4;
    const int64_t o = w ? i : i - mW4;
    const float4 x = reinterpret_cast<const float4*>(w ? d.W : d.H)[o];
    const float4 g = reinterpret_cast<const float4*>(w ? d.gW : d.gH)[o];
    const float4 D = reinterpret_cast<const float4*>(w ? d.DW : d.DH)[o];
    if (phase == 0) {
      const float4 gp = reinterpret_cast<const float4*>(w ? d.gWp : d.gHp)[o];
      a0 += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
      a1 += g.x * g.x + g.y * g.y + g.z * g.z + g.w * g.w;
      a2 += g.x * gp.x + g.y * gp.y + g.z * gp.z + g.w * gp.w;
      a3 += D.x * g.x + D.y * g.y + D.z * g.z + D.w * g.w;
    } else {
      a0 += g.x * D.x + g.y * D.y + g.z * D.z + g.w * D.w;
      a1 += D.x * D.x + D.y * D.y + D.z * D.z + D.w * D.w;
    }
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  sh[3][threadIdx.x] = a3;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) {
    const int t = (int)threadIdx.x;
    const int col = phase == 0 ? t : (t < 2 ? P_GD + t : -1);
    if (col >= 0) part[((int64_t)blockIdx.y * kSlabs + blockIdx.x) * 8 + col] = sh[threadIdx.x][0];
  }
}

// Per-problem sums of segment partials (one block per problem): the CSR loss
// (phase 0) or the four line-search sums (phase 1).
__global__ void k_seg_sums_batch(const DenseP* __restrict__ dp, int phase, double* __restrict__ scal) {
  __shared__ double sh[4][256];
  const DenseP& d = dp[blockIdx.x];
  double a[4] = {0, 0, 0, 0};
  const int64_t nseg = phase == 0 ? d.nseg_csr : d.nseg_ls;
  for (int64_t i = threadIdx.x; i < nseg; i += blockDim.x) {
    if (phase == 0) a[0] += d.fseg_csr[i];
    else for (int q = 0; q < 4; ++q) a[q] += d.fseg_ls[i * 4 + q];
  }
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* s = scal + (int64_t)blockIdx.x * kScal;
    if (phase == 0) s[S_F_F] = sh[0][0];
    else for (int q = 0; q < 4; ++q) s[S_LS0 + q] = sh[q][0];
  }
}

__device__ double sum_part(const double* part, int p, int col) {
  double s = 0;
  for (int b = 0; b < kSlabs; ++b) s += part[((int64_t)p * kSlabs + b) * 8 + col];
  return s;
}

// Objective, Polak-Ribiere+ coefficient with the descent safeguard.
__global__ void k_ctrl_dir(const DenseP* __restrict__ dp, const double* __restrict__ part, double* __restrict__ scal,
                           int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  double* s = scal + (int64_t)p * kScal;
  const double nw = sum_part(part, p, P_NW), gg = sum_part(part, p, P_GG);
  const double gp = sum_part(part, p, P_GP), dog = sum_part(part, p, P_DOG);
  const double F = s[S_F_F] + 0.5 * dp[p].lam * nw;
  s[S_F] = F;
  double beta = 0.0;
  if (s[S_FIRST] != 0.0) {
    s[S_FENTRY] = F;
  } else if (s[S_GGPREV] > 0) {
    beta = fmax(0.0, (gg - gp) / s[S_GGPREV]);
    if (beta > 0 && -gg + beta * dog >= 0) beta = 0.0;  // not a descent direction: restart
  }
  s[S_BETA] = beta;
  s[S_GGPREV] = gg;
  s[S_FIRST] = 0.0;
}

// D = -g + beta D (beta per problem)
__global__ void k_dir_batch(const DenseP* __restrict__ dp, const double* __restrict__ scal) {
  const DenseP& d = dp[blockIdx.y];
  const float beta = (float)scal[(int64_t)blockIdx.y * kScal + S_BETA];
  const int64_t n4 = (d.mW + d.nH) / 4, mW4 = d.mW / 4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const bool w = i < mW4;
    const int64_t o = w ? i : i - mW4;
    float4* D = reinterpret_cast<float4*>(w ? d.DW : d.DH) + o;
    const float4 g = reinterpret_cast<const float4*>(w ? d.gW : d.gH)[o];
    float4 v = beta != 0.f ? *D : make_float4(0.f, 0.f, 0.f, 0.f);
    v.x = fmaf(beta, v.x, -g.x);
    v.y = fmaf(beta, v.y, -g.y);
    v.z = fmaf(beta, v.z, -g.z);
    v.w = fmaf(beta, v.w, -g.w);
    *D = v;
  }
}

__global__ void k_ctrl_step(const DenseP* __restrict__ dp, const double* __restrict__ part, double* __restrict__ scal,
                            int count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  double* s = scal + (int64_t)p * kScal;
  const double lam = dp[p].lam;
  const double gd = sum_part(part, p, P_GD), dd = sum_part(part, p, P_DD);
  double c[5];
  c[0] = s[S_F];
  c[1] = gd;  // phi'(0) = <grad F, D>
  c[2] = 0.5 * s[S_LS1] + 0.5 * lam * dd;
  c[3] = s[S_LS2];
  c[4] = 0.5 * s[S_LS3];
  const double st = quartic_argmin_d(c);
  s[S_STEP] = st;
  s[S_FLAST] = st > 0 ? poly4d(c, st) : c[0];
}

// W += s DW, H += s DH; g_prev = g
__global__ void k_update_batch(const DenseP* __restrict__ dp, const double* __restrict__ scal) {
  const DenseP& d = dp[blockIdx.y];
  const float st = (float)scal[(int64_t)blockIdx.y * kScal + S_STEP];
  const int64_t n4 = (d.mW + d.nH) / 4, mW4 = d.mW / 4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const bool w = i < mW4;
    const int64_t o = w ? i : i - mW4;
    float4* X = reinterpret_cast<float4*>(w ? d.W : d.H) + o;
    const float4 D = reinterpret_cast<const float4*>(w ? d.DW : d.DH)[o];
    float4 x = *X;
    x.x = fmaf(st, D.x, x.x);
    x.y = fmaf(st, D.y, x.y);
    x.z = fmaf(st, D.z, x.z);
    x.w = fmaf(st, D.w, x.w);
    *X = x;
    reinterpret_cast<float4*>(w ? d.gWp : d.gHp)[o] = reinterpret_cast<const float4*>(w ? d.gW : d.gH)[o];
  }
}

// BF16 copies: which = 0: W and H; which = 1: DH
__global__ void k_bf16_batch(const DenseP* __restrict__ dp, int which) {
  const DenseP& d = dp[blockIdx.y];
  if (d.ldb == 0) return;  // this problem gathers FP32
  const int64_t m = d.mW / d.ld, n = d.nH / d.ld;
  const int64_t rows = which == 0 ? m + n : n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * d.ldb;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / d.ldb;
    const int c = (int)(t - r * d.ldb);
    const float* src;
    uint16_t* dst;
    int64_t rr;
    if (which == 1) {
      src = d.DH; dst = d.DHb; rr = r;
    } else if (r < m) {
      src = d.W; dst = d.Wb; rr = r;
    } else {
      src = d.H; dst = d.Hb; rr = r - m;
    }
    const float x = c < d.ld ? src[rr * d.ld + c] : 0.f;
    dst[rr * d.ldb + c] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
  }
}

struct Group {  // problems that share a row width and gather type (one batched launch per pass)
  int nchunk;
  bool bf;
  std::vector<int> members;
  DevBuf<PipeArgs> a_csr, a_csc, a_ls;
  DevBuf<int64_t> pre_csr, pre_csc, pre_ls;
  int64_t tot_csr = 0, tot_csc = 0, tot_ls = 0;
  int64_t nnz = 0;                   // entries of the members (each pass visits all of them)
};

}  // namespace

struct bm_batch_ctx {
  std::vector<bm_ctx*> hs;
  int count = 0;
  cudaStream_t stream = nullptr;
  bool bf = false;
  std::vector<uintptr_t> sig;        // ranks and device pointers the tables / graph were built for
  std::vector<std::unique_ptr<Group>> groups;
  DevBuf<DenseP> dense;
  DevBuf<FixP> fix_csr, fix_csc;
  DevBuf<int64_t> fpre_csr, fpre_csc;
  int64_t ftot_csr = 0, ftot_csc = 0;
  int nfix_csr = 0, nfix_csc = 0;
  DevBuf<double> part, scal;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bm::SpmmCombiner* comb = nullptr;  // shared SpMM launches of bm_batch_prox_step
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

void build_tables(bm_batch_ctx& b) {
  b.groups.clear();
  std::vector<DenseP> dps(b.count);
  std::vector<FixP> fc, fh;
  std::vector<int64_t> fpc{0}, fph{0};
  for (int p = 0; p < b.count; ++p) {
    bm_ctx& h = *b.hs[p];
    const Index& ix = h.ix;
    DenseP& d = dps[p];
    d.W = h.W.get(); d.H = h.H.get(); d.gW = h.gW.get(); d.gH = h.gH.get();
    d.DW = h.DW.get(); d.DH = h.DH.get(); d.gWp = h.gWp.get(); d.gHp = h.gHp.get();
    d.mW = ix.m * h.ld;
    d.nH = ix.n * h.ld;
    d.lam = h.lambda;
    d.fseg_csr = h.sc.fseg.get();
    d.nseg_csr = pass_segs(ix, kPassGradCsr).nseg;
    d.fseg_ls = h.sc.fseg.get();
    d.nseg_ls = pass_segs(ix, kPassLsCsr).nseg;
    d.ld = h.ld;
    d.ldb = ((h.ld + 7) / 8) * 8;
    d.Wb = h.Wb.get(); d.Hb = h.Hb.get(); d.DHb = h.DHb.get();
    const int nch = h.ld / 4;
    const bool pbf = h.bf_active();
    if (!pbf) d.ldb = 0;   // no BF16 copies for this problem
    Group* gr = nullptr;
    for (auto& g : b.groups) if (g->nchunk == nch && g->bf == pbf) gr = g.get();
    if (!gr) {
      b.groups.emplace_back(new Group());
      gr = b.groups.back().get();
      gr->nchunk = nch;
      gr->bf = pbf;
    }
    gr->members.push_back(p);
    gr->nnz += ix.nnz;
    for (int pass = 0; pass < 2; ++pass) {
      const Segs& sg = pass_segs(ix, pass == 0 ? kPassGradCsr : kPassGradCsc);
      if (!sg.nmulti) continue;
      FixP f{sg.mrow.get(), sg.mfirst.get(), sg.mcount.get(), sg.nmulti, h.sc.partial.get(),
             pass == 0 ? h.W.get() : h.H.get(), h.ld, (float)h.lambda, pass == 0 ? h.gW.get() : h.gH.get()};
      // the CSR and CSC passes of a handle share its partial buffer, so their
      // fix-ups run after the respective pass
      (pass == 0 ? fc : fh).push_back(f);
      (pass == 0 ? fpc : fph).push_back((pass == 0 ? fpc : fph).back() + sg.nmulti * h.ld);
    }
  }
  for (auto& gp : b.groups) {
    Group& g = *gp;
    std::vector<PipeArgs> ac, ah, al;
    std::vector<int64_t> pc{0}, ph{0}, pl{0};
    for (int p : g.members) {
      bm_ctx& h = *b.hs[p];
      const Index& ix = h.ix;
      for (int pass = 0; pass < 3; ++pass) {
        const Segs& sg = pass_segs(ix, pass == 0 ? kPassGradCsr : (pass == 1 ? kPassGradCsc : kPassLsCsr));
        PipeArgs a{};
        a.seg_row = sg.row.get();
        a.seg_beg = sg.beg.get();
        a.seg_end = sg.end.get();
        a.seg_slot = sg.slot.get();
        a.nseg = sg.nseg;
        a.idx = pass == 1 ? ix.row.get() : ix.col.get();
        a.ld = h.ld;
        a.nchunk = h.ld / 4;
        a.ldb = ((h.ld + 7) / 8) * 8;
        a.lam = (float)h.lambda;
        a.partial = h.sc.partial.get();
        a.ld_part = h.ld;
        a.ld_out = h.ld;
        if (pass == 0) {            // loss/gradient, CSR
          a.scal = ix.val.get(); a.o0 = h.W.get(); a.g0 = h.H.get(); a.g0b = h.Hb.get();
          a.scal8 = ix.codec ? ix.val8.get() : nullptr; a.scal_off = ix.code_off;
          a.out = h.gW.get(); a.fseg = h.sc.fseg.get(); a.r_out = h.r_csr.get();
          ac.push_back(a);
          pc.push_back(pc.back() + sg.nseg);
        } else if (pass == 1) {     // loss/gradient, CSC
          a.scal = ix.cval.get(); a.o0 = h.H.get(); a.g0 = h.W.get(); a.g0b = h.Wb.get();
          a.scal8 = ix.codec ? ix.cval8.get() : nullptr; a.scal_off = ix.code_off;
          a.out = h.gH.get();
          ah.push_back(a);
          ph.push_back(ph.back() + sg.nseg);
        } else {                    // line search, CSR
          a.scal = h.r_csr.get(); a.o0 = h.W.get(); a.o1 = h.DW.get(); a.g0 = h.H.get(); a.g1 = h.DH.get();
          a.g0b = h.Hb.get(); a.g1b = h.DHb.get(); a.fseg = h.sc.fseg.get();
          al.push_back(a);
          pl.push_back(pl.back() + sg.nseg);
        }
      }
    }
    const size_t np = g.members.size();
    g.a_csr.alloc(np); g.a_csc.alloc(np); g.a_ls.alloc(np);
    g.pre_csr.alloc(np + 1); g.pre_csc.alloc(np + 1); g.pre_ls.alloc(np + 1);
    BM_CUDA(cudaMemcpyAsync(g.a_csr.get(), ac.data(), np * sizeof(PipeArgs), cudaMemcpyHostToDevice, b.stream));
    BM_CUDA(cudaMemcpyAsync(g.a_csc.get(), ah.data(), np * sizeof(PipeArgs), cudaMemcpyHostToDevice, b.stream));
    BM_CUDA(cudaMemcpyAsync(g.a_ls.get(), al.data(), np * sizeof(PipeArgs), cudaMemcpyHostToDevice, b.stream));
    BM_CUDA(cudaMemcpyAsync(g.pre_csr.get(), pc.data(), (np + 1) * 8, cudaMemcpyHostToDevice, b.stream));
    BM_CUDA(cudaMemcpyAsync(g.pre_csc.get(), ph.data(), (np + 1) * 8, cudaMemcpyHostToDevice, b.stream));
    BM_CUDA(cudaMemcpyAsync(g.pre_ls.get(), pl.data(), (np + 1) * 8, cudaMemcpyHostToDevice, b.stream));
    g.tot_csr = pc.back();
    g.tot_csc = ph.back();
    g.tot_ls = pl.back();
    BM_CUDA(cudaStreamSynchronize(b.stream));
  }
  b.dense.alloc(b.count);
  BM_CUDA(cudaMemcpyAsync(b.dense.get(), dps.data(), b.count * sizeof(DenseP), cudaMemcpyHostToDevice, b.stream));
  b.fix_csr.alloc(std::max<size_t>(1, fc.size()));
  b.fix_csc.alloc(std::max<size_t>(1, fh.size()));
  b.fpre_csr.alloc(fpc.size());
  b.fpre_csc.alloc(fph.size());
  if (!fc.empty()) BM_CUDA(cudaMemcpyAsync(b.fix_csr.get(), fc.data(), fc.size() * sizeof(FixP), cudaMemcpyHostToDevice, b.stream));
  if (!fh.empty()) BM_CUDA(cudaMemcpyAsync(b.fix_csc.get(), fh.data(), fh.size() * sizeof(FixP), cudaMemcpyHostToDevice, b.stream));
  BM_CUDA(cudaMemcpyAsync(b.fpre_csr.get(), fpc.data(), fpc.size() * 8, cudaMemcpyHostToDevice, b.stream));
  BM_CUDA(cudaMemcpyAsync(b.fpre_csc.get(), fph.data(), fph.size() * 8, cudaMemcpyHostToDevice, b.stream));
  b.ftot_csr = fpc.back();
  b.ftot_csc = fph.back();
  b.nfix_csr = (int)fc.size();
  b.nfix_csc = (int)fh.size();
  b.part.alloc((size_t)b.count * kSlabs * 8);
  b.scal.alloc((size_t)b.count * kScal);
  BM_CUDA(cudaStreamSynchronize(b.stream));
}

// What the tables and the captured graph of one handle depend on: its rank,
// precision state, sizes and every device pointer build_tables() records.
void append_signature(const bm_ctx& h, std::vector<uintptr_t>& sig) {
  const Index& ix = h.ix;
  const uintptr_t v[] = {(uintptr_t)h.k, (uintptr_t)h.ld, (uintptr_t)h.bf_active(), (uintptr_t)ix.m,
                         (uintptr_t)ix.n, (uintptr_t)ix.nnz, (uintptr_t)ix.codec,
                         (uintptr_t)h.W.get(), (uintptr_t)h.H.get(), (uintptr_t)h.gW.get(), (uintptr_t)h.gH.get(),
                         (uintptr_t)h.DW.get(), (uintptr_t)h.DH.get(), (uintptr_t)h.gWp.get(),
                         (uintptr_t)h.gHp.get(), (uintptr_t)h.Wb.get(), (uintptr_t)h.Hb.get(),
                         (uintptr_t)h.DHb.get(), (uintptr_t)h.r_csr.get(), (uintptr_t)h.sc.fseg.get(),
                         (uintptr_t)h.sc.partial.get(), (uintptr_t)ix.col.get(), (uintptr_t)ix.row.get(),
                         (uintptr_t)ix.val.get(), (uintptr_t)ix.cval.get(), (uintptr_t)ix.val8.get(),
                         (uintptr_t)ix.cval8.get()};
  sig.insert(sig.end(), std::begin(v), std::end(v));
  for (int kind : {kPassGradCsr, kPassGradCsc, kPassLsCsr}) {
    const Segs& sg = pass_segs(ix, kind);
    const uintptr_t w[] = {(uintptr_t)sg.nseg, (uintptr_t)sg.nmulti, (uintptr_t)sg.row.get(),
                           (uintptr_t)sg.beg.get(), (uintptr_t)sg.end.get(), (uintptr_t)sg.slot.get(),
                           (uintptr_t)sg.mrow.get(), (uintptr_t)sg.mfirst.get(), (uintptr_t)sg.mcount.get()};
    sig.insert(sig.end(), std::begin(w), std::end(w));
  }
}

int grid_for_work(int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)num_sms() * 8));
}

// One epoch for every problem, launches only (captured into the graph).
void enqueue_epoch(bm_batch_ctx& b) {
  cudaStream_t st = b.stream;
  const dim3 gdense(std::max(1, num_sms() * 4 / std::max(1, b.count)), b.count);
  if (b.bf) {
    k_bf16_batch<<<gdense, 256, 0, st>>>(b.dense.get(), 0);
    BM_CHECK_LAUNCH();
  }
  for (auto& g : b.groups)
    launch_direct_batch<0>(g->a_csr.get(), g->pre_csr.get(), (int)g->members.size(), g->tot_csr, g->nchunk, g->bf,
                           long_segments(g->nnz, g->tot_csr), st);
  BM_CHECK_LAUNCH();
  if (b.nfix_csr) {
    k_fix_batch<<<grid_for_work(b.ftot_csr), 256, 0, st>>>(b.fix_csr.get(), b.fpre_csr.get(), b.nfix_csr);
    BM_CHECK_LAUNCH();
  }
  k_seg_sums_batch<<<b.count, 256, 0, st>>>(b.dense.get(), 0, b.scal.get());
  BM_CHECK_LAUNCH();
  for (auto& g : b.groups)
    launch_direct_batch<0>(g->a_csc.get(), g->pre_csc.get(), (int)g->members.size(), g->tot_csc, g->nchunk, g->bf,
                           long_segments(g->nnz, g->tot_csc), st);
  BM_CHECK_LAUNCH();
  if (b.nfix_csc) {
    k_fix_batch<<<grid_for_work(b.ftot_csc), 256, 0, st>>>(b.fix_csc.get(), b.fpre_csc.get(), b.nfix_csc);
    BM_CHECK_LAUNCH();
  }
  k_dots_batch<<<dim3(kSlabs, b.count), 256, 0, st>>>(b.dense.get(), 0, b.part.get());
  BM_CHECK_LAUNCH();
  k_ctrl_dir<<<(b.count + 127) / 128, 128, 0, st>>>(b.dense.get(), b.part.get(), b.scal.get(), b.count);
  BM_CHECK_LAUNCH();
  k_dir_batch<<<gdense, 256, 0, st>>>(b.dense.get(), b.scal.get());
  BM_CHECK_LAUNCH();
  if (b.bf) {
    k_bf16_batch<<<gdense, 256, 0, st>>>(b.dense.get(), 1);
    BM_CHECK_LAUNCH();
  }
  for (auto& g : b.groups)
    launch_direct_batch<2>(g->a_ls.get(), g->pre_ls.get(), (int)g->members.size(), g->tot_ls, g->nchunk, g->bf,
                           long_segments(g->nnz, g->tot_ls), st);
  BM_CHECK_LAUNCH();
  k_seg_sums_batch<<<b.count, 256, 0, st>>>(b.dense.get(), 1, b.scal.get());
  BM_CHECK_LAUNCH();
  k_dots_batch<<<dim3(kSlabs, b.count), 256, 0, st>>>(b.dense.get(), 1, b.part.get());
  BM_CHECK_LAUNCH();
  k_ctrl_step<<<(b.count + 127) / 128, 128, 0, st>>>(b.dense.get(), b.part.get(), b.scal.get(), b.count);
  BM_CHECK_LAUNCH();
  k_update_batch<<<gdense, 256, 0, st>>>(b.dense.get(), b.scal.get());
  BM_CHECK_LAUNCH();
}

template <class Fn>
bm_status batch_guarded(bm_batch_ctx* b, Fn&& fn) {
  try {
    fn();
    return BM_OK;
  } catch (const Error& e) {
    (b ? b->err : g_batch_error) = e.msg;
    return e.code;
  } catch (...) {
    (b ? b->err : g_batch_error) = "unexpected exception";
    return BM_ERR_CUDA;
  }
}

void drop_graph(bm_batch_ctx& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b.exec = nullptr;
  b.graph = nullptr;
}

}  // namespace

extern "C" {

bm_status bm_batch_create(bm_handle* hs, int32_t count, bm_batch* out) {
  if (!out) return BM_ERR_INVALID;
  *out = nullptr;
  bm_batch_ctx* b = nullptr;
  bm_status st = batch_guarded(nullptr, [&] {
    BM_REQUIRE(hs && count >= 1, BM_ERR_INVALID, "bm_batch_create: need at least one handle");
    b = new bm_batch_ctx();
    b->count = count;
    const int prec = hs[0] ? hs[0]->opt.precision : 0;
    for (int p = 0; p < count; ++p) {
      BM_REQUIRE(hs[p], BM_ERR_INVALID, "bm_batch_create: NULL handle");
      BM_REQUIRE(hs[p]->device == hs[0]->device, BM_ERR_INVALID, "bm_batch_create: handles on different devices");
      BM_REQUIRE(hs[p]->opt.precision == prec, BM_ERR_INVALID, "bm_batch_create: mixed precision modes");
      for (int q = 0; q < p; ++q)
        BM_REQUIRE(hs[q] != hs[p], BM_ERR_INVALID, "bm_batch_create: a handle appears twice");
      b->hs.push_back(hs[p]);
    }
    b->bf = prec == 1;
    BM_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  });
  if (st != BM_OK) {
    if (b) bm_batch_destroy(b);
    return st;
  }
  *out = b;
  return BM_OK;
}

void bm_batch_destroy(bm_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(*b);
  spmm_combiner_destroy(b->comb);
  cudaStream_t s = b->stream;
  delete b;
  if (s) cudaStreamDestroy(s);
}

const char* bm_batch_last_error(bm_batch b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

bm_status bm_batch_bm_phase(bm_batch b, int32_t epochs, double* F) {
  if (!b) return BM_ERR_INVALID;
  return batch_guarded(b, [&] {
    BM_REQUIRE(epochs >= 0, BM_ERR_INVALID, "bm_batch_bm_phase: epochs must be >= 0");
    std::vector<uintptr_t> sig;
    for (int p = 0; p < b->count; ++p) {
      bm_ctx& h = *b->hs[p];
      BM_CUDA(cudaStreamSynchronize(h.stream));
      BM_REQUIRE(h.k >= 1, BM_ERR_INVALID, "bm_batch_bm_phase: every handle needs rank >= 1 (run bm_init)");
      if (b->bf) {
        BM_REQUIRE(h.Wb.get() && h.DHb.get(), BM_ERR_INVALID, "bm_batch_bm_phase: BF16 copies missing");
      }
      append_signature(h, sig);
    }
    // rebuild the tables and the graph when a rank or any buffer they captured changed
    if (sig != b->sig || !b->exec) {
      drop_graph(*b);
      build_tables(*b);
      b->sig = sig;
      BM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      try {
        enqueue_epoch(*b);
      } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      BM_CUDA(cudaStreamEndCapture(b->stream, &b->graph));
      BM_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    // first epoch of the phase: steepest descent
    std::vector<double> init((size_t)b->count * kScal, 0.0);
    for (int p = 0; p < b->count; ++p) init[(size_t)p * kScal + S_FIRST] = 1.0;
    BM_CUDA(cudaMemcpyAsync(b->scal.get(), init.data(), init.size() * sizeof(double), cudaMemcpyHostToDevice,
                            b->stream));
    for (int e = 0; e < epochs; ++e) BM_CUDA(cudaGraphLaunch(b->exec, b->stream));
    std::vector<double> sc((size_t)b->count * kScal);
    BM_CUDA(cudaMemcpyAsync(sc.data(), b->scal.get(), sc.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BM_CUDA(cudaStreamSynchronize(b->stream));
    for (int p = 0; p < b->count; ++p) {
      bm_ctx& h = *b->hs[p];
      if (epochs > 0) {
        h.bm_changed = true;
        h.bf_dirty = true;
      }
      const double Fp = epochs > 0 ? sc[(size_t)p * kScal + S_FLAST] : NAN;
      BM_REQUIRE(epochs == 0 || std::isfinite(Fp), BM_ERR_NUMERIC, "bm_batch_bm_phase: objective is not finite");
      if (F) F[p] = Fp;
    }
  });
}

bm_status bm_batch_prox_step(bm_batch b, double alpha, bm_prox_info* info, bm_status* status) {
  if (!b) return BM_ERR_INVALID;
  return batch_guarded(b, [&] {
    for (int p = 0; p < b->count; ++p)
      BM_REQUIRE(!b->hs[p]->comb, BM_ERR_INVALID, "bm_batch_prox_step: a handle is already in a batched PG step");
    if (!b->comb) b->comb = spmm_combiner_create(b->count);
    int dev = 0;
    BM_CUDA(cudaGetDevice(&dev));
    std::vector<bm_status> st(b->count, BM_OK);
    std::vector<bm_prox_info> tmp(b->count);
    spmm_combiner_begin(b->comb, b->count);
    {
      // the handles leave the batched step however it ends
      struct Release {
        bm_batch_ctx* b;
        ~Release() {
          for (int p = 0; p < b->count; ++p) b->hs[p]->comb = nullptr;
        }
      } release{b};
      for (int p = 0; p < b->count; ++p) b->hs[p]->comb = b->comb;
      // one host thread per handle: each runs its PG step on its own stream,
      // the residual SpMMs meet in the combiner
      std::vector<std::thread> th;
      th.reserve(b->count);
      for (int p = 0; p < b->count; ++p) {
        try {
          th.emplace_back([&, p] {
            cudaSetDevice(dev);
            st[p] = bm_prox_step(b->hs[p], alpha, info ? &info[p] : &tmp[p]);
            spmm_combiner_leave(b->comb);
          });
        } catch (...) {
          // no thread for this handle: it leaves at once, so that the others
          // do not wait for its products
          b->hs[p]->err = "bm_batch_prox_step: could not start a host thread";
          st[p] = BM_ERR_INVALID;
          spmm_combiner_leave(b->comb);
        }
      }
      for (auto& t : th) t.join();
    }
    if (status)
      for (int p = 0; p < b->count; ++p) status[p] = st[p];
    for (int p = 0; p < b->count; ++p)
      if (st[p] != BM_OK)
        throw Error{st[p], "bm_batch_prox_step: handle " + std::to_string(p) + ": " + b->hs[p]->err};
  });
}

bm_status bm_batch_stats(bm_batch b, int64_t* spmm_products, int64_t* spmm_launches) {
  if (!b) return BM_ERR_INVALID;
  if (spmm_products) *spmm_products = spmm_combiner_products(b->comb);
  if (spmm_launches) *spmm_launches = spmm_combiner_launches(b->comb);
  return BM_OK;
}

}  // extern "C"
