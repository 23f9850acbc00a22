// Sparse passes over a segment split (one warp per segment).
//
// A warp walks its segments (grid-stride); each segment is a run of at most
// 1,024 entries of one row (CSR) or column (CSC).  The rows the segment owns
// stay in registers; for every entry a group of lanes gathers the other
// factor's row with float4 loads straight into registers.  Rows split over
// several segments write partial sums that a fix-up kernel combines in
// segment order (deterministic).
//
// MODE 0 (loss/gradient, Eq. "mf"):   r_e = <own_i, oth_j> - a_e,
//                                      out_i = sum_e r_e oth_j + lam own_i,  f += r^2 / 2
// MODE 1 (residual SpMM of Z products): out_i += gamma * sum_e v_e X_j
// MODE 2 (exact line search):          b_e = <DW_i, H_j> + <W_i, DH_j>, c_e = <DW_i, DH_j>,
//                                      sums of r b, b^2 + 2 r c, b c, c^2
#pragma once
#include "ctx.cuh"

namespace bm {

struct PipeArgs {
  const int32_t* seg_row;
  const int64_t* seg_beg;
  const int64_t* seg_end;
  const int32_t* seg_slot;
  int64_t nseg;
  const int32_t* idx;     // gathered row of each entry (pass order)
  const float* scal;      // per-entry scalar: A_e (MODE 0), v_e (MODE 1), r_e (MODE 2)
  const float* g0;        // gathered matrix (MODE 2: H)
  const float* g1;        // MODE 2: DH
  const float* o0;        // owned matrix (MODE 0: W or H; MODE 2: W)
  const float* o1;        // MODE 2: DW
  int ld, nchunk;         // row stride of the matrices (floats), chunks of 4 floats used per row
  float lam;              // MODE 0
  float gamma;            // MODE 1
  float* out;             // MODE 0 / 1 output rows (ld_out)
  int ld_out;
  float* partial;         // partial sums of multi-segment rows (ld_part)
  int ld_part;
  double* fseg;           // MODE 0: per-segment 1/2 sum r^2 (nullable); MODE 2: 4 sums per segment
  float* r_out;           // MODE 0: residual in pass order (nullable)
  const void* g0b;        // BF16 copies of g0 / g1 (row stride ldb elements, ldb % 8 == 0,
  const void* g1b;        //   zero padded) used instead of g0 / g1 when gathering in BF16
  int ldb;
  const uint8_t* scal8;   // MODE 0 value codec (nullable): A_e = scal8[e] + scal_off
  float scal_off;
};

// the per-entry scalar of entry e: one byte through the value codec, else FP32
__device__ __forceinline__ float load_scal(const PipeArgs& a, int64_t e) {
  return a.scal8 ? (float)__ldg(a.scal8 + e) + a.scal_off : __ldg(a.scal + e);
}

__device__ __forceinline__ float bf16lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }

__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ----------------------------------------------------------------------------
// One warp per segment, 32 / L entries per step, L lanes per entry loading V
// float4 chunks of the gathered row straight into registers, two steps
// unrolled.
// ----------------------------------------------------------------------------
template <bool BF>
__device__ __forceinline__ float4 gather4(const float* g, const void* gb, int64_t j, int ld, int ldb, int c) {
  if (BF) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const unsigned short*>(gb) + j * ldb) + c);
    return make_float4(bf16lo(u.x), bf16hi(u.x), bf16lo(u.y), bf16hi(u.y));
  }
  return __ldg(reinterpret_cast<const float4*>(g + j * ld) + c);
}

// Lanes that share one entry (its row split into float4 chunks l, l + L, ...)
// and resident blocks per SM, by pass mode: the loss/gradient pass runs
// fastest with four lanes per entry and three blocks per SM; the line-search
// pass (two gathered rows, three dot products) and the q-wide SpMM (up to
// 2 (k_max + 1) columns) with eight lanes and four blocks (measured on the
// recommendation-scale workload at k = 64).
template <int MODE>
constexpr int lanes_per_entry() { return MODE == 0 ? 4 : 8; }
template <int MODE>
constexpr int direct_blocks_per_sm() { return MODE == 0 ? 3 : 4; }

// One segment s of a pass (the warp's lanes cooperate).  EX: the row width is
// exactly 4 V chunks of 4 floats, so no chunk needs a bounds test.
template <int MODE, int V, bool BF, bool EX>
__device__ __forceinline__ void direct_segment(const PipeArgs& a, int64_t s) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int kLanesPerEntry = lanes_per_entry<MODE>();
  constexpr int EPS = 32 / kLanesPerEntry;   // entries per step
  const int lane = threadIdx.x & 31, g = lane / kLanesPerEntry, l = lane % kLanesPerEntry;
  const int nch = a.nchunk;
  const int i = a.seg_row[s];
  const int64_t beg = a.seg_beg[s], end = a.seg_end[s];
  float4 w[V], dw[V], acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int c = l + kLanesPerEntry * v;
    const bool in = (EX || c < nch);
    w[v] = (MODE != 1 && in) ? __ldg(reinterpret_cast<const float4*>(a.o0 + (int64_t)i * a.ld) + c)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    dw[v] = (MODE == 2 && in) ? __ldg(reinterpret_cast<const float4*>(a.o1 + (int64_t)i * a.ld) + c)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float fs = 0.f, s_rb = 0.f, s_bb = 0.f, s_bc = 0.f, s_cc = 0.f;
  for (int64_t e0 = beg; e0 < end; e0 += 32) {
    const int64_t e = e0 + lane;
    const bool valid = e < end;
    const int j = valid ? __ldg(a.idx + e) : 0;
    const float sv = valid ? load_scal(a, e) : 0.f;
#pragma unroll 2
    for (int t = 0; t < kLanesPerEntry; ++t) {
      const int src = t * EPS + g;
      const int64_t jj = __shfl_sync(FULL, j, src);
      const float sc = __shfl_sync(FULL, sv, src);
      const bool ok = e0 + src < end;
      if (MODE == 0) {
        float4 hv[V];
        float d = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + kLanesPerEntry * v;
          hv[v] = (EX || c < nch) ? gather4<BF>(a.g0, a.g0b, jj, a.ld, a.ldb, c) : make_float4(0.f, 0.f, 0.f, 0.f);
          d = fmaf(w[v].x, hv[v].x, fmaf(w[v].y, hv[v].y, fmaf(w[v].z, hv[v].z, fmaf(w[v].w, hv[v].w, d))));
        }
#pragma unroll
        for (int mk = 1; mk < kLanesPerEntry; mk <<= 1) d += __shfl_xor_sync(FULL, d, mk);
        const float r = ok ? d - sc : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          acc[v].x = fmaf(r, hv[v].x, acc[v].x);
          acc[v].y = fmaf(r, hv[v].y, acc[v].y);
          acc[v].z = fmaf(r, hv[v].z, acc[v].z);
          acc[v].w = fmaf(r, hv[v].w, acc[v].w);
        }
        if (l == 0) {
          fs = fmaf(r, r, fs);
          if (a.r_out && ok) a.r_out[e0 + src] = r;
        }
      } else if (MODE == 1) {
        const float vv = ok ? sc : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + kLanesPerEntry * v;
          if ((EX || c < nch)) {
            const float4 x = gather4<BF>(a.g0, a.g0b, jj, a.ld, a.ldb, c);
            acc[v].x = fmaf(vv, x.x, acc[v].x);
            acc[v].y = fmaf(vv, x.y, acc[v].y);
            acc[v].z = fmaf(vv, x.z, acc[v].z);
            acc[v].w = fmaf(vv, x.w, acc[v].w);
          }
        }
      } else {
        float b = 0.f, c2 = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + kLanesPerEntry * v;
          if ((EX || c < nch)) {
            const float4 h = gather4<BF>(a.g0, a.g0b, jj, a.ld, a.ldb, c);
            const float4 dh = gather4<BF>(a.g1, a.g1b, jj, a.ld, a.ldb, c);
            b = fmaf(dw[v].x, h.x, fmaf(dw[v].y, h.y, fmaf(dw[v].z, h.z, fmaf(dw[v].w, h.w, b))));
            b = fmaf(w[v].x, dh.x, fmaf(w[v].y, dh.y, fmaf(w[v].z, dh.z, fmaf(w[v].w, dh.w, b))));
            c2 = fmaf(dw[v].x, dh.x, fmaf(dw[v].y, dh.y, fmaf(dw[v].z, dh.z, fmaf(dw[v].w, dh.w, c2))));
          }
        }
#pragma unroll
        for (int mk = 1; mk < kLanesPerEntry; mk <<= 1) {
          b += __shfl_xor_sync(FULL, b, mk);
          c2 += __shfl_xor_sync(FULL, c2, mk);
        }
        if (ok && l == 0) {
          s_rb = fmaf(sc, b, s_rb);
          s_bb = fmaf(b, b, fmaf(2.f * sc, c2, s_bb));
          s_bc = fmaf(b, c2, s_bc);
          s_cc = fmaf(c2, c2, s_cc);
        }
      }
    }
  }
  if (MODE != 2) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
#pragma unroll
      for (int mk = kLanesPerEntry; mk < 32; mk <<= 1) {
        acc[v].x += __shfl_xor_sync(FULL, acc[v].x, mk);
        acc[v].y += __shfl_xor_sync(FULL, acc[v].y, mk);
        acc[v].z += __shfl_xor_sync(FULL, acc[v].z, mk);
        acc[v].w += __shfl_xor_sync(FULL, acc[v].w, mk);
      }
    }
    if (g == 0) {
      const int slot = a.seg_slot[s];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = l + kLanesPerEntry * v;
        if ((EX || c < nch)) {
          if (slot < 0) {
            float4* op = reinterpret_cast<float4*>(a.out + (int64_t)i * a.ld_out + 4 * c);
            float4 o;
            if (MODE == 0) {
              o = acc[v];
              o.x = fmaf(a.lam, w[v].x, o.x);
              o.y = fmaf(a.lam, w[v].y, o.y);
              o.z = fmaf(a.lam, w[v].z, o.z);
              o.w = fmaf(a.lam, w[v].w, o.w);
            } else {
              o = *op;
              o.x = fmaf(a.gamma, acc[v].x, o.x);
              o.y = fmaf(a.gamma, acc[v].y, o.y);
              o.z = fmaf(a.gamma, acc[v].z, o.z);
              o.w = fmaf(a.gamma, acc[v].w, o.w);
            }
            *op = o;
          } else {
            *reinterpret_cast<float4*>(a.partial + (int64_t)slot * a.ld_part + 4 * c) = acc[v];
          }
        }
      }
    }
    if (MODE == 0 && a.fseg) {
#pragma unroll
      for (int mk = 16; mk > 0; mk >>= 1) fs += __shfl_xor_sync(FULL, fs, mk);
      if (lane == 0) a.fseg[s] = 0.5 * (double)fs;
    }
  } else {
#pragma unroll
    for (int mk = 16; mk > 0; mk >>= 1) {
      s_rb += __shfl_xor_sync(FULL, s_rb, mk);
      s_bb += __shfl_xor_sync(FULL, s_bb, mk);
      s_bc += __shfl_xor_sync(FULL, s_bc, mk);
      s_cc += __shfl_xor_sync(FULL, s_cc, mk);
    }
    if (lane == 0) {
      a.fseg[s * 4 + 0] = s_rb;
      a.fseg[s * 4 + 1] = s_bb;
      a.fseg[s * 4 + 2] = s_bc;
      a.fseg[s * 4 + 3] = s_cc;
    }
  }
}

template <int MODE, int V, bool BF, bool EX>
__global__ void __launch_bounds__(256, direct_blocks_per_sm<MODE>()) k_direct(PipeArgs a) {
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nseg; s += nwarps)
    direct_segment<MODE, V, BF, EX>(a, s);
}

// The same pass over several problems in one launch: segment sg of the
// concatenated segment lists belongs to problem p with
// prefix[p] <= sg < prefix[p + 1].
template <int MODE, int V, bool BF, bool EX>
__global__ void __launch_bounds__(256, direct_blocks_per_sm<MODE>()) k_direct_batch(const PipeArgs* __restrict__ args,
                                                         const int64_t* __restrict__ prefix, int count) {
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = prefix[count];
  for (int64_t sg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sg < total; sg += nwarps) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= sg) lo = mid; else hi = mid;
    }
    direct_segment<MODE, V, BF, EX>(args[lo], sg - prefix[lo]);
  }
}

// Launch k_direct_batch for problems with the same chunk count; total_segs =
// prefix[count] (host copy) sizes the grid.
template <int MODE>
void launch_direct_batch(const PipeArgs* args_d, const int64_t* prefix_d, int count, int64_t total_segs,
                         int nchunk, bool bf, cudaStream_t st) {
  constexpr int kLanesPerEntry = lanes_per_entry<MODE>();
  const int V = (nchunk + kLanesPerEntry - 1) / kLanesPerEntry;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(total_segs, 1), 8),
                                                               (int64_t)num_sms() * 24));
  const bool ex = nchunk == kLanesPerEntry * V;
#define BM_DBATCH_CASE(VV)                                                                          \
  case VV:                                                                                          \
    if (bf) {                                                                                       \
      if (ex) k_direct_batch<MODE, VV, true, true><<<grid, 256, 0, st>>>(args_d, prefix_d, count);  \
      else k_direct_batch<MODE, VV, true, false><<<grid, 256, 0, st>>>(args_d, prefix_d, count);    \
    } else {                                                                                        \
      if (ex) k_direct_batch<MODE, VV, false, true><<<grid, 256, 0, st>>>(args_d, prefix_d, count); \
      else k_direct_batch<MODE, VV, false, false><<<grid, 256, 0, st>>>(args_d, prefix_d, count);   \
    }                                                                                               \
    break;
  switch (V) {
    BM_DBATCH_CASE(1)
    BM_DBATCH_CASE(2)
    BM_DBATCH_CASE(3)
    BM_DBATCH_CASE(4)
    BM_DBATCH_CASE(5)
    BM_DBATCH_CASE(6)
    BM_DBATCH_CASE(7)
    BM_DBATCH_CASE(8)
    default:
      throw Error{BM_ERR_INVALID, "batched pass: more than 128 columns"};
  }
#undef BM_DBATCH_CASE
}

// Launch k_direct<MODE, V, BF, EX> with V = ceil(nchunk / L) (<= 8); BF selects
// the BF16 copies (a.g0b, a.g1b) for the gathered rows.
template <int MODE>
void launch_pipe(const PipeArgs& a, cudaStream_t st, bool bf = false) {
  constexpr int kLanesPerEntry = lanes_per_entry<MODE>();
  const int V = (a.nchunk + kLanesPerEntry - 1) / kLanesPerEntry;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(a.nseg, 1), 8),
                                                               (int64_t)num_sms() * 24));
  const bool ex = a.nchunk == kLanesPerEntry * V;
#define BM_DIRECT_CASE(VV)                                                \
  case VV:                                                                \
    if (bf) {                                                             \
      if (ex) k_direct<MODE, VV, true, true><<<grid, 256, 0, st>>>(a);    \
      else k_direct<MODE, VV, true, false><<<grid, 256, 0, st>>>(a);      \
    } else {                                                              \
      if (ex) k_direct<MODE, VV, false, true><<<grid, 256, 0, st>>>(a);   \
      else k_direct<MODE, VV, false, false><<<grid, 256, 0, st>>>(a);     \
    }                                                                     \
    return;
  switch (V) {
    BM_DIRECT_CASE(1)
    BM_DIRECT_CASE(2)
    BM_DIRECT_CASE(3)
    BM_DIRECT_CASE(4)
    BM_DIRECT_CASE(5)
    BM_DIRECT_CASE(6)
    BM_DIRECT_CASE(7)
    BM_DIRECT_CASE(8)
    default:
      break;
  }
#undef BM_DIRECT_CASE
  throw Error{BM_ERR_INVALID, "sparse pass: more than 128 columns"};
}

}  // namespace bm
