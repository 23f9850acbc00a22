// Sparse passes over a segment split (one lane group per segment).
//
// Each segment is a run of at most 1,024 entries of one row (CSR) or column
// (CSC); a group of lanes of a warp owns one segment (k_sparse below).  The
// rows the segment owns stay in registers; for every entry the group gathers
// the other factor's row with float4 loads straight into registers.  Rows
// split over several segments write partial sums that a fix-up kernel
// combines in segment order (deterministic).
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

// One gathered row's chunk c (4 values): FP32 rows hold 4 floats per chunk,
// BF16 copies 4 bfloat16 (8 bytes) per chunk.
template <bool BF>
__device__ __forceinline__ float4 gather4(const float* g, const void* gb, int64_t j, int ld, int ldb, int c) {
  if (BF) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const unsigned short*>(gb) + j * ldb) + c);
    return make_float4(bf16lo(u.x), bf16hi(u.x), bf16lo(u.y), bf16hi(u.y));
  }
  return __ldg(reinterpret_cast<const float4*>(g + j * ld) + c);
}

// ----------------------------------------------------------------------------
// Group-per-segment kernel.  A warp holds 32 / L groups of L lanes; each
// group owns one segment and walks its entries one per step, the L lanes
// splitting the rows into float4 chunks c = l, l + L, ... (V chunks per lane).
// The rows the segment owns stay in registers, the gathered row of each
// entry is loaded with float4 loads straight into registers, and the group's
// sums never leave the group (no cross-group reduction).  Segments are
// ordered by length within a panel, so the groups of one warp walk segments
// of about the same length.
// ----------------------------------------------------------------------------
// Lanes per group and resident 256-thread blocks per SM requested from the
// compiler, by pass mode and layout (chosen by measurement on GB300, k = 64).
#ifndef BM_LANES_GRAD
#define BM_LANES_GRAD 8      // group-per-segment layout
#endif
#ifndef BM_LANES_SPMM
#define BM_LANES_SPMM 8
#endif
#ifndef BM_LANES_LS
#define BM_LANES_LS 8
#endif
#ifndef BM_WS_LANES_GRAD
#define BM_WS_LANES_GRAD 8   // warp-per-segment layout
#endif
#ifndef BM_WS_LANES_SPMM
#define BM_WS_LANES_SPMM 8
#endif
#ifndef BM_WS_LANES_LS
#define BM_WS_LANES_LS 8
#endif
#ifndef BM_BPS_GRAD
#define BM_BPS_GRAD 4
#endif
#ifndef BM_BPS_SPMM
#define BM_BPS_SPMM 4
#endif
#ifndef BM_BPS_LS
#define BM_BPS_LS 4
#endif
#ifndef BM_WS_BPS_GRAD
#define BM_WS_BPS_GRAD 4
#endif
#ifndef BM_WS_BPS_SPMM
#define BM_WS_BPS_SPMM 4
#endif
#ifndef BM_WS_BPS_LS
#define BM_WS_BPS_LS 4
#endif
#ifndef BM_UNROLL
#define BM_UNROLL 2          // entries of a group unrolled per loop trip
#endif

constexpr int kUnroll = BM_UNROLL;

template <int MODE, bool WS>
constexpr int pass_lanes() {
  return WS ? (MODE == 0 ? BM_WS_LANES_GRAD : (MODE == 1 ? BM_WS_LANES_SPMM : BM_WS_LANES_LS))
            : (MODE == 0 ? BM_LANES_GRAD : (MODE == 1 ? BM_LANES_SPMM : BM_LANES_LS));
}

// Widest row a pass handles, in float4 chunks: factor rows hold at most 128
// floats (k_max + 1 <= 128), the q-wide blocks of the PG step at most 256.
template <int MODE>
constexpr int max_chunks() { return MODE == 1 ? 64 : 32; }

// Resident blocks per SM for V chunks per lane: the base figure for narrow
// rows, fewer for wider rows so that their registers do not spill.
template <int MODE, int V, bool WS>
constexpr int pass_blocks_per_sm() {
  constexpr int base = WS ? (MODE == 0 ? BM_WS_BPS_GRAD : (MODE == 1 ? BM_WS_BPS_SPMM : BM_WS_BPS_LS))
                          : (MODE == 0 ? BM_BPS_GRAD : (MODE == 1 ? BM_BPS_SPMM : BM_BPS_LS));
  constexpr int cap = MODE == 1 ? (V <= 5 ? base : 3) : (V <= 2 ? base : (V <= 4 ? 3 : 2));
  return base < cap ? base : cap;
}

// One segment s.  WS = false: the group owns segment s (s < 0: an idle group
// that only joins the warp's shuffles) and takes one entry per step.  WS =
// true: every group of the warp works on the same segment s, group g taking
// entries g, g + 32/L, ... of each run of 32, and the groups' sums are added
// at the end (long segments).  EX: the row width is exactly L * V chunks, so
// no chunk needs a bounds test.
template <int MODE, int L, int V, bool BF, bool EX, bool WS>
__device__ __forceinline__ void group_segment(const PipeArgs& a, int64_t s) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int GPW = 32 / L;
  constexpr int TRIP = WS ? 32 : L;          // entries fetched per loop trip
  const int lane = threadIdx.x & 31, l = lane % L, g = lane / L;
  const int fl = WS ? lane : l;              // this lane fetches entry t0 + fl
  const int nch = a.nchunk;
  // factor rows (MODE 0, 2) of an exact width have a compile-time stride
  constexpr int kW = 4 * L * V;
  const int ld = (MODE != 1 && EX) ? kW : a.ld;
  const int ldb = (MODE != 1 && EX && kW % 8 == 0) ? kW : a.ldb;
  const bool live = s >= 0;
  const int i = live ? a.seg_row[s] : 0;
  const int64_t beg = live ? a.seg_beg[s] : 0;
  const int len = live ? (int)(a.seg_end[s] - beg) : 0;
  // every group of the warp takes the same number of steps (the longest segment)
  int steps = len;
  if (!WS) {
#pragma unroll
    for (int mk = L; mk < 32; mk <<= 1) steps = max(steps, __shfl_xor_sync(FULL, steps, mk));
  }
  float4 w[V], dw[V], acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int c = l + L * v;
    const bool in = live && (EX || c < nch);
    w[v] = (MODE != 1 && in) ? __ldg(reinterpret_cast<const float4*>(a.o0 + (int64_t)i * ld) + c)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    dw[v] = (MODE == 2 && in) ? __ldg(reinterpret_cast<const float4*>(a.o1 + (int64_t)i * ld) + c)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float fs = 0.f, s_rb = 0.f, s_bb = 0.f, s_bc = 0.f, s_cc = 0.f;
  for (int t0 = 0; t0 < steps; t0 += TRIP) {
    const bool valid = t0 + fl < len;
    const int64_t e = beg + t0 + fl;
    const int j = valid ? __ldg(a.idx + e) : 0;
    const float sv = valid ? load_scal(a, e) : 0.f;
    float r_mine = 0.f;
#pragma unroll kUnroll
    for (int u = 0; u < L; ++u) {
      const int src = WS ? u * GPW + g : u;    // entry t0 + src of the run
      const int jj = __shfl_sync(FULL, j, src, TRIP);
      const float sc = __shfl_sync(FULL, sv, src, TRIP);
      const bool ok = t0 + src < len;
      if (MODE == 0) {
        float4 hv[V];
        float d = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + L * v;
          hv[v] = (EX || c < nch) ? gather4<BF>(a.g0, a.g0b, jj, ld, ldb, c) : make_float4(0.f, 0.f, 0.f, 0.f);
          d = fmaf(w[v].x, hv[v].x, fmaf(w[v].y, hv[v].y, fmaf(w[v].z, hv[v].z, fmaf(w[v].w, hv[v].w, d))));
        }
#pragma unroll
        for (int mk = 1; mk < L; mk <<= 1) d += __shfl_xor_sync(FULL, d, mk);
        const float r = ok ? d - sc : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          acc[v].x = fmaf(r, hv[v].x, acc[v].x);
          acc[v].y = fmaf(r, hv[v].y, acc[v].y);
          acc[v].z = fmaf(r, hv[v].z, acc[v].z);
          acc[v].w = fmaf(r, hv[v].w, acc[v].w);
        }
        fs = fmaf(r, r, fs);            // every lane of the group holds the same r
        if (WS) {
          if (a.r_out && ok && l == 0) a.r_out[beg + t0 + src] = r;
        } else if (l == u) {
          r_mine = r;
        }
      } else if (MODE == 1) {
        const float vv = ok ? sc : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + L * v;
          if (EX || c < nch) {
            const float4 x = gather4<BF>(a.g0, a.g0b, jj, ld, ldb, c);
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
          const int c = l + L * v;
          if (EX || c < nch) {
            const float4 h = gather4<BF>(a.g0, a.g0b, jj, ld, ldb, c);
            const float4 dh = gather4<BF>(a.g1, a.g1b, jj, ld, ldb, c);
            b = fmaf(dw[v].x, h.x, fmaf(dw[v].y, h.y, fmaf(dw[v].z, h.z, fmaf(dw[v].w, h.w, b))));
            b = fmaf(w[v].x, dh.x, fmaf(w[v].y, dh.y, fmaf(w[v].z, dh.z, fmaf(w[v].w, dh.w, b))));
            c2 = fmaf(dw[v].x, dh.x, fmaf(dw[v].y, dh.y, fmaf(dw[v].z, dh.z, fmaf(dw[v].w, dh.w, c2))));
          }
        }
#pragma unroll
        for (int mk = 1; mk < L; mk <<= 1) {
          b += __shfl_xor_sync(FULL, b, mk);
          c2 += __shfl_xor_sync(FULL, c2, mk);
        }
        if (ok) {
          s_rb = fmaf(sc, b, s_rb);
          s_bb = fmaf(b, b, fmaf(2.f * sc, c2, s_bb));
          s_bc = fmaf(b, c2, s_bc);
          s_cc = fmaf(c2, c2, s_cc);
        }
      }
    }
    // residual of entry t0 + l, one coalesced store per group and L entries
    if (!WS && MODE == 0 && a.r_out && valid) a.r_out[e] = r_mine;
  }
  if (WS) {                                  // add the groups' sums
#pragma unroll
    for (int mk = L; mk < 32; mk <<= 1) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        acc[v].x += __shfl_xor_sync(FULL, acc[v].x, mk);
        acc[v].y += __shfl_xor_sync(FULL, acc[v].y, mk);
        acc[v].z += __shfl_xor_sync(FULL, acc[v].z, mk);
        acc[v].w += __shfl_xor_sync(FULL, acc[v].w, mk);
      }
      fs += __shfl_xor_sync(FULL, fs, mk);
      s_rb += __shfl_xor_sync(FULL, s_rb, mk);
      s_bb += __shfl_xor_sync(FULL, s_bb, mk);
      s_bc += __shfl_xor_sync(FULL, s_bc, mk);
      s_cc += __shfl_xor_sync(FULL, s_cc, mk);
    }
    if (g != 0) return;
  }
  if (!live) return;
  if (MODE != 2) {
    const int slot = a.seg_slot[s];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = l + L * v;
      if (EX || c < nch) {
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
    if (MODE == 0 && a.fseg && l == 0) a.fseg[s] = 0.5 * (double)fs;
  } else if (l == 0) {
    a.fseg[s * 4 + 0] = s_rb;
    a.fseg[s * 4 + 1] = s_bb;
    a.fseg[s * 4 + 2] = s_bc;
    a.fseg[s * 4 + 3] = s_cc;
  }
}

template <int MODE, int V, bool BF, bool EX, bool WS>
__global__ void __launch_bounds__(256, pass_blocks_per_sm<MODE, V, WS>()) k_sparse(PipeArgs a) {
  constexpr int L = pass_lanes<MODE, WS>();
  constexpr int SPW = WS ? 1 : 32 / L;   // segments per warp and trip
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int g = WS ? 0 : (threadIdx.x & 31) / L;
  // the warp's trip count is uniform: every group stays until the warp's last segment
  for (int64_t w0 = warp * SPW; w0 < a.nseg; w0 += nwarps * SPW) {
    const int64_t s = w0 + g;
    group_segment<MODE, L, V, BF, EX, WS>(a, s < a.nseg ? s : -1);
  }
}

// The same pass over several problems in one launch: segment sg of the
// concatenated segment lists belongs to problem p with
// prefix[p] <= sg < prefix[p + 1].
template <int MODE, int V, bool BF, bool EX, bool WS>
__global__ void __launch_bounds__(256, pass_blocks_per_sm<MODE, V, WS>()) k_sparse_batch(
    const PipeArgs* __restrict__ args, const int64_t* __restrict__ prefix, int count) {
  constexpr int L = pass_lanes<MODE, WS>();
  constexpr int SPW = WS ? 1 : 32 / L;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int g = WS ? 0 : (threadIdx.x & 31) / L;
  const int64_t total = prefix[count];
  for (int64_t w0 = warp * SPW; w0 < total; w0 += nwarps * SPW) {
    const int64_t sg = w0 + g;
    int lo = 0;
    if (sg < total) {
      int hi = count;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= sg) lo = mid; else hi = mid;
      }
    }
    group_segment<MODE, L, V, BF, EX, WS>(args[lo], sg < total ? sg - prefix[lo] : -1);
  }
}

// Grid of a sparse pass over nseg segments: enough warps for every segment,
// at most the resident blocks of the whole GPU.
template <int MODE, int V, bool WS>
int sparse_grid(int64_t nseg) {
  constexpr int SPW = WS ? 1 : 32 / pass_lanes<MODE, WS>();
  const int64_t warps = ceil_div(std::max<int64_t>(nseg, 1), SPW);
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps, 8),
                                                     (int64_t)num_sms() * pass_blocks_per_sm<MODE, V, WS>()));
}

// Layout for a pass over `segs`: warp-per-segment when the segments are long
// on average (a whole warp keeps enough rows in flight on one segment), else
// group-per-segment.  The autotuner may override it per pass kind.
constexpr int64_t kLongSegment = 512;
inline bool long_segments(int64_t nnz, int64_t nseg) { return nseg > 0 && nnz >= kLongSegment * nseg; }

// One instance of k_sparse / k_sparse_batch for row width V (chunks per lane).
template <int MODE, int VV, bool WS>
bool launch_sparse_v(const PipeArgs* one, const PipeArgs* args_d, const int64_t* prefix_d, int count,
                     int64_t nseg, int nchunk, bool bf, cudaStream_t st) {
  constexpr int L = pass_lanes<MODE, WS>();
  if constexpr ((VV - 1) * L < max_chunks<MODE>()) {
    if ((nchunk + L - 1) / L != VV) return false;
    const int grid = sparse_grid<MODE, VV, WS>(nseg);
    const bool ex = nchunk == L * VV;
#define BM_SPARSE_GO(BFV, EXV)                                                                              \
  if (one) k_sparse<MODE, VV, BFV, EXV, WS><<<grid, 256, 0, st>>>(*one);                                   \
  else k_sparse_batch<MODE, VV, BFV, EXV, WS><<<grid, 256, 0, st>>>(args_d, prefix_d, count);
    if (bf) {
      if (ex) { BM_SPARSE_GO(true, true) } else { BM_SPARSE_GO(true, false) }
    } else {
      if (ex) { BM_SPARSE_GO(false, true) } else { BM_SPARSE_GO(false, false) }
    }
#undef BM_SPARSE_GO
    return true;
  } else {
    (void)one; (void)args_d; (void)prefix_d; (void)count; (void)nseg; (void)nchunk; (void)bf; (void)st;
    return false;
  }
}

template <int MODE, bool WS>
void launch_sparse(const PipeArgs* one, const PipeArgs* args_d, const int64_t* prefix_d, int count, int64_t nseg,
                   int nchunk, bool bf, cudaStream_t st) {
  if (launch_sparse_v<MODE, 1, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 2, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 3, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 4, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 5, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 6, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 7, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  if (launch_sparse_v<MODE, 8, WS>(one, args_d, prefix_d, count, nseg, nchunk, bf, st)) return;
  throw Error{BM_ERR_INVALID, "sparse pass: row wider than the kernel instances"};
}

// Launch a batched pass for problems with the same chunk count; total_segs =
// prefix[count] (host copy) sizes the grid.
template <int MODE>
void launch_direct_batch(const PipeArgs* args_d, const int64_t* prefix_d, int count, int64_t total_segs,
                         int nchunk, bool bf, bool ws, cudaStream_t st) {
  if (ws) launch_sparse<MODE, true>(nullptr, args_d, prefix_d, count, total_segs, nchunk, bf, st);
  else launch_sparse<MODE, false>(nullptr, args_d, prefix_d, count, total_segs, nchunk, bf, st);
}

// Launch one pass; BF selects the BF16 copies (a.g0b, a.g1b) for the gathered
// rows, ws the warp-per-segment layout.
template <int MODE>
void launch_pipe(const PipeArgs& a, cudaStream_t st, bool bf, bool ws) {
  if (ws) launch_sparse<MODE, true>(&a, nullptr, nullptr, 0, a.nseg, a.nchunk, bf, st);
  else launch_sparse<MODE, false>(&a, nullptr, nullptr, 0, a.nseg, a.nchunk, bf, st);
}

}  // namespace bm
