// Pipelined sparse passes over a segment split.
//
// A warp walks its segments (grid-stride) in batches of 32 entries (16 for the
// two-row line-search pass).  For every
// batch the rows it gathers (and, at the first batch of a segment, the rows the
// segment owns) are copied into a per-warp ring of shared-memory stages with
// cp.async, two batches ahead of the batch being computed, so the
// latency of the row gathers overlaps the arithmetic of earlier batches.
// Lane L copies the row(s) of entry L of a batch; for the arithmetic four lanes
// share one entry (8 entries per round), each lane holding V float4 chunks.  Rows split over several segments write partial sums that a
// fix-up kernel combines in segment order (deterministic).
//
// MODE 0 (loss/gradient, Eq. "mf"):   r_e = <own_i, oth_j> - a_e,
//                                      out_i = sum_e r_e oth_j + lam own_i,  f += r^2 / 2
// MODE 1 (residual SpMM of Z products): out_i += gamma * sum_e v_e X_j
// MODE 2 (exact line search):          b_e = <DW_i, H_j> + <W_i, DH_j>, c_e = <DW_i, DH_j>,
//                                      sums of r b, b^2 + 2 r c, b c, c^2
#pragma once
#include "ctx.cuh"

namespace bm {

// Pipeline shape (compile-time; chosen by measurement on GB300).
#ifndef BM_PIPE_BATCH
#define BM_PIPE_BATCH 16   // entries per batch of the one-row passes (halved for two rows)
#endif
#ifndef BM_PIPE_STAGES
#define BM_PIPE_STAGES 3   // ring stages (BM_PIPE_STAGES - 1 batches in flight)
#endif
#ifndef BM_PIPE_WARPS
#define BM_PIPE_WARPS 4    // warps per block
#endif
constexpr int kPipeWarps = BM_PIPE_WARPS;

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
};

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

template <int MODE>
struct PipeShape {
  static constexpr int NG = MODE == 2 ? 2 : 1;                    // gathered rows per entry
  static constexpr int NO = MODE == 1 ? 0 : (MODE == 2 ? 2 : 1);  // owned rows per segment
  static constexpr int BATCH = MODE == 2 ? (BM_PIPE_BATCH > 8 ? BM_PIPE_BATCH / 2 : 8) : BM_PIPE_BATCH;
  static constexpr int S = BM_PIPE_STAGES;
};

// floats of one stage: BATCH entries x NG slots + NO owned slots (each 4*nchunk + 4
// floats; the pad spreads the slots over the banks), + BATCH scalars
__host__ __device__ inline int pipe_stage_floats(int mode, int nchunk) {
  const int ng = mode == 2 ? 2 : 1;
  const int no = mode == 1 ? 0 : (mode == 2 ? 2 : 1);
  const int batch = mode == 2 ? (BM_PIPE_BATCH > 8 ? BM_PIPE_BATCH / 2 : 8) : BM_PIPE_BATCH;
  return (batch * ng + no) * (4 * nchunk + 4) + batch;
}

inline size_t pipe_smem_bytes(int mode, int nchunk) {
  return (size_t)kPipeWarps * BM_PIPE_STAGES * pipe_stage_floats(mode, nchunk) * sizeof(float);
}

template <int MODE, int V>
__global__ void __launch_bounds__(kPipeWarps * 32) k_pipe(PipeArgs a) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NG = PipeShape<MODE>::NG, NO = PipeShape<MODE>::NO, S = PipeShape<MODE>::S;
  constexpr int BATCH = PipeShape<MODE>::BATCH, ROUNDS = BATCH / 8;
  extern __shared__ __align__(16) float pipe_sm[];
  const int lane = threadIdx.x & 31, g = lane >> 2, l = lane & 3;
  const int nch = a.nchunk;
  const int SL = 4 * nch + 4;
  const int SF = (BATCH * NG + NO) * SL + BATCH;
  float* ring = pipe_sm + (size_t)(threadIdx.x >> 5) * S * SF;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;

  // issue cursor (segment bounds cached in registers)
  int64_t is = warp0, ib = 0, i_beg = 0, i_end = 0, i_nb = 0;
  int i_row = 0;
  if (is < a.nseg) {
    i_beg = a.seg_beg[is];
    i_end = a.seg_end[is];
    i_nb = max((int64_t)1, (i_end - i_beg + BATCH - 1) / BATCH);
    i_row = a.seg_row[is];
  }
  auto issue = [&](int stage) {
    if (is < a.nseg) {
      float* st = ring + stage * SF;
      const int64_t e0 = i_beg + (int64_t)BATCH * ib;
      const int cnt = (int)min((int64_t)BATCH, i_end - e0);
      if (lane < BATCH) {
        const bool v = lane < cnt;
        const int j = v ? __ldg(a.idx + e0 + lane) : 0;
        st[(BATCH * NG + NO) * SL + lane] = v ? __ldg(a.scal + e0 + lane) : 0.f;
        const float* s0 = a.g0 + (int64_t)j * a.ld;
        float* d0 = st + lane * NG * SL;
        for (int c = 0; c < nch; ++c) cp_async16(d0 + 4 * c, s0 + 4 * c, v);
        if (NG == 2) {
          const float* s1 = a.g1 + (int64_t)j * a.ld;
          for (int c = 0; c < nch; ++c) cp_async16(d0 + SL + 4 * c, s1 + 4 * c, v);
        }
      }
      if (NO > 0 && ib == 0) {
        for (int u = lane; u < NO * nch; u += 32) {
          const int oi = NO == 2 ? (u >= nch ? 1 : 0) : 0;
          const int c = u - oi * nch;
          const float* src = (oi == 0 ? a.o0 : a.o1) + (int64_t)i_row * a.ld + 4 * c;
          cp_async16(st + (BATCH * NG + oi) * SL + 4 * c, src, true);
        }
      }
      if (++ib >= i_nb) {
        ib = 0;
        is += nwarps;
        if (is < a.nseg) {
          i_beg = a.seg_beg[is];
          i_end = a.seg_end[is];
          i_nb = max((int64_t)1, (i_end - i_beg + BATCH - 1) / BATCH);
          i_row = a.seg_row[is];
        }
      }
    }
    cp_async_commit();
  };

#pragma unroll 1
  for (int s = 0; s < S - 1; ++s) issue(s);

  // compute cursor
  int64_t cs = warp0, cb = 0, c_beg = 0, c_end = 0, c_nb = 0;
  int c_row = 0, c_slot = -1;
  if (cs < a.nseg) {
    c_beg = a.seg_beg[cs];
    c_end = a.seg_end[cs];
    c_nb = max((int64_t)1, (c_end - c_beg + BATCH - 1) / BATCH);
    c_row = a.seg_row[cs];
    c_slot = a.seg_slot[cs];
  }
  int stage = 0;
  float4 w[V], dw[V], acc[V];
  float fs = 0.f, s_rb = 0.f, s_bb = 0.f, s_bc = 0.f, s_cc = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) w[v] = dw[v] = acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  while (cs < a.nseg) {
    issue((stage + S - 1) % S);
    cp_async_wait<S - 1>();
    __syncwarp();
    const float* st = ring + stage * SF;
    const int64_t e0 = c_beg + (int64_t)BATCH * cb;
    const int cnt = (int)min((int64_t)BATCH, c_end - e0);
    if (cb == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int c = l + 4 * v;
        if (NO >= 1) w[v] = c < nch ? *reinterpret_cast<const float4*>(st + BATCH * NG * SL + 4 * c)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        if (NO == 2) dw[v] = c < nch ? *reinterpret_cast<const float4*>(st + (BATCH * NG + 1) * SL + 4 * c)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      fs = s_rb = s_bb = s_bc = s_cc = 0.f;
    }
#pragma unroll
    for (int t = 0; t < ROUNDS; ++t) {
      const int ent = t * 8 + g;
      const bool ok = ent < cnt;
      const float sc = st[(BATCH * NG + NO) * SL + ent];
      const float* r0 = st + (ent * NG) * SL;
      if (MODE == 0) {
        float4 hv[V];
        float d = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + 4 * v;
          hv[v] = c < nch ? *reinterpret_cast<const float4*>(r0 + 4 * c) : make_float4(0.f, 0.f, 0.f, 0.f);
          d = fmaf(w[v].x, hv[v].x, fmaf(w[v].y, hv[v].y, fmaf(w[v].z, hv[v].z, fmaf(w[v].w, hv[v].w, d))));
        }
        d += __shfl_xor_sync(FULL, d, 1);
        d += __shfl_xor_sync(FULL, d, 2);
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
          if (a.r_out && ok) a.r_out[e0 + ent] = r;
        }
      } else if (MODE == 1) {
        const float vv = ok ? sc : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + 4 * v;
          if (c < nch) {
            const float4 x = *reinterpret_cast<const float4*>(r0 + 4 * c);
            acc[v].x = fmaf(vv, x.x, acc[v].x);
            acc[v].y = fmaf(vv, x.y, acc[v].y);
            acc[v].z = fmaf(vv, x.z, acc[v].z);
            acc[v].w = fmaf(vv, x.w, acc[v].w);
          }
        }
      } else {
        const float* r1 = r0 + SL;
        float b = 0.f, c2 = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int c = l + 4 * v;
          if (c < nch) {
            const float4 h = *reinterpret_cast<const float4*>(r0 + 4 * c);
            const float4 dh = *reinterpret_cast<const float4*>(r1 + 4 * c);
            b = fmaf(dw[v].x, h.x, fmaf(dw[v].y, h.y, fmaf(dw[v].z, h.z, fmaf(dw[v].w, h.w, b))));
            b = fmaf(w[v].x, dh.x, fmaf(w[v].y, dh.y, fmaf(w[v].z, dh.z, fmaf(w[v].w, dh.w, b))));
            c2 = fmaf(dw[v].x, dh.x, fmaf(dw[v].y, dh.y, fmaf(dw[v].z, dh.z, fmaf(dw[v].w, dh.w, c2))));
          }
        }
        b += __shfl_xor_sync(FULL, b, 1);
        b += __shfl_xor_sync(FULL, b, 2);
        c2 += __shfl_xor_sync(FULL, c2, 1);
        c2 += __shfl_xor_sync(FULL, c2, 2);
        if (ok && l == 0) {
          s_rb = fmaf(sc, b, s_rb);
          s_bb = fmaf(b, b, fmaf(2.f * sc, c2, s_bb));
          s_bc = fmaf(b, c2, s_bc);
          s_cc = fmaf(c2, c2, s_cc);
        }
      }
    }
    if (cb + 1 >= c_nb) {
      // segment complete: reduce across the 8 groups and write
      if (MODE != 2) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
          for (int mk = 4; mk < 32; mk <<= 1) {
            acc[v].x += __shfl_xor_sync(FULL, acc[v].x, mk);
            acc[v].y += __shfl_xor_sync(FULL, acc[v].y, mk);
            acc[v].z += __shfl_xor_sync(FULL, acc[v].z, mk);
            acc[v].w += __shfl_xor_sync(FULL, acc[v].w, mk);
          }
        }
        if (g == 0) {
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int c = l + 4 * v;
            if (c < nch) {
              if (c_slot < 0) {
                float4* op = reinterpret_cast<float4*>(a.out + (int64_t)c_row * a.ld_out + 4 * c);
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
                *reinterpret_cast<float4*>(a.partial + (int64_t)c_slot * a.ld_part + 4 * c) = acc[v];
              }
            }
          }
        }
        if (MODE == 0 && a.fseg) {
#pragma unroll
          for (int mk = 16; mk > 0; mk >>= 1) fs += __shfl_xor_sync(FULL, fs, mk);
          if (lane == 0) a.fseg[cs] = 0.5 * (double)fs;
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
          a.fseg[cs * 4 + 0] = s_rb;
          a.fseg[cs * 4 + 1] = s_bb;
          a.fseg[cs * 4 + 2] = s_bc;
          a.fseg[cs * 4 + 3] = s_cc;
        }
      }
      cb = 0;
      cs += nwarps;
      if (cs < a.nseg) {
        c_beg = a.seg_beg[cs];
        c_end = a.seg_end[cs];
        c_nb = max((int64_t)1, (c_end - c_beg + BATCH - 1) / BATCH);
        c_row = a.seg_row[cs];
        c_slot = a.seg_slot[cs];
      }
    } else {
      ++cb;
    }
    __syncwarp();
    stage = stage + 1 == S ? 0 : stage + 1;
  }
  cp_async_wait<0>();
}

// Launch k_pipe<MODE, V> with V = ceil(nchunk / 4) (<= 8).
template <int MODE>
void launch_pipe(const PipeArgs& a, cudaStream_t st) {
  const int V = (a.nchunk + 3) / 4;
  const size_t smem = pipe_smem_bytes(MODE, a.nchunk);
  const int warps = kPipeWarps;
  const int blocks_per_sm = (int)std::max<size_t>(1, (200 * 1024) / std::max<size_t>(smem, 1));
  const int64_t need = ceil_div(std::max<int64_t>(a.nseg, 1), warps);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * blocks_per_sm));
#define BM_PIPE_CASE(VV)                                                                          \
  case VV: {                                                                                      \
    static bool attr = false;                                                                     \
    if (!attr) {                                                                                  \
      BM_CUDA(cudaFuncSetAttribute(k_pipe<MODE, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   200 * 1024));                                                  \
      attr = true;                                                                                \
    }                                                                                             \
    k_pipe<MODE, VV><<<grid, warps * 32, smem, st>>>(a);                                          \
    break;                                                                                        \
  }
  switch (V) {
    BM_PIPE_CASE(1)
    BM_PIPE_CASE(2)
    BM_PIPE_CASE(3)
    BM_PIPE_CASE(4)
    BM_PIPE_CASE(5)
    BM_PIPE_CASE(6)
    BM_PIPE_CASE(7)
    BM_PIPE_CASE(8)
    default:
      throw Error{BM_ERR_INVALID, "sparse pass: more than 128 columns"};
  }
#undef BM_PIPE_CASE
}

}  // namespace bm
