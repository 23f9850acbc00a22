// Index build for Omega: validation, CSR by (row, col), CSC by (col, row),
// the CSR->CSC map and the segment work splits.  Sorting is an LSD radix sort
// (8-bit digits, stable per pass) written for this library.
#include <climits>
#include <algorithm>

#include "ctx.cuh"

namespace bm {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096 keys per tile
constexpr int kRsWarps = kRsThreads / 32;

// ---------------------------------------------------------------- validation
__global__ void k_validate(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                           const float* __restrict__ vals, int64_t nnz, int64_t m, int64_t n,
                           int* __restrict__ flags) {
  int bad_range = 0, bad_val = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = rows[e], c = cols[e];
    if (r < 0 || r >= m || c < 0 || c >= n) bad_range = 1;
    if (!isfinite(vals[e])) bad_val = 1;
  }
  if (__any_sync(0xffffffffu, bad_range) && (threadIdx.x & 31) == 0) atomicOr(flags + 0, 1);
  if (__any_sync(0xffffffffu, bad_val) && (threadIdx.x & 31) == 0) atomicOr(flags + 1, 1);
}

// key = internal_row * n_int + internal_col; value = COO position
__global__ void k_make_keys(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                            int64_t nnz, bool transpose, uint64_t nint,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ pos) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = (uint64_t)(transpose ? cols[e] : rows[e]);
    uint64_t c = (uint64_t)(transpose ? rows[e] : cols[e]);
    keys[e] = r * nint + c;
    pos[e] = (uint32_t)e;
  }
}

// ---------------------------------------------------------------- radix sort
// Digit histogram of each tile, stored digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                       int shift, uint32_t* __restrict__ hist,
                                                       int64_t ntiles) {
  __shared__ uint32_t h[256];
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = tile * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
      int64_t e = base + i;
      if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + tile] = h[threadIdx.x];
    __syncthreads();
  }
}

// Stable scatter: element order inside a tile is (warp, round, lane); a
// key's rank among equal digits = earlier rounds of its warp + earlier lanes
// of its round (match.any) + the counts of earlier warps.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs, int64_t ntiles) {
  __shared__ uint32_t wcnt[kRsWarps][256];
  __shared__ uint32_t base[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][threadIdx.x] = 0;
    base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + tile];
    __syncthreads();
    uint64_t key[kRsItems];
    uint32_t val[kRsItems];
    uint32_t rank[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
      int64_t e = tile * kRsTile + (int64_t)warp * (32 * kRsItems) + r * 32 + lane;
      bool valid = e < n;
      key[r] = valid ? kin[e] : 0;
      val[r] = valid ? vin[e] : 0;
      int d = valid ? (int)((key[r] >> shift) & 255u) : 256;
      unsigned peers = __match_any_sync(0xffffffffu, d);
      int leader = __ffs(peers) - 1;
      uint32_t before = valid ? wcnt[warp][d] : 0;
      rank[r] = before + __popc(peers & lt_mask);
      __syncwarp();
      if (valid && lane == leader) wcnt[warp][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      uint32_t run = 0;
      for (int w = 0; w < kRsWarps; ++w) {
        uint32_t t = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = run;
        run += t;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
      int64_t e = tile * kRsTile + (int64_t)warp * (32 * kRsItems) + r * 32 + lane;
      if (e < n) {
        int d = (int)((key[r] >> shift) & 255u);
        uint32_t p = base[d] + wcnt[warp][d] + rank[r];
        kout[p] = key[r];
        vout[p] = val[r];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- exclusive scan (uint32)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t* total) {
  // sh: 32 entries
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = (lane < (blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  uint32_t warp_off = warp ? sh[warp - 1] : 0;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                             uint32_t* __restrict__ bsum) {
  __shared__ uint32_t sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = base + (int64_t)threadIdx.x * kScanItems + i;
    if (e < n) s += in[e];
  }
  uint32_t tot;
  block_excl_scan(s, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_single(uint32_t* __restrict__ a, int64_t n) {
  __shared__ uint32_t sh[32];
  uint32_t carry = 0;
  for (int64_t b = 0; b < n; b += kScanThreads) {
    int64_t e = b + threadIdx.x;
    uint32_t v = e < n ? a[e] : 0;
    uint32_t tot;
    uint32_t ex = block_excl_scan(v, sh, &tot);
    if (e < n) a[e] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const uint32_t* __restrict__ in, int64_t n,
                                                            const uint32_t* __restrict__ boff,
                                                            uint32_t* __restrict__ out) {
  __shared__ uint32_t sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v[kScanItems];
  uint32_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = base + (int64_t)threadIdx.x * kScanItems + i;
    v[i] = e < n ? in[e] : 0;
    s += v[i];
  }
  uint32_t tot;
  uint32_t ex = block_excl_scan(s, sh, &tot) + boff[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = base + (int64_t)threadIdx.x * kScanItems + i;
    if (e < n) out[e] = ex;
    ex += v[i];
  }
}

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, DevBuf<uint32_t>& tmp,
                        cudaStream_t st) {
  int64_t nb = ceil_div(n, kScanTile);
  tmp.alloc(nb);
  k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, tmp.get());
  BM_CHECK_LAUNCH();
  k_scan_single<<<1, kScanThreads, 0, st>>>(tmp.get(), nb);
  BM_CHECK_LAUNCH();
  k_scan_final<<<nb, kScanThreads, 0, st>>>(in, n, tmp.get(), out);
  BM_CHECK_LAUNCH();
}

// Sort (keys, vals) ascending by the low `bits` bits of the key; result in
// (k0, v0) (buffers are swapped internally).
void radix_sort_pairs(DevBuf<uint64_t>& k0, DevBuf<uint32_t>& v0, DevBuf<uint64_t>& k1,
                      DevBuf<uint32_t>& v1, int64_t n, int bits, cudaStream_t st) {
  if (n <= 1) return;
  int64_t ntiles = ceil_div(n, kRsTile);
  DevBuf<uint32_t> hist, scan_tmp;
  hist.alloc(256 * ntiles);
  int grid = (int)std::min<int64_t>(ntiles, 65535);
  uint64_t* ka = k0.get();
  uint64_t* kb = k1.get();
  uint32_t* va = v0.get();
  uint32_t* vb = v1.get();
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<grid, kRsThreads, 0, st>>>(ka, n, shift, hist.get(), ntiles);
    BM_CHECK_LAUNCH();
    exclusive_scan_u32(hist.get(), hist.get(), 256 * ntiles, scan_tmp, st);
    k_rs_scatter<<<grid, kRsThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist.get(), ntiles);
    BM_CHECK_LAUNCH();
    std::swap(ka, kb);
    std::swap(va, vb);
    ++passes;
  }
  if (passes & 1) {
    BM_CUDA(cudaMemcpyAsync(k0.get(), ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    BM_CUDA(cudaMemcpyAsync(v0.get(), va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  }
  BM_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------------- finalisation
__global__ void k_csr_finalize(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                               const float* __restrict__ vals, int64_t nnz, uint64_t nint, uint64_t mint,
                               int32_t* __restrict__ col, float* __restrict__ val,
                               uint64_t* __restrict__ key2, uint32_t* __restrict__ pos2,
                               int* __restrict__ flags) {
  int dup = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = sk[e];
    uint64_t r = key / nint;
    uint64_t c = key - r * nint;
    col[e] = (int32_t)c;
    val[e] = vals[sv[e]];
    key2[e] = c * mint + r;
    pos2[e] = (uint32_t)e;
    if (e > 0 && sk[e - 1] == key) dup = 1;
  }
  if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(flags + 2, 1);
}

__global__ void k_csc_finalize(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                               const float* __restrict__ val, int64_t nnz, uint64_t mint,
                               int32_t* __restrict__ row, float* __restrict__ cval,
                               int64_t* __restrict__ csr2csc, int32_t* __restrict__ csc2csr) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
       q += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = sk[q];
    uint64_t c = key / mint;
    row[q] = (int32_t)(key - c * mint);
    uint32_t e = sv[q];
    cval[q] = val[e];
    csr2csc[e] = q;
    csc2csr[q] = (int32_t)e;
  }
}

// ptr[i] = first position with key >= i * stride (lower bound), i = 0..count
__global__ void k_lower_bounds(const uint64_t* __restrict__ keys, int64_t nnz, uint64_t stride,
                               int64_t count, int64_t* __restrict__ ptr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= count;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t target = (uint64_t)i * stride;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < target) lo = mid + 1; else hi = mid;
    }
    ptr[i] = lo;
  }
}

int grid_for(int64_t n, int threads) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 32));
}

// bounds[i * (P + 1) + p] = first entry of row i whose index is >= p * pw
// (p = 0: the row start, p = P: the row end).
__global__ void k_panel_bounds(const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx, int64_t rows,
                               int P, int64_t pw, int64_t* __restrict__ bounds) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * (P + 1);
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / (P + 1);
    const int p = (int)(t - i * (P + 1));
    int64_t lo = ptr[i], hi = ptr[i + 1];
    if (p == P) {
      bounds[t] = hi;
      continue;
    }
    const int64_t target = (int64_t)p * pw;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)idx[mid] < target) lo = mid + 1; else hi = mid;
    }
    bounds[t] = lo;
  }
}

// Segments of at most kSegNnz entries within each (row, panel) piece,
// emitted panel by panel.  A row with no entries gets one empty segment (its
// output is written all the same); a row with several segments owns
// consecutive partial slots in entry order.  Within a panel the segments are
// ordered by decreasing length (ties in row order), so that the lane groups
// of one warp, which take consecutive segments, walk about as many entries
// each; the order changes no result (every segment's sums and slots are its
// own).
void build_segs_from_bounds(Segs& s, const std::vector<int64_t>& bnd, int64_t rows, int P, cudaStream_t st) {
  const int W = P + 1;
  std::vector<int32_t> cnt(rows), first(rows, -1), used(rows, 0);
  std::vector<int32_t> srow, sslot, mrow, mfirst, mcount;
  std::vector<int64_t> sbeg, send;
  int64_t nslots = 0;
  for (int64_t i = 0; i < rows; ++i) {
    int64_t c = 0;
    for (int p = 0; p < P; ++p) c += ceil_div(bnd[i * W + p + 1] - bnd[i * W + p], kSegNnz);
    cnt[i] = (int32_t)std::max<int64_t>(1, c);
    if (cnt[i] > 1) {
      first[i] = (int32_t)nslots;
      mrow.push_back((int32_t)i);
      mfirst.push_back((int32_t)nslots);
      mcount.push_back(cnt[i]);
      nslots += cnt[i];
    }
  }
  BM_REQUIRE(nslots < ((int64_t)1 << 31), BM_ERR_INVALID, "index: too many partial slots");
  for (int p = 0; p < P; ++p) {
    const size_t first_seg = srow.size();
    for (int64_t i = 0; i < rows; ++i) {
      const int64_t b = bnd[i * W + p], e = bnd[i * W + p + 1];
      if (b == e) {
        if (p == 0 && bnd[i * W] == bnd[i * W + P]) {  // empty row
          srow.push_back((int32_t)i);
          sbeg.push_back(b);
          send.push_back(b);
          sslot.push_back(-1);
        }
        continue;
      }
      for (int64_t sb = b; sb < e; sb += kSegNnz) {
        srow.push_back((int32_t)i);
        sbeg.push_back(sb);
        send.push_back(std::min(e, sb + kSegNnz));
        sslot.push_back(cnt[i] > 1 ? first[i] + used[i]++ : -1);
      }
    }
    // this panel's segments by decreasing length
    const size_t cnt_p = srow.size() - first_seg;
    std::vector<size_t> ord(cnt_p);
    for (size_t q = 0; q < cnt_p; ++q) ord[q] = first_seg + q;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](size_t x, size_t y) { return send[x] - sbeg[x] > send[y] - sbeg[y]; });
    std::vector<int32_t> r2(cnt_p), sl2(cnt_p);
    std::vector<int64_t> b2(cnt_p), e2(cnt_p);
    for (size_t q = 0; q < cnt_p; ++q) {
      r2[q] = srow[ord[q]];
      b2[q] = sbeg[ord[q]];
      e2[q] = send[ord[q]];
      sl2[q] = sslot[ord[q]];
    }
    std::copy(r2.begin(), r2.end(), srow.begin() + first_seg);
    std::copy(b2.begin(), b2.end(), sbeg.begin() + first_seg);
    std::copy(e2.begin(), e2.end(), send.begin() + first_seg);
    std::copy(sl2.begin(), sl2.end(), sslot.begin() + first_seg);
  }
  s.nseg = (int64_t)srow.size();
  s.nmulti = (int64_t)mrow.size();
  s.nslots = nslots;
  s.row.alloc(s.nseg);
  s.beg.alloc(s.nseg);
  s.end.alloc(s.nseg);
  s.slot.alloc(s.nseg);
  BM_CUDA(cudaMemcpyAsync(s.row.get(), srow.data(), s.nseg * 4, cudaMemcpyHostToDevice, st));
  BM_CUDA(cudaMemcpyAsync(s.beg.get(), sbeg.data(), s.nseg * 8, cudaMemcpyHostToDevice, st));
  BM_CUDA(cudaMemcpyAsync(s.end.get(), send.data(), s.nseg * 8, cudaMemcpyHostToDevice, st));
  BM_CUDA(cudaMemcpyAsync(s.slot.get(), sslot.data(), s.nseg * 4, cudaMemcpyHostToDevice, st));
  s.mrow.alloc(std::max<int64_t>(1, s.nmulti));
  s.mfirst.alloc(std::max<int64_t>(1, s.nmulti));
  s.mcount.alloc(std::max<int64_t>(1, s.nmulti));
  if (s.nmulti) {
    BM_CUDA(cudaMemcpyAsync(s.mrow.get(), mrow.data(), s.nmulti * 4, cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaMemcpyAsync(s.mfirst.get(), mfirst.data(), s.nmulti * 4, cudaMemcpyHostToDevice, st));
    BM_CUDA(cudaMemcpyAsync(s.mcount.get(), mcount.data(), s.nmulti * 4, cudaMemcpyHostToDevice, st));
  }
  BM_CUDA(cudaStreamSynchronize(st));
}

void build_segs(Segs& s, const DevBuf<int64_t>& ptr_d, int64_t rows, cudaStream_t st) {
  std::vector<int64_t> ptr(rows + 1);
  BM_CUDA(cudaMemcpyAsync(ptr.data(), ptr_d.get(), (rows + 1) * sizeof(int64_t),
                          cudaMemcpyDeviceToHost, st));
  BM_CUDA(cudaStreamSynchronize(st));
  std::vector<int64_t> bnd(2 * rows);
  for (int64_t i = 0; i < rows; ++i) bnd[2 * i] = ptr[i], bnd[2 * i + 1] = ptr[i + 1];
  build_segs_from_bounds(s, bnd, rows, 1, st);
}

int bits_for(uint64_t v) {  // number of bits to represent values < v
  int b = 0;
  while (b < 64 && (v - 1) >> b) ++b;
  return std::max(b, 1);
}

}  // namespace

// flags[0] = 1 if some value is not an integer; lo/hi = min/max as ordered int bits
__global__ void k_codec_scan(const float* __restrict__ v, int64_t n, int* __restrict__ flags,
                             int* __restrict__ lohi) {
  int lo = INT_MAX, hi = INT_MIN, bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float x = v[e];
    if (!(x == rintf(x)) || fabsf(x) >= 16777216.f) {
      bad = 1;
    } else {
      const int xi = (int)x;
      lo = min(lo, xi);
      hi = max(hi, xi);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(flags, 1);
    atomicMin(lohi, lo);
    atomicMax(lohi + 1, hi);
  }
}

__global__ void k_codec_encode(const float* __restrict__ v, int64_t n, int off, uint8_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (uint8_t)((int)v[e] - off);
}

void build_codec(bm_ctx& h) {
  Index& ix = h.ix;
  cudaStream_t st = h.stream;
  ix.codec = false;
  if (ix.nnz == 0 || h.opt.value_codec == 0) return;
  DevBuf<int> fl;
  fl.alloc(4);
  const int init[4] = {0, INT_MAX, INT_MIN, 0};
  BM_CUDA(cudaMemcpyAsync(fl.get(), init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_codec_scan<<<grid_for(ix.nnz, 256), 256, 0, st>>>(ix.val.get(), ix.nnz, fl.get(), fl.get() + 1);
  BM_CHECK_LAUNCH();
  int hf[4];
  BM_CUDA(cudaMemcpyAsync(hf, fl.get(), sizeof(hf), cudaMemcpyDeviceToHost, st));
  BM_CUDA(cudaStreamSynchronize(st));
  if (hf[0] || (int64_t)hf[2] - (int64_t)hf[1] > 255) return;
  ix.val8.alloc(ix.nnz);
  ix.cval8.alloc(ix.nnz);
  k_codec_encode<<<grid_for(ix.nnz, 256), 256, 0, st>>>(ix.val.get(), ix.nnz, hf[1], ix.val8.get());
  BM_CHECK_LAUNCH();
  k_codec_encode<<<grid_for(ix.nnz, 256), 256, 0, st>>>(ix.cval.get(), ix.nnz, hf[1], ix.cval8.get());
  BM_CHECK_LAUNCH();
  BM_CUDA(cudaStreamSynchronize(st));
  ix.code_off = (float)hf[1];
  ix.codec = true;
}

void build_index(bm_ctx& h, int64_t m, int64_t n, int64_t nnz, const int32_t* rows_d,
                 const int32_t* cols_d, const float* vals_d) {
  cudaStream_t st = h.stream;
  Index& ix = h.ix;
  ix.transposed = m > n;
  ix.m = ix.transposed ? n : m;
  ix.n = ix.transposed ? m : n;
  ix.nnz = nnz;
  DevBuf<int> flags;
  flags.alloc(4);
  BM_CUDA(cudaMemsetAsync(flags.get(), 0, 4 * sizeof(int), st));
  if (nnz > 0) {
    k_validate<<<grid_for(nnz, 256), 256, 0, st>>>(rows_d, cols_d, vals_d, nnz, m, n, flags.get());
    BM_CHECK_LAUNCH();
  }
  int hflags[4];
  BM_CUDA(cudaMemcpyAsync(hflags, flags.get(), sizeof(hflags), cudaMemcpyDeviceToHost, st));
  BM_CUDA(cudaStreamSynchronize(st));
  BM_REQUIRE(!hflags[0], BM_ERR_INVALID, "bm_create: row or column index out of range");
  BM_REQUIRE(!hflags[1], BM_ERR_INVALID, "bm_create: non-finite observed value");

  ix.row_ptr.alloc(ix.m + 1);
  ix.col_ptr.alloc(ix.n + 1);
  ix.col.alloc(nnz);
  ix.row.alloc(nnz);
  ix.val.alloc(nnz);
  ix.cval.alloc(nnz);
  ix.csr2csc.alloc(nnz);
  ix.csc2csr.alloc(nnz);
  {
    DevBuf<uint64_t> k0, k1;
    DevBuf<uint32_t> v0, v1;
    k0.alloc(nnz); k1.alloc(nnz); v0.alloc(nnz); v1.alloc(nnz);
    const uint64_t M = (uint64_t)ix.m, N = (uint64_t)ix.n;
    if (nnz > 0) {
      k_make_keys<<<grid_for(nnz, 256), 256, 0, st>>>(rows_d, cols_d, nnz, ix.transposed, N, k0.get(),
                                                      v0.get());
      BM_CHECK_LAUNCH();
    }
    const int bits = bits_for(M * N);
    radix_sort_pairs(k0, v0, k1, v1, nnz, bits, st);
    k_lower_bounds<<<grid_for(ix.m + 1, 256), 256, 0, st>>>(k0.get(), nnz, N, ix.m, ix.row_ptr.get());
    BM_CHECK_LAUNCH();
    if (nnz > 0) {
      // CSR arrays and CSC keys (col * m + row, value = CSR position) into (k1, v1)
      k_csr_finalize<<<grid_for(nnz, 256), 256, 0, st>>>(k0.get(), v0.get(), vals_d, nnz, N, M,
                                                         ix.col.get(), ix.val.get(), k1.get(), v1.get(),
                                                         flags.get());
      BM_CHECK_LAUNCH();
      BM_CUDA(cudaMemcpyAsync(hflags, flags.get(), sizeof(hflags), cudaMemcpyDeviceToHost, st));
      BM_CUDA(cudaStreamSynchronize(st));
      BM_REQUIRE(!hflags[2], BM_ERR_INVALID, "bm_create: repeated (row, col) entry in Omega");
    }
    radix_sort_pairs(k1, v1, k0, v0, nnz, bits, st);
    k_lower_bounds<<<grid_for(ix.n + 1, 256), 256, 0, st>>>(k1.get(), nnz, M, ix.n, ix.col_ptr.get());
    BM_CHECK_LAUNCH();
    if (nnz > 0) {
      k_csc_finalize<<<grid_for(nnz, 256), 256, 0, st>>>(k1.get(), v1.get(), ix.val.get(), nnz, M,
                                                         ix.row.get(), ix.cval.get(), ix.csr2csc.get(),
                                                         ix.csc2csr.get());
      BM_CHECK_LAUNCH();
    }
    BM_CUDA(cudaStreamSynchronize(st));
  }
  build_segs(ix.rs, ix.row_ptr, ix.m, st);
  build_segs(ix.cs, ix.col_ptr, ix.n, st);
  build_codec(h);
}

}  // namespace bm

namespace bm {
// Shared with the distance-geometry index build (edm.cu).
void sort_pairs_ext(DevBuf<uint64_t>& k0, DevBuf<uint32_t>& v0, DevBuf<uint64_t>& k1, DevBuf<uint32_t>& v1,
                    int64_t n, int bits, cudaStream_t st) {
  radix_sort_pairs(k0, v0, k1, v1, n, bits, st);
}
void build_segs_ext(Segs& s, const DevBuf<int64_t>& ptr_d, int64_t rows, cudaStream_t st) {
  build_segs(s, ptr_d, rows, st);
}
void lower_bounds_ext(const uint64_t* keys, int64_t nnz, uint64_t stride, int64_t count, int64_t* ptr,
                      cudaStream_t st) {
  k_lower_bounds<<<grid_for(count + 1, 256), 256, 0, st>>>(keys, nnz, stride, count, ptr);
  BM_CHECK_LAUNCH();
}
int key_bits_ext(uint64_t v) { return bits_for(v); }

void ensure_panel_segs(bm_ctx& h, bool csr, int P) {
  Index& ix = h.ix;
  auto& mp = csr ? ix.rsp : ix.csp;
  if (P <= 1 || mp.count(P)) return;
  const int64_t rows = csr ? ix.m : ix.n, other = csr ? ix.n : ix.m;
  const int64_t pw = ceil_div(std::max<int64_t>(other, 1), P);
  DevBuf<int64_t> bd;
  bd.alloc(rows * (P + 1));
  k_panel_bounds<<<grid_for(rows * (P + 1), 256), 256, 0, h.stream>>>(
      csr ? ix.row_ptr.get() : ix.col_ptr.get(), csr ? ix.col.get() : ix.row.get(), rows, P, pw, bd.get());
  BM_CHECK_LAUNCH();
  std::vector<int64_t> bnd(rows * (P + 1));
  BM_CUDA(cudaMemcpyAsync(bnd.data(), bd.get(), bnd.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, h.stream));
  BM_CUDA(cudaStreamSynchronize(h.stream));
  std::unique_ptr<Segs> s(new Segs());
  build_segs_from_bounds(*s, bnd, rows, P, h.stream);
  mp[P] = std::move(s);
  ensure_pass_scratch(h, 0);
}

int64_t max_slots(const Index& ix) {
  int64_t s = std::max(ix.rs.nslots, ix.cs.nslots);
  for (const auto& kv : ix.rsp) s = std::max(s, kv.second->nslots);
  for (const auto& kv : ix.csp) s = std::max(s, kv.second->nslots);
  return s;
}

int64_t max_segs(const Index& ix) {
  int64_t s = std::max(ix.rs.nseg, ix.cs.nseg);
  for (const auto& kv : ix.rsp) s = std::max(s, kv.second->nseg);
  for (const auto& kv : ix.csp) s = std::max(s, kv.second->nseg);
  return s;
}

void ensure_pass_scratch(bm_ctx& h, int ld_part) {
  h.sc.ld_part = std::max({h.sc.ld_part, ld_part, h.ldmax});
  const int64_t need_p = std::max<int64_t>(1, max_slots(h.ix)) * h.sc.ld_part;
  if ((int64_t)h.sc.partial.n < need_p) {
    h.sc.partial.release();
    h.sc.partial.alloc(need_p);
  }
  const int64_t need_f = max_segs(h.ix) * 4 + 4;
  if ((int64_t)h.sc.fseg.n < need_f) {
    h.sc.fseg.release();
    h.sc.fseg.alloc(need_f);
  }
}
}  // namespace bm
