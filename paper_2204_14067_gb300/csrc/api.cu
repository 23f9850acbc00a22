// The C ABI (include/bm.h): argument checks, host/device marshalling,
// handle lifetime, the BM phase and Algorithm 1 orchestration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <set>

#include "ctx.cuh"

namespace bm {

int num_sms() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

void allow_max_smem(const void* kernel) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, kernel})) return;
  int optin = 0;
  BM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  BM_CUDA(cudaFuncGetAttributes(&fa, kernel));
  // static and dynamic shared memory together may not exceed the opt-in limit
  BM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes));
  done.insert({dev, kernel});
}

bool is_device_ptr(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

Profiler::~Profiler() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

cudaEvent_t Profiler::next() {
  if (used == pool.size()) {
    cudaEvent_t e;
    BM_CUDA(cudaEventCreate(&e));
    pool.push_back(e);
  }
  return pool[used++];
}

void Profiler::begin(const char* name, cudaStream_t st) {
  cudaEvent_t a = next();
  BM_CUDA(cudaEventRecord(a, st));
  marks.push_back({name, {a, nullptr}});
}

void Profiler::end(cudaStream_t st) {
  cudaEvent_t b = next();
  BM_CUDA(cudaEventRecord(b, st));
  marks.back().second.second = b;
}

namespace {

thread_local std::string g_last_error;

template <class Fn>
bm_status guarded(bm_ctx* h, Fn&& fn) {
  return guard_call(h ? h->err : g_last_error, std::forward<Fn>(fn));
}

// Copy `count` elements to a device buffer if `src` is host memory.
template <typename T>
const T* to_device(const T* src, int64_t count, DevBuf<T>& tmp, cudaStream_t st) {
  if (count == 0) return src;
  if (is_device_ptr(src)) return src;
  tmp.alloc(count);
  BM_CUDA(cudaMemcpyAsync(tmp.get(), src, count * sizeof(T), cudaMemcpyHostToDevice, st));
  return tmp.get();
}

cudaMemcpyKind kind_to(const void* dst) { return is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }
cudaMemcpyKind kind_from(const void* src) { return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

// Caller-orientation factor pointers map to internal (W, H) swapped when transposed.
// Rows of k floats between a caller buffer (row stride k) and a device block
// (row stride ld >= k); with no padding (k == ld) one contiguous copy, which
// the copy engines move much faster than a pitched copy of short rows.
void copy_out_rows(bm_ctx& h, float* dst, const float* src, int64_t rows, int k) {
  if (!dst || rows == 0 || k == 0) return;
  if (k == h.ld) {
    BM_CUDA(cudaMemcpyAsync(dst, src, (size_t)rows * k * sizeof(float), kind_to(dst), h.stream));
    return;
  }
  BM_CUDA(cudaMemcpy2DAsync(dst, k * sizeof(float), src, h.ld * sizeof(float), k * sizeof(float), rows,
                            kind_to(dst), h.stream));
}

void copy_in_rows(bm_ctx& h, float* dst, const float* src, int64_t rows, int k) {
  if (src && rows > 0 && k > 0 && k == h.ld) {
    BM_CUDA(cudaMemcpyAsync(dst, src, (size_t)rows * k * sizeof(float), kind_from(src), h.stream));
    return;
  }
  BM_CUDA(cudaMemsetAsync(dst, 0, rows * h.ld * sizeof(float), h.stream));
  if (!src || rows == 0 || k == 0) return;
  BM_CUDA(cudaMemcpy2DAsync(dst, h.ld * sizeof(float), src, k * sizeof(float), k * sizeof(float), rows,
                            kind_from(src), h.stream));
}

void set_rank(bm_ctx& h, int k) {
  h.k = k;
  h.ld = std::max(4, round_up4(k));
  h.bf_dirty = true;
}

// Real roots of c1 + 2 c2 s + 3 c3 s^2 + 4 c4 s^3 = 0; pick the argmin of
// phi(s) = c0 + c1 s + ... + c4 s^4 over s = 0 and the positive roots.
double poly4(const double c[5], double s) { return (((c[4] * s + c[3]) * s + c[2]) * s + c[1]) * s + c[0]; }
double dpoly4(const double c[5], double s) { return ((4 * c[4] * s + 3 * c[3]) * s + 2 * c[2]) * s + c[1]; }
double ddpoly4(const double c[5], double s) { return (12 * c[4] * s + 6 * c[3]) * s + 2 * c[2]; }

double quartic_argmin(const double c[5]) {
  std::vector<double> roots;
  const double a3 = 4 * c[4], a2 = 3 * c[3], a1 = 2 * c[2], a0 = c[1];
  const double scale = std::max({std::fabs(a3), std::fabs(a2), std::fabs(a1), std::fabs(a0), 1e-300});
  if (std::fabs(a3) > 1e-14 * scale) {
    // s^3 + p2 s^2 + p1 s + p0 = 0, depressed with s = t - p2/3
    const double p2 = a2 / a3, p1 = a1 / a3, p0 = a0 / a3;
    const double q = (3 * p1 - p2 * p2) / 9.0;
    const double r = (9 * p2 * p1 - 27 * p0 - 2 * p2 * p2 * p2) / 54.0;
    const double disc = q * q * q + r * r;
    if (disc > 0) {
      const double sq = std::sqrt(disc);
      const double s1 = std::cbrt(r + sq), s2 = std::cbrt(r - sq);
      roots.push_back(s1 + s2 - p2 / 3.0);
    } else {
      const double th = std::acos(std::max(-1.0, std::min(1.0, q < 0 ? r / std::sqrt(-q * q * q) : 0.0)));
      const double m = 2.0 * std::sqrt(std::max(0.0, -q));
      for (int t = 0; t < 3; ++t) roots.push_back(m * std::cos((th + 2.0 * M_PI * t) / 3.0) - p2 / 3.0);
    }
  } else if (std::fabs(a2) > 1e-14 * scale) {
    const double d = a1 * a1 - 4 * a2 * a0;
    if (d >= 0) {
      const double sq = std::sqrt(d);
      const double qq = -0.5 * (a1 + (a1 >= 0 ? sq : -sq));
      if (qq != 0) roots.push_back(qq / a2), roots.push_back(a0 / qq);
      else roots.push_back(0.0);
    }
  } else if (std::fabs(a1) > 0) {
    roots.push_back(-a0 / a1);
  }
  double best_s = 0.0, best = poly4(c, 0.0);
  for (double s : roots) {
    for (int it = 0; it < 3; ++it) {  // Newton polish on phi'
      const double d2 = ddpoly4(c, s);
      if (d2 == 0) break;
      s -= dpoly4(c, s) / d2;
    }
    if (!(s > 0) || !std::isfinite(s)) continue;
    const double v = poly4(c, s);
    if (v < best) best = v, best_s = s;
  }
  return best_s;
}

double objective_now(bm_ctx& h, double* f_out = nullptr) {
  LossOut o = loss_grad_dev(h, false, false);
  if (f_out) *f_out = o.f;
  return o.f + 0.5 * h.lambda * (o.nW2 + o.nH2);
}

// `epochs` BM iterations.  Returns F at entry (from the first loss evaluation);
// *F_out receives F after the last step, read off the line-search quartic
// (exact in exact arithmetic), so no extra loss pass is spent on it.
double bm_phase_dev(bm_ctx& h, int epochs, double* F_out) {
  const Index& ix = h.ix;
  double F = 0.0, F_entry = 0.0;
  double gg_prev = 0.0;
  bool have_prev = false;
  if (epochs <= 0 || h.k == 0) {
    F_entry = objective_now(h);
    if (F_out) *F_out = F_entry;
    return F_entry;
  }
  for (int e = 0; e < epochs; ++e) {
    const int64_t mW = ix.m * h.ld, nH = ix.n * h.ld;
    LossOut o = loss_grad_dev(h, true, true);
    F = o.f + 0.5 * h.lambda * (o.nW2 + o.nH2);
    BM_REQUIRE(std::isfinite(F), BM_ERR_NUMERIC, "bm_bm_phase: objective is not finite");
    if (e == 0) F_entry = F;
    const double gg = dot_dev(h, h.gW.get(), h.gW.get(), mW) + dot_dev(h, h.gH.get(), h.gH.get(), nH);
    double beta = 0.0;
    if (have_prev && gg_prev > 0) {
      const double gp = dot_dev(h, h.gW.get(), h.gWp.get(), mW) + dot_dev(h, h.gH.get(), h.gHp.get(), nH);
      beta = std::max(0.0, (gg - gp) / gg_prev);
    }
    if (!have_prev) {
      BM_CUDA(cudaMemsetAsync(h.DW.get(), 0, mW * sizeof(float), h.stream));
      BM_CUDA(cudaMemsetAsync(h.DH.get(), 0, nH * sizeof(float), h.stream));
    }
    xpby_dev(h, h.DW.get(), h.gW.get(), (float)beta, mW);  // D = -g + beta D
    xpby_dev(h, h.DH.get(), h.gH.get(), (float)beta, nH);
    if (beta > 0) {
      const double dg = dot_dev(h, h.DW.get(), h.gW.get(), mW) + dot_dev(h, h.DH.get(), h.gH.get(), nH);
      if (dg >= 0) {
        xpby_dev(h, h.DW.get(), h.gW.get(), 0.0f, mW);
        xpby_dev(h, h.DH.get(), h.gH.get(), 0.0f, nH);
      }
    }
    double c[5];
    c[0] = F;
    line_search_coeffs_dev(h, c);
    const double s = quartic_argmin(c);
    if (s > 0) {
      axpy_dev(h, h.W.get(), h.DW.get(), (float)s, mW);
      axpy_dev(h, h.H.get(), h.DH.get(), (float)s, nH);
      h.bm_changed = true;
      h.bf_dirty = true;
      F = poly4(c, s);
    }
    if (e + 1 < epochs) {
      BM_CUDA(cudaMemcpyAsync(h.gWp.get(), h.gW.get(), mW * sizeof(float), cudaMemcpyDeviceToDevice, h.stream));
      BM_CUDA(cudaMemcpyAsync(h.gHp.get(), h.gH.get(), nH * sizeof(float), cudaMemcpyDeviceToDevice, h.stream));
    }
    gg_prev = gg;
    have_prev = true;
  }
  if (F_out) *F_out = F;
  BM_CUDA(cudaStreamSynchronize(h.stream));
  return F_entry;
}

}  // namespace
}  // namespace bm

using namespace bm;

namespace bm {
void profile_report(Profiler& prof, int32_t cap, char* names, int64_t* launches, double* total_ms,
                    int32_t* count) {
  std::vector<std::string> keys;
  std::vector<int64_t> cnt;
  std::vector<double> ms;
  for (auto& mk : prof.marks) {
    if (!mk.second.second) continue;
    float t = 0.f;
    BM_CUDA(cudaEventElapsedTime(&t, mk.second.first, mk.second.second));
    size_t i = 0;
    while (i < keys.size() && keys[i] != mk.first) ++i;
    if (i == keys.size()) keys.push_back(mk.first), cnt.push_back(0), ms.push_back(0.0);
    cnt[i] += 1;
    ms[i] += t;
  }
  if (count) *count = (int32_t)keys.size();
  for (size_t i = 0; i < keys.size() && (int32_t)i < cap; ++i) {
    if (names) {
      std::snprintf(names + 48 * i, 48, "%s", keys[i].c_str());
    }
    if (launches) launches[i] = cnt[i];
    if (total_ms) total_ms[i] = ms[i];
  }
}
}  // namespace bm

extern "C" {

bm_status bm_default_options(bm_options* o) {
  if (!o) return BM_ERR_INVALID;
  o->alpha = 1.99;
  o->bm_epochs = 3;
  o->pg_steps = 1;
  o->lmsvd_p = 1;
  o->lmsvd_imax = 50;
  o->lmsvd_min_iter = 2;
  o->lmsvd_tol = 1e-5;
  o->tau = 1e-6;
  o->ritz_rel = 1e-6;
  o->psi0 = 0.1;
  o->k_init = 8;
  o->precision = 0;
  o->autotune = 0;
  o->step_rule = 0;
  o->value_codec = 1;
  o->bm_solver = 0;
  o->tensor_grams = 1;
  o->pad_ = 0;
  o->seed = 0;
  return BM_OK;
}

bm_status bm_create(int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                    const float* vals, double lambda, int32_t k_max, const bm_options* opt,
                    bm_handle* out) {
  if (!out) {
    g_last_error = "bm_create: out is NULL";
    return BM_ERR_INVALID;
  }
  *out = nullptr;
  bm_ctx* h = nullptr;
  bm_status st = guarded(nullptr, [&] {
    BM_REQUIRE(m >= 1 && n >= 1, BM_ERR_INVALID, "bm_create: m and n must be >= 1");
    BM_REQUIRE(m < (1LL << 31) && n < (1LL << 31), BM_ERR_INVALID, "bm_create: m and n must be < 2^31");
    BM_REQUIRE(nnz >= 0 && nnz < (1LL << 31), BM_ERR_INVALID, "bm_create: nnz must be in [0, 2^31)");
    BM_REQUIRE(nnz == 0 || (rows && cols && vals), BM_ERR_INVALID, "bm_create: NULL index or value array");
    BM_REQUIRE(std::isfinite(lambda) && lambda > 0, BM_ERR_INVALID, "bm_create: lambda must be finite and > 0");
    BM_REQUIRE(k_max >= 1 && k_max <= std::min(m, n) && k_max <= 127, BM_ERR_INVALID,
               "bm_create: k_max must be in [1, min(m, n)] and <= 127");
    bm_options o;
    if (opt) o = *opt; else bm_default_options(&o);
    BM_REQUIRE(o.alpha > 0 && std::isfinite(o.alpha), BM_ERR_INVALID, "bm_create: alpha must be > 0");
    BM_REQUIRE(o.lmsvd_p >= 0 && o.lmsvd_p <= 1, BM_ERR_INVALID, "bm_create: lmsvd_p must be 0 or 1");
    BM_REQUIRE(o.precision == 0 || o.precision == 1, BM_ERR_INVALID, "bm_create: precision must be 0 or 1");
    BM_REQUIRE(o.step_rule == 0 || o.step_rule == 1, BM_ERR_INVALID, "bm_create: step_rule must be 0 or 1");
    BM_REQUIRE(o.value_codec == 0 || o.value_codec == 1, BM_ERR_INVALID, "bm_create: value_codec must be 0 or 1");
    BM_REQUIRE(o.bm_solver == 0 || o.bm_solver == 1, BM_ERR_INVALID, "bm_create: bm_solver must be 0 or 1");
    BM_REQUIRE(o.tensor_grams == 0 || o.tensor_grams == 1, BM_ERR_INVALID, "bm_create: tensor_grams must be 0 or 1");
    BM_REQUIRE(o.lmsvd_imax >= 1 && o.k_init >= 1 && o.bm_epochs >= 0 && o.pg_steps >= 0, BM_ERR_INVALID,
               "bm_create: iteration counts out of range");
    h = new bm_ctx();
    h->opt = o;
    h->lambda = lambda;
    h->k_max = k_max;
    BM_CUDA(cudaGetDevice(&h->device));
    BM_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    DevBuf<int32_t> tr, tc;
    DevBuf<float> tv;
    const int32_t* rd = to_device(rows, nnz, tr, h->stream);
    const int32_t* cd = to_device(cols, nnz, tc, h->stream);
    const float* vd = to_device(vals, nnz, tv, h->stream);
    build_index(*h, m, n, nnz, rd, cd, vd);
    const Index& ix = h->ix;
    h->ldmax = round_up4(k_max + 1);
    const int64_t mW = ix.m * h->ldmax, nH = ix.n * h->ldmax;
    h->W.alloc(mW); h->H.alloc(nH);
    h->gW.alloc(mW); h->gH.alloc(nH);
    h->DW.alloc(mW); h->DH.alloc(nH);
    h->gWp.alloc(mW); h->gHp.alloc(nH);
    h->r_csr.alloc(std::max<int64_t>(1, nnz));
    h->r_csc.alloc(std::max<int64_t>(1, nnz));
    if (o.precision == 1) {
      const int64_t ldb = ((h->ldmax + 7) / 8) * 8;
      h->Wb.alloc(ix.m * ldb);
      h->Hb.alloc(ix.n * ldb);
      h->DHb.alloc(ix.n * ldb);
    }
    ensure_pass_scratch(*h, h->ldmax);
    h->sc.red.alloc(4096);
    h->sc.scal.alloc(64);
    set_rank(*h, 0);
    BM_CUDA(cudaMemsetAsync(h->W.get(), 0, mW * sizeof(float), h->stream));
    BM_CUDA(cudaMemsetAsync(h->H.get(), 0, nH * sizeof(float), h->stream));
    prox_create(*h);
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
  if (st != BM_OK) {
    if (h) bm_destroy(h);
    return st;
  }
  *out = h;
  return BM_OK;
}

void bm_destroy(bm_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  prox_destroy(*h);
  bb_destroy(h->bb);
  h->bb = nullptr;
  bcd_destroy(h->bcd);
  h->bcd = nullptr;
  if (h->side_stream) {
    cudaStreamSynchronize(h->side_stream);
    cudaStreamDestroy(h->side_stream);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  cudaStream_t own = h->own_stream;
  delete h;
  if (own) cudaStreamDestroy(own);
}

const char* bm_last_error(bm_handle h) { return h ? h->err.c_str() : g_last_error.c_str(); }

bm_status bm_set_stream(bm_handle h, void* stream) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    BM_CUDA(cudaStreamSynchronize(h->stream));
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  });
}

bm_status bm_dims(bm_handle h, int64_t* m, int64_t* n, int64_t* nnz, int32_t* transposed, int32_t* k) {
  if (!h) return BM_ERR_INVALID;
  if (m) *m = h->ix.m;
  if (n) *n = h->ix.n;
  if (nnz) *nnz = h->ix.nnz;
  if (transposed) *transposed = h->ix.transposed ? 1 : 0;
  if (k) *k = h->k;
  return BM_OK;
}

bm_status bm_get_codes(bm_handle h, int32_t* active, float* offset, uint8_t* csr_codes, uint8_t* csc_codes) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    const Index& ix = h->ix;
    if (active) *active = ix.codec ? 1 : 0;
    if (offset) *offset = ix.code_off;
    if (ix.codec && ix.nnz) {
      if (csr_codes)
        BM_CUDA(cudaMemcpyAsync(csr_codes, ix.val8.get(), ix.nnz, kind_to(csr_codes), h->stream));
      if (csc_codes)
        BM_CUDA(cudaMemcpyAsync(csc_codes, ix.cval8.get(), ix.nnz, kind_to(csc_codes), h->stream));
    }
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
}

bm_status bm_get_index(bm_handle h, int64_t* row_ptr, int32_t* col, float* val, int64_t* col_ptr,
                       int32_t* row, float* cval, int64_t* csr2csc) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    const Index& ix = h->ix;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (dst && bytes) BM_CUDA(cudaMemcpyAsync(dst, src, bytes, kind_to(dst), h->stream));
    };
    cp(row_ptr, ix.row_ptr.get(), (ix.m + 1) * 8);
    cp(col_ptr, ix.col_ptr.get(), (ix.n + 1) * 8);
    cp(col, ix.col.get(), ix.nnz * 4);
    cp(val, ix.val.get(), ix.nnz * 4);
    cp(row, ix.row.get(), ix.nnz * 4);
    cp(cval, ix.cval.get(), ix.nnz * 4);
    cp(csr2csc, ix.csr2csc.get(), ix.nnz * 8);
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
}

bm_status bm_set_factors(bm_handle h, int32_t k, const float* W, const float* H) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    BM_REQUIRE(k >= 0 && k <= h->k_max, BM_ERR_INVALID, "bm_set_factors: k must be in [0, k_max]");
    BM_REQUIRE(k == 0 || (W && H), BM_ERR_INVALID, "bm_set_factors: NULL factor");
    set_rank(*h, k);
    h->refine = false;
    const float* Wi = h->ix.transposed ? H : W;
    const float* Hi = h->ix.transposed ? W : H;
    copy_in_rows(*h, h->W.get(), Wi, h->ix.m, k);
    copy_in_rows(*h, h->H.get(), Hi, h->ix.n, k);
    prox_reset(*h);
    h->bm_changed = true;
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
}

namespace {
// Checkpoint layout: this header, W (m x k) and H (n x k) in the internal
// orientation with rows packed, then the PG-step state.
struct StateHeader {
  char magic[8];
  int64_t m, n, nnz;
  int32_t k, k_max;
  int32_t bm_changed, refine;
  int32_t panels[kPassKinds];
  int32_t pad_;
  int64_t prox_bytes;
};
constexpr char kStateMagic[8] = {'B', 'M', 'S', 'T', 'A', 'T', 'E', '1'};
}  // namespace

bm_status bm_get_state(bm_handle h, void* buf, size_t* len) {
  if (!h || !len) return BM_ERR_INVALID;
  return guarded(h, [&] {
    const size_t pb = prox_state_bytes(*h);
    const size_t fb = ((size_t)h->ix.m + (size_t)h->ix.n) * (size_t)h->k * sizeof(float);
    const size_t need = sizeof(StateHeader) + fb + pb;
    if (!buf) {
      *len = need;
      return;
    }
    BM_REQUIRE(*len >= need, BM_ERR_INVALID, "bm_get_state: buffer too small (pass buf = NULL to get the size)");
    StateHeader hd{};
    std::memcpy(hd.magic, kStateMagic, sizeof(kStateMagic));
    hd.m = h->ix.m;
    hd.n = h->ix.n;
    hd.nnz = h->ix.nnz;
    hd.k = h->k;
    hd.k_max = h->k_max;
    hd.bm_changed = h->bm_changed ? 1 : 0;
    hd.refine = h->refine ? 1 : 0;
    for (int i = 0; i < kPassKinds; ++i) hd.panels[i] = h->ix.panels[i];
    hd.prox_bytes = (int64_t)pb;
    uint8_t* p = static_cast<uint8_t*>(buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    copy_out_rows(*h, reinterpret_cast<float*>(p), h->W.get(), h->ix.m, h->k);
    p += (size_t)h->ix.m * h->k * sizeof(float);
    copy_out_rows(*h, reinterpret_cast<float*>(p), h->H.get(), h->ix.n, h->k);
    p += (size_t)h->ix.n * h->k * sizeof(float);
    BM_CUDA(cudaStreamSynchronize(h->stream));
    prox_state_save(*h, p);
    *len = need;
  });
}

bm_status bm_set_state(bm_handle h, const void* buf, size_t len) {
  if (!h || !buf) return BM_ERR_INVALID;
  return guarded(h, [&] {
    BM_REQUIRE(len >= sizeof(StateHeader), BM_ERR_INVALID, "bm_set_state: truncated state");
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    BM_REQUIRE(std::memcmp(hd.magic, kStateMagic, sizeof(kStateMagic)) == 0, BM_ERR_INVALID,
               "bm_set_state: not a state written by bm_get_state");
    BM_REQUIRE(hd.m == h->ix.m && hd.n == h->ix.n && hd.nnz == h->ix.nnz && hd.k_max == h->k_max, BM_ERR_INVALID,
               "bm_set_state: the state belongs to a problem of other dimensions or rank cap");
    BM_REQUIRE(hd.k >= 0 && hd.k <= h->k_max && hd.prox_bytes >= 0, BM_ERR_INVALID, "bm_set_state: invalid state");
    for (int i = 0; i < kPassKinds; ++i)
      BM_REQUIRE(hd.panels[i] >= 1 && hd.panels[i] <= BM_MAX_PANELS, BM_ERR_INVALID, "bm_set_state: invalid state");
    const size_t fb = ((size_t)hd.m + (size_t)hd.n) * (size_t)hd.k * sizeof(float);
    BM_REQUIRE(len == sizeof(StateHeader) + fb + (size_t)hd.prox_bytes, BM_ERR_INVALID,
               "bm_set_state: state size mismatch");
    const uint8_t* p = static_cast<const uint8_t*>(buf) + sizeof(hd);
    set_rank(*h, hd.k);
    copy_in_rows(*h, h->W.get(), reinterpret_cast<const float*>(p), h->ix.m, hd.k);
    p += (size_t)hd.m * hd.k * sizeof(float);
    copy_in_rows(*h, h->H.get(), reinterpret_cast<const float*>(p), h->ix.n, hd.k);
    p += (size_t)hd.n * hd.k * sizeof(float);
    BM_CUDA(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < kPassKinds; ++i) {
      ensure_panel_segs(*h, pass_is_csr(i), hd.panels[i]);
      h->ix.panels[i] = hd.panels[i];
    }
    prox_reset(*h);
    prox_state_load(*h, p, (size_t)hd.prox_bytes);
    h->bm_changed = hd.bm_changed != 0;
    h->refine = hd.refine != 0;
  });
}

bm_status bm_get_factors(bm_handle h, int32_t* k, float* W, float* H) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    if (k) *k = h->k;
    float* Wo = h->ix.transposed ? H : W;
    float* Ho = h->ix.transposed ? W : H;
    copy_out_rows(*h, Wo, h->W.get(), h->ix.m, h->k);
    copy_out_rows(*h, Ho, h->H.get(), h->ix.n, h->k);
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
}

bm_status bm_loss_grad(bm_handle h, double* f, double* F, float* gW, float* gH) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    const bool want = gW || gH;
    LossOut o = loss_grad_dev(*h, want, false);
    const double Fv = o.f + 0.5 * h->lambda * (o.nW2 + o.nH2);
    BM_REQUIRE(std::isfinite(Fv), BM_ERR_NUMERIC, "bm_loss_grad: objective is not finite");
    if (f) *f = o.f;
    if (F) *F = Fv;
    float* gWo = h->ix.transposed ? gH : gW;
    float* gHo = h->ix.transposed ? gW : gH;
    copy_out_rows(*h, gWo, h->gW.get(), h->ix.m, h->k);
    copy_out_rows(*h, gHo, h->gH.get(), h->ix.n, h->k);
    BM_CUDA(cudaStreamSynchronize(h->stream));
  });
}

bm_status bm_bm_phase(bm_handle h, int32_t epochs, double* F) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    BM_REQUIRE(epochs >= 0, BM_ERR_INVALID, "bm_bm_phase: epochs must be >= 0");
    bm_phase_dev(*h, epochs, F);
  });
}

bm_status bm_init(bm_handle h, bm_prox_info* info) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] { init_step_dev(*h, info); });
}

bm_status bm_prox_step(bm_handle h, double alpha, bm_prox_info* info) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    const double a = alpha > 0 ? alpha : h->opt.alpha;
    BM_REQUIRE(std::isfinite(a), BM_ERR_INVALID, "bm_prox_step: alpha must be finite");
    prox_step_dev(*h, a, info);
  });
}

bm_status bm_solve(bm_handle h, const bm_solve_opts* o, bm_solve_info* info) {
  if (!h) return BM_ERR_INVALID;
  bool converged = false;
  bm_status st = guarded(h, [&] {
    bm_solve_opts so{100, 0, 1e-10, 0.0, 0.0};
    if (o) so = *o;
    BM_REQUIRE(so.max_outer >= 0, BM_ERR_INVALID, "bm_solve: max_outer must be >= 0");
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&] {
      return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    bm_prox_info pi;
    if (h->k == 0) init_step_dev(*h, nullptr);
    if (h->opt.autotune && !h->tuned && h->k > 0) autotune_dev(*h, BM_MAX_PANELS, nullptr);
    // F(X_t) is read from the first loss pass of each BM phase; the BM output
    // X~_t (F from its line search) is an iterate too and may end the solve.
    double F_prev = 0.0, F = 0.0;
    bool have_prev = false;
    int outer = 0;
    for (outer = 1; outer <= so.max_outer; ++outer) {
      double F_bm = 0.0;
      F = h->opt.bm_solver == 1 ? bcd_phase_dev(*h, h->opt.bm_epochs, &F_bm)
                                : bm_phase_dev(*h, h->opt.bm_epochs, &F_bm);
      BM_REQUIRE(std::isfinite(F), BM_ERR_NUMERIC, "bm_solve: objective is not finite");
      if (have_prev) {
        if (so.F_target > 0 && F <= so.F_target) { converged = true; break; }
        const double rel = std::fabs(F_prev - F) / (1.0 + std::fabs(F_prev));
        if (rel < so.tol) { converged = true; break; }
        // BF16 gathers: the final iterations run in FP32 once progress reaches
        // the BF16 noise level (relative change < 3e-3 or no decrease)
        if (h->opt.precision == 1 && !h->refine && (rel < 3e-3 || F >= F_prev)) h->refine = true;
      }
      if (so.F_target > 0 && F_bm <= so.F_target) { converged = true; break; }
      F_prev = F;
      have_prev = true;
      for (int x = 0; x < h->opt.pg_steps; ++x) {
        if (h->opt.step_rule == 1)
          prox_step_bb_dev(*h, nullptr, nullptr);
        else
          prox_step_dev(*h, h->opt.alpha, nullptr);
      }
      if (so.time_limit_s > 0 && elapsed() > so.time_limit_s) { ++outer; break; }
    }
    F = objective_now(*h);
    if (!converged && so.F_target > 0 && F <= so.F_target) converged = true;
    if (info) {
      info->outer = std::min(outer, so.max_outer);
      info->k = h->k;
      info->converged = converged ? 1 : 0;
      info->F = F;
      info->seconds = elapsed();
    }
    (void)pi;
  });
  if (st == BM_OK && !converged) {
    h->err = "bm_solve: stopped on max_outer or time_limit_s";
    return BM_ERR_NOT_CONVERGED;
  }
  return st;
}

}  // extern "C" (solve)

extern "C" {

bm_status bm_profile_enable(bm_handle h, int32_t enable) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    BM_CUDA(cudaStreamSynchronize(h->stream));
    h->prof.marks.clear();
    h->prof.used = 0;
    h->prof.on = enable != 0;
  });
}

bm_status bm_profile_read(bm_handle h, int32_t cap, char* names, int64_t* launches, double* total_ms,
                          int32_t* count) {
  if (!h) return BM_ERR_INVALID;
  return guarded(h, [&] {
    BM_CUDA(cudaStreamSynchronize(h->stream));
    profile_report(h->prof, cap, names, launches, total_ms, count);
  });
}

}  // extern "C"

namespace bm {
// exported for prox.cu
void set_rank_ext(bm_ctx& h, int k) { set_rank(h, k); }
double quartic_argmin_ext(const double c[5]) { return quartic_argmin(c); }
double objective_ext(bm_ctx& h) { return objective_now(h); }
}  // namespace bm
