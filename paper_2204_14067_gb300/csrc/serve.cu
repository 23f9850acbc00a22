// Continuous-batching server for many matrix-completion solves.
//
// A server thread admits queued requests while a slot is free and the
// device-memory estimate fits, initialises them (bm_create + bm_init), and
// advances all active solves cycle by cycle (Algorithm 1): in batched mode the
// BM phases of all active solves run as one bm_batch (CUDA-graph replay,
// one launch per sparse pass), then their PG steps run concurrently from a
// pool of host threads, each solve on its own stream.  Requests that arrive
// while others are on the GPU join at the next cycle; finished solves leave
// and free their slot and memory.  The plain mode runs one solve at a time
// with bm_solve.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int64_t m, n;
  std::vector<int32_t> rows, cols;
  std::vector<float> vals;
  double lambda;
  int32_t k_max;
  double t_submit;
};

struct Active {
  Request req;
  bm_handle h = nullptr;
  double t_start = 0;
  double F_prev = NAN, F = NAN;
  int outer = 0;
  size_t mem = 0;
};

thread_local std::string g_server_error;

}  // namespace

struct KeptFactors {
  int32_t k = 0;
  std::vector<float> W, H;   // caller orientation, m x k and n x k
};

struct bm_server_ctx {
  bm_server_opts o{};
  std::map<int64_t, KeptFactors> kept;   // keep_factors: finished solves' factors by request id
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request> queue;
  std::vector<bm_request_result> done;
  std::atomic<bool> stop{false};
  std::atomic<int> in_system{0};
  int64_t next_id = 0;
  size_t mem_used = 0;
  int device = 0;
  std::thread th;
  std::string err;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Device bytes a solve needs (index, factors and their work copies, PG
// blocks), with a margin; used for admission.
size_t estimate_bytes(const Request& r, int prec) {
  const int64_t m = std::min(r.m, r.n), n = std::max(r.m, r.n), nnz = (int64_t)r.rows.size();
  const int64_t ld = (r.k_max + 1 + 3) / 4 * 4, ld2 = (2 * (r.k_max + 1) + 3) / 4 * 4;
  size_t b = (size_t)nnz * (4 + 4 + 4 + 4 + 8 + 4 + 4 + 4);       // index, map, residual in both orders
  b += (size_t)nnz * 24;                                          // radix-sort scratch during create
  b += (size_t)(m + n) * ld * 4 * 8;                               // W, H, gradients, directions
  b += (size_t)m * ld2 * 4 * 17 + (size_t)n * ld * 4 * 2 + (size_t)n * ld2 * 4;  // PG blocks
  if (prec == 1) b += (size_t)(m + n) * ld * 2 * 3 + (size_t)std::max(m * ld2, n * ld) * 2;
  return b + b / 4 + (64u << 20);
}

void finish(bm_server_ctx& s, Active& a, bm_status st) {
  if (st != BM_OK) {
    // keep the failing request's message for bm_server_last_error
    const std::string msg = "request " + std::to_string(a.req.id) + ": " + bm_last_error(a.h);
    std::lock_guard<std::mutex> lk(s.mu);
    s.err = msg;
  }
  bm_request_result r{};
  r.id = a.req.id;
  r.status = st;
  r.outer = a.outer;
  r.F = a.F;
  int32_t k = 0;
  if (a.h) bm_dims(a.h, nullptr, nullptr, nullptr, nullptr, &k);
  r.k = k;
  r.t_submit = a.req.t_submit;
  r.t_start = a.t_start;
  r.t_done = s.now();
  KeptFactors kf;
  bool keep = false;
  if (s.o.keep_factors && st == BM_OK && a.h) {
    kf.k = k;
    try {
      kf.W.resize((size_t)a.req.m * k);
      kf.H.resize((size_t)a.req.n * k);
      int32_t kk = 0;
      if (bm_get_factors(a.h, &kk, kf.W.data(), kf.H.data()) == BM_OK && kk == k) keep = true;
      else r.status = BM_ERR_CUDA;
    } catch (...) {
      r.status = BM_ERR_OOM;   // no host memory for the kept factors
    }
  }
  if (a.h) bm_destroy(a.h);
  a.h = nullptr;
  std::lock_guard<std::mutex> lk(s.mu);
  if (keep) s.kept[r.id] = std::move(kf);
  s.mem_used -= a.mem;
  s.done.push_back(r);
  s.in_system--;
  s.cv.notify_all();
}

bool admit_one(bm_server_ctx& s, std::vector<Active>& act) {
  Request req;
  size_t need = 0;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    if (s.queue.empty() || (int)act.size() >= s.o.max_active) return false;
    need = estimate_bytes(s.queue.front(), s.o.precision);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t budget = s.o.mem_budget_gb > 0 ? (size_t)(s.o.mem_budget_gb * 1e9) : total_b;
    if (!act.empty() && (s.mem_used + need > budget || need + (1u << 30) > free_b)) return false;
    req = std::move(s.queue.front());
    s.queue.pop_front();
    s.mem_used += need;
  }
  Active a;
  a.req = std::move(req);
  a.mem = need;
  a.t_start = s.now();
  bm_options o;
  bm_default_options(&o);
  o.precision = s.o.precision;
  bm_status st = bm_create(a.req.m, a.req.n, (int64_t)a.req.rows.size(), a.req.rows.data(), a.req.cols.data(),
                           a.req.vals.data(), a.req.lambda, a.req.k_max, &o, &a.h);
  if (st == BM_OK) st = bm_init(a.h, nullptr);
  if (st != BM_OK) {
    finish(s, a, st);
    return true;
  }
  // release the host copy of the request data
  std::vector<int32_t>().swap(a.req.rows);
  std::vector<int32_t>().swap(a.req.cols);
  std::vector<float>().swap(a.req.vals);
  act.push_back(std::move(a));
  return true;
}

void run_plain(bm_server_ctx& s) {
  std::vector<Active> act;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s.mu);
      s.cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return s.stop.load() || !s.queue.empty(); });
      if (s.stop && s.queue.empty()) return;
    }
    if (!admit_one(s, act)) continue;
    if (act.empty()) continue;
    Active& a = act.back();
    bm_solve_opts so{s.o.max_outer, 0, s.o.tol, 0.0, 0.0};
    bm_solve_info info{};
    bm_status st = bm_solve(a.h, &so, &info);
    if (st == BM_ERR_NOT_CONVERGED) st = BM_OK;
    a.outer = info.outer;
    a.F = info.F;
    finish(s, a, st);
    act.clear();
  }
}

void run_batched(bm_server_ctx& s) {
  std::vector<Active> act;
  bm_batch bt = nullptr;
  std::vector<bm_handle> bt_set;
  const int nw = std::max(1, s.o.workers);
  while (true) {
    while (admit_one(s, act)) {
    }
    if (act.empty()) {
      std::unique_lock<std::mutex> lk(s.mu);
      if (s.stop && s.queue.empty()) break;
      s.cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return s.stop.load() || !s.queue.empty(); });
      continue;
    }
    // BM phase of every active solve of rank >= 1 as one batch (a rank-0
    // iterate has no factors to move; its next PG step starts from X = 0)
    std::vector<bm_handle> set;
    std::vector<size_t> in_batch;
    for (size_t i = 0; i < act.size(); ++i) {
      int32_t k = 0;
      bm_dims(act[i].h, nullptr, nullptr, nullptr, nullptr, &k);
      if (k >= 1) set.push_back(act[i].h), in_batch.push_back(i);
    }
    if (set != bt_set) {
      if (bt) bm_batch_destroy(bt);
      bt = nullptr;
      if (!set.empty() && bm_batch_create(set.data(), (int32_t)set.size(), &bt) != BM_OK) bt = nullptr;
      bt_set = set;
    }
    std::vector<double> Fb(set.size(), NAN);
    std::vector<bm_status> sts(act.size(), BM_OK);
    if (bt) {
      const bm_status st = bm_batch_bm_phase(bt, 3, Fb.data());
      if (st != BM_OK)
        for (size_t i : in_batch) sts[i] = st;
    }
    // PG steps concurrently, each solve on its own stream; the server thread
    // is one of the workers (a worker thread that cannot be started leaves
    // its share to the others)
    std::atomic<size_t> next{0};
    auto work = [&] {
      cudaSetDevice(s.device);
      for (size_t i = next++; i < act.size(); i = next++) {
        if (sts[i] != BM_OK) continue;
        bm_prox_info pi{};
        sts[i] = bm_prox_step(act[i].h, 0.0, &pi);
        act[i].F_prev = act[i].F;
        act[i].F = pi.F;
        act[i].outer++;
        // BF16 gathers: the final iterations run in FP32 once progress stalls
        if (std::isfinite(act[i].F_prev) && act[i].h->opt.precision == 1 && !act[i].h->refine &&
            (std::fabs(act[i].F_prev - act[i].F) / (1.0 + std::fabs(act[i].F_prev)) < 3e-3 ||
             act[i].F >= act[i].F_prev))
          act[i].h->refine = true;
      }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < std::min<int>(nw, (int)act.size()); ++w) {
      try {
        pool.emplace_back(work);
      } catch (...) {
        break;
      }
    }
    work();
    for (auto& t : pool) t.join();
    // retire finished solves.  A batch must not outlive its handles: when a
    // member retires the batch is destroyed first (a later bm_create may
    // return the freed handle's address, so the handle list alone cannot
    // tell an old batch from a new one).
    std::vector<Active> keep;
    for (size_t i = 0; i < act.size(); ++i) {
      Active& a = act[i];
      const bool conv = std::isfinite(a.F_prev) && (a.h->opt.precision == 0 || a.h->refine) &&
                        std::fabs(a.F_prev - a.F) / (1.0 + std::fabs(a.F_prev)) < s.o.tol;
      if (sts[i] != BM_OK || conv || a.outer >= s.o.max_outer) {
        if (bt && std::find(bt_set.begin(), bt_set.end(), a.h) != bt_set.end()) {
          bm_batch_destroy(bt);
          bt = nullptr;
          bt_set.clear();
        }
        finish(s, a, sts[i]);
      } else {
        keep.push_back(std::move(a));
      }
    }
    act.swap(keep);
  }
  if (bt) bm_batch_destroy(bt);
}

}  // namespace

extern "C" {

bm_status bm_server_create(const bm_server_opts* o, bm_server* out) {
  if (!o || !out) return BM_ERR_INVALID;
  if (o->max_active < 1 || o->max_outer < 1 || (o->precision != 0 && o->precision != 1) ||
      (o->keep_factors != 0 && o->keep_factors != 1)) {
    g_server_error = "bm_server_create: max_active, max_outer >= 1, precision and keep_factors 0 or 1 required";
    return BM_ERR_INVALID;
  }
  bm_server_ctx* s = nullptr;
  try {
    s = new bm_server_ctx();
    s->o = *o;
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    s->th = std::thread([s] {
      cudaSetDevice(s->device);
      if (s->o.batched) run_batched(*s);
      else run_plain(*s);
    });
  } catch (...) {
    delete s;
    g_server_error = "bm_server_create: could not allocate the server or start its thread";
    return BM_ERR_OOM;
  }
  *out = s;
  return BM_OK;
}

bm_status bm_server_submit(bm_server s, int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                           const float* vals, double lambda, int32_t k_max, int64_t* id) {
  if (!s) return BM_ERR_INVALID;
  if (m < 1 || n < 1 || nnz < 0 || (nnz && (!rows || !cols || !vals)) || !(lambda > 0) || k_max < 1 ||
      k_max > std::min<int64_t>(std::min(m, n), 127)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "bm_server_submit: invalid request";
    return BM_ERR_INVALID;
  }
  Request r;
  r.m = m;
  r.n = n;
  try {
    r.rows.assign(rows, rows + nnz);
    r.cols.assign(cols, cols + nnz);
    r.vals.assign(vals, vals + nnz);
  } catch (...) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "bm_server_submit: no host memory for the request's copy";
    return BM_ERR_OOM;
  }
  r.lambda = lambda;
  r.k_max = k_max;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r.id = s->next_id++;
    r.t_submit = s->now();
    if (id) *id = r.id;
    s->queue.push_back(std::move(r));
    s->in_system++;
  }
  s->cv.notify_all();
  return BM_OK;
}

bm_status bm_server_drain(bm_server s, double timeout_s) {
  if (!s) return BM_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
                                 [&] { return s->in_system.load() == 0; });
  if (!ok) {
    s->err = "bm_server_drain: timed out";
    return BM_ERR_TIMEOUT;
  }
  return BM_OK;
}

bm_status bm_server_results(bm_server s, bm_request_result* out, int32_t cap, int32_t* count) {
  if (!s) return BM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (count) *count = (int32_t)s->done.size();
  for (int32_t i = 0; out && i < cap && i < (int32_t)s->done.size(); ++i) out[i] = s->done[i];
  return BM_OK;
}

bm_status bm_server_factors(bm_server s, int64_t id, int32_t* k, float* W, float* H) {
  if (!s) return BM_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->kept.find(id);
  if (it == s->kept.end()) {
    s->err = "bm_server_factors: no factors kept for request " + std::to_string(id);
    return BM_ERR_INVALID;
  }
  if (k) *k = it->second.k;
  if (!W && !H) return BM_OK;
  if (W) std::copy(it->second.W.begin(), it->second.W.end(), W);
  if (H) std::copy(it->second.H.begin(), it->second.H.end(), H);
  s->kept.erase(it);
  return BM_OK;
}

double bm_server_now(bm_server s) { return s ? s->now() : 0.0; }

const char* bm_server_last_error(bm_server s) { return s ? s->err.c_str() : g_server_error.c_str(); }

void bm_server_destroy(bm_server s) {
  if (!s) return;
  s->stop = true;
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  delete s;
}

}  // extern "C"
