// Handle state and the device routines shared between translation units.
#pragma once
#include <map>
#include <memory>
#include <new>
#include <utility>

#include "common.cuh"

namespace bm {

// Work split of one sparse pass: each segment is a run of at most kSegNnz
// consecutive entries of one row (CSR) or column (CSC).  A warp processes one
// segment; rows spanning several segments write partial sums that a fix-up
// kernel adds in segment order (deterministic results).
constexpr int64_t kSegNnz = 1024;

struct Segs {
  int64_t nseg = 0;
  int64_t nmulti = 0;          // rows with more than one segment
  DevBuf<int32_t> row;         // [nseg] owning row
  DevBuf<int64_t> beg, end;    // [nseg] entry range
  DevBuf<int32_t> slot;        // [nseg] partial slot (-1: single-segment row)
  DevBuf<int32_t> mrow;        // [nmulti] row id
  DevBuf<int32_t> mfirst;      // [nmulti] first partial slot
  DevBuf<int32_t> mcount;      // [nmulti] number of partial slots
  int64_t nslots = 0;
};

// Sparse passes whose work split is chosen separately (bm_autotune).
enum PassKind : int {
  kPassGradCsr = 0,   // loss / gradient, rows (gathers H)
  kPassGradCsc = 1,   // gradient, columns (gathers W)
  kPassLsCsr = 2,     // line-search sums, rows (gathers H and D_H)
  kPassSpmmCsr = 3,   // q-wide SpMM R Y, rows (gathers the n-side block)
  kPassSpmmCsc = 4,   // q-wide SpMM R^T U, columns (gathers the m-side block)
  kPassKinds = 5
};
inline bool pass_is_csr(int kind) { return kind == kPassGradCsr || kind == kPassLsCsr || kind == kPassSpmmCsr; }

struct Index {
  int64_t m = 0, n = 0, nnz = 0;  // internal orientation, m <= n
  bool transposed = false;
  DevBuf<int64_t> row_ptr, col_ptr;
  DevBuf<int32_t> col, row;       // CSR column ids, CSC row ids
  DevBuf<float> val, cval;        // A in CSR and in CSC order
  // Value codec: when every observed value is an integer and they span at most
  // 255, the loss/gradient passes read one byte per entry, a_e = code_e + code_off
  // (exact in FP32 for |a| < 2^24); val / cval stay for the other uses.
  bool codec = false;
  float code_off = 0.f;
  DevBuf<uint8_t> val8, cval8;
  DevBuf<int64_t> csr2csc;        // CSC position of CSR entry e
  DevBuf<int32_t> csc2csr;        // CSR position of CSC entry q (residual permutation)
  Segs rs, cs;                    // CSR (rows) and CSC (columns) work splits
  // Panel-ordered splits by panel count P >= 2: the gathered side is cut into
  // P equal index ranges and the segments are ordered panel by panel (rows
  // in order within a panel), so the warps running at any moment gather from
  // one panel's rows, which can stay in L2.  A row's segments keep
  // consecutive partial slots in entry order (same deterministic fix-up).
  std::map<int, std::unique_ptr<Segs>> rsp, csp;
  int panels[kPassKinds] = {1, 1, 1, 1, 1};   // panel count used by each pass kind
  // Kernel layout of each pass kind: -1 automatic (warp per segment when the
  // segments hold >= 512 entries on average, else a lane group per segment),
  // 0 group per segment, 1 warp per segment (set by bm_autotune).
  int layout[kPassKinds] = {-1, -1, -1, -1, -1};
};

// The work split a pass kind uses (the natural one when its panel count is 1).
inline const Segs& pass_segs(const Index& ix, int kind) {
  const bool csr = pass_is_csr(kind);
  const int P = ix.panels[kind];
  if (P > 1) {
    const auto& mp = csr ? ix.rsp : ix.csp;
    auto it = mp.find(P);
    if (it != mp.end()) return *it->second;
  }
  return csr ? ix.rs : ix.cs;
}

// Whether a pass kind runs warp-per-segment (see Index::layout).
inline bool pass_ws(const Index& ix, int kind) {
  if (ix.layout[kind] >= 0) return ix.layout[kind] == 1;
  const Segs& sg = pass_segs(ix, kind);
  return sg.nseg > 0 && ix.nnz >= 512 * sg.nseg;
}

// Scratch reused across calls (sized once for the handle's k_max).
struct Scratch {
  int ld_part = 4;                // row width (floats) the partial buffer is sized for
  DevBuf<float> partial;          // segment partial sums
  DevBuf<float> partial2;         // those of a pass running beside the first (loss/gradient call)
  DevBuf<double> fseg;            // per-segment loss partials
  DevBuf<double> red;             // block partials of dense reductions
  DevBuf<double> scal;            // small device scalars
  DevBuf<int> sel_cols;           // column lists of small transforms
  DevBuf<double> sel_scale;       // and their scales
  DevBuf<double> eig_glob;        // eigensolver storage when a matrix exceeds shared memory
};

struct ProxState;  // defined in prox.cu
struct BbState;    // defined in sparsa.cu (SpaRSA step rule)
struct BcdState;   // defined in bcd.cu (column-block BM solver)
struct SpmmCombiner;  // defined in dense.cu (shared SpMM launches of batched PG steps)

// Optional per-kernel event timing (bm_profile_enable).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  ~Profiler();
  void begin(const char* name, cudaStream_t st);  // call before a launch
  void end(cudaStream_t st);                      // call after it
  cudaEvent_t next();
};

}  // namespace bm

struct bm_ctx {
  bm::Index ix;
  double lambda = 0;
  int k_max = 0;
  bm_options opt{};
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t side_stream = nullptr;         // work that overlaps the sparse passes (created on first use)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int device = 0;

  int k = 0;                     // current rank
  int ld = 4;                    // leading dimension of W, H (round_up4(k), >= 4)
  int ldmax = 4;                 // capacity: round_up4(k_max + 1)
  bm::DevBuf<float> W, H;        // m x ld, n x ld (padding columns are zero)
  bm::DevBuf<float> gW, gH;      // gradients
  bm::DevBuf<float> DW, DH;      // BM search directions
  bm::DevBuf<float> gWp, gHp;    // previous gradients (Polak-Ribiere)
  bm::DevBuf<float> r_csr, r_csc;  // residual R on Omega in CSR / CSC order
  bm::Scratch sc;
  bm::ProxState* ps = nullptr;
  bm::BbState* bb = nullptr;     // SpaRSA step-rule state (created on first use)
  bm::BcdState* bcd = nullptr;   // column-block BM solver scratch (created on first use)
  bm::SpmmCombiner* comb = nullptr;  // set while a batched PG step runs: SpMMs go through it
  bm::Profiler prof;
  std::string err;
  bool bm_changed = false;       // BM phase moved since the last PG step
  // BF16 gathers (bm_options.precision == 1): copies of W, H and D_H, row
  // stride ldb = round_up(ld, 8) elements, zero padded.
  bool refine = false;           // bm_solve switched to FP32 for the final iterations
  bool bf_dirty = true;          // W/H changed since the copies were made
  int ldb = 8;
  bm::DevBuf<uint16_t> Wb, Hb, DHb;
  bool bf_active() const { return opt.precision == 1 && !refine; }
  bool tuned = false;            // panel counts chosen (bm_autotune / bm_set_panels)
};

namespace bm {

// Run fn; a thrown Error, allocation failure or other exception becomes the
// returned status and the message in err.
template <class Fn>
bm_status guard_call(std::string& err, Fn&& fn) {
  try {
    fn();
    return BM_OK;
  } catch (const Error& e) {
    err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    err = "host allocation failed";
    return BM_ERR_OOM;
  } catch (...) {
    err = "unexpected exception";
    return BM_ERR_CUDA;
  }
}

// Wrap a kernel launch with profiler events when profiling is on.
#define BM_LAUNCH(h, name, ...)                              \
  do {                                                       \
    if ((h).prof.on) (h).prof.begin(name, (h).stream);       \
    __VA_ARGS__;                                             \
    BM_CHECK_LAUNCH();                                       \
    if ((h).prof.on) (h).prof.end((h).stream);               \
  } while (0)

// index.cu
void build_index(bm_ctx& h, int64_t m, int64_t n, int64_t nnz, const int32_t* rows_d,
                 const int32_t* cols_d, const float* vals_d);
// Build (once) the P-panel split of one side and grow the partial / segment
// scratch to fit it.
void ensure_panel_segs(bm_ctx& h, bool csr, int P);
// Largest slot and segment counts over all built splits.
int64_t max_slots(const Index& ix);
int64_t max_segs(const Index& ix);
// Partial scratch for slot rows of width ld_part floats, segment scratch for
// 4 doubles per segment (grown, never shrunk).
void ensure_pass_scratch(bm_ctx& h, int ld_part);

// grad.cu
struct LossOut {
  double f;      // 1/2 sum r^2
  double nW2;    // ||W||^2
  double nH2;    // ||H||^2
};
// f, gradients (written to h.gW/h.gH when want_grad), residual stored in
// h.r_csr / h.r_csc when store_r.  Stream-ordered; returns after a sync.
LossOut loss_grad_dev(bm_ctx& h, bool want_grad, bool store_r);
// Work beside the handle's stream: side_fork makes the side stream (created
// on first use) wait for the handle's stream so far; launches issued while an
// OnSideStream lives go to the side stream; side_join makes the handle's
// stream wait for everything issued on the side stream before it.  A
// SideScope forks on construction and joins when it goes out of scope, also
// when an exception leaves it, so that no later work on the handle's stream
// can overtake side-stream work of a failed call.
void side_fork(bm_ctx& h);
void side_join(bm_ctx& h) noexcept;
struct SideScope {
  bm_ctx& h;
  explicit SideScope(bm_ctx& hh) : h(hh) { side_fork(h); }
  ~SideScope() { side_join(h); }
  SideScope(const SideScope&) = delete;
  SideScope& operator=(const SideScope&) = delete;
};
struct OnSideStream {
  bm_ctx& h;
  cudaStream_t main;
  explicit OnSideStream(bm_ctx& hh) : h(hh), main(hh.stream) { h.stream = h.side_stream; }
  ~OnSideStream() { h.stream = main; }
};
// BF16 copy of a row-major block (rows x ld floats -> rows x ldb bfloat16, padded with 0)
void to_bf16_dev(bm_ctx& h, const float* src, int64_t rows, int ld, uint16_t* dst, int ldb);
// Refresh the BF16 copies of W and H if they are stale.
void ensure_bf16(bm_ctx& h);
// Residual r at the current factors in CSR order (CSR pass) and in CSC order
// (permutation gather); returns f = 1/2 sum r^2.
double residual_dev(bm_ctx& h);
// Quartic coefficients c0..c4 of phi(s) along (h.DW, h.DH), using h.r_csr.
void line_search_coeffs_dev(bm_ctx& h, double c[5]);
// One launch of a sparse pass kind on the current state, for timing (loss /
// gradient and line-search kinds; outputs land in the usual scratch).
void tuning_pass_dev(bm_ctx& h, int kind);
// Dense helpers over m x ld / n x ld arrays (deterministic FP64 reductions).
double dot_dev(bm_ctx& h, const float* x, const float* y, int64_t count);
void axpy_dev(bm_ctx& h, float* y, const float* x, float a, int64_t count);          // y += a x
void xpby_dev(bm_ctx& h, float* y, const float* x, float b, int64_t count);          // y = -x + b y
void copy_pad_dev(bm_ctx& h, float* dst, int ldd, const float* src, int lds, int64_t rows,
                  int cols, cudaMemcpyKind kind);

// api.cu: argmin over s >= 0 of c0 + c1 s + ... + c4 s^4 (0 or a real root of the derivative)
// Per-name launch counts and device milliseconds of the recorded marks (synchronise first).
void profile_report(Profiler& prof, int32_t cap, char* names, int64_t* launches, double* total_ms, int32_t* count);
double quartic_argmin_ext(const double c[5]);

// prox.cu
void prox_create(bm_ctx& h);
void prox_destroy(bm_ctx& h);
void prox_reset(bm_ctx& h);
// One inexact PG step with step size alpha; info->F (an extra loss pass) only with eval_F.
void prox_step_dev(bm_ctx& h, double alpha, bm_prox_info* info, bool eval_F = true);
// One PG step with the SpaRSA step rule (sparsa.cu); bb_reset forgets the previous point.
void prox_step_bb_dev(bm_ctx& h, bm_prox_info* info, bm_bb_info* bb);
void bb_reset(bm_ctx& h);
void bb_destroy(BbState* s);
// `epochs` sweeps of the column-block BM solver (bcd.cu); returns F at entry,
// *F_out = F after the sweeps.
double bcd_phase_dev(bm_ctx& h, int epochs, double* F_out);
void bcd_destroy(BcdState* s);
void init_step_dev(bm_ctx& h, bm_prox_info* info);
// Checkpoint of the PG-step state (warm start and safeguard): size, save
// into host memory, load from host memory (validated; BM_ERR_INVALID).
size_t prox_state_bytes(const bm_ctx& h);
void prox_state_save(bm_ctx& h, uint8_t* out);
void prox_state_load(bm_ctx& h, const uint8_t* in, size_t len);
// One q-wide SpMM of the PG step (CSR: R Y, CSC: R^T U) on scratch blocks of
// width min(k_max + 1, k + 1), for timing.
void tuning_spmm_dev(bm_ctx& h, bool csr);
// Time every pass kind with panel counts 1..max_panels (only where the
// gathered side exceeds a quarter of L2) and keep the fastest.
void autotune_dev(bm_ctx& h, int max_panels, bm_tune_info* info);

}  // namespace bm

namespace bm {
// index.cu helpers shared with edm.cu
void sort_pairs_ext(DevBuf<uint64_t>& k0, DevBuf<uint32_t>& v0, DevBuf<uint64_t>& k1, DevBuf<uint32_t>& v1,
                    int64_t n, int bits, cudaStream_t st);
void build_segs_ext(Segs& s, const DevBuf<int64_t>& ptr_d, int64_t rows, cudaStream_t st);
void lower_bounds_ext(const uint64_t* keys, int64_t nnz, uint64_t stride, int64_t count, int64_t* ptr,
                      cudaStream_t st);
int key_bits_ext(uint64_t v);
}  // namespace bm
