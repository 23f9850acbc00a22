/*
 * bm.h -- C ABI of the GB300 (sm_103a) implementation of the data-parallel
 * hot path of BM-Global (Lee, Liang, Tang & Toh, arXiv 2204.14067) for
 * nuclear-norm regularised matrix completion
 *
 *     min_X  F(X) = 1/2 ||P_Omega(X - A)||_F^2 + lambda ||X||_*      (Eq. "MC")
 *
 * solved through the factorisation X = W H^T                          (Eq. "MF")
 *
 *     min_{W,H}  1/2 ||P_Omega(W H^T - A)||_F^2 + lambda/2 (||W||^2 + ||H||^2)
 *
 * alternating BM phases with inexact proximal-gradient steps (Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Orientation: callers pass an m x n matrix.  If m > n the library stores
 *    the transpose internally (the paper assumes m <= n, Sec. 1); factors,
 *    gradients and index dumps that are documented as "caller orientation"
 *    are mapped back, those documented as "internal" are not.
 *  - Indexing is 0-based; indices are int32, counts int64.
 *  - Dense factors are row-major with leading dimension k (W[i*k + c]).
 *  - Pointers may be host or device memory; the library detects which
 *    (cudaPointerGetAttributes) and copies as needed.  Inputs are copied
 *    and never retained; output buffers are owned by the caller.
 *  - Every call returns a bm_status and never aborts or throws.  The text
 *    of the last failure on a handle is returned by bm_last_error(h);
 *    failures without a handle are reported by bm_last_error(NULL).
 *  - A handle owns its device memory and a CUDA stream; handles are
 *    independent, one handle must not be used by two threads at once.
 */
#ifndef BM_GB300_H
#define BM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bm_ctx* bm_handle;

typedef enum {
  BM_OK = 0,
  BM_ERR_INVALID = 1,       /* bad argument: sizes, indices, duplicates, non-finite values */
  BM_ERR_OOM = 2,           /* device allocation failed */
  BM_ERR_CUDA = 3,          /* a CUDA call failed */
  BM_ERR_TIMEOUT = 4,       /* a bounded device wait ran out */
  BM_ERR_NUMERIC = 5,       /* NaN/Inf in the objective or a small eigenproblem */
  BM_ERR_NOT_CONVERGED = 6  /* bm_solve stopped on max_outer or time_limit */
} bm_status;

/* Solver parameters.  Defaults (bm_default_options) follow the paper where
 * it gives a value and the design notes where it does not. */
typedef struct {
  double alpha;          /* PG step size; 1.99 (Sec. 5.1: L = 1, alpha < 2 delta / L) */
  int32_t bm_epochs;     /* y: BM iterations per cycle; 3 (Sec. 5.1.1, x = 1, y = 3) */
  int32_t pg_steps;      /* x: inexact PG steps per cycle; 1 */
  int32_t lmsvd_p;       /* LmSVD memory p_t (Algorithm 2); 1 */
  int32_t lmsvd_imax;    /* LmSVD iteration cap; 50 */
  int32_t lmsvd_min_iter;/* Rayleigh-Ritz steps before the stop test; 2 */
  double lmsvd_tol;      /* stop when max |theta - theta_prev| <= tol * theta_1; 1e-5 (FP32
                            resolves the Ritz values to about eps32 * theta_1; a tighter test
                            spends iterations on rounding) */
  double tau;            /* orth(): drop Gram eigenvalues <= tau (Eq. "orth-W"); 1e-6 */
  double ritz_rel;       /* Algorithm 2 J_s: keep s_j > ritz_rel * s_1; 1e-6 */
  double psi0;           /* safeguard noise level psi_0 (Sec. "Ensuring sufficient precision"); 0.1 */
  int32_t k_init;        /* k_{-1}: sketch size of the initial PG step (Sec. "Initialization"); 8 */
  int32_t precision;     /* 0: FP32 factors; 1: BF16 factor copies for the gathers */
  uint64_t seed;         /* counter-based RNG key for the sketch and xi_t */
  int32_t autotune;      /* 1: bm_solve runs bm_autotune once before its first cycle; 0 */
  int32_t step_rule;     /* PG step size in bm_solve: 0 fixed alpha; 1 the SpaRSA rule of
                            bm_prox_step_bb (supplement Sec. "The SpaRSA variant"); 0 */
  int32_t value_codec;   /* 1: when every observed value is an integer and they span at most
                            255, the loss/gradient passes read one byte per entry
                            (a = code + offset, exact); 0: always FP32 values; 1 */
  int32_t bm_solver;     /* BM phase of bm_solve: 0 Polak-Ribiere+ CG on all of (W, H) with
                            the exact line search; 1 column-block coordinate descent
                            (bm_bcd_phase); 0 */
  int32_t tensor_grams;  /* 1: the PG step's symmetric plain Gram (the Rayleigh-Ritz matrix
                            (Z^T Q)^T (Z^T Q) of LmSVD) runs on the tensor cores from
                            bfloat16 slices (see bm_dense_gram, mode 2); the thin products
                            W^T U, H^T Y (faster on the FP32 pipes at these widths) and the
                            Grams that need compensated sums (orthonormalisation, B B^T,
                            W^T W, H^T H) stay on the FP32 pipes; 0: every Gram on the FP32
                            pipes; 1 */
  int32_t pad_;
} bm_options;

/* Result of one inexact PG step (Eq. "inexactpg", "truncate"). */
typedef struct {
  int32_t k_new;         /* rank of X_{t+1}: singular values surviving the threshold */
  int32_t warm_cols;     /* columns of the LmSVD warm start U^{t,0} */
  int32_t lmsvd_iters;   /* Rayleigh-Ritz steps taken */
  int32_t n_L;           /* LmSVD block products with Z^T (each block of L(U) = Z Z^T U costs one) */
  int32_t cap_hit;       /* 1 if more than k_max values survived (rank capped) */
  int32_t pad_;
  double eps;            /* ||Z_t - Z~_t||_F (Sec. "Inexact PG step", monitoring formula) */
  double F;              /* objective F(X_{t+1}) = f + lambda * sum(Sigma) */
} bm_prox_info;

typedef struct {
  int32_t max_outer;     /* cycles of Algorithm 1; default 100 */
  int32_t pad_;
  double tol;            /* stop when |F_t - F_{t-1}| / (1 + |F_{t-1}|) < tol; default 1e-10 */
  double F_target;       /* stop when F <= F_target (<= 0: unused) */
  double time_limit_s;   /* wall-clock limit (<= 0: none) */
} bm_solve_opts;

typedef struct {
  int32_t outer;         /* cycles run */
  int32_t k;             /* final rank */
  int32_t converged;     /* 1 if tol or F_target was met */
  int32_t pad_;
  double F;              /* final objective */
  double seconds;        /* wall time of the solve */
} bm_solve_info;

/* Fill *o with the defaults listed in bm_options.  Never fails for o != NULL. */
bm_status bm_default_options(bm_options* o);

/*
 * bm_create -- upload Omega and A, build the index structures.
 * Paper: Omega is an index set and P_Omega the sampling operator (Sec. 1,
 * Eq. "MC"); the m <= n convention (Sec. 1).
 *   m, n        caller's matrix size, both >= 1.
 *   nnz         |Omega| >= 0 (< 2^31).
 *   rows, cols  int32[nnz], 0 <= rows < m, 0 <= cols < n, no repeated pair.
 *   vals        float32[nnz] observed values A_ij, finite.
 *   lambda      nuclear-norm weight, > 0.
 *   k_max       rank cap, 1 <= k_max <= min(m, n).
 *   opt         solver options (NULL: defaults).
 *   out         receives the handle.
 * Builds, on the device, CSR sorted by (row, col) and CSC sorted by (col, row)
 * of the internal orientation (bit-exact canonical order).  Factors start at
 * k = 0 (X = 0).  Errors: BM_ERR_INVALID for bad sizes, out-of-range or
 * repeated indices, non-finite values; BM_ERR_OOM; BM_ERR_CUDA.
 */
bm_status bm_create(int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                    const float* vals, double lambda, int32_t k_max, const bm_options* opt,
                    bm_handle* out);

/* Free all device memory of h (NULL is ignored). */
void bm_destroy(bm_handle h);

/* Text of the last failure on h (or of the last failure without a handle if
 * h is NULL).  The pointer stays valid until the next call on h. */
const char* bm_last_error(bm_handle h);

/* Run the handle's work on `stream` (a cudaStream_t; NULL restores the
 * handle's own stream).  The stream must outlive its use by h. */
bm_status bm_set_stream(bm_handle h, void* stream);

/* Sizes: internal m <= n, nnz, whether the caller's matrix was transposed,
 * current rank k.  Any output pointer may be NULL. */
bm_status bm_dims(bm_handle h, int64_t* m, int64_t* n, int64_t* nnz, int32_t* transposed,
                  int32_t* k);

/*
 * bm_get_index -- copy the index structures (internal orientation) into
 * caller buffers (host or device; any may be NULL):
 *   row_ptr int64[m+1], col int32[nnz], val float[nnz]        CSR by (row, col)
 *   col_ptr int64[n+1], row int32[nnz], cval float[nnz]       CSC by (col, row)
 *   csr2csc int64[nnz]  CSC position of each CSR entry
 */
bm_status bm_get_index(bm_handle h, int64_t* row_ptr, int32_t* col, float* val, int64_t* col_ptr,
                       int32_t* row, float* cval, int64_t* csr2csc);

/*
 * bm_get_codes -- the value codec (bm_options.value_codec): *active = 1 if
 * the loss/gradient passes read one-byte codes, *offset the integer added to
 * a code; csr_codes / csc_codes (uint8[nnz], host or device, nullable)
 * receive the codes in CSR and CSC order when active.  Any pointer may be NULL.
 */
bm_status bm_get_codes(bm_handle h, int32_t* active, float* offset, uint8_t* csr_codes, uint8_t* csc_codes);

/*
 * bm_set_factors -- set X = W H^T (caller orientation): W float[m*k],
 * H float[n*k], row-major, 0 <= k <= k_max.  Resets the safeguard state of
 * the PG steps (the next bm_prox_step warm-starts from orth(W)).
 */
bm_status bm_set_factors(bm_handle h, int32_t k, const float* W, const float* H);

/* bm_get_factors -- copy the current factors (caller orientation) into
 * W float[m*k], H float[n*k] (either may be NULL); *k receives the rank. */
bm_status bm_get_factors(bm_handle h, int32_t* k, float* W, float* H);

/*
 * bm_loss_grad -- the sparse loss and gradient of (MF)/(BM-nuclear) at the
 * current factors (Eq. "mf"):
 *   f  = 1/2 sum_{(i,j) in Omega} (<W_i, H_j> - A_ij)^2
 *   F  = f + lambda/2 (||W||_F^2 + ||H||_F^2)
 *   gW = R H + lambda W,  gH = R^T W + lambda H,  R = P_Omega(W H^T - A)
 * f, F: host doubles (either may be NULL).  gW float[m*k], gH float[n*k]
 * in caller orientation, host or device, may be NULL.  FP32 arithmetic with
 * FP64 reduction of f.  Errors: BM_ERR_NUMERIC if f is not finite.
 */
bm_status bm_loss_grad(bm_handle h, double* f, double* F, float* gW, float* gH);

/*
 * bm_bm_phase -- `epochs` iterations of the BM-phase solver: nonlinear
 * conjugate gradient (Polak-Ribiere+) on (MF) with an exact line search on
 * the quartic phi(s) = F~(W + s D_W, H + s D_H).  Each iteration keeps the
 * non-increase condition (Eq. "nonincrease").  *F (nullable) receives the
 * objective after the last iteration.
 */
bm_status bm_bm_phase(bm_handle h, int32_t epochs, double* F);

/*
 * bm_init -- the initial point: one inexact PG step from X_{-1} = 0 with
 * alpha = 1/L = 1, using the HMT range finder on k_init Gaussian columns and
 * the Nystrom approximation (Sec. "Initialization", Eq. "nys"), then
 * Eq. "exactSVD", "approxSVD", "truncate".  info may be NULL.
 */
bm_status bm_init(bm_handle h, bm_prox_info* info);

/*
 * bm_prox_step -- one inexact PG step from X~ = W H^T (Eq. "inexactpg"):
 * Z = X~ - alpha R; LmSVD (Algorithm 2) on L(U) = Z Z^T U warm-started from
 * orth([U_t, W]) plus the safeguard column (Eq. "rt0", "rt"); exact SVD of
 * U^T Z (Eq. "exactSVD"); soft-threshold by lambda*alpha (Eq. "truncate");
 * W <- U sqrt(Sigma), H <- V sqrt(Sigma) (Algorithm 1).  alpha <= 0 uses
 * the handle's option.  info may be NULL.
 */
bm_status bm_prox_step(bm_handle h, double alpha, bm_prox_info* info);

/*
 * bm_solve -- Algorithm 1: bm_init if k = 0, then cycles of bm_epochs BM
 * iterations and pg_steps PG steps until a stopping rule of *o holds
 * (o NULL: defaults).  info may be NULL.  Returns BM_ERR_NOT_CONVERGED if
 * max_outer or time_limit_s ended the solve.
 */
bm_status bm_solve(bm_handle h, const bm_solve_opts* o, bm_solve_info* info);

/*
 * Checkpoint / resume (no counterpart in the paper).  bm_get_state writes the
 * solve state into a caller-owned host buffer: the rank, W and H, the PG
 * step's warm-start and safeguard state (U_t, U_{t-1}, the truncated vector
 * u, psi_t, the rank history, t) and the work-split choice; with buf = NULL
 * it only stores the required size in *len (BM_ERR_INVALID if *len is too
 * small).  bm_set_state restores such a state into a handle created for the
 * same problem (same m, n, |Omega| and k_max; BM_ERR_INVALID otherwise, or
 * for a damaged buffer).  A solve continued after bm_set_state takes the
 * same steps as one that was never interrupted.
 */
bm_status bm_get_state(bm_handle h, void* buf, size_t* len);
bm_status bm_set_state(bm_handle h, const void* buf, size_t len);

/*
 * Work-split tuning of the sparse passes (no counterpart in the paper; it
 * changes the order of work, not the arithmetic of Eq. (MF) and (ZZ)).
 * Pass kinds, in array order: 0 loss/gradient over rows (gathers H), 1
 * gradient over columns (gathers W), 2 line-search sums over rows (gathers H
 * and D_H), 3 the PG step's SpMM R Y over rows, 4 its SpMM R^T U over
 * columns.  With P panels a pass visits its segments in P groups, each
 * gathering from one P-th of the gathered block's rows, so the rows in use at
 * any moment fit the 129 MB L2.  Results differ between panel counts only in
 * the order of floating-point additions.
 *
 * bm_autotune times every kind with one panel and, where the gathered block
 * exceeds a quarter of L2, with 2, 3, 4, 6, 8, 12, 16 panels (up to
 * max_panels), each in both kernel layouts (bm_set_layout), and keeps the
 * fastest; it needs factors (k >= 1), overwrites
 * the gradient, search-direction and PG scratch buffers (not W, H or the PG
 * warm-start state) and takes about 20 launches per kind.  info (nullable)
 * receives the choice.  bm_set_panels fixes the counts (each in
 * [1, BM_MAX_PANELS]); bm_get_panels reads them.  A batch (bm_batch_create)
 * reads the counts when it is created.  Errors: BM_ERR_INVALID for a bad
 * count or empty factors.
 */
#define BM_PASS_KINDS 5
#define BM_MAX_PANELS 16
typedef struct {
  int32_t panels[BM_PASS_KINDS];   /* chosen panel count per pass kind */
  int32_t timed;                   /* timed candidates */
  double ms[BM_PASS_KINDS];        /* one launch with the chosen split (ms, fastest of 3) */
  double ms_single[BM_PASS_KINDS]; /* one launch with one panel and the automatic layout (ms) */
  int32_t layout[BM_PASS_KINDS];   /* chosen kernel layout per pass kind (see bm_set_layout) */
  int32_t pad_;
} bm_tune_info;
bm_status bm_autotune(bm_handle h, int32_t max_panels, bm_tune_info* info);
bm_status bm_set_panels(bm_handle h, const int32_t* panels);
bm_status bm_get_panels(bm_handle h, int32_t* panels);
/*
 * Kernel layout of each pass kind: 0 = a group of lanes per segment (several
 * segments per warp; suits many short rows or columns), 1 = a whole warp per
 * segment (suits long ones), -1 = automatic (1 when the pass's segments hold
 * 512 or more entries on average).  bm_autotune also times both layouts and
 * keeps the faster.  bm_get_layout reports the layout each kind runs with
 * (0 or 1).  Results differ between layouts only in the order of
 * floating-point additions.  Errors: BM_ERR_INVALID for a value outside
 * {-1, 0, 1}.
 */
bm_status bm_set_layout(bm_handle h, const int32_t* layout);
bm_status bm_get_layout(bm_handle h, int32_t* layout);
/*
 * bm_gather_roof -- measurement aid for the roofline of the sparse passes
 * (no counterpart in the paper).  Times a gather-only pass over the entries of
 * pass kind `kind` in its index order (CSR kinds gather rows of H, CSC kinds
 * rows of W, FP32, the handle's current row stride): every entry loads its
 * whole row and nothing is computed or stored per entry.  *ms (nullable)
 * receives the fastest of three launches after a warm-up, *gbs (nullable) the
 * gathered bytes per second in GB/s.  A pass that gathers the same rows cannot
 * run faster without reusing rows; the ratio of the two times is the pass's
 * fraction of this roof.  Needs factors (k >= 1); allocates a small output
 * buffer.  Errors: BM_ERR_INVALID for an unknown kind or no factors.
 */
bm_status bm_gather_roof(bm_handle h, int32_t kind, double* ms, double* gbs);

/*
 * bm_dense_gram -- C = A^T B of two tall FP32 blocks, the dense k-wide
 * product of the PG step (Eq. "PUi"/"orth-W" Grams; Algorithm 2's
 * Rayleigh-Ritz matrix), exposed for callers and tests.
 *   A      float[L * lda] device, row-major L x a (a columns used)
 *   B      float[L * ldb] device, row-major L x b
 *   C      double[a * b] device, row-major (written)
 *   mode   0: FP32 pipes, FP32 sums over 32-row tiles added as FP32 pairs;
 *          1: FP32 pipes, compensated (error-free products and sums, about
 *             FP64 accuracy); 2: tensor cores (tcgen05.mma, kind::f16):
 *             each value split into three bfloat16 slices, six slice
 *             products per 16-row step accumulated in FP32 per block slab,
 *             the slab sums added in FP64 -- about FP32 accuracy.
 *   stream cudaStream_t (NULL: default stream); the call returns after it
 *          has finished.  Scratch is allocated on first use and kept for
 *          later calls, one set per host thread.
 * Requirements: L >= 0, 1 <= a, b; lda, ldb multiples of 4 with lda >= a,
 * ldb >= b; A, B 16-byte aligned; mode 2 also a, b <= 256.  Errors:
 * BM_ERR_INVALID for bad arguments, BM_ERR_CUDA for a launch failure,
 * BM_ERR_NUMERIC if a tensor-core wait ran out of time (C is then NaN).
 */
bm_status bm_dense_gram(const float* A, int64_t L, int32_t a, int32_t lda, const float* B, int32_t b, int32_t ldb,
                        double* C, int32_t mode, void* stream);
const char* bm_dense_last_error(void);

/*
 * bm_sym_eig -- eigen-decomposition S = V diag(evals) V^T of a small
 * symmetric matrix on one thread block, the q x q eigenproblems of the PG
 * step (Algorithm 2's Rayleigh-Ritz matrix Q^T L Q, the Gram B B^T of the
 * exact small SVD, Eq. "orth-W"), exposed for callers and tests.
 *   S      double[n * n] device, row-major; (S + S^T) / 2 is used
 *   evals  double[n] device (written), descending
 *   evecs  double[n * n] device (written), row-major, column j = vector j
 *   mode   0: FP32 Householder tridiagonalisation + implicit QL, with one
 *             divide-and-conquer level (QL on the two halves, merge through
 *             the secular equation) for 24 <= n <= 150 (eigenvalue errors
 *             about eps32 * ||S||); 1: mode 0's vectors made orthogonal by
 *             one FP64 Newton-Schulz step (V), then S' = V^T S V in FP64 and
 *             FP32 Jacobi sweeps on S' to a
 *             relative threshold (eigenvalues of a positive definite S to
 *             about eps32 relative), for n <= 160; 2: as 1 with FP64 sweeps,
 *             for n <= 112.  Modes 1 and 2 beyond those sizes run the
 *             Householder + QL of mode 0 in FP64.
 *   stream cudaStream_t (NULL: default stream); returns after it finished.
 * Requirements: 1 <= n <= 256.  Errors: BM_ERR_INVALID for bad arguments,
 * BM_ERR_NUMERIC for a non-finite eigenvalue or a QL that did not converge,
 * BM_ERR_CUDA for a launch failure.
 */
bm_status bm_sym_eig(const double* S, int32_t n, double* evals, double* evecs, int32_t mode, void* stream);

/*
 * Batched BM phase over many solves.  A batch groups handles on one device
 * (same precision mode, each with rank >= 1).  bm_batch_bm_phase runs
 * `epochs` iterations of the BM-phase solver of bm_bm_phase on every handle
 * in lockstep: each sparse pass (loss/gradient CSR and CSC, exact line
 * search) of all handles with the same row width is one launch over their
 * concatenated segment lists, and the direction, step length and update run
 * as batched device kernels, so an epoch is one CUDA graph replay (captured
 * on first use and re-captured when a rank, the work split or a buffer it
 * captured changes).  F (double[count],
 * nullable) receives each handle's objective after the last iteration.
 * The batch owns a stream; the handles' own streams are synchronised first.
 * A handle must not be used elsewhere while its batch call runs, and must
 * outlive the batch.
 *
 * bm_batch_create -- hs: bm_handle[count] (read during the call; the batch
 *   keeps the handles, not the array), count >= 1; *out receives the batch
 *   (NULL on failure).  Errors: BM_ERR_INVALID for a NULL array, output or
 *   handle, handles on different devices or in different precision modes,
 *   a handle listed twice; BM_ERR_CUDA if its stream cannot be created.
 * bm_batch_destroy -- waits for the batch's stream, then frees the batch,
 *   its graph and its stream (not the handles).  NULL is ignored.
 * bm_batch_last_error -- the message of the batch's last failed call (b =
 *   NULL: of this thread's last failed bm_batch_create).
 */
typedef struct bm_batch_ctx* bm_batch;
bm_status bm_batch_create(bm_handle* hs, int32_t count, bm_batch* out);
void bm_batch_destroy(bm_batch b);
const char* bm_batch_last_error(bm_batch b);
bm_status bm_batch_bm_phase(bm_batch b, int32_t epochs, double* F);
/*
 * bm_batch_prox_step -- one inexact PG step (Eq. "inexactpg", as
 * bm_prox_step with step size alpha, <= 0: each handle's option) on every
 * handle of the batch at once.  Each handle's step runs on its own host
 * thread and stream; the q-wide residual SpMMs of Eq. "ZZ" (the sparse part
 * of the products Z^T U and Z Y of Algorithm 2) meet: when every handle
 * still inside its step has one ready, they run as shared launches over the
 * concatenated segment lists (one per orientation, row width and layout),
 * and the results are bit for bit those of bm_prox_step.  Handles of any rank
 * may take part.  info (bm_prox_info[count], nullable) receives each
 * handle's result, status (bm_status[count], nullable) each handle's status
 * (a handle whose own step fails leaves and does not stop the others; a
 * shared launch that fails fails every handle's step still in the batch).
 * Errors: the first failing handle's status, with its message in
 * bm_batch_last_error.
 *
 * bm_batch_stats -- the products handed to the shared launches so far and
 * the launches made for them (nullable outputs).
 */
bm_status bm_batch_prox_step(bm_batch b, double alpha, bm_prox_info* info, bm_status* status);
bm_status bm_batch_stats(bm_batch b, int64_t* spmm_products, int64_t* spmm_launches);

/*
 * Serving: a continuous-batching request loop for many completion solves.
 * bm_server_create starts a server thread on the current device.  Requests
 * (bm_server_submit copies the COO data) wait in a FIFO queue and are
 * admitted while fewer than max_active solves are running and the
 * device-memory estimate of the request fits mem_budget_gb (0: the whole
 * device) and the free memory.  Each admitted solve gets its own handle
 * (bm_create + bm_init with the server's precision) and stays resident
 * until it finishes.  batched = 1: every cycle runs the BM phases (3
 * iterations) of all active solves as one bm_batch and then their PG steps
 * concurrently from `workers` host threads, each on its own stream (measured
 * faster here than bm_batch_prox_step's shared SpMM launches, whose
 * rendezvous holds every solve to the slowest one's pace); a solve finishes
 * when the
 * relative change of F between cycles is below tol or after max_outer
 * cycles, and requests that arrived meanwhile join at the next cycle.
 * batched = 0: one solve at a time with bm_solve.
 */
typedef struct bm_server_ctx* bm_server;
typedef struct {
  int32_t max_active;    /* slots (batched = 0 uses one) */
  int32_t precision;     /* bm_options.precision of every solve */
  int32_t batched;       /* 1: batched BM phases + concurrent PG steps; 0: one solve at a time */
  int32_t workers;       /* host threads for the PG steps */
  double mem_budget_gb;  /* admission budget (0: device size) */
  int32_t max_outer;     /* cycles per solve */
  int32_t keep_factors;  /* 1: keep each finished solve's factors for bm_server_factors */
  double tol;            /* relative change of F that ends a solve */
} bm_server_opts;
typedef struct {
  int64_t id;            /* from bm_server_submit */
  int32_t status;        /* bm_status of the solve */
  int32_t k;             /* final rank */
  int32_t outer;         /* cycles run */
  int32_t pad_;
  double F;              /* final objective */
  double t_submit;       /* seconds since bm_server_create */
  double t_start;        /* admission time */
  double t_done;         /* completion time (latency = t_done - t_submit) */
} bm_request_result;
bm_status bm_server_create(const bm_server_opts* o, bm_server* out);
bm_status bm_server_submit(bm_server s, int64_t m, int64_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                           const float* vals, double lambda, int32_t k_max, int64_t* id);
/* Wait until every submitted request has finished (BM_ERR_TIMEOUT after timeout_s > 0). */
bm_status bm_server_drain(bm_server s, double timeout_s);
/* Copy up to cap results (completion order); *count receives the number finished. */
bm_status bm_server_results(bm_server s, bm_request_result* out, int32_t cap, int32_t* count);
/*
 * With keep_factors = 1 the server copies each successfully finished solve's
 * factors to host memory before it frees the solve's device state.
 * bm_server_factors copies request id's factors (caller orientation, the
 * request's m x k and n x k, row-major) into W float[m*k] and H float[n*k]
 * and releases the server's copy; with W = H = NULL it only reports *k and
 * keeps the copy.  BM_ERR_INVALID if no factors are kept for id.
 */
bm_status bm_server_factors(bm_server s, int64_t id, int32_t* k, float* W, float* H);
double bm_server_now(bm_server s);
const char* bm_server_last_error(bm_server s);
void bm_server_destroy(bm_server s);

/*
 * Distance-geometry (PSD) factorised loss, Eq. "EDM" of the supplement (BM
 * formulation of the kernel-estimation / molecular-conformation QSDP):
 *   g(V) = 1/2 sum_{(i,j) in Omega} w_ij (<E_ij, V V^T> - d_ij^2)^2 + lambda ||V||_F^2
 *   grad g(V) = 2 (sum_{(i,j)} w_ij r_ij E_ij + lambda I) V
 * with E_ij = (e_i - e_j)(e_i - e_j)^T, so <E_ij, V V^T> = ||v_i - v_j||^2,
 * and r_ij = ||v_i - v_j||^2 - d_ij^2.  lambda may be negative (trace
 * regulariser on the PSD cone).  Weights w_ij = 2 give the unhalved sum
 * sum r_ij^2.
 */
typedef struct bm_edm_ctx* bm_edm_handle;

/* n points (>= 2); npairs pairs (i[p], j[p]), 0 <= i, j < n, i != j, each
 * unordered pair at most once; d[p] >= 0 finite; w[p] finite (w NULL: all 1).
 * Arrays host or device, copied.  1 <= k_max <= min(128, n).  Builds a
 * symmetric CSR (both directions of every pair) on the device.
 * Errors: BM_ERR_INVALID for bad indices, repeated pairs, bad values. */
bm_status bm_edm_create(int64_t n, int64_t npairs, const int32_t* i, const int32_t* j, const float* d,
                        const float* w, double lambda, int32_t k_max, bm_edm_handle* out);
void bm_edm_destroy(bm_edm_handle h);
const char* bm_edm_last_error(bm_edm_handle h);
/* V float[n*k] row-major (host or device), 1 <= k <= k_max. */
bm_status bm_edm_set_factor(bm_edm_handle h, int32_t k, const float* V);
/* *g (host, nullable) = g(V); gV float[n*k] (host or device, nullable) = grad g(V).
 * Errors: BM_ERR_NUMERIC if g is not finite. */
bm_status bm_edm_loss_grad(bm_edm_handle h, double* g, float* gV);
/* Run the handle's calls on `stream` (a cudaStream_t; NULL: the handle's own
 * stream).  Work queued on the previous stream is finished first. */
bm_status bm_edm_set_stream(bm_edm_handle h, void* stream);

/*
 * Algorithm 1 on the distance-geometry QSDP (Eq. "QSDP": minimise
 * 1/2 sum w_ij (X_ii + X_jj - 2 X_ij - d_ij^2)^2 + lambda <I, X> over X
 * positive semidefinite with <E, X> = 0), factored as X = V V^T, V^T e = 0
 * (Eq. "EDM").  BM phase: Polak-Ribiere+ with the exact quartic line search
 * (every direction keeps V^T e = 0).  PG step: by Lemma "PiX" and
 * Eq. "proxsym", X+ = P_S+(V V^T - alpha L_{w r} - alpha lambda J) with
 * L_c = sum c_ij E_ij, J = I - e e^T / n, alpha = 1/L (Gershgorin bound of
 * ||A* A||); the leading eigenpairs come from LmSVD (Algorithm 2) on the
 * operator shifted to be positive semidefinite; V+ = U diag(sqrt(mu_+)).
 * Rank rule: k eigenpairs are computed; all positive -> the next step
 * computes k + floor(n / 20) (at most k_max), else the number of positive
 * ones.  The initial point is one PG step from X = 0 with
 * k_0 = min(100, floor(0.15 n), k_max) pairs.
 *
 * The factor (bm_edm_set_factor or a PG step) is expected to satisfy
 * V^T e = 0; setting a factor forgets the warm start and the rank schedule,
 * and the next PG step then computes min(k + 1, k_max) eigenpairs.
 *
 * bm_edm_set_options: bm_epochs, lmsvd_p (0 or 1), lmsvd_imax,
 *   lmsvd_min_iter, lmsvd_tol, tau and seed of *o are used (defaults:
 *   bm_default_options).
 * bm_edm_init: the initial PG step (the factor becomes X_0's).
 * bm_edm_bm_phase: `epochs` BM iterations; *F (nullable) = g(V) after them.
 * bm_edm_prox_step: one PG step; info (nullable): k_new = rank of X+,
 *   warm_cols = eigenpairs computed, lmsvd_iters, n_L = eigenpairs the next
 *   step computes, cap_hit = 1 if all computed eigenvalues were positive,
 *   eps = the shift sigma, F = g(V+).
 * bm_edm_solve: bm_edm_init if the factor is empty, then cycles of bm_epochs
 *   BM iterations and one PG step until |F_t - F_{t-1}| / (1 + |F_{t-1}|) <
 *   tol, F <= F_target (if nonzero) or max_outer / time_limit_s
 *   (BM_ERR_NOT_CONVERGED).
 * bm_edm_get_factor: *k (nullable) = rank; V (nullable, n x k row-major,
 *   host or device) = the factor.
 */
bm_status bm_edm_set_options(bm_edm_handle h, const bm_options* o);
bm_status bm_edm_init(bm_edm_handle h, bm_prox_info* info);
bm_status bm_edm_bm_phase(bm_edm_handle h, int32_t epochs, double* F);
bm_status bm_edm_prox_step(bm_edm_handle h, bm_prox_info* info);
bm_status bm_edm_solve(bm_edm_handle h, const bm_solve_opts* o, bm_solve_info* info);
bm_status bm_edm_get_factor(bm_edm_handle h, int32_t* k, float* V);
/* Kernel timing of the handle's launches, as bm_profile_enable / bm_profile_read. */
bm_status bm_edm_profile_enable(bm_edm_handle h, int32_t enable);
bm_status bm_edm_profile_read(bm_edm_handle h, int32_t cap, char* names, int64_t* launches, double* total_ms,
                              int32_t* count);

/*
 * bm_loss_grad_csr_noalloc -- the loss and W-side gradient of (MF) for
 * callers that cannot allocate device memory.  The paper has no counterpart;
 * this exists for code that may not call cudaMalloc where it needs a
 * gradient: kernels driven from inside another framework's memory pool,
 * allocation-free real-time or graph-replay loops, and callers that only
 * hold buffers handed to them.  It allocates nothing: no cudaMalloc,
 * cudaFree or allocating library call.  Its one scratch array (a loss
 * partial per row) is a fixed file-scope device array of
 * BM_NOALLOC_MAX_ROWS doubles (2 MiB) that every GPU loading the library
 * keeps until the process exits.
 *   m, n      matrix size (internal orientation, any m, n >= 1); m must not
 *             exceed BM_NOALLOC_MAX_ROWS (else BM_ERR_INVALID).
 *   row_ptr   int64[m+1], col int32[nnz], val float[nnz]: CSR of Omega and A
 *             (columns < n; the arrays are trusted, not validated).
 *   W, H      float[m*ld], float[n*ld] row-major, 1 <= k <= ld <= 128,
 *             ld % 4 == 0; columns k..ld-1 must be zero.  W, H and gW must
 *             start on a 16-byte boundary (rows are moved as float4), else
 *             BM_ERR_INVALID; lambda must be finite in FP32.
 *   gW        float[m*ld] out: R H + lambda W (columns k..ld-1 written as 0).
 *   f         double* out (device): 1/2 sum r_e^2.
 *   stream    cudaStream_t the work is queued on (NULL: default stream).
 * Every pointer must be device memory.  The call is asynchronous: results
 * are ready when `stream` reaches them.  The first call on a device looks up
 * the scratch array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  Every
 * call shares the scratch array and overwrites the rows it reads, so calls
 * that overlap on the GPU (other streams, other threads) race; serialise them.
 * Failures return a status; the message is in bm_noalloc_last_error().
 */
#define BM_NOALLOC_MAX_ROWS 262144
bm_status bm_loss_grad_csr_noalloc(int64_t m, int64_t n, const int64_t* row_ptr, const int32_t* col,
                                   const float* val, const float* W, const float* H, int32_t k, int32_t ld,
                                   double lambda, float* gW, double* f, void* stream);
const char* bm_noalloc_last_error(void);

/*
 * bm_bcd_phase -- `epochs` sweeps of column-block coordinate descent on (MF):
 * the form of polyMF-SS the paper adopts for the BM phase of matrix
 * completion (matrix completion experiments: each block is one column of W
 * and the same column of H, exact line search).  Block c: g_w = R h_c +
 * lambda w_c, g_h = R^T w_c + lambda h_c, direction -(g_w, g_h), step = the
 * minimiser over s >= 0 of the objective's quartic along it (the rule of
 * bm_bm_phase); columns in order 0..k-1.  *F (nullable) = F after the last
 * block.  Errors: BM_ERR_INVALID for epochs < 0; BM_ERR_NUMERIC.
 */
bm_status bm_bcd_phase(bm_handle h, int32_t epochs, double* F);

/*
 * The SpaRSA step rule for the PG step (supplement Sec. "The SpaRSA variant
 * for Matrix Completion").  alpha_BB of Eq. "proxBB" from the last two points
 * X~_{t-1}, X~_t at which a PG step was taken, read as the step length
 * ||dX||_F^2 / <dX, dG> (the printed ratio is its reciprocal, a curvature),
 * with <dX, dG> = ||r_t - r_{t-1}||^2 over Omega and ||dX||_F^2 from k x k
 * Grams (Eq. "trace" with its last term's sign corrected), clipped to
 * [alpha_min, alpha_max]; the first step (no previous point, or after
 * bm_set_factors / bm_set_state) starts from bm_options.alpha, clipped alike.  Then the
 * smallest i >= 0 such that alpha = alpha_BB beta^i gives an X_{t+1}
 * satisfying Eq. "back" or Eq. "decrease" (delta); each rejected trial
 * restores X~_t and the warm-start / safeguard state exactly.  After
 * max_backtracks reductions the last trial is kept (accepted_by = 0).
 *   bm_bb_default_options: alpha_min 1e-3, alpha_max 1e3, beta 0.5,
 *     delta 0.995, max_backtracks 30.
 *   bm_set_bb_options: BM_ERR_INVALID unless 0 < alpha_min <= alpha_max
 *     (finite), beta and delta in (0, 1), max_backtracks >= 0.
 *   bm_prox_step_bb: info (nullable) as bm_prox_step, F = F(X_{t+1});
 *     bb (nullable) receives the step record.
 * Device memory: two extra copies of the factors and two residual arrays.
 */
typedef struct {
  double alpha_min;
  double alpha_max;
  double beta;
  double delta;
  int32_t max_backtracks;
  int32_t pad_;
} bm_bb_options;

typedef struct {
  double alpha_bb;       /* Eq. "proxBB" value before backtracking */
  double alpha;          /* step length taken */
  int32_t backtracks;    /* reductions by beta */
  int32_t accepted_by;   /* 1 Eq. "back", 2 Eq. "decrease" only, 0 none within max_backtracks */
} bm_bb_info;

bm_status bm_bb_default_options(bm_bb_options* o);
bm_status bm_set_bb_options(bm_handle h, const bm_bb_options* o);
bm_status bm_prox_step_bb(bm_handle h, bm_prox_info* info, bm_bb_info* bb);

/*
 * Kernel timing for measurement.  While enabled, the library records a pair
 * of CUDA events on the handle's stream around every launch of its kernels
 * (no extra synchronisation).  bm_profile_read synchronises, then reports per
 * kernel name: launches and total device milliseconds since the last enable.
 *   names     char[cap * 48], NUL-terminated names (may be NULL)
 *   launches  int64[cap], total_ms double[cap] (may be NULL)
 *   count     receives the number of kernel names (<= cap written)
 */
bm_status bm_profile_enable(bm_handle h, int32_t enable);
bm_status bm_profile_read(bm_handle h, int32_t cap, char* names, int64_t* launches, double* total_ms,
                          int32_t* count);

#ifdef __cplusplus
}
#endif
#endif /* BM_GB300_H */
