// Dense thin-block routines used by the proximal step: Grams C = A^T B over a
// long dimension, thin products Y = beta*Y + gamma*A*C, the q-wide SpMM of
// the residual, the symmetric eigensolver and small helpers.
#pragma once
#include "ctx.cuh"

namespace bm {

// A tall row-major block: rows x cols with leading dimension ld (multiple of 4).
struct Tall {
  float* p = nullptr;
  int64_t rows = 0;
  int cols = 0;
  int ld = 4;
  float* row(int64_t i) const { return p + i * ld; }
};

// Scratch for the dense routines (owned by the prox state).
struct DenseWork {
  DevBuf<double> gram_part;   // slab partials of Grams
  DevBuf<int> status;         // eigensolver status flags
  DevBuf<int> tc_status;      // tensor-core Gram: 1 after a barrier wait ran out (results poisoned with NaN)
  DevBuf<double> scratch;     // eigensolver work matrices
};

// C (a x b, FP64, row-major ldc = b) = A^T B, A: L x a, B: L x b.
// compensated: FP32 two-product/two-sum within a row tile (near-exact sums).
void gram_dev(bm_ctx& h, DenseWork& w, const Tall& A, const Tall& B, double* C, bool compensated,
              const char* tag);

// Tensor-core form of a plain Gram (gram_tc.cu): bfloat16 slices, six slice
// products per row step on tcgen05.mma, FP32 accumulation per block slab,
// FP64 sum of the slabs.  Returns false, launching nothing, when the shape
// does not fit it (a or b > 256, unaligned rows or bases).
bool gram_tc_dev(bm_ctx& h, DenseWork& w, const Tall& A, const Tall& B, double* C, const char* tag);

// C (a x b FP64) = sum over `slabs` FP32-pair slab partials (slab-major,
// a x b each, row-major), added in slab order; sym: read (j, i) for i > j.
void gram_reduce_dev(bm_ctx& h, const float2* part, int slabs, int a, int b, int sym, double* C);

// Y = beta * Y + gamma * A * C, A: L x a, C: a x b FP32 (row-major, ldc), Y: L x b.
void gemm_dev(bm_ctx& h, const Tall& A, const float* C, int ldc, const Tall& Y, float beta, float gamma,
              const char* tag);

// Shared launches of the q-wide residual SpMMs of several handles' PG steps,
// each running on its own host thread and stream (bm_batch_prox_step).  While
// h.comb is set, spmm_dev hands its product to the combiner and waits: when
// every participant still inside its PG step has handed one in (or the
// first waiting product has waited 100 us), the products that have arrived
// run as batched passes over the concatenated segment lists (one launch per
// orientation, row width and layout) on the combiner's stream, ordered after
// each participant's earlier work, and each participant's stream then waits
// for them.  A participant that finishes its PG step calls
// spmm_combiner_leave.  The products are the same, bit for bit, as those of
// separate launches.
SpmmCombiner* spmm_combiner_create(int participants_max);
void spmm_combiner_destroy(SpmmCombiner* c);
void spmm_combiner_begin(SpmmCombiner* c, int participants);
void spmm_combiner_leave(SpmmCombiner* c);
int64_t spmm_combiner_launches(const SpmmCombiner* c);   // batched launches so far
int64_t spmm_combiner_products(const SpmmCombiner* c);   // products handed in so far

// Sparse part of Z products: Out(i,:) += gamma * sum_e v_e X(idx_e,:) over a
// segment split (CSR: i = row, idx = col; CSC: i = col, idx = row).  Blocks
// wider than kSpmmCols run as several launches over column slices.
constexpr int kSpmmCols = 256;
void spmm_dev(bm_ctx& h, bool csr, const float* vals, const Tall& X, const Tall& Out, float gamma);

// Accuracy modes of the symmetric eigensolver.
//  kEigFast: FP32 Householder tridiagonalisation, then implicit QL, with one
//    divide-and-conquer level for 24 <= n <= 150 (the halves by QL, merged
//    through the secular equation); eigenvalue errors ~ eps32 * ||S||.
//  kEigRelative: kEigFast vectors V0, one FP64 Newton-Schulz step to an
//    orthogonal V, S' = V^T S V in FP64, then FP32 Jacobi
//    sweeps on S' with the relative rotation test |s_pq| > eps sqrt(s_pp s_qq);
//    for positive semidefinite S this resolves each eigenvalue to a relative
//    accuracy set by the conditioning of the diagonally scaled S' (Demmel and
//    Veselic, "Jacobi's method is more accurate than QR", 1992), so small
//    eigenvalues far below eps32 * ||S|| stay accurate.
//  kEigDouble: as kEigRelative with FP64 Jacobi sweeps.
enum EigMode { kEigFast = 0, kEigRelative = 1, kEigDouble = 2 };

// Symmetric eigendecomposition of S (n x n FP64, row-major, symmetrised on
// load): eigenvalues descending into evals[n] (FP64), eigenvectors into evecs
// (n x n FP64 row-major, column j = vector j).  Throws BM_ERR_NUMERIC if the
// iteration fails.
void sym_eig_dev(bm_ctx& h, DenseWork& w, const double* S, int n, double* evals, double* evecs, EigMode mode);

// T (n x n FP32, ld ldt) = R^{-1}, R^T R = S (S FP64 n x n, positive definite).
// Throws BM_ERR_NUMERIC if a pivot is not positive.
void chol_inv_dev(bm_ctx& h, DenseWork& w, const double* S, int n, float* T, int ldt);
// As chol_inv_dev, returning false instead of throwing when a pivot is not
// positive; on success *inv_fro2 = ||R^{-1}||_F^2, so lambda_min(S) >= 1 / *inv_fro2.
bool chol_inv_try_dev(bm_ctx& h, DenseWork& w, const double* S, int n, float* T, int ldt, double* inv_fro2);

// T (rows x cols FP32, ld) = E(0:rows, cols_idx) * diag(scale)  (E FP64 n x n)
void select_scale_dev(bm_ctx& h, const double* E, int n, int rows, const int* cols_h, const double* scale_h,
                      int cols, float* T, int ldt);

// FP64 -> FP32 copy of a small matrix with new leading dimension.
void small_to_f32_dev(bm_ctx& h, const double* S, int rows, int cols, int lds, float* T, int ldt);

// C = A * B (FP64 small matrices, row-major, dims r x s times s x t) and
// C = A * B^T (r x s times t x s).
void small_mm_dev(bm_ctx& h, const double* A, const double* B, double* C, int r, int s, int t, bool transB);

// x(count) = counter-based standard normals (SplitMix64 + Box-Muller, FP64) as FP32,
// written into column `col` of the tall block.
void counter_normal_dev(bm_ctx& h, uint64_t seed, uint64_t stream, int64_t count, const Tall& X, int col);

// Fill `val` with -A (CSR and CSC order).
void negate_values_dev(bm_ctx& h, const float* a, float* out, int64_t count);

// sums over Omega: out[0] = sum r^2, out[1] = sum r*a  (CSR order)
void residual_sums_dev(bm_ctx& h, const float* r, const float* a, int64_t nnz, double out[2]);

// column copy: dst(:, d0:d0+c) = src(:, s0:s0+c)
void copy_cols_dev(bm_ctx& h, const Tall& src, int s0, const Tall& dst, int d0, int c);

// set all of a tall block to zero (rows x ld)
void zero_dev(bm_ctx& h, const Tall& X);

}  // namespace bm
