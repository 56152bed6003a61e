// Internal host interface between the C ABI layer and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/lrs.h"

#include <vector>

struct lrs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int coop_ok = 0;
  char err[512] = {0};
  // workspace: one device arena, bump-allocated per call and reset at call entry
  char* ws = nullptr;
  size_t ws_cap = 0;
  size_t ws_top = 0;
  size_t ws_limit = 0;      // lrs_set_workspace_limit (0: none)
  // small pinned host buffer for scalar read-back
  void* host_scratch = nullptr;
  // side buffer for split-K partial sums of the CUDA-core GEMM (independent of
  // the workspace arena, which callers lay out before the GEMM runs)
  void* aux = nullptr;
  size_t aux_cap = 0;
  int64_t launches = 0;
  // a second stream for independent work inside one call (forked from and
  // joined back into `stream` with the two events); created on first use
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  // Record / replay of a call sequence (the batch graph, batch.cu).  replay
  // 0: every host read-back as usual.  1 (record): the same, and each value
  // read back is appended to `log`.  2 (capture): the stream is being
  // captured into a CUDA graph; a read-back takes the next logged value
  // instead of waiting, and a guard kernel in its place ORs 1 into
  // *cap_guard when the graph runs and the device holds another value; the
  // error estimates are written to cap_err[0] (SVD) and cap_err[1] (ID) on
  // the device.
  int replay = 0;
  std::vector<int32_t> log;
  size_t log_pos = 0;
  int* cap_guard = nullptr;
  double* cap_err = nullptr;
  // optional timing of the A-pass kernel (lrs_set_kernel_timing)
  int time_kernels = 0;
  cudaEvent_t kev0 = nullptr, kev1 = nullptr;
  double last_kernel_ms = -1.0;
};

lrs_status lrs_fail(lrs_ctx* ctx, lrs_status st, const char* fmt, ...);

namespace lrs {

// kernel attributes ---------------------------------------------------------
// Raise (never lower) func's dynamic shared-memory limit on ctx's device; safe
// across threads.  Every launch with more than 48 KB of dynamic shared memory
// goes through it.
lrs_status raise_dyn_smem(lrs_ctx* ctx, const void* func, size_t bytes);

// record / replay of host read-backs (lrs_ctx::replay) -----------------------
constexpr int kReplayRecord = 1, kReplayCapture = 2;
// out[i] = the host value of the device int dev[i], i < n (n <= 8), as the
// context's replay mode says; synchronises unless capturing
lrs_status replay_ints(lrs_ctx* ctx, int n, const int32_t* const* dev, int32_t* out);
// capture mode: err = sqrt(sum_{i >= kk} s_i^2 / fro2) (0 when fro2 <= 0 or
// NULL) into *out on the device, as svd_finish computes it on the host
lrs_status launch_err_tail(lrs_ctx* ctx, const double* s, int64_t r, int64_t kk, const double* fro2, double* out);
// capture mode: err = sqrt(max(tail2, 0) / nrm2) (0 when nrm2 <= 0) into *out
lrs_status launch_err_ratio(lrs_ctx* ctx, const double* tail2, const double* nrm2, double* out);

// workspace ---------------------------------------------------------------
lrs_status ws_reserve(lrs_ctx* ctx, size_t bytes);           // grow (only between calls)
lrs_status aux_reserve(lrs_ctx* ctx, size_t bytes);          // grow ctx->aux (synchronises when it grows)
void* ws_alloc(lrs_ctx* ctx, size_t bytes);                   // 256-B aligned, nullptr if full

// sketch.cu ----------------------------------------------------------------
struct GridDev {
  int ndim, kind;
  int64_t N[3];
  int32_t s[3];
  int64_t Nc[3];
  int64_t n, l;
};
bool grid_from_abi(const lrs_grid* g, GridDev* out, char* why, size_t nwhy);
// Y[m x l] (FP64) = A D
lrs_status launch_sketch(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                         const GridDev& g, double* Y, int64_t ldy);
// W[m x |I|] (FP64) = A(:, I)  with I the injection points of grid g
lrs_status launch_gather(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                         const GridDev& g, double* W, int64_t ldw);
// *out = sum of part[0..np) (device, one block, fixed order)
lrs_status launch_sum(lrs_ctx* ctx, const double* part, int np, double* out);
// W (m x |I|) and W^T (|I| x m), FP32, from one pass over A (WT NULL: W alone)
lrs_status launch_gather32_both(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                                const GridDev& g, float* W, int64_t ldw, float* WT, int64_t ldwt);
// sum of squares of A (m x n), FP64, into *out (device).  FP32 rows are
// summed in FP32 per thread segment unless exact = 1 (every square in FP64:
// for a difference of two such sums, e.g. 1 - ||Q^T A||^2 / ||A||^2)
lrs_status launch_fro2(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t n,
                       int64_t lda, double* out, int exact = 0);

// gemm_simt.cu / gemm_tc.cu -----------------------------------------------
// C (M x N) = X^T A ; X: K x M (ldx), A: K x N (lda); row-major everything.
struct GemmArgs {
  int64_t M, N, K;
  const void* X; int32_t xdt; int64_t ldx;
  const void* A; int32_t adt; int64_t lda;
  void* C; int c_f64; int c_trans; int64_t ldc;
  double alpha;            // C = alpha * X^T A
  int accum = 0;           // 1: C += alpha * X^T A
};
lrs_status launch_gemm_simt(lrs_ctx* ctx, const GemmArgs& a, int fp64);
// lrs_api.cu: the precision dispatch of every product (FP64 / FP32 CUDA cores, tensor-core forms)
lrs_status gemm_prec(lrs_ctx* ctx, int prec, int64_t M, int64_t N, int64_t K, const void* X, int32_t xdt, int64_t ldx,
                     const void* A, int32_t adt, int64_t lda, void* C, int c_f64, int c_trans, int64_t ldc);
// the SVD of a given B (r x n, row stride n; FP64 when prec is FP64, else FP32)
// with rows in the basis Q (m x r): U = Q U_B, S, V = B^T U_B S^-1, as lrs_svd_k
size_t svd_from_b_ws(int64_t r, int64_t n, int64_t m, int64_t kk, int32_t prec, int num_sms);
lrs_status svd_from_b(lrs_ctx* ctx, const void* B, int64_t r, int64_t n, const double* Q, int64_t ldq, int64_t m,
                      int32_t k, int32_t prec, double* U, int64_t ldu, double* S, void* V, int64_t ldv,
                      const double* fro2, double* err_est);
// fro2_out (device, may be NULL): also ||A||_F^2 of the operand A, fused (M <= 128 only)
lrs_status launch_gemm_tc(lrs_ctx* ctx, const GemmArgs& a, int prec, double* fro2_out = nullptr);
// apass_tc.cu: the same product for a narrow X (M <= 256) and a wide FP32/BF16
// A, with A's slabs staged by TMA.  launch_gemm_tc dispatches here whenever
// apass_eligible holds.
bool apass_eligible(const GemmArgs& a, int prec);
size_t apass_workspace(int64_t M, int64_t K, int prec);
lrs_status launch_apass(lrs_ctx* ctx, const GemmArgs& a, int prec, double* fro2_out);
// workspace bytes the tensor-core path needs for an M x K operand X (0 for SIMT modes)
size_t gemm_tc_workspace(int64_t M, int64_t K, int prec);
// extra workspace that lets the generic tensor-core product split its K x N
// operand A once instead of once per row tile (used when available)
size_t gemm_tc_a_workspace(int64_t N, int64_t K, int prec);
// extra workspace of the split-K partial sums for an M x N x K product (0 when not split)
size_t gemm_tc_splitk_workspace(int64_t M, int64_t N, int64_t K, int num_sms);

// cpqr.cu --------------------------------------------------------------------
// Householder CPQR of the p x c matrix M stored COLUMN-major (column j at
// M + j*ldm), in place, FP64.  Stops after kmax steps or when the largest
// remaining column norm <= rtol * |R_00|.
struct CpqrOut {
  int32_t* perm;     // device, c entries: position -> original column
  double* R;         // device, kmax x c, row-major (row stride c), pivoted column order
  double* V;         // device, Householder vectors, p x kmax column-major (unit norm)
  double* tail2;     // device, 1: squared Frobenius norm of the trailing block
  int32_t* rank;     // device, 1: steps taken
};
lrs_status launch_cpqr(lrs_ctx* ctx, double* M, int64_t p, int64_t c, int64_t ldm,
                       int64_t kmax, double rtol, const CpqrOut& o);
// exact workspace bytes launch_cpqr allocates for these sizes
size_t cpqr_scratch_bytes(int64_t p, int64_t c, int64_t kmax, int num_sms);
// Q (p x r, row-major ldq) = H_0 ... H_{r-1} [I_r; 0]
lrs_status launch_form_q(lrs_ctx* ctx, const double* V, int64_t p, int64_t r,
                         double* Q, int64_t ldq);
// workspace launch_form_q takes for p rows and r columns (0 when a column fits
// in shared memory)
inline size_t form_q_ws(int64_t p, int64_t r) {
  return 8 * (size_t)p > 200 * 1024 ? ((8 * (size_t)(p * r) + 255) & ~size_t(255)) : 0;
}
// ID: P (m x k) from R (k x m, pivoted order) and perm.
lrs_status launch_id_coeffs(lrs_ctx* ctx, const double* R, int64_t k, int64_t m,
                            const int32_t* perm, int32_t* J, double* P, int64_t ldp);

// orth_gram.cu ------------------------------------------------------------------
// Orthonormal basis of a tall-skinny M (p x c row-major, p >= 4c, c <= 128)
// by pivoted Cholesky of the FP64 Gram (CPQR's pivots and stop rule) and one
// Cholesky-QR refinement.  Only for rtol >= kOrthGramRtolMin (the Gram squares
// the condition number).  Returns LRS_ERANK (nothing reported) when the
// refinement breaks down; the caller then runs Householder CPQR.  Synchronises.
constexpr double kOrthGramRtolMin = 1e-6;
bool orth_gram_eligible(int64_t p, int64_t c, double rtol);
size_t orth_gram_ws(int64_t p, int64_t c, int num_sms);
// refine = false: skip the Cholesky-QR2 pass (well-conditioned basis of the
// same range, orthonormal only to ~u cond^2; for intermediate C-PWR iterates)
// the range finder of lrs_range_find on M (p x c, row stride ldi) into Q
// (p x r, row stride ldq), with its workspace bound; callers reserve first.
// kcap > 0: at most kcap pivoted Householder steps (r <= kcap)
size_t orth_ws_of(int64_t p, int64_t c, int num_sms);
lrs_status orth_basis(lrs_ctx* ctx, const double* M, int64_t p, int64_t c, int64_t ldi, double rtol, double* Q,
                      int64_t ldq, int64_t* r_out, int64_t kcap = 0);
// spc.cu: C[i][j] = (sum_t a(i,t) b(t,j)) / div[i] (div may be NULL), FP64, with
// a(i,t) = A[i*a_si + t*a_st], b(t,j) = B[t*b_st + col(j)*b_sj], col(j) = cols ? cols[j] : j
lrs_status spc_small_gemm(lrs_ctx* ctx, int64_t M, int64_t N, int64_t K, const double* A, int64_t a_si, int64_t a_st,
                          const double* B, int64_t b_st, int64_t b_sj, const int32_t* cols, const double* div,
                          double* C, int64_t ldc);
// spc.cu: eps_hat[i] = cf lambda_max(B_f B_f^T - taus[i] B_c B_c^T) from kept rows
// B_f (mc x n, storage dtype, row stride ldb) and B_c (mc x l FP64, row stride ldc);
// taus / eps_hat host arrays; synchronises
lrs_status spc_err_from_rows(lrs_ctx* ctx, const void* Bf, int32_t dtype, int64_t mc, int64_t n, int64_t ldb,
                             const double* Bc, int64_t l, int64_t ldc, double cf, const double* taus, int32_t ntau,
                             double* eps_hat);
// rdiag (optional, device): |R_ii| of the pivoted factor, i < r
// Rt (optional, device, r x c row-major): the factor in original column
// order, M ~= Q Rt (with the refinement folded in)
lrs_status launch_orth_gram(lrs_ctx* ctx, const double* M, int64_t p, int64_t c, int64_t ldm, double rtol,
                            double* Q, int64_t ldq, int64_t* r_out, bool refine = true, double* rdiag = nullptr,
                            double* Rt = nullptr);
// one-block Cholesky of a c x c PSD G (pivot = 1: pivoted, CPQR's rules),
// R (rows 0..rank-1, row stride ldr, pivoted order, zeros below the diagonal)
lrs_status launch_pchol(lrs_ctx* ctx, const double* G, int c, int kmax, double rtol, int pivot, int32_t* perm,
                        double* R, int64_t ldr, int32_t* rank);
// G (c x c, full, row-major) = M^T M for M p x c (row stride ldm, c <= 128);
// workspace num_sms * c (c + 1) / 2 doubles
lrs_status launch_gram(lrs_ctx* ctx, const double* M, int64_t p, int c, int64_t ldm, double* G);
// Q (p x r, row stride ldq) = M(:, perm[0..r)) R^{-1}, R the leading r x r
// upper triangle of an ldr-strided matrix (perm NULL: the first r columns)
lrs_status launch_trsm_rows(lrs_ctx* ctx, const double* M, int64_t p, int64_t ldm, const int32_t* perm,
                            const double* R, int64_t ldr, int r, double* Q, int64_t ldq);
// Rt(t, perm[j]) = R(t, j) for the pivoted factor R (rows 0..r-1, row stride ldr)
lrs_status launch_rt_scatter(lrs_ctx* ctx, const double* R, int64_t ldr, const int32_t* perm, int64_t r, int64_t c,
                             double* Rt);
// the same for a WIDE (or square) M (c > 128 columns): left-looking pivoted
// Cholesky that forms only the pivots' Gram columns (one cooperative launch),
// then the tall-skinny tail (Q_1 = M(:, piv) R_11^{-1}, one Cholesky-QR
// refinement).  LRS_ERANK (nothing reported) when the rank exceeds 128 or the
// refinement breaks down: the caller then runs Householder CPQR.
bool orth_wide_eligible(int64_t p, int64_t c, double rtol, int num_sms);
size_t orth_wide_ws(int64_t p, int64_t c, int num_sms);
lrs_status launch_orth_wide(lrs_ctx* ctx, const double* M, int64_t p, int64_t c, int64_t ldm, double rtol,
                            double* Q, int64_t ldq, int64_t* r_out, bool refine, double* rdiag, double* Rt = nullptr);
// out[i] = |R[i * ld + i]|, i < r (device pointers)
lrs_status launch_abs_diag(lrs_ctx* ctx, const double* R, int64_t ld, int64_t r, double* out);

// R (r x r upper, row-major, positive diagonal) with R^T R = B B^T for a wide
// FP32 B (r x n, r <= 128): exact-slice Gram on the tensor cores + FP64
// Cholesky.  With perm_out (device, r entries) the Cholesky is pivoted:
// P^T B B^T P = R^T R, perm_out[pos] = row of B.  LRS_ERANK (nothing
// reported) when the Cholesky breaks down; the caller then runs TSQR.
// Synchronises.
size_t r_of_bt_gram_ws(int64_t r, int num_sms);
// G (r x r FP64, both triangles) = B B^T for B r x n FP32 (row stride ldb),
// r <= 128: an exact-slice product on the tensor cores (~2^-46 relative);
// workspace gram_oz_ws(r, num_sms).  Synchronises (error flag).
size_t gram_oz_ws(int64_t r, int num_sms);
lrs_status launch_gram_oz(lrs_ctx* ctx, const float* B, int64_t r, int64_t n, int64_t ldb, double* G);
lrs_status launch_r_of_bt_gram(lrs_ctx* ctx, const float* B, int64_t r, int64_t n, int64_t ldb, double* R,
                               int32_t* perm_out = nullptr);

// svd_small.cu ------------------------------------------------------------------
// R factor (r x r, row-major) of B^T where B is r x n row-major in FP32 or FP64.
lrs_status launch_tsqr(lrs_ctx* ctx, const void* B, int b_f64, int64_t r, int64_t n,
                       int64_t ldb, double* R);
// FP64 one-sided Jacobi on the columns of R (r x r): R V = U_R diag(s); returns
// V (r x r, row-major) and s (r), sorted descending.
lrs_status launch_jacobi(lrs_ctx* ctx, double* R, int64_t r, double* V, double* s);
// workspace of the multi-SM FP64 Jacobi on r columns of length len (launch_jacobi
// falls back to one block without it)
size_t jacobi_ws(int64_t r, int64_t len);
// jacobi_cluster.cu: FP64 one-sided Jacobi on the rows of R (r x r upper
// triangular, row stride ldr) on one thread-block cluster: U_B (r x r
// row-major, row perm[i] <- position i; perm NULL = identity) and s (r),
// descending.  LRS_ERANK (nothing launched) when no cluster fits or r is out
// of range [8, 1024]; workspace jacobi_rows_ws(r).
size_t jacobi_rows_ws(int64_t r);
lrs_status launch_jacobi_rows(lrs_ctx* ctx, const double* R, int64_t r, int64_t ldr, const int32_t* perm,
                              double* Ub, double* s);

// misc.cu -------------------------------------------------------------------------
// transposed copy of a row-major FP64 matrix: dst (cols x rows) = src^T
lrs_status launch_transpose(lrs_ctx* ctx, const double* src, int64_t rows, int64_t cols,
                            int64_t lds, double* dst, int64_t ldd);
// the same for FP32
lrs_status launch_transpose32(lrs_ctx* ctx, const float* src, int64_t rows, int64_t cols, int64_t lds,
                              float* dst, int64_t ldd);
// two-block cooperative launch whose barrier wait runs out (lrs_selftest_barrier_timeout)
lrs_status launch_barrier_selftest(lrs_ctx* ctx, int64_t spin_limit);
// FP32 -> FP64 copy of n contiguous values (exact)
lrs_status launch_widen_f32(lrs_ctx* ctx, const float* src, int64_t n, double* dst);
// FP64 -> FP32 copy (round to nearest)
lrs_status launch_to_f32(lrs_ctx* ctx, const double* src, int64_t rows, int64_t cols, int64_t lds,
                         float* dst, int64_t ldd);
// U columns sign fix (largest |entry| positive, lowest row on ties): flips U
// (m x k) in place and writes the applied signs (+1/-1) to sign_out (k)
lrs_status launch_sign_fix(lrs_ctx* ctx, double* U, int64_t m, int64_t k, int64_t ldu, double* sign_out);
// W[:, j] = sign[j] * V[:, j] / s[j]  (r x k, FP64; sign may be NULL)
lrs_status launch_scale_cols(lrs_ctx* ctx, const double* V, int64_t r, int64_t ldv,
                             const double* s, const double* sign, int64_t k, double* W, int64_t ldw);

}  // namespace lrs
