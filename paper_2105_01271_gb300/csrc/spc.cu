// SPC-ID lifting (Sec. 4, Alg. 5) and its single-pass error estimate
// SPC-ID-ERR (Alg. 6), declared in include/lrs.h.
//
// Lifting.  With the SVD of the sketch A_c = Y (U_r, S_r, V_r: its leading r
// triplets) and the row ID's skeleton rows J, the lifted skeleton is
//     S_f = A_c(J,:) T_r = A_c(J,:) V_r S_r^-1 U_r^T A_f = X^T A_f,
//     X   = U_r S_r^-1 V_r^T A_c(J,:)^T                       (m x k)
// (T_r = A_c^+ U_r U_r^T A_f, the form Alg. 5's operator takes once
// H^T = A_c^T A_f is substituted).  A_f is resident in HBM here, so the
// sketch is known before the one full read, and that read contracts A_f
// with the k columns of X instead of accumulating H (n x l) and forming
// T_r (l x n): S_r^-1 is applied once, not twice.
//
// Error estimate.  Every c-th snapshot, B_f = A_f(J,:), B_c = A_c(J,:):
//     eps_hat(tau) = c lambda_max(B_f B_f^T - tau B_c B_c^T)
// for each tau of a caller-given grid.  The m_c x m_c Grams are FP64 (FP32
// data: the exact-slice Gram of the SVD path), and lambda_max comes from one
// block per tau: Householder tridiagonalisation in shared memory, then
// bisection on Sturm counts.
#include "common.cuh"
#include "internal.h"

#include <math.h>

namespace lrs {
namespace {

constexpr int kEigMax = 128;    // largest m_c (the matrix lives in shared memory)

// C[i][j] = (sum_t a(i,t) b(t,j)) / div[i] (div may be NULL), FP64,
//   a(i,t) = A[i*a_si + t*a_st],  b(t,j) = B[t*b_st + col(j)*b_sj],  col(j) = cols ? cols[j] : j.
// 16 x 16 output tile per block, K staged through shared memory 16 at a time.
__global__ void k_small_gemm(int64_t M, int64_t N, int64_t K, const double* __restrict__ A, int64_t a_si,
                             int64_t a_st, const double* __restrict__ B, int64_t b_st, int64_t b_sj,
                             const int32_t* __restrict__ cols, const double* __restrict__ div,
                             double* __restrict__ C, int64_t ldc) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * 16, j0 = (int64_t)blockIdx.x * 16;
  const int64_t bj = j0 + tx;
  const int64_t bcol = bj < N ? (cols ? (int64_t)cols[bj] : bj) : 0;
  // four interleaved partial sums (one FP64 FMA chain would wait ~64 cycles
  // per term), combined in a fixed order
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
  for (int64_t t0 = 0; t0 < K; t0 += 16) {
    const int64_t ai = i0 + ty, at = t0 + tx, bt = t0 + ty;
    As[ty][tx] = (ai < M && at < K) ? A[ai * a_si + at * a_st] : 0.0;
    Bs[ty][tx] = (bt < K && bj < N) ? B[bt * b_st + bcol * b_sj] : 0.0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u += 4) {
      acc0 = fma(As[ty][u], Bs[u][tx], acc0);
      acc1 = fma(As[ty][u + 1], Bs[u + 1][tx], acc1);
      acc2 = fma(As[ty][u + 2], Bs[u + 2][tx], acc2);
      acc3 = fma(As[ty][u + 3], Bs[u + 3][tx], acc3);
    }
    __syncthreads();
  }
  const double acc = (acc0 + acc1) + (acc2 + acc3);
  const int64_t i = i0 + ty;
  if (i < M && bj < N) C[i * ldc + bj] = div ? acc / div[i] : acc;
}

lrs_status small_gemm(lrs_ctx* ctx, int64_t M, int64_t N, int64_t K, const double* A, int64_t a_si, int64_t a_st,
                      const double* B, int64_t b_st, int64_t b_sj, const int32_t* cols, const double* div,
                      double* C, int64_t ldc) {
  if (M < 1 || N < 1) return LRS_OK;
  const dim3 grid((unsigned)((N + 15) / 16), (unsigned)((M + 15) / 16));
  if (grid.y > 65535u) return lrs_fail(ctx, LRS_EINVAL, "spc: %lld rows exceed the small-product grid", (long long)M);
  k_small_gemm<<<grid, 256, 0, ctx->stream>>>(M, N, K, A, a_si, a_st, B, b_st, b_sj, cols, div, C, ldc);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// Row Gram, partial over a column slab: part[b][e] = sum_{t in slab b} B(i,t) B(j,t)
// for the packed upper-triangle entry e = (i, j), i <= j < r.  B(i, t) =
// B[i * ldb + t] in storage type dt.  32 columns are staged in shared memory
// (FP64) at a time; thread x owns the entries x, x + 256, ...
constexpr int kRgCols = 32;
constexpr int kRgPer = 33;      // ceil(128 * 129 / 2 / 256)

__global__ void __launch_bounds__(256) k_row_gram(const void* __restrict__ B, int32_t dt, int r, int64_t n,
                                                  int64_t ldb, int64_t cols_b, double* __restrict__ part) {
  extern __shared__ double rg[];                   // r x (kRgCols + 1)
  const int T = r * (r + 1) / 2;
  const int64_t c0 = (int64_t)blockIdx.x * cols_b;
  const int64_t c1 = min(n, c0 + cols_b);
  int ei[kRgPer], ej[kRgPer];
  double acc[kRgPer];
#pragma unroll
  for (int u = 0; u < kRgPer; ++u) {
    const int e = threadIdx.x + 256 * u;
    int i = 0, rem = e;
    while (i < r && rem >= r - i) { rem -= r - i; ++i; }       // row i holds r - i entries (i..r-1)
    ei[u] = i;
    ej[u] = i + rem;
    acc[u] = 0.0;
  }
  for (int64_t a0 = c0; a0 < c1; a0 += kRgCols) {
    const int nc = (int)min((int64_t)kRgCols, c1 - a0);
    __syncthreads();
    for (int e = threadIdx.x; e < r * kRgCols; e += blockDim.x) {
      const int i = e / kRgCols, t = e - i * kRgCols;
      rg[i * (kRgCols + 1) + t] = t < nc ? ld_f64(B, dt, (int64_t)i * ldb + a0 + t) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kRgPer; ++u) {
      if (threadIdx.x + 256 * u < T) {
        const double* xi = rg + ei[u] * (kRgCols + 1);
        const double* xj = rg + ej[u] * (kRgCols + 1);
        double s = acc[u];
        for (int t = 0; t < kRgCols; ++t) s = fma(xi[t], xj[t], s);
        acc[u] = s;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kRgPer; ++u) {
    const int e = threadIdx.x + 256 * u;
    if (e < T) part[(int64_t)blockIdx.x * T + e] = acc[u];
  }
}

// G (r x r, both triangles) = sum over blocks of the packed partials, in block order
__global__ void k_row_gram_reduce(const double* __restrict__ part, int nb, int r, double* __restrict__ G) {
  const int T = r * (r + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < T; e += gridDim.x * blockDim.x) {
    int i = 0, rem = e;
    while (rem >= r - i) { rem -= r - i; ++i; }
    const int j = i + rem;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * T + e];
    G[i * r + j] = s;
    G[j * r + i] = s;
  }
}

size_t row_gram_ws(int64_t r, int num_sms) {
  return sizeof(double) * (size_t)(2 * num_sms) * (size_t)(r * (r + 1) / 2) + 512;
}

lrs_status row_gram(lrs_ctx* ctx, const void* B, int32_t dt, int64_t r, int64_t n, int64_t ldb, double* G) {
  int64_t nb = 2 * (int64_t)ctx->num_sms;
  int64_t cols_b = (n + nb - 1) / nb;
  cols_b = ((cols_b + kRgCols - 1) / kRgCols) * kRgCols;
  nb = (n + cols_b - 1) / cols_b;
  const int64_t T = r * (r + 1) / 2;
  double* part = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(nb * T));
  if (!part) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (row gram)");
  const size_t dyn = sizeof(double) * (size_t)(r * (kRgCols + 1));
  k_row_gram<<<(unsigned)nb, 256, dyn, ctx->stream>>>(B, dt, (int)r, n, ldb, cols_b, part);
  k_row_gram_reduce<<<(unsigned)((T + 255) / 256), 256, 0, ctx->stream>>>(part, (int)nb, (int)r, G);
  ctx->launches += 2;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// Sturm count of the symmetric tridiagonal (d, e): the number of its
// eigenvalues below x, from the signs of the LDL^T pivots of T - x I.
__device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// out[b] = c * lambda_max(Gf - taus[b] Gc) (n x n symmetric, n <= kEigMax), one
// block per tau: Householder reduction of the matrix to tridiagonal form in
// shared memory (Golub & Van Loan, Sec. 8.3.1), then bisection on the Sturm
// count (Sec. 8.4.1) with kEigPts points per pass, so each pass narrows the
// bracket of lambda_max by kEigPts + 1; 10 passes reach the rounding level.
constexpr int kEigPts = 64;
constexpr int kEigPasses = 10;

__global__ void __launch_bounds__(256) k_eig_max(const double* __restrict__ Gf, const double* __restrict__ Gc,
                                                 int n, const double* __restrict__ taus, double c,
                                                 double* __restrict__ out) {
  extern __shared__ double em[];
  const int ld = n + 1;
  double* M = em;                 // n x ld
  double* v = M + n * ld;         // Householder vector
  double* w = v + n;              // p, then w = p - K v
  double* d = w + n;              // tridiagonal: diagonal
  double* e = d + n;              //              sub-diagonal, e[i] couples i and i + 1
  __shared__ double red[32];
  __shared__ double s_lo, s_hi;
  __shared__ int s_cnt[kEigPts];
  const double tau = taus[blockIdx.x];
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int i = q / n, j = q - i * n;
    M[i * ld + j] = Gf[q] - tau * Gc[q];
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int len = n - k - 1;                                   // column k below the diagonal
    double xs = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const double x = M[(k + 1 + i) * ld + k];
      xs += x * x;
    }
    xs = block_sum(xs, red);
    const double x0 = M[(k + 1) * ld + k];
    if (threadIdx.x == 0) d[k] = M[k * ld + k];
    if (xs == 0.0) {                                             // already reduced (block-uniform)
      if (threadIdx.x == 0) e[k] = 0.0;
      __syncthreads();
      continue;
    }
    const double nx = sqrt(xs);
    const double alpha = x0 >= 0.0 ? -nx : nx;                   // H x = alpha e_1
    const double beta = 1.0 / (xs - alpha * x0);                 // 2 / (v^T v), v = x - alpha e_1
    for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = i == 0 ? x0 - alpha : M[(k + 1 + i) * ld + k];
    if (threadIdx.x == 0) e[k] = alpha;
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {       // p = beta A22 v
      const double* row = M + (k + 1 + i) * ld + (k + 1);
      double acc = 0.0;
      for (int j = 0; j < len; ++j) acc = fma(row[j], v[j], acc);
      w[i] = beta * acc;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) pv += w[i] * v[i];
    pv = block_sum(pv, red);
    const double K = 0.5 * beta * pv;
    for (int i = threadIdx.x; i < len; i += blockDim.x) w[i] -= K * v[i];
    __syncthreads();
    for (int q = threadIdx.x; q < len * len; q += blockDim.x) {  // A22 -= v w^T + w v^T
      const int i = q / len, j = q - i * len;
      M[(k + 1 + i) * ld + (k + 1 + j)] -= v[i] * w[j] + w[i] * v[j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = M[(n - 2) * ld + (n - 2)];
      e[n - 2] = M[(n - 1) * ld + (n - 2)];
    }
    d[n - 1] = M[(n - 1) * ld + (n - 1)];
    // Gershgorin bracket of the spectrum
    double lo = d[0], hi = d[0], emax = 0.0;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      if (i + 1 < n) emax = fmax(emax, fabs(e[i]));
    }
    const double pad = 1e-15 * fmax(fabs(lo), fabs(hi)) + 1e-300;
    s_lo = lo - pad;
    s_hi = hi + pad;
    red[0] = 1e-290 * fmax(1.0, emax * emax);                    // smallest pivot magnitude
  }
  __syncthreads();
  const double pivmin = red[0];
  __syncthreads();
  for (int pass = 0; pass < kEigPasses; ++pass) {
    const double lo = s_lo, hi = s_hi;
    if (threadIdx.x < kEigPts) {
      const double x = lo + (hi - lo) * (double)(threadIdx.x + 1) / (double)(kEigPts + 1);
      s_cnt[threadIdx.x] = sturm_count(d, e, n, x, pivmin);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // count(x) = n exactly when lambda_max < x: keep the last point below it
      int t = -1;
      while (t + 1 < kEigPts && s_cnt[t + 1] < n) ++t;
      const double step = (hi - lo) / (double)(kEigPts + 1);
      s_lo = t < 0 ? lo : lo + step * (double)(t + 1);
      s_hi = t + 1 < kEigPts ? lo + step * (double)(t + 2) : hi;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = c * 0.5 * (s_lo + s_hi);
}

size_t eig_smem(int n) { return sizeof(double) * ((size_t)n * (size_t)(n + 1) + 4 * (size_t)n); }

bool spc_dtype_ok(int32_t dt) { return dt == LRS_F64 || dt == LRS_F32 || dt == LRS_BF16; }

// eps_hat[i] = cf * lambda_max(B_f B_f^T - taus[i] B_c B_c^T) for kept rows
// B_f (mc x n, storage dt, row stride ldb) and B_c (mc x l FP64, row stride ldc)
lrs_status spc_err_rows(lrs_ctx* ctx, const void* Bf, int32_t dtype, int64_t mc, int64_t n, int64_t ldb,
                        const double* Bc, int64_t l, int64_t ldc, double cf, const double* taus, int32_t ntau,
                        double* eps_hat) {
  if (ntau < 1 || ntau > 65535) return lrs_fail(ctx, LRS_EINVAL, "spc_err: %d taus", ntau);
  if (mc < 1 || mc > kEigMax)
    return lrs_fail(ctx, LRS_EINVAL, "spc_err: m_c = %lld kept rows outside [1, %d]", (long long)mc, kEigMax);
  for (int32_t i = 0; i < ntau; ++i)
    if (!(taus[i] >= 0.0) || !isfinite(taus[i])) return lrs_fail(ctx, LRS_EINVAL, "spc_err: tau[%d] = %g", i, taus[i]);
  const size_t gram_ws = dtype == LRS_F32 ? gram_oz_ws(mc, ctx->num_sms) : row_gram_ws(mc, ctx->num_sms);
  const size_t need = 2 * 8 * (size_t)(mc * mc) + 16 * (size_t)ntau + 4 * (size_t)ntau + gram_ws +
                      row_gram_ws(mc, ctx->num_sms) + 8192;
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  double* Gf = (double*)ws_alloc(ctx, 8 * (size_t)(mc * mc));
  double* Gc = (double*)ws_alloc(ctx, 8 * (size_t)(mc * mc));
  double* dtau = (double*)ws_alloc(ctx, 8 * (size_t)ntau);
  double* dout = (double*)ws_alloc(ctx, 8 * (size_t)ntau);
  if (!Gf || !Gc || !dtau || !dout) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (spc_err)");
  const size_t mark = ctx->ws_top;
  if (dtype == LRS_F32) st = launch_gram_oz(ctx, (const float*)Bf, mc, n, ldb, Gf);
  else st = row_gram(ctx, Bf, dtype, mc, n, ldb, Gf);
  if (st) return st;
  ctx->ws_top = mark;
  st = row_gram(ctx, Bc, LRS_F64, mc, l, ldc, Gc);
  if (st) return st;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(dtau, taus, 8 * (size_t)ntau, cudaMemcpyHostToDevice, ctx->stream));
  const size_t smem = eig_smem((int)mc);
  if (smem > 48 * 1024) {
    st = raise_dyn_smem(ctx, (const void*)k_eig_max, smem);
    if (st) return st;
  }
  k_eig_max<<<(unsigned)ntau, 256, smem, ctx->stream>>>(Gf, Gc, (int)mc, dtau, cf, dout);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(eps_hat, dout, 8 * (size_t)ntau, cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return LRS_OK;
}

constexpr int64_t kSketchSvdDirs = 112;   // the FP64 Jacobi tile of lrs_svd_k holds r <= 112

}  // namespace

lrs_status spc_small_gemm(lrs_ctx* ctx, int64_t M, int64_t N, int64_t K, const double* A, int64_t a_si, int64_t a_st,
                          const double* B, int64_t b_st, int64_t b_sj, const int32_t* cols, const double* div,
                          double* C, int64_t ldc) {
  return small_gemm(ctx, M, N, K, A, a_si, a_st, B, b_st, b_sj, cols, div, C, ldc);
}

lrs_status spc_err_from_rows(lrs_ctx* ctx, const void* Bf, int32_t dtype, int64_t mc, int64_t n, int64_t ldb,
                             const double* Bc, int64_t l, int64_t ldc, double cf, const double* taus, int32_t ntau,
                             double* eps_hat) {
  return spc_err_rows(ctx, Bf, dtype, mc, n, ldb, Bc, l, ldc, cf, taus, ntau, eps_hat);
}

}  // namespace lrs

using namespace lrs;

extern "C" {

lrs_status lrs_spc_lift(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                        const double* Y, int64_t l, int64_t ldy, const double* U, int64_t ldu, const double* S,
                        const double* V, int64_t ldv, int64_t r, const int32_t* J, int32_t k, int32_t prec,
                        void* Sf, int64_t ldsf) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!A || !Y || !U || !S || !V || !J || !Sf) return lrs_fail(ctx, LRS_EINVAL, "spc_lift: NULL pointer");
  if (!spc_dtype_ok(dtype) || prec < LRS_PREC_FP64 || prec > LRS_PREC_BF16X3)
    return lrs_fail(ctx, LRS_EINVAL, "spc_lift: bad dtype/prec");
  if (m < 1 || n < 1 || l < 1 || k < 1 || r < k || r > (m < l ? m : l))
    return lrs_fail(ctx, LRS_EINVAL, "spc_lift: need 1 <= k <= r <= min(m, l) (m=%lld l=%lld r=%lld k=%d)",
                    (long long)m, (long long)l, (long long)r, k);
  if (lda < n || ldy < l || ldu < r || ldv < r || ldsf < n)
    return lrs_fail(ctx, LRS_EINVAL, "spc_lift: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // the r-th singular value must be nonzero: S_r^-1 enters the operator
  double* h = (double*)ctx->host_scratch;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 12, S + (r - 1), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (!(h[12] > 0.0)) return lrs_fail(ctx, LRS_EINVAL, "spc_lift: s_r = %g is not positive", h[12]);
  const bool tc = prec >= LRS_PREC_SPLIT_BF16;
  const size_t need = 8 * (size_t)(r * k) + 8 * (size_t)(m * k) + 4096 +
                      (tc ? gemm_tc_workspace(k, m, prec) + gemm_tc_splitk_workspace(k, n, m, ctx->num_sms) : 0);
  lrs_status st = ws_reserve(ctx, need);
  if (st) return st;
  double* Mk = (double*)ws_alloc(ctx, 8 * (size_t)(r * k));      // S_r^-1 V_r^T A_c(J,:)^T  (r x k)
  double* X = (double*)ws_alloc(ctx, 8 * (size_t)(m * k));       // U_r Mk                   (m x k)
  if (!Mk || !X) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (spc_lift)");
  // Mk(q, j) = (1 / S_q) sum_t V(t, q) Y(J_j, t)
  st = small_gemm(ctx, r, k, l, V, 1, ldv, Y, 1, ldy, J, S, Mk, k);
  if (st) return st;
  // X(i, j) = sum_q U(i, q) Mk(q, j)
  st = small_gemm(ctx, m, k, r, U, ldu, 1, Mk, k, 1, nullptr, nullptr, X, k);
  if (st) return st;
  // S_f = X^T A_f: the one full read of A_f
  GemmArgs g{k, n, m, X, LRS_F64, k, A, dtype, lda, Sf, prec == LRS_PREC_FP64 ? 1 : 0, 0, ldsf, 1.0};
  if (prec == LRS_PREC_FP64) return launch_gemm_simt(ctx, g, 1);
  if (prec == LRS_PREC_FP32) return launch_gemm_simt(ctx, g, 0);
  return launch_gemm_tc(ctx, g, prec);
}

lrs_status lrs_sketch_svd(lrs_ctx* ctx, const double* Y, int64_t m, int64_t l, int64_t ldy, double rtol, double* Q,
                          int64_t ldq, int32_t r, double* U, int64_t ldu, double* S, double* V, int64_t ldv,
                          int64_t* rank_out) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!Y || !Q || !U || !S || !V || !rank_out) return lrs_fail(ctx, LRS_EINVAL, "sketch_svd: NULL pointer");
  const int64_t mn = m < l ? m : l;
  if (m < 1 || l < 1 || r < 1 || r > kSketchSvdDirs || r > mn)
    return lrs_fail(ctx, LRS_EINVAL, "sketch_svd: need 1 <= r <= min(m, l, %lld) (r=%d)", (long long)kSketchSvdDirs, r);
  if (ldy < l || ldq < mn || ldu < r || ldv < r) return lrs_fail(ctx, LRS_EINVAL, "sketch_svd: strides too small");
  if (!(rtol >= 0.0) || rtol >= 1.0) return lrs_fail(ctx, LRS_EINVAL, "sketch_svd: rtol=%g not in [0,1)", rtol);
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int64_t pmax = mn < kSketchSvdDirs ? mn : kSketchSvdDirs;
  const size_t iter_ws = 8 * (size_t)(l * m) + 8 * (size_t)(l * pmax) + 8 * (size_t)(m * pmax) + 1024 +
                         orth_ws_of(m, pmax, ctx->num_sms);
  const size_t ow = orth_ws_of(m, l, ctx->num_sms);
  lrs_status st = ws_reserve(ctx, ow > iter_ws ? ow : iter_ws);
  if (st) return st;
  // the pivoted QR, stopped at rtol or after pmax steps (only the leading
  // directions enter the SVD)
  int64_t rank = 0;
  st = orth_basis(ctx, Y, m, l, ldy, rtol, Q, ldq, &rank, pmax);
  if (st) return st;
  *rank_out = rank;
  if (rank < r) return lrs_fail(ctx, LRS_ERANK, "sketch_svd: numerical rank %lld < r = %d", (long long)rank, r);
  const int64_t p = rank;
  if (p == pmax && pmax < mn) {
    // The sketch may have more directions than the Jacobi tile holds: refine
    // the leading p by two steps of subspace iteration, Q_p <- orth(Y Y^T Q_p),
    // which shrinks their angle to the dominant p-dimensional singular
    // subspace by (s_{p+1} / s_p)^2 per step; the SVD below is then the
    // Rayleigh-Ritz step on that subspace.
    ctx->ws_top = 0;                                    // Q is the caller's; nothing else is live
    double* Yt = (double*)ws_alloc(ctx, 8 * (size_t)(l * m));
    double* T = (double*)ws_alloc(ctx, 8 * (size_t)(l * p));
    double* Z = (double*)ws_alloc(ctx, 8 * (size_t)(m * p));
    if (!Yt || !T || !Z) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (sketch_svd)");
    st = launch_transpose(ctx, Y, m, l, ldy, Yt, m);   // Yt = Y^T (l x m, row-major)
    if (st) return st;
    const size_t mark = ctx->ws_top;
    for (int it = 0; it < 2; ++it) {
      st = small_gemm(ctx, l, p, m, Yt, m, 1, Q, ldq, 1, nullptr, nullptr, T, p);   // T = Y^T Q_p
      if (st) return st;
      st = small_gemm(ctx, m, p, l, Y, ldy, 1, T, p, 1, nullptr, nullptr, Z, p);    // Z = Y T
      if (st) return st;
      int64_t rz = 0;
      ctx->ws_top = mark;
      st = orth_basis(ctx, Z, m, p, p, 0.0, Q, ldq, &rz, p);
      if (st) return st;
      if (rz != p) return lrs_fail(ctx, LRS_ERANK, "sketch_svd: subspace iteration lost rank (%lld of %lld)",
                                   (long long)rz, (long long)p);
    }
  }
  st = lrs_svd_k(ctx, Y, LRS_F64, m, l, ldy, Q, ldq, p, r, LRS_PREC_FP64, U, ldu, S, V, ldv, nullptr);
  return st == LRS_ERANK ? LRS_OK : st;
}

lrs_status lrs_spc_err(lrs_ctx* ctx, const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda,
                       const double* Y, int64_t l, int64_t ldy, int32_t c, const double* taus, int32_t ntau,
                       double* eps_hat) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!A || !Y || !taus || !eps_hat) return lrs_fail(ctx, LRS_EINVAL, "spc_err: NULL pointer");
  if (!spc_dtype_ok(dtype)) return lrs_fail(ctx, LRS_EINVAL, "spc_err: bad dtype");
  if (m < 1 || n < 1 || l < 1 || c < 1) return lrs_fail(ctx, LRS_EINVAL, "spc_err: bad sizes");
  if (lda < n || ldy < l) return lrs_fail(ctx, LRS_EINVAL, "spc_err: strides too small");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // B_f = A_f(J,:), J = c-1, 2c-1, ...: rows at stride c * lda from row c - 1
  const size_t esz = dtype == LRS_F64 ? 8 : (dtype == LRS_F32 ? 4 : 2);
  const char* Bf = (const char*)A + (size_t)(c - 1) * (size_t)lda * esz;
  return spc_err_rows(ctx, Bf, dtype, m / c, n, (int64_t)c * lda, Y + (size_t)(c - 1) * (size_t)ldy, l,
                      (int64_t)c * ldy, (double)c, taus, ntau, eps_hat);
}

}  // extern "C"
