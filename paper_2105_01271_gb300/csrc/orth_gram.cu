// Orthonormal basis of a TALL-SKINNY p x c matrix M (p >= 4c, c <= 128) with
// the rank-revealing truncation of the paper's QR(.) (Algs. 2/3/7), without a
// p-row Householder sweep per pivot:
//
//   1. G = M^T M in FP64 (split over row blocks, fixed-order sum).
//   2. Pivoted Cholesky of G: G(piv, piv) = R^T R.  Column pivoting of M by
//      largest remaining 2-norm depends on M only through G (the remaining
//      norm^2 of a column is the diagonal of the Schur complement), so the
//      pivots, the stop step r (|R_jj| <= rtol |R_00|) and |R_jj| are those of
//      Householder CPQR in exact arithmetic; ties go to the lowest current
//      position with the same swap rule as cpqr.cu.
//   3. Q_1 = M(:, piv[0:r]) R_11^{-1}   (row-wise triangular solve).
//   4. One refinement (Cholesky-QR2): G_2 = Q_1^T Q_1 = R_2^T R_2,
//      Q = Q_1 R_2^{-1}.  Q spans M(:, piv[0:r]); its R factor
//      (R_2 R_11) has a positive diagonal.
//   Q_1 alone spans the same range with |Q_1^T Q_1 - I| ~ u cond(M_r)^2
//   (<= ~1e-4 at rtol = 1e-6): callers whose basis only feeds a product that
//   is orthonormalised again skip step 4 (refine = false).
//
// Forming G squares the condition number, so this route is only taken when
// rtol^2 stays far above the FP64 rounding of G (rtol >= 1e-6); otherwise the
// Householder CPQR in cpqr.cu runs.
#include "common.cuh"
#include "internal.h"

namespace lrs {

namespace {

constexpr int kGramRows = 32;           // rows of M staged per pass
constexpr int kMaxC = 128;

// packed upper-triangle index e -> (i, j), row i holding entries (i, i..c-1)
__device__ __forceinline__ void tri_ij(int e, int c, int& i, int& j) {
  int ii = 0, base = 0;
  while (base + (c - ii) <= e) { base += c - ii; ++ii; }
  i = ii;
  j = ii + (e - base);
}

// This block's rows' contribution to the upper triangle of M^T M.  Entries
// are dealt round-robin to the 256 threads (KPER per thread, fully unrolled,
// so every lane of every warp keeps the FP64 pipes busy); packed layout
// part[blockIdx.x * ntri + e].
template <int KPER>
__global__ void __launch_bounds__(256) k_gram_partial(const double* __restrict__ M, int64_t p, int c,
                                                      int64_t ldm, int64_t rows_b, double* __restrict__ part) {
  extern __shared__ double tile[];                 // kGramRows x c
  const int ntri = c * (c + 1) / 2;
  const int64_t r0 = (int64_t)blockIdx.x * rows_b;
  const int64_t r1 = min(p, r0 + rows_b);
  double acc[KPER];
  int ii[KPER], jj[KPER];
#pragma unroll
  for (int q = 0; q < KPER; ++q) {
    const int e = threadIdx.x + q * 256;
    acc[q] = 0.0;
    if (e < ntri) tri_ij(e, c, ii[q], jj[q]);
    else { ii[q] = 0; jj[q] = 0; }
  }
  for (int64_t a0 = r0; a0 < r1; a0 += kGramRows) {
    const int nr = (int)min((int64_t)kGramRows, r1 - a0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * c; e += blockDim.x) {
      const int rr = e / c, cc = e - rr * c;
      tile[rr * c + cc] = M[(a0 + rr) * ldm + cc];
    }
    __syncthreads();
    for (int rr = 0; rr < nr; ++rr) {
      const double* row = tile + rr * c;
#pragma unroll
      for (int q = 0; q < KPER; ++q) acc[q] = fma(row[ii[q]], row[jj[q]], acc[q]);
    }
  }
  double* out = part + (int64_t)blockIdx.x * ntri;
#pragma unroll
  for (int q = 0; q < KPER; ++q) {
    const int e = threadIdx.x + q * 256;
    if (e < ntri) out[e] = acc[q];
  }
}

// G (c x c, full symmetric, row-major) = sum over the nb block partials: a
// warp per packed entry, lanes over blocks (four loads in flight each), then a
// fixed shuffle tree -- the same order in every run.
__global__ void k_gram_reduce(const double* __restrict__ part, int nb, int c, double* __restrict__ G) {
  const int ntri = c * (c + 1) / 2;
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwt = (gridDim.x * blockDim.x) >> 5;
  for (int e = w0; e < ntri; e += nwt) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nb; b += 128) {
      a0 += part[(int64_t)b * ntri + e];
      a1 += part[(int64_t)(b + 32) * ntri + e];
      a2 += part[(int64_t)(b + 64) * ntri + e];
      a3 += part[(int64_t)(b + 96) * ntri + e];
    }
    for (; b < nb; b += 32) a0 += part[(int64_t)b * ntri + e];
    const double sum = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) {
      int i, j;
      tri_ij(e, c, i, j);
      G[i * c + j] = sum;
      G[j * c + i] = sum;
    }
  }
}

__device__ __forceinline__ bool better(double a, int pa, double b, int pb) { return pivot_better(a, pa, b, pb); }

// Pivoted (pivot = 1) or plain Cholesky of the c x c PSD G, one block, in
// POSITION order: the pivot moves to position j by the symmetric swap of
// positions j and piv (the transposition cpqr.cu applies), so the remaining
// block is always [j+1, c)^2 and row j of the working matrix becomes row j of
// R (rows < j hold R, and their columns j and piv are swapped with the rest).
// Only the upper triangle is stored and updated (sym(a, b) = G[min][max]).
// Per step, two block barriers:
//   swap and scale row j (each thread owns one index a and the two cells of a)
//   | Schur update of the remaining upper triangle: warp 0 takes the diagonal
//     and, from the values it just wrote, the next pivot (the largest remaining
//     diagonal, lowest position on ties), its inverse square root and the stop
//     test; warps 1.. take the entries above the diagonal, rows k and n-2-k of
//     the n remaining paired into one run of n entries so every run is as long.
// Outputs: perm[pos] = physical column, R (rows 0..rank-1, row-major ldr,
// pivoted order, zero below the diagonal), *rank.
__global__ void __launch_bounds__(256) k_pchol(const double* __restrict__ Gin, int c, int kmax, double rtol,
                                               int pivot, int32_t* __restrict__ perm, double* __restrict__ R,
                                               int64_t ldr, int32_t* __restrict__ rank) {
  extern __shared__ double sm[];
  const int ld = c + 1;
  double* G = sm;                                   // c x ld, upper triangle by position
  int* phys_at = reinterpret_cast<int*>(G + c * ld);
  __shared__ int s_piv, s_stop;
  __shared__ double s_ljj, s_inv, s_top;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a = wid; a < c; a += nw)
    for (int b2 = lane; b2 < c; b2 += 32) G[a * ld + b2] = Gin[a * c + b2];
  for (int q = threadIdx.x; q < c; q += blockDim.x) phys_at[q] = q;
  __syncthreads();

  // the pivot of step jn from the remaining diagonal, one warp; the lane
  // holding position q has its (just written) value in dval when mine(q)
  auto decide = [&](int jn, double bv, int bp) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (better(ov, op, bv, bp)) { bv = ov; bp = op; }
    }
    if (lane == 0) {
      if (!pivot) { bp = jn; bv = jn < c ? G[jn * ld + jn] : -1.0; }
      // R_jj = sqrt(d), 1 / R_jj = rsqrt(d); the stop test |R_jj| <= rtol |R_00|
      // is taken on the squares, d <= rtol^2 d_0
      const double y = bv > 0.0 ? rsqrt_fast(bv) : 0.0;
      if (jn == 0) s_top = bv;
      const bool stop = (jn >= kmax) || jn >= c || !(bv > 0.0) || (jn > 0 && bv <= rtol * rtol * s_top);
      s_stop = stop ? 1 : 0;
      if (!stop) {
        if (bp != jn) { const int t = phys_at[jn]; phys_at[jn] = phys_at[bp]; phys_at[bp] = t; }
        s_piv = bp; s_ljj = bv * y; s_inv = y;
      }
    }
  };
  if (wid == 0) {
    double bv = -1.0;
    int bp = 0x7fffffff;
    if (pivot)
      for (int q = lane; q < c; q += 32) {
        const double d = G[q * ld + q];
        if (norm_key(d) > norm_key(bv)) { bv = d; bp = q; }
      }
    decide(0, bv, bp);
  }
  __syncthreads();
  int j = 0;
  for (;; ++j) {
    if (s_stop) break;
    const int pv = s_piv;
    const double inv = s_inv;
    // ---- swap positions j and pv, scale row j beyond the diagonal -------------
    // thread a exchanges sym(a, j) and sym(a, pv); for a > j the new sym(j, a)
    // is row j of R and is stored scaled.
    for (int a = threadIdx.x; a < c; a += blockDim.x) {
      if (a == j) {
        if (pv != j) G[pv * ld + pv] = G[j * ld + j];
        G[j * ld + j] = s_ljj;
      } else if (a == pv) {
        G[j * ld + pv] *= inv;                      // sym(j, pv) is unchanged by the swap
      } else if (a < j) {
        if (pv != j) {                              // finished rows: swap columns j and pv
          const double t = G[a * ld + j];
          G[a * ld + j] = G[a * ld + pv];
          G[a * ld + pv] = t;
        }
      } else {
        // a > j, a != pv: new sym(j, a) = old sym(pv, a); new sym(pv, a) = old sym(j, a)
        if (pv != j) {
          double* cpa = (a < pv) ? &G[a * ld + pv] : &G[pv * ld + a];
          const double old_j = G[j * ld + a], old_p = *cpa;
          G[j * ld + a] = old_p * inv;
          *cpa = old_j;
        } else {
          G[j * ld + a] *= inv;
        }
      }
    }
    __syncthreads();
    // ---- Schur complement, upper triangle: S_ab -= R_ja R_jb (j < a <= b) -----
    const int n = c - j - 1;
    if (wid == 0) {
      // the diagonal, then the next pivot from it
      double bv = -1.0;
      int bp = 0x7fffffff;
      for (int a = j + 1 + lane; a < c; a += 32) {
        const double rja = G[j * ld + a];
        const double d = fma(-rja, rja, G[a * ld + a]);
        G[a * ld + a] = d;
        if (pivot && norm_key(d) > norm_key(bv)) { bv = d; bp = a; }
      }
      __syncwarp();
      decide(j + 1, bv, bp);
    } else if (n > 1) {
      // above the diagonal: row k (a = j+1+k) has n-1-k entries; rows k and
      // n-2-k together have n, k < n-1-k (the middle row alone when n is even)
      const int runs = n / 2;                       // pairs, plus the middle row when n is even
      for (int v = wid - 1; v < runs; v += nw - 1) {
        const int k2 = n - 2 - v;
        const int len0 = n - 1 - v;                 // entries of row v
        const int len = (k2 == v) ? len0 : n;       // the middle row is alone
        const int a0 = j + 1 + v, a1 = j + 1 + k2;
        const double r0 = G[j * ld + a0], r1 = G[j * ld + a1];
        for (int e = lane; e < len; e += 32) {
          int a, b2;
          double ra;
          if (e < len0) { a = a0; b2 = a0 + 1 + e; ra = r0; }
          else { a = a1; b2 = a1 + 1 + (e - len0); ra = r1; }
          G[a * ld + b2] = fma(-ra, G[j * ld + b2], G[a * ld + b2]);
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *rank = j;
  for (int q = threadIdx.x; q < c; q += blockDim.x) perm[q] = phys_at[q];
  for (int a = wid; a < j; a += nw)
    for (int b2 = lane; b2 < c; b2 += 32) R[(int64_t)a * ldr + b2] = (b2 < a) ? 0.0 : G[a * ld + b2];
}

// Q (p x r, row-major ldq) = M(:, perm[0:r]) R^{-1}, R upper triangular
// (r x r leading block of the ldr-strided R).  A team of T threads (T = 1..32,
// a power of two) solves one row q R = m right-looking: lane t mod T owns
// unknowns t; at step j the owner of j finishes q_j = m_j / R_jj and hands it
// to the team with one shuffle, and every lane subtracts q_j R_jt from its own
// unknowns t > j.  No FP64 reduction across lanes, so p * T threads keep every
// SM's FP64 units on useful work even when p is small.  The block's rows live
// in shared memory during the substitution.  perm may be NULL.
__global__ void __launch_bounds__(256) k_trsm_rows(const double* __restrict__ M, int64_t p, int64_t ldm,
                                                   const int32_t* __restrict__ perm,
                                                   const double* __restrict__ R, int64_t ldr, int r, int T,
                                                   double* __restrict__ Q, int64_t ldq) {
  extern __shared__ double sm[];
  double* Rs = sm;                                  // r x r
  double* dinv = Rs + r * r;                        // r: 1 / R_jj
  double* qs = dinv + r;                            // rows x (r + 1)
  const int rows = blockDim.x / T;
  const int ld = r + 1;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Rs[e] = R[(int64_t)(e / r) * ldr + (e % r)];
  for (int j = threadIdx.x; j < r; j += blockDim.x) dinv[j] = 1.0 / R[(int64_t)j * ldr + j];
  const int64_t i0 = (int64_t)blockIdx.x * rows;
  for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
    const int rr = e / r, t = e - rr * r;
    const int64_t i = i0 + rr;
    const int col = perm ? perm[t] : t;
    qs[rr * ld + t] = (i < p) ? M[i * ldm + col] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tm = threadIdx.x & (T - 1);
  const unsigned tmask = (T == 32 ? 0xffffffffu : ((1u << T) - 1u)) << (lane & ~(T - 1));
  const int base = lane & ~(T - 1);
  double* q = qs + (threadIdx.x / T) * ld;
  for (int jx = 0; jx < r; ++jx) {
    const int owner = jx & (T - 1);
    double qj = 0.0;
    if (tm == owner) { qj = q[jx] * dinv[jx]; q[jx] = qj; }
    qj = __shfl_sync(tmask, qj, base + owner);
    const double* Rrow = Rs + jx * r;
    // unknowns t > jx owned by this lane: t = tm, tm + T, ...
    int t = tm + ((jx + 1 - tm + T - 1) / T) * T;
    if (jx + 1 <= tm) t = tm;
    for (; t < r; t += T) q[t] = fma(-qj, Rrow[t], q[t]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * r; e += blockDim.x) {
    const int rr = e / r, t = e - rr * r;
    const int64_t i = i0 + rr;
    if (i < p) Q[i * ldq + t] = qs[rr * ld + t];
  }
}

// the partial-Gram kernel with KPER the smallest listed count >= per: every
// unrolled slot is an issued FP64 FMA, so slots past the last entry are pure
// waste on the narrow FP64 pipe (per = 11 at c = 72, 13 at c = 79; the
// counts whose unrolled form spills are left out)
template <int K, int... Ks>
void gram_partial_dispatch(int per, unsigned nb, size_t dyn, cudaStream_t s, const double* M, int64_t p, int c,
                           int64_t ldm, int64_t rows_b, double* part) {
  if constexpr (sizeof...(Ks) == 0) {
    k_gram_partial<K><<<nb, 256, dyn, s>>>(M, p, c, ldm, rows_b, part);
  } else {
    if (per <= K) k_gram_partial<K><<<nb, 256, dyn, s>>>(M, p, c, ldm, rows_b, part);
    else gram_partial_dispatch<Ks...>(per, nb, dyn, s, M, p, c, ldm, rows_b, part);
  }
}

lrs_status gram(lrs_ctx* ctx, const double* M, int64_t p, int c, int64_t ldm, double* G) {
  if (c < 1 || c > kMaxC) return lrs_fail(ctx, LRS_EINVAL, "gram: %d columns (1..%d)", c, kMaxC);
  // one block per SM with an equal share of the rows (at least 8): a few
  // thousand rows still spread over every SM's FP64 units
  int64_t nb = ctx->num_sms;
  int64_t rows_b = (p + nb - 1) / nb;
  if (rows_b < 8) rows_b = 8;
  nb = (p + rows_b - 1) / rows_b;
  const int ntri = c * (c + 1) / 2;
  double* part = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(nb * ntri));
  if (!part) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (gram)");
  const size_t dyn = sizeof(double) * (size_t)(kGramRows * c);
  const int per = (ntri + 255) / 256;
  gram_partial_dispatch<2, 6, 8, 10, 11, 13, 14, 16, 20, 24, 28, 33>(per, (unsigned)nb, dyn, ctx->stream, M,
                                                                          p, c, ldm, rows_b, part);
  ctx->launches++;
  k_gram_reduce<<<(ntri + 7) / 8, 256, 0, ctx->stream>>>(part, (int)nb, c, G);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

size_t pchol_smem(int c) { return sizeof(double) * (size_t)(c * (c + 1)) + sizeof(int) * (size_t)c; }

lrs_status pchol(lrs_ctx* ctx, const double* G, int c, int kmax, double rtol, int pivot, int32_t* perm,
                 double* R, int64_t ldr, int32_t* rank) {
  const size_t dyn = pchol_smem(c);
  if (dyn > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_pchol, (size_t)(dyn)); if (_s) return _s; }
  k_pchol<<<1, 256, dyn, ctx->stream>>>(G, c, kmax, rtol, pivot, perm, R, ldr, rank);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status trsm_rows(lrs_ctx* ctx, const double* M, int64_t p, int64_t ldm, const int32_t* perm, const double* R,
                     int64_t ldr, int r, double* Q, int64_t ldq) {
  // team size: enough threads (p * T) for ~8 FP64-busy warps per SM
  const int64_t want = (int64_t)ctx->num_sms * 8 * 32;
  int T = 1;
  while (T < 32 && p * T < want) T <<= 1;
  // the block's rows (256 / T of them) and R must fit in shared memory: for a
  // wide R, teams grow (fewer rows per block) until they do
  auto dyn_of = [&](int t) { return sizeof(double) * (size_t)(r * r + r + (256 / t) * (r + 1)); };
  while (T < 32 && dyn_of(T) > 200 * 1024) T <<= 1;
  const int rows = 256 / T;
  const size_t dyn = dyn_of(T);
  if (dyn > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_trsm_rows, (size_t)(dyn)); if (_s) return _s; }
  const unsigned nb = (unsigned)((p + rows - 1) / rows);
  k_trsm_rows<<<nb, 256, dyn, ctx->stream>>>(M, p, ldm, perm, R, ldr, r, T, Q, ldq);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// R factors in the original column order, for callers that chain them:
// Rt (r x c, row-major) with M ~= Q Rt.
// From a pivoted factor R (rows 0..r-1, pivoted column order, row stride
// ldr) and perm[pos] = original column: Rt(t, perm[j]) = R(t, j) (j >= t).
__global__ void k_rt_scatter(const double* __restrict__ R, int64_t ldr, const int32_t* __restrict__ perm, int64_t r,
                             int64_t c, double* __restrict__ Rt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * c) return;
  const int64_t t = e / c, j = e - t * c;
  Rt[t * c + perm[j]] = j >= t ? R[t * ldr + j] : 0.0;
}
// From the left-looking factor L (by original column, L[i * kmax + t]):
// Rt(t, i) = L(i, t).
__global__ void k_rt_from_l(const double* __restrict__ L, int64_t kmax, int64_t r, int64_t c, double* __restrict__ Rt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * c) return;
  const int64_t t = e / c, i = e - t * c;
  Rt[t * c + i] = L[i * kmax + t];
}
// out = U X for U (r x r upper triangular, row stride r) and X (r x c):
// out(t, i) = sum_{s >= t} U(t, s) X(s, i), FP64, fixed order
__global__ void k_trmm_upper(const double* __restrict__ U, int64_t r, const double* __restrict__ X, int64_t c,
                             double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * c) return;
  const int64_t t = e / c, i = e - t * c;
  double acc = 0.0;
  for (int64_t s = t; s < r; ++s) acc = fma(U[t * r + s], X[s * c + i], acc);
  out[t * c + i] = acc;
}

lrs_status launch_rt_scatter(lrs_ctx* ctx, const double* R, int64_t ldr, const int32_t* perm, int64_t r, int64_t c,
                             double* Rt) {
  if (r < 1 || c < 1) return LRS_OK;
  k_rt_scatter<<<(unsigned)((r * c + 255) / 256), 256, 0, ctx->stream>>>(R, ldr, perm, r, c, Rt);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

static lrs_status launch_trmm_upper(lrs_ctx* ctx, const double* U, int64_t r, const double* X, int64_t c,
                                    double* out) {
  k_trmm_upper<<<(unsigned)((r * c + 255) / 256), 256, 0, ctx->stream>>>(U, r, X, c, out);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_pchol(lrs_ctx* ctx, const double* G, int c, int kmax, double rtol, int pivot, int32_t* perm,
                        double* R, int64_t ldr, int32_t* rank) {
  return pchol(ctx, G, c, kmax, rtol, pivot, perm, R, ldr, rank);
}

lrs_status launch_gram(lrs_ctx* ctx, const double* M, int64_t p, int c, int64_t ldm, double* G) {
  return gram(ctx, M, p, c, ldm, G);
}

lrs_status launch_trsm_rows(lrs_ctx* ctx, const double* M, int64_t p, int64_t ldm, const int32_t* perm,
                            const double* R, int64_t ldr, int r, double* Q, int64_t ldq) {
  return trsm_rows(ctx, M, p, ldm, perm, R, ldr, r, Q, ldq);
}

bool orth_gram_eligible(int64_t p, int64_t c, double rtol) {
  return c >= 1 && c <= kMaxC && p >= 4 * c && rtol >= kOrthGramRtolMin;
}

size_t orth_gram_ws(int64_t p, int64_t c, int num_sms) {
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t b = 0;
  b += a256(sizeof(double) * (size_t)num_sms * (size_t)(c * (c + 1) / 2));   // Gram partials (one pass at a time)
  b += 2 * a256(sizeof(double) * (size_t)(c * c));       // G, R
  b += a256(4 * (size_t)c) + a256(8);                    // perm, rank
  b += a256(sizeof(double) * (size_t)(p * c));           // Q_1
  b += a256(sizeof(double) * (size_t)(c * c));           // the first factor (original column order)
  return b + 1024;
}

lrs_status launch_orth_gram(lrs_ctx* ctx, const double* M, int64_t p, int64_t c, int64_t ldm, double rtol,
                            double* Q, int64_t ldq, int64_t* r_out, bool refine, double* rdiag, double* Rt) {
  const int ci = (int)c;
  double* G = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(c * c));
  double* R = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(c * c));
  int32_t* perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)c);
  int32_t* rank = (int32_t*)ws_alloc(ctx, 8);
  double* Q1 = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(p * c));
  // the first factor in original column order when it is refined afterwards
  double* R1t = (Rt && refine) ? (double*)ws_alloc(ctx, sizeof(double) * (size_t)(c * c)) : Rt;
  if (!G || !R || !perm || !rank || !Q1 || (Rt && !R1t))
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (orth_gram)");
  const size_t mark = ctx->ws_top;
  lrs_status st = gram(ctx, M, p, ci, ldm, G);
  if (st) return st;
  ctx->ws_top = mark;
  st = pchol(ctx, G, ci, ci, rtol, 1, perm, R, c, rank);
  if (st) return st;
  int32_t* h = (int32_t*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {rank};
    st = replay_ints(ctx, 1, d, h + 40);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 40, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  const int r = h[40];
  *r_out = r;
  if (r == 0) return LRS_OK;
  if (rdiag) {
    st = launch_abs_diag(ctx, R, c, r, rdiag);
    if (st) return st;
  }
  // M(:, perm) = Q_1 R: the factor in original column order, before the
  // refinement reuses R and perm (then Rt <- R_2 Rt)
  if (Rt) {
    st = launch_rt_scatter(ctx, R, c, perm, r, c, R1t);
    if (st) return st;
  }
  if (!refine) return trsm_rows(ctx, M, p, ldm, perm, R, c, r, Q, ldq);
  st = trsm_rows(ctx, M, p, ldm, perm, R, c, r, Q1, r);
  if (st) return st;
  // refinement: G_2 = Q_1^T Q_1 = R_2^T R_2 (plain Cholesky), Q = Q_1 R_2^{-1}
  st = gram(ctx, Q1, p, r, r, G);
  if (st) return st;
  ctx->ws_top = mark;
  st = pchol(ctx, G, r, r, 0.0, 0, perm, R, r, rank);
  if (st) return st;
  if (ctx->replay) {
    const int32_t* d[1] = {rank};
    st = replay_ints(ctx, 1, d, h + 41);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 41, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  // Q_1 has full column rank r by construction; a breakdown here means the
  // first pass lost it to rounding: the caller falls back to Householder CPQR
  if (h[41] != r) return LRS_ERANK;
  if (Rt) {
    st = launch_trmm_upper(ctx, R, r, R1t, c, Rt);
    if (st) return st;
  }
  return trsm_rows(ctx, Q1, p, r, nullptr, R, r, r, Q, ldq);
}

}  // namespace lrs

namespace lrs {

size_t r_of_bt_gram_ws(int64_t r, int num_sms) {
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  return gram_oz_ws(r, num_sms) + a256(sizeof(double) * (size_t)(r * r)) + a256(4 * (size_t)r) + a256(8) + 512;
}

lrs_status launch_r_of_bt_gram(lrs_ctx* ctx, const float* B, int64_t r, int64_t n, int64_t ldb, double* R,
                               int32_t* perm_out) {
  if (r < 1 || r > kMaxC) return lrs_fail(ctx, LRS_EINVAL, "svd: r=%lld out of range for the Gram route", (long long)r);
  const int ri = (int)r;
  double* G = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(r * r));
  int32_t* perm = perm_out ? perm_out : (int32_t*)ws_alloc(ctx, 4 * (size_t)r);
  int32_t* rank = (int32_t*)ws_alloc(ctx, 8);
  if (!G || !perm || !rank) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (svd gram)");
  lrs_status gs = launch_gram_oz(ctx, B, r, n, ldb, G);
  if (gs) return gs;
  // pivoted when the caller takes the permutation (P^T B B^T P = R^T R)
  lrs_status st = pchol(ctx, G, ri, ri, 0.0, perm_out ? 1 : 0, perm, R, r, rank);
  if (st) return st;
  int32_t* h = (int32_t*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {rank};
    st = replay_ints(ctx, 1, d, h + 42);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 42, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return h[42] == ri ? LRS_OK : LRS_ERANK;
}

}  // namespace lrs

namespace lrs {

// ---------------------------------------------------------------------------
// WIDE (or square) M, c > 128 columns: left-looking pivoted Cholesky of
// G = M^T M without forming G.  Step j needs only the pivot's column of the
// Schur complement,
//     S(:, piv) = M^T m_piv - L(:, 0:j) L(piv, 0:j)^T,
// one FP64 matrix-vector product over the ORIGINAL columns (p c FMAs, against
// 3 (p-j)(c-j) for a Householder step), then L(:, j) = S(:, piv) / sqrt(d_piv)
// and the remaining norms^2 are down-dated, d_i -= L(i, j)^2.  The pivot and
// tie rules and the stop test are those of k_pchol (and so of cpqr.cu).
//
// One persistent cooperative launch.  Block b owns a contiguous range of
// physical columns (all p rows, in shared memory) and their d_i; L lives in
// global memory by physical column, L[i * kmax + t].  One grid barrier per
// step: each block publishes its best remaining candidate (double-buffered by
// step parity, so a block still reading step j's candidates never sees step
// j+1's), and every block reduces the candidates itself in block order, so
// all blocks take the same decision and apply the same position swap to their
// own copy of the permutation.
// ---------------------------------------------------------------------------
namespace {

constexpr int kLpThreads = 512;
constexpr int kLpMaxCpb = 16;           // owned columns per block

struct LpcholState {
  const double* Mc; int64_t p, c, ldm;  // column-major copy of M (column i at Mc + i * ldm)
  int64_t kmax; double rtol;
  int64_t cpb;                          // columns owned per block
  double* L;                            // c x kmax, by physical column
  int32_t* perm; double* R; int64_t ldr; int32_t* rank;
  PivotCand* cand;                      // 2 x nb
  GridBarrier bar;
};

__global__ void __launch_bounds__(kLpThreads, 1) k_lpchol(LpcholState s) {
  extern __shared__ double lsm[];
  const int nb = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t o_lo = min(s.c, (int64_t)b * s.cpb), o_hi = min(s.c, o_lo + s.cpb);
  const int nown = (int)(o_hi - o_lo);
  const int64_t p = s.p;
  double* slab = lsm;                               // nown x p: owned columns
  double* xpiv = slab + s.cpb * p;                  // p: the pivot column
  double* lpiv = xpiv + p;                          // kmax: L(piv, 0:j)
  double* d = lpiv + s.kmax;                        // nown: remaining norms^2
  double* lown = d + kLpMaxCpb;                     // cpb x kmax: L rows of the owned columns
  int32_t* pos_of = reinterpret_cast<int32_t*>(lown + s.cpb * s.kmax);
  int32_t* phys_at = pos_of + s.c;
  __shared__ double sv[32];
  __shared__ int sp[32], sf[32];
  __shared__ int s_piv, s_stop;
  __shared__ double s_ljj, s_inv, s_top;
  __shared__ unsigned char s_done[kLpMaxCpb];

  for (int64_t e = threadIdx.x; e < (int64_t)nown * p; e += blockDim.x) {
    const int64_t cc = e / p, i = e - cc * p;
    slab[cc * p + i] = s.Mc[(o_lo + cc) * s.ldm + i];
  }
  for (int64_t q = threadIdx.x; q < s.c; q += blockDim.x) { pos_of[q] = (int)q; phys_at[q] = (int)q; }
  if (threadIdx.x < kLpMaxCpb) s_done[threadIdx.x] = 0;
  __syncthreads();
  // d_i = ||m_i||^2, a warp per owned column (fixed order)
  for (int cc = wid; cc < nown; cc += nw) {
    double a = 0.0;
    for (int64_t i = lane; i < p; i += 32) a = fma(slab[cc * p + i], slab[cc * p + i], a);
    a = warp_sum(a);
    if (lane == 0) d[cc] = a;
  }
  __syncthreads();

  // publish this block's best remaining candidate into buffer `buf`
  auto publish = [&](int buf) {
    double bv = -1.0; int bp = 0x7fffffff, bf = -1;
    if (threadIdx.x < 32) {
      for (int cc = lane; cc < nown; cc += 32) {
        if (s_done[cc]) continue;
        const int ph = (int)(o_lo + cc);
        if (pivot_better(d[cc], pos_of[ph], bv, bp)) { bv = d[cc]; bp = pos_of[ph]; bf = ph; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        const int of = __shfl_xor_sync(0xffffffffu, bf, o);
        if (pivot_better(ov, op, bv, bp)) { bv = ov; bp = op; bf = of; }
      }
      if (lane == 0) cand_store(s.cand + buf * nb + b, bv, bp, bf);
    }
  };
  // every block: the winner of buffer `buf` (block order, same result everywhere)
  auto decide = [&](int buf, int64_t j) {
    double bv = -1.0; int bp = 0x7fffffff, bf = -1;
    for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) {
      double v; int pp, pf;
      cand_load(s.cand + buf * nb + bb, v, pp, pf);
      if (pivot_better(v, pp, bv, bp)) { bv = v; bp = pp; bf = pf; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int op = __shfl_xor_sync(0xffffffffu, bp, o);
      const int of = __shfl_xor_sync(0xffffffffu, bf, o);
      if (pivot_better(ov, op, bv, bp)) { bv = ov; bp = op; bf = of; }
    }
    if (lane == 0) { sv[wid] = bv; sp[wid] = bp; sf[wid] = bf; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nw; ++w)
        if (pivot_better(sv[w], sp[w], bv, bp)) { bv = sv[w]; bp = sp[w]; bf = sf[w]; }
      if (j == 0) s_top = bv;
      const bool stop = (j >= s.kmax) || bf < 0 || !(bv > 0.0) || (j > 0 && bv <= s.rtol * s.rtol * s_top);
      s_stop = stop ? 1 : 0;
      if (!stop) {
        // move the pivot to position j (the transposition of cpqr.cu)
        const int pj = phys_at[j];
        phys_at[j] = bf; phys_at[bp] = pj;
        pos_of[bf] = (int)j; pos_of[pj] = bp;
        // L(piv, j) = sqrt(d_piv) and its reciprocal, once per step
        const double y = rsqrt_fast(bv);
        s_piv = bf; s_ljj = bv * y; s_inv = y;
        if (bf >= o_lo && bf < o_hi) s_done[bf - o_lo] = 1;
      }
    }
    __syncthreads();
  };

  publish(0);
  if (!grid_sync(s.bar)) return;
  int64_t j = 0;
  for (;; ++j) {
    decide((int)(j & 1), j);
    if (s_stop) break;
    const int piv = s_piv;
    const double ljj = s_ljj, inv = s_inv;
    // the pivot column and L(piv, 0:j)
    for (int64_t i = threadIdx.x; i < p; i += blockDim.x) xpiv[i] = __ldcg(s.Mc + (int64_t)piv * s.ldm + i);
    for (int64_t t = threadIdx.x; t < j; t += blockDim.x) lpiv[t] = __ldcg(s.L + (int64_t)piv * s.kmax + t);
    __syncthreads();
    // a warp per owned column: m_i . m_piv - L(i, 0:j) L(piv, 0:j), fixed
    // order (four interleaved partial sums per lane, then the shuffle tree)
    for (int cc = wid; cc < nown; cc += nw) {
      const int64_t ph = o_lo + cc;
      const bool live = !s_done[cc];
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, corr = 0.0;
      if (live) {
        const double* col = slab + (int64_t)cc * p;
        int64_t i = lane;
        for (; i + 96 < p; i += 128) {
          a0 = fma(xpiv[i], col[i], a0);
          a1 = fma(xpiv[i + 32], col[i + 32], a1);
          a2 = fma(xpiv[i + 64], col[i + 64], a2);
          a3 = fma(xpiv[i + 96], col[i + 96], a3);
        }
        for (; i < p; i += 32) a0 = fma(xpiv[i], col[i], a0);
        for (int64_t t = lane; t < j; t += 32) corr = fma(lown[cc * s.kmax + t], lpiv[t], corr);
      }
      const double g = warp_sum((a0 + a1) + (a2 + a3));
      corr = warp_sum(corr);
      if (lane == 0) {
        double lij;
        if (ph == piv) lij = ljj;
        else if (!live) lij = 0.0;
        else {
          lij = (g - corr) * inv;
          d[cc] = fma(-lij, lij, d[cc]);
        }
        s.L[ph * s.kmax + j] = lij;
        lown[cc * s.kmax + j] = lij;
      }
    }
    __syncthreads();
    publish((int)((j + 1) & 1));
    if (!grid_sync(s.bar)) return;
  }

  // epilogue: rank, permutation, the leading r x r block of R (pivoted order)
  const int64_t r = j;
  if (b == 0) {
    if (threadIdx.x == 0) *s.rank = (int32_t)r;
    for (int64_t q = threadIdx.x; q < s.c; q += blockDim.x) s.perm[q] = phys_at[q];
  }
  for (int64_t e = (int64_t)b * blockDim.x + threadIdx.x; e < r * r; e += (int64_t)nb * blockDim.x) {
    const int64_t i = e / r, q = e - i * r;
    s.R[i * s.ldr + q] = (q < i) ? 0.0 : __ldcg(s.L + (int64_t)phys_at[q] * s.kmax + i);
  }
}

struct LpGeom { int64_t nb, cpb; size_t smem; };

LpGeom lp_geom(int64_t p, int64_t c, int64_t kmax, int num_sms) {
  LpGeom g{};
  g.cpb = (c + num_sms - 1) / num_sms;
  if (g.cpb < 1) g.cpb = 1;
  g.nb = (c + g.cpb - 1) / g.cpb;
  g.smem = sizeof(double) * (size_t)(g.cpb * p + p + kmax + kLpMaxCpb + g.cpb * kmax) +
           sizeof(int32_t) * (size_t)(2 * c);
  return g;
}

constexpr int64_t kLpMaxRank = 128;     // the refinement's Gram kernels take up to 128 columns

}  // namespace

bool orth_wide_eligible(int64_t p, int64_t c, double rtol, int num_sms) {
  if (c <= kMaxC || p < 1 || !(rtol >= kOrthGramRtolMin)) return false;
  const int64_t kmax = min(min(p, c), kLpMaxRank + 1);
  const LpGeom g = lp_geom(p, c, kmax, num_sms);
  return g.cpb <= kLpMaxCpb && g.smem <= 200 * 1024;
}

size_t orth_wide_ws(int64_t p, int64_t c, int num_sms) {
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const int64_t kmax = min(min(p, c), kLpMaxRank + 1);
  const LpGeom g = lp_geom(p, c, kmax, num_sms);
  size_t b = 0;
  b += a256(sizeof(double) * (size_t)(p * c));           // column-major copy
  b += a256(sizeof(double) * (size_t)(c * kmax));        // L
  b += a256(sizeof(double) * (size_t)(kmax * kmax));     // R
  b += a256(4 * (size_t)c) + a256(8);                    // perm, rank
  b += a256(sizeof(PivotCand) * (size_t)(2 * g.nb)) + 256;   // candidates, barrier
  // then the tall-skinny tail (Q_1 and the refinement's Gram) on p x r, r <= 128
  b += orth_gram_ws(p, kLpMaxRank, num_sms);
  b += a256(sizeof(double) * (size_t)(kmax * c));        // the factor in original column order
  return b + 1024;
}

lrs_status launch_orth_wide(lrs_ctx* ctx, const double* M, int64_t p, int64_t c, int64_t ldm, double rtol,
                            double* Q, int64_t ldq, int64_t* r_out, bool refine, double* rdiag, double* Rt) {
  if (!ctx->coop_ok) return LRS_ERANK;               // the caller's Householder route reports it
  const int64_t kmax_full = min(p, c);
  const int64_t kmax = min(kmax_full, kLpMaxRank + 1);
  const LpGeom g = lp_geom(p, c, kmax, ctx->num_sms);
  double* Mc = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(p * c));
  double* L = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(c * kmax));
  double* R = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(kmax * kmax));
  int32_t* perm = (int32_t*)ws_alloc(ctx, 4 * (size_t)c);
  int32_t* rank = (int32_t*)ws_alloc(ctx, 8);
  PivotCand* cand = (PivotCand*)ws_alloc(ctx, sizeof(PivotCand) * (size_t)(2 * g.nb));
  unsigned* bar = (unsigned*)ws_alloc(ctx, 256);
  if (!Mc || !L || !R || !perm || !rank || !cand || !bar)
    return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (orth_wide)");
  lrs_status st = launch_transpose(ctx, M, p, c, ldm, Mc, p);
  if (st) return st;
  LpcholState s{};
  s.Mc = Mc; s.p = p; s.c = c; s.ldm = p; s.kmax = kmax; s.rtol = rtol; s.cpb = g.cpb;
  s.L = L; s.perm = perm; s.R = R; s.ldr = kmax; s.rank = rank;
  s.cand = cand;
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, 256, ctx->stream));
  s.bar.count = bar; s.bar.gen = bar + 1; s.bar.err = (int*)(bar + 2);
  if (g.smem > 48 * 1024)
    { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_lpchol, g.smem); if (_s) return _s; }
  int per_sm = 0;
  LRS_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lpchol, kLpThreads, g.smem));
  if (per_sm < 1 || g.nb > (int64_t)per_sm * ctx->num_sms) return LRS_ERANK;
  void* args[] = {&s};
  LRS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_lpchol, dim3((unsigned)g.nb), dim3(kLpThreads),
                                                args, g.smem, ctx->stream));
  ctx->launches++;
  int32_t* h = (int32_t*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[2] = {rank, (const int32_t*)(bar + 2)};
    int32_t v[2];
    lrs_status rs = replay_ints(ctx, 2, d, v);
    if (rs) return rs;
    h[43] = v[0];
    h[44] = v[1];
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 43, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 44, bar + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[44] != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "orth_wide: grid barrier wait gave up");
  const int r = h[43];
  // more than 128 directions: the refinement kernels cannot take it; the
  // caller's Householder route runs instead
  if (r > kLpMaxRank) return LRS_ERANK;
  *r_out = r;
  if (r == 0) return LRS_OK;
  if (rdiag) {
    st = launch_abs_diag(ctx, R, kmax, r, rdiag);
    if (st) return st;
  }
  // M = Q_1 L^T in original column order (L is kept by original column)
  double* R1t = (Rt && refine) ? (double*)ws_alloc(ctx, sizeof(double) * (size_t)(r * c)) : Rt;
  if (Rt) {
    if (!R1t) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (orth_wide factor)");
    k_rt_from_l<<<(unsigned)((r * c + 255) / 256), 256, 0, ctx->stream>>>(L, kmax, r, c, R1t);
    ctx->launches++;
    LRS_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (!refine) return trsm_rows(ctx, M, p, ldm, perm, R, kmax, r, Q, ldq);
  double* Q1 = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(p * r));
  double* G2 = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(r * r));
  double* R2 = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(r * r));
  if (!Q1 || !G2 || !R2) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (orth_wide refine)");
  st = trsm_rows(ctx, M, p, ldm, perm, R, kmax, r, Q1, r);
  if (st) return st;
  // refinement: G_2 = Q_1^T Q_1 = R_2^T R_2 (plain Cholesky), Q = Q_1 R_2^{-1}
  const size_t mark = ctx->ws_top;
  st = gram(ctx, Q1, p, r, r, G2);
  if (st) return st;
  ctx->ws_top = mark;
  st = pchol(ctx, G2, r, r, 0.0, 0, perm, R2, r, rank);
  if (st) return st;
  if (ctx->replay) {
    const int32_t* d[1] = {rank};
    st = replay_ints(ctx, 1, d, h + 45);
    if (st) return st;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 45, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[45] != r) return LRS_ERANK;
  if (Rt) {
    st = launch_trmm_upper(ctx, R2, r, R1t, c, Rt);
    if (st) return st;
  }
  return trsm_rows(ctx, Q1, p, r, nullptr, R2, r, r, Q, ldq);
}

}  // namespace lrs
