// Pieces of the SVD of B (r x n, r small) for TPC-SVD (paper Alg. 2,
// "SVD(B)") without squaring its condition number:
//   1. R = the R factor of B^T by Householder TSQR: each block factors a
//      chunk of C columns of B (a C x r slab of B^T) in shared memory and
//      writes its r x r triangle; the triangles of all chunks, laid side by
//      side, form a new r x (chunks * r) matrix that the same kernel reduces
//      again, until one chunk remains.  In the working precision T of B (the
//      R form of lrs_slab_factor, and the fallback when the Gram's Cholesky
//      of an FP32 B breaks down).
//   2. FP64 one-sided (Hestenes) Jacobi on the columns of R: R V = U_R
//      diag(s).  Since B = R^T Q_T^T = V diag(s) (Q_T U_R)^T, the left
//      singular vectors of B are V and its singular values s.  One block, or
//      one warp per pair across the SMs (cooperative) from r = 24 on.
// Shared memory bounds r: r*C*sizeof(T) <= ~200 KB for TSQR and
// 2*r*r*8 <= ~200 KB for the one-block Jacobi.  The usual FP32-data route
// (exact-slice Gram, pivoted Cholesky, the cluster Jacobi on the rows of R)
// is in gram_oz.cu, orth_gram.cu and jacobi_cluster.cu.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <vector>

namespace lrs {

constexpr int kTsqrThreads = 1024;
constexpr size_t kSmemCap = 200 * 1024;

// tile[i][t] holds column i of the C x r slab (row i of B's chunk), t < C.
template <typename T>
__global__ void __launch_bounds__(kTsqrThreads, 1)
k_tsqr_leaf(const void* __restrict__ B, int b_f64, int64_t r, int64_t n, int64_t ldb, int64_t C,
            T* __restrict__ out, int64_t ldo, double* __restrict__ Rfinal) {
  extern __shared__ unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ T s_scal[2];
  const int64_t j0 = (int64_t)blockIdx.x * C;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // load: row i of B, columns j0 .. j0+C-1 (zero beyond n)
  for (int64_t e = threadIdx.x; e < r * C; e += blockDim.x) {
    const int64_t i = e / C, t = e - i * C;
    const int64_t col = j0 + t;
    T v = T(0);
    if (col < n) {
      v = b_f64 ? (T)reinterpret_cast<const double*>(B)[i * ldb + col]
                : (T)reinterpret_cast<const float*>(B)[i * ldb + col];
    }
    tile[i * C + t] = v;
  }
  __syncthreads();
  __shared__ T red[32];
  const int64_t steps = r < C ? r : C;
  for (int64_t i = 0; i < steps; ++i) {
    T* x = tile + i * C;
    // ||x||^2 over the whole block
    T a = T(0);
    for (int64_t t = i + threadIdx.x; t < C; t += blockDim.x) a = fma(x[t], x[t], a);
    a = block_sum(a, red);
    const T alpha = sqrt(a);
    const T x0 = x[i];
    const T sgn = x0 >= T(0) ? T(1) : T(-1);
    const T v0 = x0 + sgn * alpha;
    // ||v||^2 = ||x||^2 - x0^2 + v0^2
    const T vn2 = a - x0 * x0 + v0 * v0;
    const T inv = vn2 > T(0) ? T(1) / sqrt(vn2) : T(0);
    for (int64_t t = i + 1 + threadIdx.x; t < C; t += blockDim.x) x[t] *= inv;
    if (threadIdx.x == 0) { s_scal[0] = -sgn * alpha; s_scal[1] = v0 * inv; }
    __syncthreads();
    const T rii = s_scal[0];
    const T v0n = s_scal[1];
    // apply H = I - 2 v v^T to columns c > i ; v = (v0n, x[i+1..C-1])
    for (int64_t c = i + 1 + wid; c < r; c += nw) {
      T* y = tile + c * C;
      T w = (lane == 0) ? v0n * y[i] : T(0);
      for (int64_t t = i + 1 + lane; t < C; t += 32) w = fma(x[t], y[t], w);
      w = warp_sum(w);
      const T tw = T(2) * w;
      if (lane == 0) y[i] = fma(-tw, v0n, y[i]);
      for (int64_t t = i + 1 + lane; t < C; t += 32) y[t] = fma(-tw, x[t], y[t]);
    }
    __syncthreads();
    if (threadIdx.x == 0) x[i] = rii;
    __syncthreads();
  }
  // column c of R (rows 0..c) sits in tile[c][0..c]
  if (Rfinal) {
    for (int64_t e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int64_t i = e / r, c = e - i * r;        // R[i][c]
      Rfinal[i * r + c] = (i <= c && i < C) ? (double)tile[c * C + i] : 0.0;
    }
  } else {
    // next level: row c, columns blockIdx*r .. +r-1 hold R[0..r-1][c]
    for (int64_t e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int64_t c = e / r, t = e - c * r;
      out[c * ldo + (int64_t)blockIdx.x * r + t] = (t <= c && t < C) ? tile[c * C + t] : T(0);
    }
  }
}

template <typename T>
static lrs_status tsqr_impl(lrs_ctx* ctx, const void* B, int b_f64, int64_t r, int64_t n,
                            int64_t ldb, double* R) {
  int64_t C = (int64_t)(kSmemCap / (sizeof(T) * (size_t)r));
  if (C > 1024) C = 1024;
  if (C < r) return lrs_fail(ctx, LRS_EINVAL, "svd: rank r=%lld too large for the TSQR tile", (long long)r);
  const size_t dyn = sizeof(T) * (size_t)(r * C);
  auto kern = k_tsqr_leaf<T>;
  { const lrs_status _s = raise_dyn_smem(ctx, (const void*)kern, (size_t)(dyn)); if (_s) return _s; }
  const void* src = B;
  int src_f64 = b_f64;
  int64_t cur_n = n, cur_ld = ldb;
  while (true) {
    const int64_t chunks = (cur_n + C - 1) / C;
    if (chunks == 1) {
      kern<<<1, kTsqrThreads, dyn, ctx->stream>>>(src, src_f64, r, cur_n, cur_ld, C, nullptr, 0, R);
      ctx->launches++;
      break;
    }
    const int64_t next_n = chunks * r;
    T* nxt = (T*)ws_alloc(ctx, sizeof(T) * (size_t)(r * next_n));
    if (!nxt) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (tsqr)");
    kern<<<(unsigned)chunks, kTsqrThreads, dyn, ctx->stream>>>(src, src_f64, r, cur_n, cur_ld, C, nxt,
                                                                 next_n, nullptr);
    ctx->launches++;
    src = nxt;
    src_f64 = sizeof(T) == 8;
    cur_n = next_n;
    cur_ld = next_n;
  }
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_tsqr(lrs_ctx* ctx, const void* B, int b_f64, int64_t r, int64_t n, int64_t ldb,
                       double* R) {
  if (b_f64) return tsqr_impl<double>(ctx, B, 1, r, n, ldb, R);
  return tsqr_impl<float>(ctx, B, 0, r, n, ldb, R);
}

// ---------------------------------------------------------------------------
// One-sided Jacobi, one block, round-robin pairing (r' = r rounded up to even
// columns; the pad column is zero and never rotates).
// ---------------------------------------------------------------------------
constexpr int kJacLanes = 16;

template <typename T>
__global__ void __launch_bounds__(1024, 1)
k_jacobi(const double* __restrict__ R, int64_t r, double* __restrict__ Vout, double* __restrict__ s_out,
         int max_sweeps) {
  extern __shared__ unsigned char smem_raw[];
  const int64_t rp = (r + 1) & ~int64_t(1);
  T* Wc = reinterpret_cast<T*>(smem_raw);             // rp columns of length r
  T* Vc = Wc + rp * r;                                // rp columns of length r
  int* order = reinterpret_cast<int*>(Vc + rp * r);   // rp
  __shared__ int s_rot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t e = threadIdx.x; e < rp * r; e += blockDim.x) {
    const int64_t c = e / r, i = e - c * r;
    Wc[e] = c < r ? (T)R[i * r + c] : T(0);
    Vc[e] = (c == i && c < r) ? T(1) : T(0);
  }
  for (int64_t c = threadIdx.x; c < rp; c += blockDim.x) order[c] = (int)c;
  __syncthreads();
  const T eps = sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08);
  // a pair counts as orthogonal once |w_p . w_q| <= tol ||w_p|| ||w_q||.  The
  // computed dot product itself carries ~sqrt(r) eps of rounding, so a
  // threshold at that level keeps re-rotating converged pairs until the sweep
  // cap; eps * max(r, 16) (the column length, as in LAPACK's one-sided
  // Jacobi) sits safely above it.
  const T tol = eps * (T)(r > 16 ? r : 16);
  // a team of kJacLanes lanes (half a warp) per pair: all pairs of a round at
  // r <= 128 run in one pass of the block, with a 4-level shuffle tree
  const int lg = threadIdx.x % kJacLanes, grp = threadIdx.x / kJacLanes, ngrp = blockDim.x / kJacLanes;
  const int ri = (int)r, rpi = (int)rp;
  const unsigned gmask = ((1u << kJacLanes) - 1u) << (lane & (32 - kJacLanes));
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < rpi - 1; ++round) {
      // round-robin: slot 0 fixed, others rotate; pairs (slot a, slot rp-1-a)
      for (int pr = grp; pr < rpi / 2; pr += ngrp) {
        const int sa = pr, sb = rpi - 1 - pr;
        auto slot = [&](int sidx) -> int {
          if (sidx == 0) return 0;
          int v = sidx - 1 + round;                  // < 2 (rp - 1): one conditional subtract
          if (v >= rpi - 1) v -= rpi - 1;
          return 1 + v;
        };
        int p = slot(sa), q = slot(sb);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        if (q >= ri) continue;                       // the zero pad column
        T* wp = Wc + p * ri; T* wq = Wc + q * ri;
        T a = T(0), b = T(0), g = T(0);
        for (int i = lg; i < ri; i += kJacLanes) {
          a = fma(wp[i], wp[i], a); b = fma(wq[i], wq[i], b); g = fma(wp[i], wq[i], g);
        }
#pragma unroll
        for (int o = kJacLanes / 2; o > 0; o >>= 1) {
          a += __shfl_xor_sync(gmask, a, o); b += __shfl_xor_sync(gmask, b, o); g += __shfl_xor_sync(gmask, g, o);
        }
        if (fabs(g) <= tol * (sqrt(a) * sqrt(b)) || g == T(0)) continue;
        const T zeta = (b - a) / (T(2) * g);
        const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        const T cs = T(1) / sqrt(T(1) + t * t);
        const T sn = cs * t;
        for (int i = lg; i < ri; i += kJacLanes) {
          const T x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y; wq[i] = sn * x + cs * y;
          T* vp = Vc + p * ri; T* vq = Vc + q * ri;
          const T u = vp[i], w = vq[i];
          vp[i] = cs * u - sn * w; vq[i] = sn * u + cs * w;
        }
        if (lg == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // singular values = column norms; sort descending (ties by index) -- r is small
  __shared__ double s_norm[1024];
  for (int64_t c = wid; c < r; c += nw) {
    T a = T(0);
    for (int64_t i = lane; i < r; i += 32) a = fma(Wc[c * r + i], Wc[c * r + i], a);
    a = warp_sum(a);
    if (lane == 0) s_norm[c] = sqrt((double)a);
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < r; c += blockDim.x) {
    int64_t rank = 0;
    const double v = s_norm[c];
    for (int64_t d = 0; d < r; ++d) {
      const double u = s_norm[d];
      if (u > v || (u == v && d < c)) ++rank;
    }
    order[rank] = (int)c;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int64_t i = e / r, k = e - i * r;           // V[i][k] = Vc[order[k]][i]
    Vout[i * r + k] = (double)Vc[(int64_t)order[k] * r + i];
  }
  for (int64_t k = threadIdx.x; k < r; k += blockDim.x) s_out[k] = s_norm[order[k]];
}

// ---------------------------------------------------------------------------
// FP64 one-sided Jacobi across the GPU: the pairs of one round-robin round
// are spread over up to one block (one warp) per SM, with a grid barrier
// between rounds.  On GB300 the FP64 pipe of one SM retires one warp-wide
// DFMA every 16 cycles, so the one-block kernel above spends ~50 us per round
// at r = 112; here each SM works on one pair per round.  The columns live in
// global memory (L2-resident: 2 r^2 doubles) and are read with ld.global.cg,
// since another SM may have rotated them in the previous round.
// ---------------------------------------------------------------------------
struct JacobiCoop {
  double* W;       // rp columns of length len (column c at c * len)
  double* Vc;      // rp columns of length r, starts as I
  const double* R; // the input: r x r row-major (by_rows = 0), or r x len row-major (by_rows = 1)
  int64_t r, rp, len, ldr;
  int by_rows;     // 1: column c of the Jacobi matrix is row c of R (B^T of a wide B)
  int max_sweeps;
  int* rot;        // rotations per sweep (max_sweeps counters, zeroed)
  int* sweeps;     // sweeps taken
  GridBarrier bar;
};

__global__ void __launch_bounds__(32) k_jacobi_coop(JacobiCoop J) {
  const int lane = threadIdx.x;
  const int64_t r = J.r, rp = J.rp, len = J.len;
  for (int64_t e = (int64_t)blockIdx.x * 32 + lane; e < rp * len; e += (int64_t)gridDim.x * 32) {
    const int64_t c = e / len, i = e - c * len;
    J.W[e] = c < r ? (J.by_rows ? J.R[c * J.ldr + i] : J.R[i * J.ldr + c]) : 0.0;
  }
  for (int64_t e = (int64_t)blockIdx.x * 32 + lane; e < rp * r; e += (int64_t)gridDim.x * 32) {
    const int64_t c = e / r, i = e - c * r;
    J.Vc[e] = (c == i && c < r) ? 1.0 : 0.0;
  }
  if (!grid_sync(J.bar)) return;
  const double eps = 1.1102230246251565e-16;
  const double tol = eps * (double)(r > 16 ? r : 16);        // as the one-block kernel
  const double tol2 = tol * tol;
  int sweep = 0;
  for (; sweep < J.max_sweeps; ++sweep) {
    for (int64_t round = 0; round < rp - 1; ++round) {
      for (int64_t pr = blockIdx.x; pr < rp / 2; pr += gridDim.x) {
        const int64_t sa = pr, sb = rp - 1 - pr;
        int64_t p = sa == 0 ? 0 : 1 + ((sa - 1 + round) % (rp - 1));
        int64_t q = 1 + ((sb - 1 + round) % (rp - 1));
        if (p > q) { const int64_t t = p; p = q; q = t; }
        if (q >= r) continue;                                  // the zero pad column
        double* wp = J.W + p * len;
        double* wq = J.W + q * len;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int64_t i = lane; i < len; i += 32) {
          const double x = __ldcg(wp + i), y = __ldcg(wq + i);
          a = fma(x, x, a); b = fma(y, y, b); g = fma(x, y, g);
        }
        a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
        if (g == 0.0 || g * g <= tol2 * (a * b)) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t);
        const double sn = cs * t;
        double* vp = J.Vc + p * r;
        double* vq = J.Vc + q * r;
        for (int64_t i = lane; i < len; i += 32) {
          const double x = __ldcg(wp + i), y = __ldcg(wq + i);
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
        for (int64_t i = lane; i < r; i += 32) {
          const double u = __ldcg(vp + i), w = __ldcg(vq + i);
          vp[i] = cs * u - sn * w;
          vq[i] = sn * u + cs * w;
        }
        if (lane == 0) atomicAdd(J.rot + sweep, 1);
      }
      if (!grid_sync(J.bar)) return;
    }
    // the barrier above orders every count of this sweep before this read
    if (ld_volatile_s32(J.rot + sweep) == 0) break;
  }
  if (blockIdx.x == 0 && lane == 0) *J.sweeps = sweep;
}

// singular values (column norms of W), descending with ties by index, and V
__global__ void __launch_bounds__(1024) k_jacobi_finish(const double* __restrict__ W, const double* __restrict__ Vc,
                                                        int64_t r, int64_t len, double* __restrict__ Vout,
                                                        double* __restrict__ s_out) {
  __shared__ double s_norm[1024];
  __shared__ int order[1024];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t c = wid; c < r; c += nw) {
    double a = 0.0;
    for (int64_t i = lane; i < len; i += 32) a = fma(W[c * len + i], W[c * len + i], a);
    a = warp_sum(a);
    if (lane == 0) s_norm[c] = sqrt(a);
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < r; c += blockDim.x) {
    int64_t rank = 0;
    const double v = s_norm[c];
    for (int64_t d = 0; d < r; ++d) {
      const double u = s_norm[d];
      if (u > v || (u == v && d < c)) ++rank;
    }
    order[rank] = (int)c;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int64_t i = e / r, k = e - i * r;
    Vout[i * r + k] = Vc[(int64_t)order[k] * r + i];
  }
  for (int64_t k = threadIdx.x; k < r; k += blockDim.x) s_out[k] = s_norm[order[k]];
}

size_t jacobi_ws(int64_t r, int64_t len) {
  const int64_t rp = (r + 1) & ~int64_t(1);
  return ((sizeof(double) * (size_t)(rp * len) + 255) & ~size_t(255)) +
         ((sizeof(double) * (size_t)(rp * r) + 255) & ~size_t(255)) + 1024;
}

// the cooperative FP64 Jacobi on the columns of R (r x r, by_rows = 0) or of
// B^T (B r x len row-major, stride ldr, by_rows = 1); false: no workspace
static bool jacobi_coop(lrs_ctx* ctx, const double* R, int64_t r, int64_t len, int64_t ldr, int by_rows, double* V,
                        double* s, lrs_status* st_out) {
  const int64_t rp = (r + 1) & ~int64_t(1);
  JacobiCoop J{};
  J.r = r; J.rp = rp; J.len = len; J.ldr = ldr; J.by_rows = by_rows; J.R = R; J.max_sweeps = 40;
  J.W = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(rp * len));
  J.Vc = (double*)ws_alloc(ctx, sizeof(double) * (size_t)(rp * r));
  unsigned* scratch = (unsigned*)ws_alloc(ctx, 512);
  if (!J.W || !J.Vc || !scratch) return false;
  *st_out = LRS_OK;
  lrs_status& st = *st_out;
  cudaError_t e = cudaMemsetAsync(scratch, 0, 512, ctx->stream);
  if (e != cudaSuccess) { st = lrs_fail(ctx, LRS_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e)); return true; }
  J.bar.count = scratch; J.bar.gen = scratch + 1; J.bar.err = (int*)(scratch + 2);
  J.sweeps = (int*)(scratch + 3);
  J.rot = (int*)(scratch + 4);                           // 40 counters
  int64_t nb = rp / 2;
  if (nb > ctx->num_sms) nb = ctx->num_sms;
  void* args[] = {&J};
  e = cudaLaunchCooperativeKernel((const void*)k_jacobi_coop, dim3((unsigned)nb), dim3(32), args, 0, ctx->stream);
  if (e != cudaSuccess) { st = lrs_fail(ctx, LRS_ECUDA, "jacobi launch: %s", cudaGetErrorString(e)); return true; }
  k_jacobi_finish<<<1, 1024, 0, ctx->stream>>>(J.W, J.Vc, r, len, V, s);
  ctx->launches += 2;
  e = cudaGetLastError();
  if (e != cudaSuccess) { st = lrs_fail(ctx, LRS_ECUDA, "jacobi: %s", cudaGetErrorString(e)); return true; }
  int* h = (int*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {(const int32_t*)J.bar.err};
    st = replay_ints(ctx, 1, d, h + 48);
    if (st) return true;
  } else {
    e = cudaMemcpyAsync(h + 48, J.bar.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  if (e != cudaSuccess) { st = lrs_fail(ctx, LRS_ECUDA, "jacobi: %s", cudaGetErrorString(e)); return true; }
  if (h[48] != 0) st = lrs_fail(ctx, LRS_ETIMEOUT, "svd: Jacobi grid barrier wait gave up");
  return true;
}


lrs_status launch_jacobi(lrs_ctx* ctx, double* R, int64_t r, double* V, double* s) {
  const int64_t rp = (r + 1) & ~int64_t(1);
  if (ctx->coop_ok && r >= 24 && r <= 1024) {
    lrs_status st = LRS_OK;
    if (jacobi_coop(ctx, R, r, r, r, 0, V, s, &st)) return st;
    // no room in the workspace: the one-block kernel below
  }
  const size_t dyn = sizeof(double) * 2 * (size_t)(rp * r) + sizeof(int) * (size_t)rp + 64;
  if (dyn > kSmemCap || r > 1024)
    return lrs_fail(ctx, LRS_EINVAL, "svd: rank r=%lld too large for the Jacobi tile", (long long)r);
  { const lrs_status _s = raise_dyn_smem(ctx, (const void*)k_jacobi<double>, (size_t)(dyn)); if (_s) return _s; }
  k_jacobi<double><<<1, 1024, dyn, ctx->stream>>>(R, r, V, s, 40);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
