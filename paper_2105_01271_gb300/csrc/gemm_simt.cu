// C = alpha * X^T A on CUDA cores (FP32 FMA or FP64 FMA).
//
// X is K x M and A is K x N, both row-major, so both operands stream along
// their contiguous dimension: a K-slab of X (BK x BM) and of A (BK x BN) are
// staged in shared memory with coalesced loads and each thread accumulates a
// TM x TN outer-product tile in registers.  This is the plain FP32 method's
// A-pass (B = Q^T A_f, paper Alg. 2) and the FP64 path for FP64 data; the
// tensor-core forms live in gemm_tc.cu.
#include "common.cuh"
#include "internal.h"

namespace lrs {

template <typename T>
__device__ __forceinline__ T ld_as(const void* p, int32_t dt, int64_t i) {
  if (dt == LRS_F64) return (T)__ldg(reinterpret_cast<const double*>(p) + i);
  if (dt == LRS_F32) return (T)__ldg(reinterpret_cast<const float*>(p) + i);
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
  return (T)__uint_as_float(((unsigned)b) << 16);
}

constexpr int BM = 64, BN = 128, BK = 16, TM = 4, TN = 8;   // 16 x 16 threads

// Split-K: block z of grid.y sums k in [z kc, (z+1) kc) and, when part is
// set, stores its raw sums to part[z][M][N]; k_gemm_sum adds the slices in
// slice order (deterministic) and applies alpha and the layout of C.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_tn(GemmArgs a, int64_t kc, T* __restrict__ part) {
  __shared__ T Xs[BK][BM];
  __shared__ T As[BK][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  // one flat grid over the (M tile, N tile) pairs, M tiles fastest: either
  // dimension can be a dof count
  const int64_t gm = (a.M + BM - 1) / BM;
  const int64_t bid = blockIdx.x;
  const int64_t m0 = (bid % gm) * BM, n0 = (bid / gm) * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  const int64_t kb = (int64_t)blockIdx.y * kc;
  const int64_t ke = min(a.K, kb + kc);
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    // X slab: BK x BM = 1024 elements, 4 per thread
#pragma unroll
    for (int e = 0; e < (BK * BM) / 256; ++e) {
      const int id = threadIdx.x + e * 256;
      const int kk = id / BM, mm = id % BM;
      const int64_t gk = k0 + kk, gm = m0 + mm;
      Xs[kk][mm] = (gk < ke && gm < a.M) ? ld_as<T>(a.X, a.xdt, gk * a.ldx + gm) : T(0);
    }
    // A slab: BK x BN = 2048 elements, 8 per thread
#pragma unroll
    for (int e = 0; e < (BK * BN) / 256; ++e) {
      const int id = threadIdx.x + e * 256;
      const int kk = id / BN, nn = id % BN;
      const int64_t gk = k0 + kk, gn = n0 + nn;
      As[kk][nn] = (gk < ke && gn < a.N) ? ld_as<T>(a.A, a.adt, gk * a.lda + gn) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T xv[TM], av[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) xv[i] = Xs[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) av[j] = As[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(xv[i], av[j], acc[i][j]);
    }
    __syncthreads();
  }
  const T alpha = (T)a.alpha;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty * TM + i;
    if (gm >= a.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= a.N) continue;
      if (part) {
        part[((int64_t)blockIdx.y * a.M + gm) * a.N + gn] = acc[i][j];
        continue;
      }
      const T v = alpha * acc[i][j];
      const int64_t off = a.c_trans ? gn * a.ldc + gm : gm * a.ldc + gn;
      if (a.c_f64) {
        double* c = reinterpret_cast<double*>(a.C) + off;
        *c = a.accum ? *c + (double)v : (double)v;
      } else {
        float* c = reinterpret_cast<float*>(a.C) + off;
        *c = a.accum ? *c + (float)v : (float)v;
      }
    }
  }
}

template <typename T>
__global__ void k_gemm_sum(const T* __restrict__ part, int64_t splits, GemmArgs a) {
  const int64_t mn = a.M * a.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int64_t z = 0; z < splits; ++z) s += part[z * mn + e];
    const int64_t gm = e / a.N, gn = e - gm * a.N;
    const T v = (T)a.alpha * s;
    const int64_t off = a.c_trans ? gn * a.ldc + gm : gm * a.ldc + gn;
    if (a.c_f64) {
      double* c = reinterpret_cast<double*>(a.C) + off;
      *c = a.accum ? *c + (double)v : (double)v;
    } else {
      float* c = reinterpret_cast<float*>(a.C) + off;
      *c = a.accum ? *c + (float)v : (float)v;
    }
  }
}

template <typename T>
lrs_status gemm_simt_impl(lrs_ctx* ctx, const GemmArgs& a) {
  const int64_t gm = (a.M + BM - 1) / BM, gn = (a.N + BN - 1) / BN;
  if (gm * gn > 0x7fffffffLL)
    return lrs_fail(ctx, LRS_EINVAL, "gemm: M=%lld N=%lld too large for the SIMT path", (long long)a.M, (long long)a.N);
  // Few output tiles and a long K (a thin product such as Q^T Y): split K so
  // that about two blocks run per SM; the slices are summed in a fixed order.
  int64_t splits = 1, kc = a.K;
  const int64_t tiles = gm * gn, want = 2 * (int64_t)ctx->num_sms;
  if (tiles < ctx->num_sms && a.K >= 8 * BK) {
    splits = (want + tiles - 1) / tiles;
    const int64_t kmax_splits = (a.K + 4 * BK - 1) / (4 * BK);        // at least 4 K-steps per slice
    if (splits > kmax_splits) splits = kmax_splits;
    if (splits > 64) splits = 64;
    kc = ((a.K + splits - 1) / splits + BK - 1) / BK * BK;
    splits = (a.K + kc - 1) / kc;
  }
  T* part = nullptr;
  if (splits > 1) {
    const lrs_status st = aux_reserve(ctx, sizeof(T) * (size_t)(splits * a.M * a.N));
    if (st) return st;
    part = reinterpret_cast<T*>(ctx->aux);
  }
  dim3 grid((unsigned)tiles, (unsigned)splits);
  k_gemm_tn<T><<<grid, 256, 0, ctx->stream>>>(a, kc, part);
  ctx->launches++;
  if (part) {
    const int64_t mn = a.M * a.N;
    const unsigned nb = (unsigned)((mn + 255) / 256 < 4096 ? (mn + 255) / 256 : 4096);
    k_gemm_sum<T><<<nb, 256, 0, ctx->stream>>>(part, splits, a);
    ctx->launches++;
  }
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_gemm_simt(lrs_ctx* ctx, const GemmArgs& a, int fp64) {
  if (a.M <= 0 || a.N <= 0) return LRS_OK;
  return fp64 ? gemm_simt_impl<double>(ctx, a) : gemm_simt_impl<float>(ctx, a);
}

}  // namespace lrs
