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

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_tn(GemmArgs a) {
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

  for (int64_t k0 = 0; k0 < a.K; k0 += BK) {
    // X slab: BK x BM = 1024 elements, 4 per thread
#pragma unroll
    for (int e = 0; e < (BK * BM) / 256; ++e) {
      const int id = threadIdx.x + e * 256;
      const int kk = id / BM, mm = id % BM;
      const int64_t gk = k0 + kk, gm = m0 + mm;
      Xs[kk][mm] = (gk < a.K && gm < a.M) ? ld_as<T>(a.X, a.xdt, gk * a.ldx + gm) : T(0);
    }
    // A slab: BK x BN = 2048 elements, 8 per thread
#pragma unroll
    for (int e = 0; e < (BK * BN) / 256; ++e) {
      const int id = threadIdx.x + e * 256;
      const int kk = id / BN, nn = id % BN;
      const int64_t gk = k0 + kk, gn = n0 + nn;
      As[kk][nn] = (gk < a.K && gn < a.N) ? ld_as<T>(a.A, a.adt, gk * a.lda + gn) : T(0);
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
      const T v = alpha * acc[i][j];
      const int64_t off = a.c_trans ? gn * a.ldc + gm : gm * a.ldc + gn;
      if (a.c_f64) reinterpret_cast<double*>(a.C)[off] = (double)v;
      else reinterpret_cast<float*>(a.C)[off] = (float)v;
    }
  }
}

lrs_status launch_gemm_simt(lrs_ctx* ctx, const GemmArgs& a, int fp64) {
  if (a.M <= 0 || a.N <= 0) return LRS_OK;
  const int64_t gm = (a.M + BM - 1) / BM, gn = (a.N + BN - 1) / BN;
  if (gm * gn > 0x7fffffffLL)
    return lrs_fail(ctx, LRS_EINVAL, "gemm: M=%lld N=%lld too large for the SIMT path", (long long)a.M, (long long)a.N);
  dim3 grid((unsigned)(gm * gn));
  if (fp64) k_gemm_tn<double><<<grid, 256, 0, ctx->stream>>>(a);
  else k_gemm_tn<float><<<grid, 256, 0, ctx->stream>>>(a);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
