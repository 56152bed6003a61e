// Small elementwise kernels of the SVD epilogue and layout changes.
#include "common.cuh"
#include "internal.h"

namespace lrs {

// dst (cols x rows, row stride ldd) = src^T, src rows x cols (row stride lds)
template <typename TI, typename TO>
__global__ void k_transpose(const TI* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                            TO* __restrict__ dst, int64_t ldd) {
  __shared__ TO tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? (TO)src[r * lds + c] : (TO)0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ldd + r] = tile[threadIdx.x][i];
  }
}

lrs_status launch_transpose(lrs_ctx* ctx, const double* src, int64_t rows, int64_t cols, int64_t lds,
                            double* dst, int64_t ldd) {
  if (rows <= 0 || cols <= 0) return LRS_OK;
  if ((rows + 31) / 32 > 65535) return lrs_fail(ctx, LRS_EINVAL, "transpose: %lld rows", (long long)rows);
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  k_transpose<double, double><<<grid, dim3(32, 8), 0, ctx->stream>>>(src, rows, cols, lds, dst, ldd);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_transpose32(lrs_ctx* ctx, const float* src, int64_t rows, int64_t cols, int64_t lds,
                              float* dst, int64_t ldd) {
  if (rows <= 0 || cols <= 0) return LRS_OK;
  if ((rows + 31) / 32 > 65535) return lrs_fail(ctx, LRS_EINVAL, "transpose: %lld rows", (long long)rows);
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  k_transpose<float, float><<<grid, dim3(32, 8), 0, ctx->stream>>>(src, rows, cols, lds, dst, ldd);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// dst (rows x cols, FP32, row stride ldd) = src (FP64, row stride lds), rounded to nearest
__global__ void k_to_f32(const double* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                         float* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / cols, c = e - r * cols;
    dst[r * ldd + c] = __double2float_rn(src[r * lds + c]);
  }
}

lrs_status launch_to_f32(lrs_ctx* ctx, const double* src, int64_t rows, int64_t cols, int64_t lds,
                         float* dst, int64_t ldd) {
  const int64_t tot = rows * cols;
  if (tot <= 0) return LRS_OK;
  int64_t nb = (tot + 255) / 256;
  if (nb > (int64_t)ctx->num_sms * 16) nb = (int64_t)ctx->num_sms * 16;
  k_to_f32<<<(unsigned)nb, 256, 0, ctx->stream>>>(src, rows, cols, lds, dst, ldd);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// One block per column: find the largest-|entry| of U[:, c] (lowest row on
// ties); if negative flip U[:, c] and V[:, c].  |entry| is compared through
// its bit pattern as a 64-bit integer (the order of non-negative doubles; NaN
// entries rank below every number, as a floating-point compare would leave
// them), on the integer pipe: an FP64 compare issues over ~64 cycles per warp
// instruction on this part.
__device__ __forceinline__ long long abs_key(double x) {
  const long long k = __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL;
  return k > 0x7FF0000000000000LL ? -2LL : k;
}

__global__ void __launch_bounds__(256) k_sign_fix(double* __restrict__ U, int64_t m, int64_t ldu,
                                                  double* __restrict__ sign_out) {
  __shared__ long long sv[32];
  __shared__ int64_t si[32];
  __shared__ double s_sign;
  const int64_t c = blockIdx.x;
  long long best = -1; int64_t bi = INT64_MAX;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const long long a = abs_key(U[i * ldu + c]);
    if (a > best || (a == best && i < bi)) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sv[wid] = best; si[wid] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long b = -1; int64_t bj = INT64_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > b || (sv[w] == b && si[w] < bj)) { b = sv[w]; bj = si[w]; }
    s_sign = (bj < m && U[bj * ldu + c] < 0.0) ? -1.0 : 1.0;
    sign_out[c] = s_sign;
  }
  __syncthreads();
  if (s_sign > 0.0) return;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) U[i * ldu + c] = -U[i * ldu + c];
}

lrs_status launch_sign_fix(lrs_ctx* ctx, double* U, int64_t m, int64_t k, int64_t ldu, double* sign_out) {
  if (k <= 0) return LRS_OK;
  k_sign_fix<<<(unsigned)k, 256, 0, ctx->stream>>>(U, m, ldu, sign_out);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

__global__ void k_scale_cols(const double* __restrict__ V, int64_t r, int64_t ldv,
                             const double* __restrict__ s, const double* __restrict__ sign, int64_t k,
                             double* __restrict__ W, int64_t ldw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * k) return;
  const int64_t i = e / k, c = e - i * k;
  const double sc = s[c];
  const double sg = sign ? sign[c] : 1.0;
  W[i * ldw + c] = sc > 0.0 ? sg * V[i * ldv + c] / sc : 0.0;
}

lrs_status launch_scale_cols(lrs_ctx* ctx, const double* V, int64_t r, int64_t ldv, const double* s,
                             const double* sign, int64_t k, double* W, int64_t ldw) {
  const int64_t tot = r * k;
  if (tot <= 0) return LRS_OK;
  k_scale_cols<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(V, r, ldv, s, sign, k, W, ldw);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded grid barrier: a two-block cooperative launch in
// which block 1 leaves without arriving, so block 0's wait runs out after
// spin_limit polls, records LRS_ETIMEOUT and returns.  The host reads the
// flag; nothing faults, traps or hangs.
__global__ void k_barrier_selftest(GridBarrier bar, long long spin_limit) {
  if (blockIdx.x != 0) return;
  grid_sync(bar, spin_limit);
}

lrs_status launch_barrier_selftest(lrs_ctx* ctx, int64_t spin_limit) {
  unsigned* bar = (unsigned*)ws_alloc(ctx, 256);
  if (!bar) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (selftest)");
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(bar, 0, 256, ctx->stream));
  GridBarrier b{};
  b.count = bar; b.gen = bar + 1; b.err = (int*)(bar + 2);
  long long lim = spin_limit;
  void* args[] = {&b, &lim};
  LRS_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(2), dim3(32), args, 0,
                                                ctx->stream));
  ctx->launches++;
  int* h = (int*)ctx->host_scratch;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 36, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (h[36] != 0) return lrs_fail(ctx, (lrs_status)h[36], "selftest: the grid barrier wait gave up");
  return LRS_OK;
}

}  // namespace lrs

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe (lrs_fp64_peak): 8 independent dependent chains
// per thread hide the FMA latency; the result feeds one store per thread so
// the chains stay live.
// ---------------------------------------------------------------------------
namespace lrs {

__global__ void __launch_bounds__(256) k_dfma_chains(int32_t iters, double seed, double* __restrict__ out) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double b = 0.999999, d = 1e-7;
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace lrs

extern "C" lrs_status lrs_fp64_peak(lrs_ctx* ctx, int32_t iters, double* tflops) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!tflops || iters < 16 || iters > (1 << 20)) return lrs_fail(ctx, LRS_EINVAL, "fp64_peak: iters=%d", iters);
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const unsigned blocks = (unsigned)ctx->num_sms * 4;
  lrs_status st = lrs::ws_reserve(ctx, sizeof(double) * (size_t)blocks * 256 + 256);
  if (st) return st;
  double* out = (double*)lrs::ws_alloc(ctx, sizeof(double) * (size_t)blocks * 256);
  if (!out) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (fp64_peak)");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LRS_CUDA_TRY(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return lrs_fail(ctx, LRS_ECUDA, "fp64_peak: event creation failed");
  }
  double best = 0.0;
  lrs_status res = LRS_OK;
  for (int rep = 0; rep < 4 && res == LRS_OK; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    lrs::k_dfma_chains<<<blocks, 256, 0, ctx->stream>>>(iters, 1.0 + rep, out);
    ctx->launches++;
    cudaEventRecord(e1, ctx->stream);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      res = lrs_fail(ctx, LRS_ECUDA, "fp64_peak: launch failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double t = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0 / (ms * 1e-3) / 1e12;
    if (rep > 0 && t > best) best = t;            // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (res == LRS_OK) *tflops = best;
  return res;
}

// ---------------------------------------------------------------------------
// record / replay of host read-backs
// ---------------------------------------------------------------------------
namespace lrs {

__global__ void k_guard_eq(const int32_t* __restrict__ v, int32_t want, int* __restrict__ flag) {
  if (*v != want) atomicOr(flag, 1);
}

// the same left-to-right sum as the host loop of svd_finish, no contraction
__global__ void k_err_tail(const double* __restrict__ s, int64_t r, int64_t kk, const double* __restrict__ fro2,
                           double* __restrict__ out) {
  double tail = 0.0;
  for (int64_t i = r - 1; i >= kk; --i) tail = __dadd_rn(tail, __dmul_rn(s[i], s[i]));
  const double f = fro2 ? *fro2 : 0.0;
  *out = f > 0.0 ? sqrt(tail / f) : 0.0;
}

__global__ void k_err_ratio(const double* __restrict__ tail2, const double* __restrict__ nrm2, double* __restrict__ out) {
  const double n = *nrm2;
  *out = n > 0.0 ? sqrt(fmax(*tail2, 0.0) / n) : 0.0;
}

lrs_status replay_ints(lrs_ctx* ctx, int n, const int32_t* const* dev, int32_t* out) {
  if (n < 1 || n > 8) return lrs_fail(ctx, LRS_EINVAL, "replay: %d values", n);
  if (ctx->replay == kReplayCapture) {
    for (int i = 0; i < n; ++i) {
      if (ctx->log_pos >= ctx->log.size())
        return lrs_fail(ctx, LRS_EINVAL, "replay: the call sequence reads more values than were recorded");
      out[i] = ctx->log[ctx->log_pos++];
      k_guard_eq<<<1, 1, 0, ctx->stream>>>(dev[i], out[i], ctx->cap_guard);
      ctx->launches++;
    }
    LRS_CUDA_TRY(ctx, cudaGetLastError());
    return LRS_OK;
  }
  int32_t* h = (int32_t*)ctx->host_scratch + 512;
  for (int i = 0; i < n; ++i)
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + i, dev[i], sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < n; ++i) {
    out[i] = h[i];
    if (ctx->replay == kReplayRecord) ctx->log.push_back(h[i]);
  }
  return LRS_OK;
}

lrs_status launch_err_tail(lrs_ctx* ctx, const double* s, int64_t r, int64_t kk, const double* fro2, double* out) {
  k_err_tail<<<1, 1, 0, ctx->stream>>>(s, r, kk, fro2, out);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_err_ratio(lrs_ctx* ctx, const double* tail2, const double* nrm2, double* out) {
  k_err_ratio<<<1, 1, 0, ctx->stream>>>(tail2, nrm2, out);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs

namespace lrs {

__global__ void k_widen_f32(const float* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}

lrs_status launch_widen_f32(lrs_ctx* ctx, const float* src, int64_t n, double* dst) {
  if (n <= 0) return LRS_OK;
  int64_t nb = (n + 255) / 256;
  if (nb > (int64_t)ctx->num_sms * 16) nb = (int64_t)ctx->num_sms * 16;
  k_widen_f32<<<(unsigned)nb, 256, 0, ctx->stream>>>(src, n, dst);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
