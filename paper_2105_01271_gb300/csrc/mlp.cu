// Learned sketch proposal: a 3-layer MLP (66 -> 128 -> 128 -> 6, ReLU,
// softmax cross-entropy) with BF16 weights and FP32 accumulation, trained and
// run by the kernels in this file (declared in include/lrs.h).
//
// Parameters live in one FP32 buffer (the master copy Adam updates) laid out
// as W1 [128 x 66] | b1 [128] | W2 [128 x 128] | b2 [128] | W3 [6 x 128] | b3 [6];
// a uint16 buffer of the same layout holds the BF16 rounding of the weight
// slots, which is what the forward and backward products read.  Every sum
// runs in a fixed order (one thread per output), so results are
// deterministic.
#include "common.cuh"
#include "internal.h"

#include <cuda_bf16.h>

namespace lrs {
namespace {

constexpr int kIn = LRS_MLP_IN, kHid = LRS_MLP_HID, kOut = LRS_MLP_OUT;
constexpr int64_t oW1 = 0, ob1 = oW1 + (int64_t)kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + (int64_t)kHid * kHid,
                  oW3 = ob2 + kHid, ob3 = oW3 + (int64_t)kOut * kHid, kParams = ob3 + kOut;

__device__ __forceinline__ float bf(const uint16_t* w, int64_t i) { return __uint_as_float(((uint32_t)w[i]) << 16); }

// Z = X W^T + b (B x N), H = relu(Z) when relu, else H = Z
__global__ void k_linear(const float* __restrict__ X, int64_t B, int K, const uint16_t* __restrict__ W,
                         const float* __restrict__ b, int N, int relu, float* __restrict__ Z, float* __restrict__ H) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= B * N) return;
  const int64_t r = id / N;
  const int n = (int)(id - r * N);
  float z = b[n];
  for (int k = 0; k < K; ++k) z = fmaf(X[r * K + k], bf(W, (int64_t)n * K + k), z);
  Z[id] = z;
  H[id] = (relu && z < 0.f) ? 0.f : z;
}

// dZ = (softmax(Z) - onehot(y)) / B, loss_row = -log softmax(Z)_y
__global__ void k_softmax_ce(const float* __restrict__ Z, const int32_t* __restrict__ y, int64_t B,
                             float* __restrict__ dZ, float* __restrict__ loss_row) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const float* z = Z + r * kOut;
  float mx = z[0];
  for (int c = 1; c < kOut; ++c) mx = fmaxf(mx, z[c]);
  float e[kOut], s = 0.f;
  for (int c = 0; c < kOut; ++c) { e[c] = expf(z[c] - mx); s += e[c]; }
  const int yc = y[r];
  for (int c = 0; c < kOut; ++c) dZ[r * kOut + c] = (e[c] / s - (c == yc ? 1.f : 0.f)) / (float)B;
  loss_row[r] = logf(s) - (z[yc] - mx);
}

// dH = (dZ W) * (Zprev > 0)   (dZ: B x N, W: N x K, Zprev: B x K)
__global__ void k_back_input(const float* __restrict__ dZ, int64_t B, int N, const uint16_t* __restrict__ W, int K,
                             const float* __restrict__ Zprev, float* __restrict__ dH) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= B * K) return;
  const int64_t r = id / K;
  const int k = (int)(id - r * K);
  float a = 0.f;
  for (int n = 0; n < N; ++n) a = fmaf(dZ[r * N + n], bf(W, (int64_t)n * K + k), a);
  dH[id] = Zprev[id] > 0.f ? a : 0.f;
}

// gW[n, k] = sum_r dZ[r, n] H[r, k]  (k < K);  gb[n] = sum_r dZ[r, n]
__global__ void k_back_weight(const float* __restrict__ dZ, const float* __restrict__ H, int64_t B, int N, int K,
                              float* __restrict__ gW, float* __restrict__ gb) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (int64_t)N * (K + 1)) return;
  const int n = (int)(id / (K + 1));
  const int k = (int)(id - (int64_t)n * (K + 1));
  float a = 0.f;
  if (k < K) {
    for (int64_t r = 0; r < B; ++r) a = fmaf(dZ[r * N + n], H[r * K + k], a);
    gW[(int64_t)n * K + k] = a;
  } else {
    for (int64_t r = 0; r < B; ++r) a += dZ[r * N + n];
    gb[n] = a;
  }
}

__global__ void k_sum_rows(const float* __restrict__ v, int64_t B, float* __restrict__ out) {
  __shared__ float red[32];
  float a = 0.f;
  for (int64_t i = threadIdx.x; i < B; i += blockDim.x) a += v[i];
  a = block_sum(a, red);
  if (threadIdx.x == 0) *out = a / (float)B;
}

__device__ __forceinline__ bool is_weight_slot(int64_t i) {
  return (i >= oW1 && i < ob1) || (i >= oW2 && i < ob2) || (i >= oW3 && i < ob3);
}

// Adam (beta 0.9 / 0.999, eps 1e-8) on the FP32 master copy; weight slots are
// re-rounded to BF16 (RNE) for the next products
__global__ void k_adam(float* __restrict__ p, uint16_t* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m1, float* __restrict__ m2, float lr, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  const float gi = g[i];
  const float a = 0.9f * m1[i] + 0.1f * gi;
  const float b = 0.999f * m2[i] + 0.001f * gi * gi;
  m1[i] = a;
  m2[i] = b;
  const float v = p[i] - lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
  p[i] = v;
  if (is_weight_slot(i)) w[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__global__ void k_round_weights(const float* __restrict__ p, uint16_t* __restrict__ w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kParams) w[i] = is_weight_slot(i) ? __bfloat16_as_ushort(__float2bfloat16_rn(p[i])) : (uint16_t)0;
}

// features of one matrix from |R_ii| (non-increasing) of the range finder's
// pivoted factor of the cheapest configuration's sketch (rank r, l columns)
__global__ void k_features(const double* __restrict__ s, int64_t ns, double r, double l, double N, double m,
                           float* __restrict__ x) {
  for (int i = threadIdx.x; i < kIn; i += blockDim.x) {
    double v = -1.0;
    if (i < LRS_MLP_NSIGMA) {
      if (i < ns && s[0] > 0.0) v = fmin(fmax(log10(fmax(s[i] / s[0], 1e-300)), -6.0), 0.0) / 6.0;
    } else if (i == LRS_MLP_NSIGMA) {
      v = log2(N) / 8.0;
    } else if (i == LRS_MLP_NSIGMA + 1) {
      v = log2(m) / 11.0;
    } else {
      v = r / fmin(m, l);
    }
    x[i] = (float)v;
  }
}

unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct Acts {
  float *Z1, *H1, *Z2, *H2, *Z3, *D3, *D2, *D1, *L;
};

lrs_status forward(lrs_ctx* ctx, const float* p, const uint16_t* w, const float* X, int64_t B, Acts& a) {
  k_linear<<<blocks_for(B * kHid), 256, 0, ctx->stream>>>(X, B, kIn, w + oW1, p + ob1, kHid, 1, a.Z1, a.H1);
  k_linear<<<blocks_for(B * kHid), 256, 0, ctx->stream>>>(a.H1, B, kHid, w + oW2, p + ob2, kHid, 1, a.Z2, a.H2);
  k_linear<<<blocks_for(B * kOut), 256, 0, ctx->stream>>>(a.H2, B, kHid, w + oW3, p + ob3, kOut, 0, a.Z3, a.Z3);
  ctx->launches += 3;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

bool alloc_acts(lrs_ctx* ctx, int64_t B, Acts& a) {
  float** f[] = {&a.Z1, &a.H1, &a.Z2, &a.H2, &a.D2, &a.D1};
  for (float** q : f) {
    *q = (float*)ws_alloc(ctx, sizeof(float) * (size_t)(B * kHid));
    if (!*q) return false;
  }
  a.Z3 = (float*)ws_alloc(ctx, sizeof(float) * (size_t)(B * kOut));
  a.D3 = (float*)ws_alloc(ctx, sizeof(float) * (size_t)(B * kOut));
  a.L = (float*)ws_alloc(ctx, sizeof(float) * (size_t)B);
  return a.Z3 && a.D3 && a.L;
}

size_t acts_bytes(int64_t B) { return sizeof(float) * (size_t)(B * (6 * kHid + 2 * kOut + 1)) + 16 * 256; }

}  // namespace
}  // namespace lrs

using namespace lrs;

extern "C" {

int64_t lrs_mlp_param_count(void) { return kParams; }

lrs_status lrs_mlp_init_bf16(lrs_ctx* ctx, const float* params, uint16_t* wbf16) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!params || !wbf16) return lrs_fail(ctx, LRS_EINVAL, "mlp: NULL pointer");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  k_round_weights<<<blocks_for(kParams), 256, 0, ctx->stream>>>(params, wbf16);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status lrs_mlp_features(lrs_ctx* ctx, const double* rdiag, int64_t ns, int64_t r, int64_t l, int64_t N, int64_t m,
                            float* x) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if ((!rdiag && ns > 0) || !x || ns < 0 || r < 0 || l < 1 || N < 1 || m < 1)
    return lrs_fail(ctx, LRS_EINVAL, "mlp_features: bad arguments");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  k_features<<<1, 128, 0, ctx->stream>>>(rdiag, ns, (double)r, (double)l, (double)N, (double)m, x);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status lrs_mlp_forward(lrs_ctx* ctx, const float* params, const uint16_t* wbf16, const float* X, int64_t B,
                           float* logits) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!params || !wbf16 || !X || !logits || B < 1) return lrs_fail(ctx, LRS_EINVAL, "mlp_forward: bad arguments");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, acts_bytes(B));
  if (st) return st;
  Acts a{};
  if (!alloc_acts(ctx, B, a)) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (mlp)");
  st = forward(ctx, params, wbf16, X, B, a);
  if (st) return st;
  LRS_CUDA_TRY(ctx, cudaMemcpyAsync(logits, a.Z3, sizeof(float) * (size_t)(B * kOut), cudaMemcpyDeviceToDevice,
                                    ctx->stream));
  return LRS_OK;
}

lrs_status lrs_mlp_loss_grad(lrs_ctx* ctx, const float* params, const uint16_t* wbf16, const float* X,
                             const int32_t* y, int64_t B, float* grad, float* loss) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!params || !wbf16 || !X || !y || !grad || !loss || B < 1)
    return lrs_fail(ctx, LRS_EINVAL, "mlp_loss_grad: bad arguments");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  lrs_status st = ws_reserve(ctx, acts_bytes(B));
  if (st) return st;
  Acts a{};
  if (!alloc_acts(ctx, B, a)) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (mlp)");
  st = forward(ctx, params, wbf16, X, B, a);
  if (st) return st;
  cudaStream_t s = ctx->stream;
  k_softmax_ce<<<blocks_for(B), 256, 0, s>>>(a.Z3, y, B, a.D3, a.L);
  k_sum_rows<<<1, 256, 0, s>>>(a.L, B, loss);
  // layer 3
  k_back_weight<<<blocks_for((int64_t)kOut * (kHid + 1)), 256, 0, s>>>(a.D3, a.H2, B, kOut, kHid, grad + oW3,
                                                                        grad + ob3);
  k_back_input<<<blocks_for(B * kHid), 256, 0, s>>>(a.D3, B, kOut, wbf16 + oW3, kHid, a.Z2, a.D2);
  // layer 2
  k_back_weight<<<blocks_for((int64_t)kHid * (kHid + 1)), 256, 0, s>>>(a.D2, a.H1, B, kHid, kHid, grad + oW2,
                                                                        grad + ob2);
  k_back_input<<<blocks_for(B * kHid), 256, 0, s>>>(a.D2, B, kHid, wbf16 + oW2, kHid, a.Z1, a.D1);
  // layer 1
  k_back_weight<<<blocks_for((int64_t)kHid * (kIn + 1)), 256, 0, s>>>(a.D1, X, B, kHid, kIn, grad + oW1,
                                                                       grad + ob1);
  ctx->launches += 7;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status lrs_mlp_adam(lrs_ctx* ctx, float* params, uint16_t* wbf16, const float* grad, float* m1, float* m2,
                        int64_t step, float lr) {
  if (!ctx) return LRS_EINVAL;
  ctx->err[0] = 0;
  if (!params || !wbf16 || !grad || !m1 || !m2 || step < 1) return lrs_fail(ctx, LRS_EINVAL, "mlp_adam: bad arguments");
  LRS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
  k_adam<<<blocks_for(kParams), 256, 0, ctx->stream>>>(params, wbf16, grad, m1, m2, lr, c1, c2);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // extern "C"
