// Deterministic sketch A_c = A_f D without forming D (paper Sec. 2, Table 1),
// the C-PWR column subsample A_f(:, I) (Alg. 7), and ||A_f||_F^2.
//
// Per axis the coarse point j sits at fine index c_j = s*j + s/2.
//   injection       : A_c[t, j] = A_f[t, c_j]                     (exact copy)
//   nearest neighbour: weights 1/4, 1/2, 1/4 at c_j-1, c_j, c_j+1, tensor
//                      product over axes; points outside the grid are zero
//   global sketch   : mean of the s^d points of the cell
// One thread produces one coarse value; a warp covers consecutive coarse x
// points of one snapshot row, so its loads walk one fine row with stride s.
// The traffic is the sectors the stencil touches (Table 1's "fraction of the
// fine grid used"), accumulated in FP64.
#include "common.cuh"
#include "internal.h"

#include <string.h>

namespace lrs {

bool grid_from_abi(const lrs_grid* g, GridDev* o, char* why, size_t nwhy) {
  if (!g) { snprintf(why, nwhy, "grid is NULL"); return false; }
  if (g->ndim < 1 || g->ndim > 3) { snprintf(why, nwhy, "grid ndim %d not in 1..3", g->ndim); return false; }
  if (g->kind < LRS_INJECT || g->kind > LRS_BLOCKAVG) { snprintf(why, nwhy, "bad stencil kind %d", g->kind); return false; }
  memset(o, 0, sizeof(*o));
  o->ndim = g->ndim; o->kind = g->kind; o->n = 1; o->l = 1;
  for (int d = 0; d < 3; ++d) {
    int64_t N = d < g->ndim ? g->N[d] : 1;
    int32_t s = d < g->ndim ? g->s[d] : 1;
    if (N < 1 || s < 1) { snprintf(why, nwhy, "axis %d: N=%lld s=%d must be >= 1", d, (long long)N, s); return false; }
    if (N % s != 0) { snprintf(why, nwhy, "axis %d: N=%lld not a multiple of s=%d", d, (long long)N, s); return false; }
    if (d < g->ndim && g->kind == LRS_FULLWEIGHT && s < 2) {
      snprintf(why, nwhy, "full weighting needs s >= 2 (axis %d has s=%d)", d, s); return false;
    }
    o->N[d] = N; o->s[d] = s; o->Nc[d] = N / s;
    o->n *= N; o->l *= N / s;
  }
  return true;
}

template <int KIND, typename OutT>
__global__ void __launch_bounds__(256) k_sketch(const void* __restrict__ A, int32_t dt, int64_t m,
                                                int64_t lda, GridDev g, OutT* __restrict__ Y,
                                                int64_t ldy) {
  const int64_t total = m * g.l;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / g.l, j = idx - t * g.l;
    const int64_t xc = j % g.Nc[0];
    const int64_t yc = (j / g.Nc[0]) % g.Nc[1];
    const int64_t zc = j / (g.Nc[0] * g.Nc[1]);
    const int64_t cx = g.s[0] * xc + g.s[0] / 2;
    const int64_t cy = g.s[1] * yc + g.s[1] / 2;
    const int64_t cz = g.s[2] * zc + g.s[2] / 2;
    const int64_t row = t * lda;
    double acc = 0.0;
    if (KIND == LRS_INJECT) {
      acc = ld_f64(A, dt, row + (cz * g.N[1] + cy) * g.N[0] + cx);
    } else if (KIND == LRS_FULLWEIGHT) {
      const int rz = g.ndim >= 3 ? 1 : 0, ry = g.ndim >= 2 ? 1 : 0;
      for (int dz = -rz; dz <= rz; ++dz) {
        const int64_t z = cz + dz;
        if (z < 0 || z >= g.N[2]) continue;
        const double wz = g.ndim >= 3 ? (dz == 0 ? 0.5 : 0.25) : 1.0;
        for (int dy = -ry; dy <= ry; ++dy) {
          const int64_t y = cy + dy;
          if (y < 0 || y >= g.N[1]) continue;
          const double wy = g.ndim >= 2 ? (dy == 0 ? 0.5 : 0.25) : 1.0;
          const int64_t base = row + (z * g.N[1] + y) * g.N[0];
          for (int dx = -1; dx <= 1; ++dx) {
            const int64_t x = cx + dx;
            if (x < 0 || x >= g.N[0]) continue;
            const double wx = dx == 0 ? 0.5 : 0.25;
            acc += (wz * (wy * wx)) * ld_f64(A, dt, base + x);
          }
        }
      }
    } else {  // block average
      const double wx = 1.0 / g.s[0], wy = g.ndim >= 2 ? 1.0 / g.s[1] : 1.0,
                   wz = g.ndim >= 3 ? 1.0 / g.s[2] : 1.0;
      const double w = wz * (wy * wx);
      for (int64_t z = g.s[2] * zc; z < g.s[2] * (zc + 1); ++z)
        for (int64_t y = g.s[1] * yc; y < g.s[1] * (yc + 1); ++y) {
          const int64_t base = row + (z * g.N[1] + y) * g.N[0];
          for (int64_t x = g.s[0] * xc; x < g.s[0] * (xc + 1); ++x) acc += w * ld_f64(A, dt, base + x);
        }
    }
    Y[t * ldy + j] = (OutT)acc;
  }
}

static int grid_blocks(lrs_ctx* ctx, int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)ctx->num_sms * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

lrs_status launch_sketch(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                         const GridDev& g, double* Y, int64_t ldy) {
  const int th = 256;
  const int nb = grid_blocks(ctx, m * g.l, th);
  switch (g.kind) {
    case LRS_INJECT: k_sketch<LRS_INJECT, double><<<nb, th, 0, ctx->stream>>>(A, dt, m, lda, g, Y, ldy); break;
    case LRS_FULLWEIGHT: k_sketch<LRS_FULLWEIGHT, double><<<nb, th, 0, ctx->stream>>>(A, dt, m, lda, g, Y, ldy); break;
    default: k_sketch<LRS_BLOCKAVG, double><<<nb, th, 0, ctx->stream>>>(A, dt, m, lda, g, Y, ldy); break;
  }
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_gather(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                         const GridDev& g, double* W, int64_t ldw) {
  GridDev gi = g;
  gi.kind = LRS_INJECT;
  return launch_sketch(ctx, A, dt, m, lda, gi, W, ldw);
}

lrs_status launch_gather32(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                           const GridDev& g, float* W, int64_t ldw) {
  GridDev gi = g;
  gi.kind = LRS_INJECT;
  const int nb = grid_blocks(ctx, m * gi.l, 256);
  k_sketch<LRS_INJECT, float><<<nb, 256, 0, ctx->stream>>>(A, dt, m, lda, gi, W, ldw);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// ---------------------------------------------------------------------------
// ||A||_F^2: per-block FP64 partials in a fixed order, then one block sums
// them (deterministic for a given device).
// ---------------------------------------------------------------------------
// rows are walked by blocks, columns by threads; float4 loads for FP32 rows
// aligned to 16 B, FP32 partial squares per row segment, FP64 across them.
__global__ void __launch_bounds__(256) k_fro2_partial(const void* __restrict__ A, int32_t dt,
                                                      int64_t m, int64_t n, int64_t lda,
                                                      double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  const bool vec = dt == LRS_F32 && (n % 4 == 0) && (lda % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  for (int64_t t = blockIdx.x; t < m; t += gridDim.x) {
    if (vec) {
      const float4* row = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(A) + t * lda);
      float s = 0.f;
      for (int64_t j = threadIdx.x; j < n / 4; j += blockDim.x) {
        const float4 v = __ldg(row + j);
        s = fmaf(v.x, v.x, s); s = fmaf(v.y, v.y, s); s = fmaf(v.z, v.z, s); s = fmaf(v.w, v.w, s);
      }
      acc += (double)s;
    } else {
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = ld_f64(A, dt, t * lda + j);
        acc = fma(v, v, acc);
      }
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_partials(const double* __restrict__ part, int np, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *out = acc;
}

lrs_status launch_sum(lrs_ctx* ctx, const double* part, int np, double* out) {
  k_sum_partials<<<1, 256, 0, ctx->stream>>>(part, np, out);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

lrs_status launch_fro2(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t n,
                       int64_t lda, double* out) {
  int64_t nb64 = m < (int64_t)ctx->num_sms * 8 ? m : (int64_t)ctx->num_sms * 8;
  const int nb = (int)(nb64 < 1 ? 1 : nb64);
  double* part = (double*)ws_alloc(ctx, sizeof(double) * nb);
  if (!part) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (fro2)");
  k_fro2_partial<<<nb, 256, 0, ctx->stream>>>(A, dt, m, n, lda, part);
  k_sum_partials<<<1, 256, 0, ctx->stream>>>(part, nb, out);
  ctx->launches += 2;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
