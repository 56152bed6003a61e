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

// One thread per coarse point j and group of kSkRows snapshots: the stencil
// offsets (32-bit: a row holds < 2^31 elements, checked on the host) are
// computed once and reused for every snapshot of the group, whose loads are
// independent and in flight together.  The accumulation order per value is
// fixed (z, then y, then x), the same for every snapshot and launch shape.
constexpr int kSkRows = 4;

template <int KIND, typename OutT>
__global__ void __launch_bounds__(256) k_sketch(const void* __restrict__ A, int32_t dt, int64_t m,
                                                int64_t lda, GridDev g, OutT* __restrict__ Y,
                                                int64_t ldy) {
  const uint32_t l = (uint32_t)g.l, Ncx = (uint32_t)g.Nc[0], Ncy = (uint32_t)g.Nc[1];
  const uint32_t Nx = (uint32_t)g.N[0], Ny = (uint32_t)g.N[1], Nz = (uint32_t)g.N[2];
  const uint32_t sx = (uint32_t)g.s[0], sy = (uint32_t)g.s[1], sz = (uint32_t)g.s[2];
  for (int64_t t0 = (int64_t)blockIdx.y * kSkRows; t0 < m; t0 += (int64_t)gridDim.y * kSkRows) {
    const int nt = (int)min((int64_t)kSkRows, m - t0);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < l; j += gridDim.x * blockDim.x) {
      const uint32_t xc = j % Ncx, rest = j / Ncx;
      const uint32_t yc = rest % Ncy, zc = rest / Ncy;
      const uint32_t cx = sx * xc + sx / 2, cy = sy * yc + sy / 2, cz = sz * zc + sz / 2;
      double acc[kSkRows];
#pragma unroll
      for (int u = 0; u < kSkRows; ++u) acc[u] = 0.0;
      if (KIND == LRS_INJECT) {
        const uint32_t off = (cz * Ny + cy) * Nx + cx;
#pragma unroll
        for (int u = 0; u < kSkRows; ++u)
          if (u < nt) {
            // an FP32 output takes the value straight through (the compiler
            // folds the widening away); an FP64 one widens on the integer pipe
            if (sizeof(OutT) == 4) acc[u] = ld_f64(A, dt, (t0 + u) * lda + off);
            else acc[u] = ld_wide(A, dt, (t0 + u) * lda + off);
          }
      } else if (KIND == LRS_FULLWEIGHT) {
        const int rz = g.ndim >= 3 ? 1 : 0, ry = g.ndim >= 2 ? 1 : 0;
        for (int dz = -rz; dz <= rz; ++dz) {
          const int64_t z = (int64_t)cz + dz;
          if (z < 0 || z >= Nz) continue;
          const double wz = g.ndim >= 3 ? (dz == 0 ? 0.5 : 0.25) : 1.0;
          for (int dy = -ry; dy <= ry; ++dy) {
            const int64_t y = (int64_t)cy + dy;
            if (y < 0 || y >= Ny) continue;
            const double wy = g.ndim >= 2 ? (dy == 0 ? 0.5 : 0.25) : 1.0;
            const uint32_t base = ((uint32_t)z * Ny + (uint32_t)y) * Nx;
            for (int dx = -1; dx <= 1; ++dx) {
              const int64_t x = (int64_t)cx + dx;
              if (x < 0 || x >= Nx) continue;
              const double w = wz * (wy * (dx == 0 ? 0.5 : 0.25));
              const uint32_t off = base + (uint32_t)x;
              double v[kSkRows];
#pragma unroll
              for (int u = 0; u < kSkRows; ++u) v[u] = u < nt ? ld_wide(A, dt, (t0 + u) * lda + off) : 0.0;
#pragma unroll
              for (int u = 0; u < kSkRows; ++u) acc[u] += w * v[u];
            }
          }
        }
      } else {  // block average
        const double wx = 1.0 / sx, wy = g.ndim >= 2 ? 1.0 / sy : 1.0, wz = g.ndim >= 3 ? 1.0 / sz : 1.0;
        const double w = wz * (wy * wx);
        for (uint32_t z = sz * zc; z < sz * (zc + 1); ++z)
          for (uint32_t y = sy * yc; y < sy * (yc + 1); ++y) {
            const uint32_t base = (z * Ny + y) * Nx;
            for (uint32_t x = sx * xc; x < sx * (xc + 1); ++x) {
#pragma unroll
              for (int u = 0; u < kSkRows; ++u)
                if (u < nt) acc[u] += w * ld_wide(A, dt, (t0 + u) * lda + base + x);
            }
          }
      }
#pragma unroll
      for (int u = 0; u < kSkRows; ++u)
        if (u < nt) Y[(t0 + u) * ldy + j] = (OutT)acc[u];
    }
  }
}

// grid: x over coarse points (256 per block), y over groups of kSkRows
// snapshots, about 16 blocks per SM in total
static dim3 sketch_grid(lrs_ctx* ctx, int64_t m, int64_t l) {
  int64_t bx = (l + 255) / 256;
  if (bx > 4096) bx = 4096;
  if (bx < 1) bx = 1;
  int64_t by = ((int64_t)ctx->num_sms * 16 + bx - 1) / bx;
  const int64_t groups = (m + kSkRows - 1) / kSkRows;
  if (by > groups) by = groups;
  if (by > 65535) by = 65535;
  if (by < 1) by = 1;
  return dim3((unsigned)bx, (unsigned)by);
}

static bool sketch_sizes_ok(lrs_ctx* ctx, const GridDev& g) {
  if (g.n >= (int64_t)1 << 31 || g.l >= (int64_t)1 << 31) {
    lrs_fail(ctx, LRS_EINVAL, "sketch: a snapshot of %lld points exceeds 2^31", (long long)g.n);
    return false;
  }
  return true;
}

lrs_status launch_sketch(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                         const GridDev& g, double* Y, int64_t ldy) {
  if (!sketch_sizes_ok(ctx, g)) return LRS_EINVAL;
  const dim3 grid = sketch_grid(ctx, m, g.l);
  switch (g.kind) {
    case LRS_INJECT: k_sketch<LRS_INJECT, double><<<grid, 256, 0, ctx->stream>>>(A, dt, m, lda, g, Y, ldy); break;
    case LRS_FULLWEIGHT: k_sketch<LRS_FULLWEIGHT, double><<<grid, 256, 0, ctx->stream>>>(A, dt, m, lda, g, Y, ldy); break;
    default: k_sketch<LRS_BLOCKAVG, double><<<grid, 256, 0, ctx->stream>>>(A, dt, m, lda, g, Y, ldy); break;
  }
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

// W = A_f(:, I) and its transpose W^T in one pass (FP32 outputs; WT NULL:
// W alone): a thread
// takes one subsample point j and 8 consecutive snapshots, writes W[t, j]
// (coalesced over j) and the 8 values W^T[j, t0..t0+7] as 32 contiguous
// bytes (two 16-byte stores when the row stride and base allow).
constexpr int kGtRows = 8;

__global__ void __launch_bounds__(256) k_gather_both(const void* __restrict__ A, int32_t dt, int64_t m,
                                                     int64_t lda, GridDev g, float* __restrict__ W, int64_t ldw,
                                                     float* __restrict__ WT, int64_t ldwt, int vec) {
  const uint32_t l = (uint32_t)g.l, Ncx = (uint32_t)g.Nc[0], Ncy = (uint32_t)g.Nc[1];
  const uint32_t Nx = (uint32_t)g.N[0], Ny = (uint32_t)g.N[1];
  const uint32_t sx = (uint32_t)g.s[0], sy = (uint32_t)g.s[1], sz = (uint32_t)g.s[2];
  for (int64_t t0 = (int64_t)blockIdx.y * kGtRows; t0 < m; t0 += (int64_t)gridDim.y * kGtRows) {
    const int nt = (int)min((int64_t)kGtRows, m - t0);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < l; j += gridDim.x * blockDim.x) {
      const uint32_t xc = j % Ncx, rest = j / Ncx;
      const uint32_t yc = rest % Ncy, zc = rest / Ncy;
      const uint32_t off = ((sz * zc + sz / 2) * Ny + (sy * yc + sy / 2)) * Nx + (sx * xc + sx / 2);
      float v[kGtRows];
#pragma unroll
      for (int u = 0; u < kGtRows; ++u) v[u] = u < nt ? (float)ld_f64(A, dt, (t0 + u) * lda + off) : 0.f;
#pragma unroll
      for (int u = 0; u < kGtRows; ++u)
        if (u < nt) W[(t0 + u) * ldw + j] = v[u];
      if (!WT) continue;                 // W alone (lrs_touch)
      float* dst = WT + (int64_t)j * ldwt + t0;
      if (vec && nt == kGtRows) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
      } else {
#pragma unroll
        for (int u = 0; u < kGtRows; ++u)
          if (u < nt) dst[u] = v[u];
      }
    }
  }
}

lrs_status launch_gather32_both(lrs_ctx* ctx, const void* A, int32_t dt, int64_t m, int64_t lda,
                                const GridDev& g, float* W, int64_t ldw, float* WT, int64_t ldwt) {
  GridDev gi = g;
  gi.kind = LRS_INJECT;
  if (!sketch_sizes_ok(ctx, gi)) return LRS_EINVAL;
  int64_t bx = (gi.l + 255) / 256;
  if (bx > 4096) bx = 4096;
  if (bx < 1) bx = 1;
  int64_t by = ((int64_t)ctx->num_sms * 16 + bx - 1) / bx;
  const int64_t groups = (m + kGtRows - 1) / kGtRows;
  if (by > groups) by = groups;
  if (by > 65535) by = 65535;
  if (by < 1) by = 1;
  const int vec = (ldwt % 4 == 0) && ((reinterpret_cast<uintptr_t>(WT) & 15) == 0) ? 1 : 0;
  k_gather_both<<<dim3((unsigned)bx, (unsigned)by), 256, 0, ctx->stream>>>(A, dt, m, lda, gi, W, ldw, WT, ldwt, vec);
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


// ---------------------------------------------------------------------------
// ||A||_F^2: per-block FP64 partials in a fixed order, then one block sums
// them (deterministic for a given device).
// ---------------------------------------------------------------------------
// rows are walked by blocks, columns by threads; float4 loads for FP32 rows
// aligned to 16 B, FP32 partial squares per row segment, FP64 across them.
__global__ void __launch_bounds__(256) k_fro2_partial(const void* __restrict__ A, int32_t dt,
                                                      int64_t m, int64_t n, int64_t lda,
                                                      double* __restrict__ part, int exact) {
  __shared__ double red[32];
  double acc = 0.0;
  const bool vec = !exact && dt == LRS_F32 && (n % 4 == 0) && (lda % 4 == 0) &&
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
                       int64_t lda, double* out, int exact) {
  int64_t nb64 = m < (int64_t)ctx->num_sms * 8 ? m : (int64_t)ctx->num_sms * 8;
  const int nb = (int)(nb64 < 1 ? 1 : nb64);
  double* part = (double*)ws_alloc(ctx, sizeof(double) * nb);
  if (!part) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (fro2)");
  k_fro2_partial<<<nb, 256, 0, ctx->stream>>>(A, dt, m, n, lda, part, exact);
  k_sum_partials<<<1, 256, 0, ctx->stream>>>(part, nb, out);
  ctx->launches += 2;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  return LRS_OK;
}

}  // namespace lrs
