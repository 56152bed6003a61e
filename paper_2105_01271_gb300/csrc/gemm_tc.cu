// Tensor-core (tcgen05) forms of C = alpha * X^T A  (the A-pass B = Q^T A_f of
// paper Alg. 2 and the C-PWR products W^T G, W T of Alg. 7).
//
// Precision: every operand is split into BF16 pieces, x = x_0 + x_1 (+ x_2),
// and the products x_i a_j with i + j below the number of pieces are summed
// by tcgen05.mma in FP32 (TMEM).  Two pieces (LRS_PREC_SPLIT_BF16) carry 16
// significant bits of each operand, three (LRS_PREC_BF16X3) 24 bits; BF16
// data is exact in one piece.
//
// Data flow of one persistent CTA (one per SM, 320 threads):
//   warps 0-7  convert: stream a 64 x 128 slab of A (row-major, 128 consecutive
//              columns per row -> coalesced) from global memory, split it and
//              write the BF16 pieces into shared memory in the K-major
//              128-byte-swizzled UMMA layout; later read the accumulator out
//              of TMEM and store C.
//   warp 8     allocates TMEM and issues the MMAs (one thread).
//   warp 9     copies the pre-split X pieces (already in the shared-memory
//              image, prepared once per call by k_prep_x) with one bulk copy
//              per stage.
// Stages are guarded by mbarriers; all waits are bounded (LRS_ETIMEOUT).
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"
#include "bf16_split.cuh"

#include <cuda_bf16.h>

namespace lrs {

using namespace tc;

constexpr int TBM = 128;          // UMMA M (X columns -> rows of C)
constexpr int TBN = 128;          // UMMA N (A columns -> columns of C)
constexpr int TBK = 64;           // K per stage (one 128-byte swizzle row of BF16)
constexpr int kPieceBytes = TBM * TBK * 2;   // 16 KB per operand piece per stage
constexpr int kConvWarps = 8;
constexpr int kThreads = (kConvWarps + 2) * 32;

// ---------------------------------------------------------------------------
// X (K x M, row-major) -> pieces in the shared-memory image:
//   out[((mt * Kt + kt) * SX + piece) * 16 KB + sw128_offset(row, k)]
// one thread per (tile row, 8-wide k chunk)
// ---------------------------------------------------------------------------
template <int SX>
__global__ void __launch_bounds__(256) k_prep_x(const void* __restrict__ X, int32_t xdt, int64_t ldx,
                                                int64_t K, int64_t M, int64_t Mt, int64_t Kt,
                                                uint8_t* __restrict__ out) {
  const int64_t total = Mt * Kt * TBM * 8;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(id % TBM);
    const int64_t rest = id / TBM;
    const int c = (int)(rest % 8);
    const int64_t tk = rest / 8;              // mt * Kt + kt
    const int64_t kt = tk % Kt, mt = tk / Kt;
    const int64_t m = mt * TBM + row;
    uint32_t w[SX][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      __nv_bfloat16 p0[SX], p1[SX];
      const int64_t k0 = kt * TBK + c * 8 + e;
      split_any<SX>(X, xdt, k0 * ldx + m, (k0 < K && m < M), p0);
      split_any<SX>(X, xdt, (k0 + 1) * ldx + m, (k0 + 1 < K && m < M), p1);
#pragma unroll
      for (int s = 0; s < SX; ++s) w[s][e >> 1] = pack2(p0[s], p1[s]);
    }
    uint8_t* blk = out + (tk * SX) * (int64_t)kPieceBytes;
#pragma unroll
    for (int s = 0; s < SX; ++s) {
      uint4* dst = reinterpret_cast<uint4*>(blk + (int64_t)s * kPieceBytes + sw128_offset(row, c * 8));
      *dst = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// ---------------------------------------------------------------------------
// main kernel
// ---------------------------------------------------------------------------
struct TcParams {
  int64_t M, N, K;
  const uint8_t* Xp;        // pre-split X pieces
  const uint8_t* Ap;        // pre-split A pieces (same image layout, by (nt, kt)); NULL: split in the CTA
  const void* A; int32_t adt; int64_t lda;
  void* C; int c_f64; int c_trans; int64_t ldc;
  double alpha;
  int accum;
  int64_t Mt, Nt, Kt;
  int64_t splits, KS;       // split-K: K-tile chunks of KS tiles; splits > 1 -> FP32 partials
  float* partial;           // splits x M x N (row-major) when splits > 1
  int* err;
  double* fro2_part;        // optional: per-CTA partial sums of A^2 (only when Mt == 1)
};

template <int ADT, int SA, int SX, int NS>
struct TcCfg {
  static constexpr int kStageBytes = (SA + SX) * kPieceBytes;
  static constexpr int kP = SA > SX ? SA : SX;
  static constexpr int kSmem = NS * kStageBytes + 1024 + 256;
};

template <int ADT>
__device__ __forceinline__ void load_a8(const void* A, int64_t lda, int64_t k0, int64_t K, int64_t n,
                                        int64_t N, float (&v)[8]) {
  const bool nok = n < N;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t k = k0 + e;
    float x = 0.f;
    if (nok && k < K) {
      if (ADT == LRS_F32) x = __ldg(reinterpret_cast<const float*>(A) + k * lda + n);
      else {
        const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(A) + k * lda + n);
        x = __uint_as_float(((unsigned)b) << 16);
      }
    }
    v[e] = x;
  }
}
__device__ __forceinline__ void load_a8_f64(const void* A, int64_t lda, int64_t k0, int64_t K, int64_t n,
                                            int64_t N, double (&v)[8]) {
  const bool nok = n < N;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t k = k0 + e;
    v[e] = (nok && k < K) ? __ldg(reinterpret_cast<const double*>(A) + k * lda + n) : 0.0;
  }
}

template <int ADT, int SA, int SX, int NS>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(TcParams P) {
  using Cfg = TcCfg<ADT, SA, SX, NS>;
  using VT = typename std::conditional<ADT == LRS_F64, double, float>::type;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_a[NS], full_x[NS], empty[NS], tmem_full[2], tmem_empty[2];
  __shared__ uint32_t tmem_base_sh;

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  uint8_t* smem = smem_raw + pad;                      // 1024-B aligned stage buffers
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = P.Mt * P.Nt * P.splits;
  // tile -> (split, mt, nt).  One row tile: nt fastest.  Several: mt fastest,
  // so the CTAs that need the same A columns (every row tile of one nt) run
  // side by side and the A slab comes from HBM once, from L2 for the others.
  const bool mfast = P.Mt > 1;
  auto tile_nt = [&](int64_t tile) -> int64_t { return mfast ? (tile / P.Mt) % P.Nt : tile % P.Nt; };
  auto tile_mt = [&](int64_t tile) -> int64_t { return mfast ? tile % P.Mt : (tile / P.Nt) % P.Mt; };
  auto kt_range = [&](int64_t tile, int64_t& lo, int64_t& hi) {
    const int64_t ks = tile / (P.Mt * P.Nt);
    lo = ks * P.KS;
    hi = min(P.Kt, lo + P.KS);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full_a[s], kConvWarps);
      mbar_init(&full_x[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tmem_full[b], 1);
      mbar_init(&tmem_empty[b], kConvWarps);
    }
    fence_mbar_init();
  }
  // two accumulators: the epilogue of one tile runs under the MMAs of the next
  if (warp == kConvWarps) tmem_alloc(&tmem_base_sh, 2 * TBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp < kConvWarps) {
    // ---------------- converters + epilogue ----------------
    const int t = threadIdx.x;
    const int nl = t & (TBN - 1);           // row of the B operand tile (column of C)
    const int ch = t >> 7;                  // 0/1: chunks {ch, ch+2, ch+4, ch+6}
    int64_t it = 0;
    int tcount = 0;
    bool ok = true;
    VT cur[4][8];
    bool have_cur = false;
    double fro2 = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tcount) {
      const int64_t nt = tile_nt(tile), mt = tile_mt(tile);
      const int64_t n = nt * TBN + nl;
      int64_t kt_lo, kt_hi;
      kt_range(tile, kt_lo, kt_hi);
      if (!have_cur && !P.Ap) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t k0 = kt_lo * TBK + (int64_t)(ch + 2 * i) * 8;
          if constexpr (ADT == LRS_F64) load_a8_f64(P.A, P.lda, k0, P.K, n, P.N, cur[i]);
          else load_a8<ADT>(P.A, P.lda, k0, P.K, n, P.N, cur[i]);
        }
      }
      for (int64_t kt = kt_lo; kt < kt_hi && !P.Ap; ++kt, ++it) {
        // prefetch the next slab (next k-tile of this tile, or the first of the next tile)
        VT nxt[4][8];
        const bool last = (kt + 1 == kt_hi);
        const int64_t ntile = tile + gridDim.x;
        const bool pf = !last || ntile < ntiles;
        if (pf) {
          int64_t kt2 = kt + 1;
          if (last) { int64_t h2; kt_range(ntile, kt2, h2); }
          const int64_t n2 = last ? (tile_nt(ntile) * TBN + nl) : n;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int64_t k0 = kt2 * TBK + (int64_t)(ch + 2 * i) * 8;
            if constexpr (ADT == LRS_F64) load_a8_f64(P.A, P.lda, k0, P.K, n2, P.N, nxt[i]);
            else load_a8<ADT>(P.A, P.lda, k0, P.K, n2, P.N, nxt[i]);
          }
        }
        const int s = (int)(it % NS);
        const uint32_t ph = (uint32_t)((it / NS) & 1);
        {
          // one lane waits, the warp follows its verdict (warp-uniform exit)
          int w_ok = 1;
          if (lane == 0) w_ok = mbar_wait(&empty[s], ph ^ 1u, P.err) ? 1 : 0;
          w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
          if (!w_ok) { ok = false; break; }
        }
        uint8_t* abase = smem + (size_t)s * Cfg::kStageBytes;
        if (P.fro2_part) {
          // ||A||_F^2 rides along with the one read of A (FP32 per slab, FP64 across slabs)
          float sq = 0.f;
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int e = 0; e < 8; ++e) sq = fmaf((float)cur[i][e], (float)cur[i][e], sq);
          fro2 += (double)sq;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = ch + 2 * i;
          uint32_t w[SA][4];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            __nv_bfloat16 p0[SA], p1[SA];
            if constexpr (ADT == LRS_F64) {
              split_f64<SA>(cur[i][e], p0);
              split_f64<SA>(cur[i][e + 1], p1);
            } else {
              split_f32<SA>(cur[i][e], p0);
              split_f32<SA>(cur[i][e + 1], p1);
            }
#pragma unroll
            for (int q = 0; q < SA; ++q) w[q][e >> 1] = pack2(p0[q], p1[q]);
          }
#pragma unroll
          for (int q = 0; q < SA; ++q) {
            uint4* dst = reinterpret_cast<uint4*>(abase + q * kPieceBytes + sw128_offset(nl, c * 8));
            *dst = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full_a[s]);
        if (pf) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int e = 0; e < 8; ++e) cur[i][e] = nxt[i][e];
        }
        have_cur = pf;
      }
      if (!ok) break;
      // ---------------- epilogue: TMEM -> C ----------------
      const int abuf = tcount & 1;
      {
        int w_ok = 1;
        if (lane == 0) w_ok = mbar_wait(&tmem_full[abuf], (uint32_t)((tcount >> 1) & 1), P.err) ? 1 : 0;
        w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
        if (!w_ok) { ok = false; break; }
      }
      tc_fence_after();
      const int q4 = warp & 3, half = warp >> 2;
      const int64_t m = mt * TBM + q4 * 32 + lane;
      // FP32 C with alpha = 1 and no accumulation: the values as they are (the
      // FP64 route below rounds 1.0 * v back to v), 16-byte stores when aligned
      const bool plain = !P.c_f64 && !P.accum && !P.c_trans && P.alpha == 1.0 && P.splits == 1;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t v[16];
        const int col = half * 64 + j * 16;
        tmem_ld16(tmem + (uint32_t)(abuf * TBN) + ((uint32_t)(q4 * 32) << 16) + (uint32_t)col, v);
        tmem_ld_wait();
        if (m < P.M) {
          const int64_t nb = nt * TBN + col;
          if (plain) {
            float* c = reinterpret_cast<float*>(P.C) + m * P.ldc + nb;
            if (nb + 16 <= P.N && ((reinterpret_cast<uintptr_t>(c) & 15u) == 0)) {
#pragma unroll
              for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4*>(c + e) = make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                                                __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (nb + e < P.N) c[e] = __uint_as_float(v[e]);
            }
          } else if (P.splits > 1) {
            float* dst = P.partial + ((tile / (P.Mt * P.Nt)) * P.M + m) * P.N;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int64_t nn = nb + e;
              if (nn >= P.N) break;
              dst[nn] = __uint_as_float(v[e]);
            }
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int64_t nn = nb + e;
              if (nn >= P.N) break;
              const double val = P.alpha * (double)__uint_as_float(v[e]);
              const int64_t off = P.c_trans ? nn * P.ldc + m : m * P.ldc + nn;
              if (P.c_f64) {
                double* c = reinterpret_cast<double*>(P.C) + off;
                *c = P.accum ? *c + val : val;
              } else {
                float* c = reinterpret_cast<float*>(P.C) + off;
                *c = P.accum ? (float)((double)*c + val) : (float)val;
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tmem_empty[abuf]);
    }
    if (P.fro2_part) {
      // per-CTA partial of ||A||_F^2 (fixed reduction order -> deterministic)
      __shared__ double red_f[kConvWarps];
      double v = warp_sum(fro2);
      if (lane == 0) red_f[warp] = v;
      asm volatile("bar.sync 1, %0;" ::"r"(kConvWarps * 32) : "memory");   // converter warps only
      if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < kConvWarps; ++w) tsum += red_f[w];
        P.fro2_part[blockIdx.x] = tsum;
      }
    }
  } else if (warp == kConvWarps) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(TBM, TBN);
      int64_t it = 0;
      int tcount = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tcount) {
        const int abuf = tcount & 1;
        if (!mbar_wait(&tmem_empty[abuf], (uint32_t)(((tcount >> 1) & 1) ^ 1), P.err)) break;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(abuf * TBN);
        int64_t kt_lo, kt_hi;
        kt_range(tile, kt_lo, kt_hi);
        for (int64_t kt = kt_lo; kt < kt_hi; ++kt, ++it) {
          const int s = (int)(it % NS);
          const uint32_t ph = (uint32_t)((it / NS) & 1);
          if (!mbar_wait(&full_x[s], ph, P.err) || (!P.Ap && !mbar_wait(&full_a[s], ph, P.err))) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + (size_t)s * Cfg::kStageBytes);   // A-data pieces (UMMA B)
          const uint32_t x0 = a0 + SA * kPieceBytes;                           // X pieces (UMMA A)
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            int first = (kt == kt_lo && kk == 0) ? 1 : 0;
#pragma unroll
            for (int i = 0; i < SA; ++i)
#pragma unroll
              for (int j = 0; j < SX; ++j) {
                if (i + j >= Cfg::kP) continue;
                const uint64_t ad = sdesc_kmajor_sw128(x0 + j * kPieceBytes + kk * 32);
                const uint64_t bd = sdesc_kmajor_sw128(a0 + i * kPieceBytes + kk * 32);
                umma_bf16(dacc, ad, bd, idesc, first ? 0u : 1u);
                first = 0;
              }
          }
          umma_commit(&empty[s]);
        }
        if (!ok) break;
        umma_commit(&tmem_full[abuf]);
      }
    }
    __syncwarp();
  } else {
    // ---------------- X-piece loader ----------------
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t mt = tile_mt(tile), nt = tile_nt(tile);
        int64_t kt_lo, kt_hi;
        kt_range(tile, kt_lo, kt_hi);
        bool ok = true;
        for (int64_t kt = kt_lo; kt < kt_hi; ++kt, ++it) {
          const int s = (int)(it % NS);
          const uint32_t ph = (uint32_t)((it / NS) & 1);
          if (!mbar_wait(&empty[s], ph ^ 1u, P.err)) { ok = false; break; }
          uint8_t* xdst = smem + (size_t)s * Cfg::kStageBytes + SA * kPieceBytes;
          const uint8_t* xsrc = P.Xp + ((mt * P.Kt + kt) * SX) * (int64_t)kPieceBytes;
          if (P.Ap) {
            // both operands pre-split: one barrier completes on both copies
            uint8_t* adst = smem + (size_t)s * Cfg::kStageBytes;
            const uint8_t* asrc = P.Ap + ((nt * P.Kt + kt) * SA) * (int64_t)kPieceBytes;
            mbar_arrive_expect_tx(&full_x[s], (SX + SA) * kPieceBytes);
            bulk_g2s(adst, asrc, SA * kPieceBytes, &full_x[s]);
          } else {
            mbar_arrive_expect_tx(&full_x[s], SX * kPieceBytes);
          }
          bulk_g2s(xdst, xsrc, SX * kPieceBytes, &full_x[s]);
        }
        if (!ok) {
          // wait (bounded) for the copies still in flight before leaving
          for (int b = 0; b < NS && it - 1 - b >= 0; ++b) {
            const int64_t j = it - 1 - b;
            mbar_wait_quiet(&full_x[j % NS], (uint32_t)((j / NS) & 1));
          }
          break;
        }
      }
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kConvWarps) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * TBN);
  }
}

// ---------------------------------------------------------------------------
// C = alpha * sum_s partial[s] in a fixed order (deterministic split-K)
__global__ void k_splitk_reduce(const float* __restrict__ part, int64_t splits, int64_t M, int64_t N,
                                double alpha, void* __restrict__ C, int c_f64, int c_trans, int64_t ldc, int accum) {
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t s = 0; s < splits; ++s) acc += (double)part[s * total + e];
    const int64_t m = e / N, nn = e - m * N;
    const int64_t off = c_trans ? nn * ldc + m : m * ldc + nn;
    if (c_f64) {
      double* c = reinterpret_cast<double*>(C) + off;
      *c = accum ? *c + alpha * acc : alpha * acc;
    } else {
      float* c = reinterpret_cast<float*>(C) + off;
      *c = accum ? (float)((double)*c + alpha * acc) : (float)(alpha * acc);
    }
  }
}

// number of K splits: enough tiles to fill the SMs, at least 8 K-tiles each
static int64_t choose_splits(int64_t tiles, int64_t Kt, int num_sms) {
  if (tiles >= num_sms / 2) return 1;
  int64_t s = num_sms / tiles;
  if (s > Kt / 8) s = Kt / 8;
  return s < 1 ? 1 : s;
}

size_t gemm_tc_splitk_workspace(int64_t M, int64_t N, int64_t K, int num_sms) {
  const int64_t tiles = ((M + TBM - 1) / TBM) * ((N + TBN - 1) / TBN);
  const int64_t s = choose_splits(tiles, (K + TBK - 1) / TBK, num_sms);
  return s > 1 ? (size_t)(s * M * N) * sizeof(float) + 256 : 0;
}

template <int ADT, int SA, int SX>
static lrs_status run_tc(lrs_ctx* ctx, const GemmArgs& a, double* fro2_out) {
  constexpr int NS = (SA + SX) <= 4 ? 3 : 2;
  using Cfg = TcCfg<ADT, SA, SX, NS>;
  // everything taken from the workspace below is dead once the launches are
  // queued (one stream): give it back on return
  const size_t ws_mark = ctx->ws_top;
  TcParams P{};
  P.M = a.M; P.N = a.N; P.K = a.K;
  P.A = a.A; P.adt = a.adt; P.lda = a.lda;
  P.C = a.C; P.c_f64 = a.c_f64; P.c_trans = a.c_trans; P.ldc = a.ldc; P.alpha = a.alpha; P.accum = a.accum;
  P.Mt = (a.M + TBM - 1) / TBM; P.Nt = (a.N + TBN - 1) / TBN; P.Kt = (a.K + TBK - 1) / TBK;
  P.splits = fro2_out ? 1 : choose_splits(P.Mt * P.Nt, P.Kt, ctx->num_sms);
  P.KS = (P.Kt + P.splits - 1) / P.splits;
  P.splits = (P.Kt + P.KS - 1) / P.KS;
  if (P.splits > 1) {
    P.partial = (float*)ws_alloc(ctx, sizeof(float) * (size_t)(P.splits * a.M * a.N));
    if (!P.partial) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (split-K partials)");
  }
  const size_t xbytes = (size_t)(P.Mt * P.Kt * SX) * kPieceBytes;
  uint8_t* Xp = (uint8_t*)ws_alloc(ctx, xbytes);
  int* err = (int*)ws_alloc(ctx, 256);
  if (!Xp || !err) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (tensor-core gemm: %zu B)", xbytes);
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 256, ctx->stream));
  {
    const int64_t total = P.Mt * P.Kt * TBM * 8;
    int64_t nb = (total + 255) / 256;
    if (nb > (int64_t)ctx->num_sms * 32) nb = (int64_t)ctx->num_sms * 32;
    k_prep_x<SX><<<(unsigned)nb, 256, 0, ctx->stream>>>(a.X, a.xdt, a.ldx, a.K, a.M, P.Mt, P.Kt, Xp);
    ctx->launches++;
  }
  P.Xp = Xp;
  P.err = err;
  // with two or more row tiles every CTA row would split the same A slabs
  // again: split A once into the same image (when the workspace has room)
  P.Ap = nullptr;
  if (P.Mt >= 2 && !fro2_out) {
    const size_t abytes = (size_t)(P.Nt * P.Kt * SA) * kPieceBytes;
    uint8_t* Ap = (uint8_t*)ws_alloc(ctx, abytes);
    if (Ap) {
      const int64_t total = P.Nt * P.Kt * TBM * 8;
      int64_t nb = (total + 255) / 256;
      if (nb > (int64_t)ctx->num_sms * 32) nb = (int64_t)ctx->num_sms * 32;
      k_prep_x<SA><<<(unsigned)nb, 256, 0, ctx->stream>>>(a.A, a.adt, a.lda, a.K, a.N, P.Nt, P.Kt, Ap);
      ctx->launches++;
      P.Ap = Ap;
    }
  }
  double* part = nullptr;
  if (fro2_out) {
    if (P.Mt != 1) return lrs_fail(ctx, LRS_EINVAL, "gemm: fused ||A||^2 needs M <= %d", TBM);
    part = (double*)ws_alloc(ctx, sizeof(double) * (size_t)ctx->num_sms);
    if (!part) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (tensor-core gemm)");
  }
  P.fro2_part = part;
  auto kern = k_gemm_tc<ADT, SA, SX, NS>;
  { const lrs_status _s = raise_dyn_smem(ctx, (const void*)kern, (size_t)(Cfg::kSmem)); if (_s) return _s; }
  const int64_t ntiles = P.Mt * P.Nt * P.splits;
  const unsigned grid = (unsigned)(ntiles < ctx->num_sms ? ntiles : ctx->num_sms);
  const bool timing = ctx->time_kernels && ctx->kev0 && ctx->kev1;
  if (timing) LRS_CUDA_TRY(ctx, cudaEventRecord(ctx->kev0, ctx->stream));
  kern<<<grid, kThreads, Cfg::kSmem, ctx->stream>>>(P);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  if (timing) LRS_CUDA_TRY(ctx, cudaEventRecord(ctx->kev1, ctx->stream));
  if (P.splits > 1) {
    const int64_t tot = a.M * a.N;
    int64_t nb = (tot + 255) / 256;
    if (nb > (int64_t)ctx->num_sms * 8) nb = (int64_t)ctx->num_sms * 8;
    k_splitk_reduce<<<(unsigned)nb, 256, 0, ctx->stream>>>(P.partial, P.splits, a.M, a.N, a.alpha, a.C,
                                                            a.c_f64, a.c_trans, a.ldc, a.accum);
    ctx->launches++;
    LRS_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (fro2_out) {
    lrs_status st = launch_sum(ctx, part, (int)grid, fro2_out);
    if (st) return st;
  }
  int* h = (int*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {(const int32_t*)err};
    const lrs_status rs = replay_ints(ctx, 1, d, h + 16);
    if (rs) return rs;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 16, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[16] != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "tensor-core gemm: a pipeline wait gave up");
  if (timing) {
    float ms = 0.f;
    LRS_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->kev0, ctx->kev1));
    ctx->last_kernel_ms = ms;
  }
  ctx->ws_top = ws_mark;
  return LRS_OK;
}

size_t gemm_tc_a_workspace(int64_t N, int64_t K, int prec) {
  const int64_t Nt = (N + TBN - 1) / TBN, Kt = (K + TBK - 1) / TBK;
  const int sa = prec == LRS_PREC_BF16X3 ? 3 : 2;
  return (size_t)(Nt * Kt * sa) * kPieceBytes + 512;
}

size_t gemm_tc_workspace(int64_t M, int64_t K, int prec) {
  const int64_t Mt = (M + TBM - 1) / TBM, Kt = (K + TBK - 1) / TBK;
  const int sx = prec == LRS_PREC_BF16X3 ? 3 : 2;
  const size_t generic = (size_t)(Mt * Kt * sx) * kPieceBytes + 1024 + 512;
  const size_t narrow = apass_workspace(M, K, prec);
  return generic > narrow ? generic : narrow;
}

lrs_status launch_gemm_tc(lrs_ctx* ctx, const GemmArgs& a, int prec, double* fro2_out) {
  if (a.M <= 0 || a.N <= 0) return LRS_OK;
  if (a.K <= 0) return lrs_fail(ctx, LRS_EINVAL, "gemm: K must be >= 1 on the tensor-core path");
  const bool three = prec == LRS_PREC_BF16X3;
  if (prec != LRS_PREC_SPLIT_BF16 && !three)
    return lrs_fail(ctx, LRS_EINVAL, "gemm: precision mode %d is not a tensor-core mode", prec);
  if (apass_eligible(a, prec)) return launch_apass(ctx, a, prec, fro2_out);
  switch (a.adt) {
    case LRS_F32: return three ? run_tc<LRS_F32, 3, 3>(ctx, a, fro2_out) : run_tc<LRS_F32, 2, 2>(ctx, a, fro2_out);
    case LRS_F64: return three ? run_tc<LRS_F64, 3, 3>(ctx, a, fro2_out) : run_tc<LRS_F64, 2, 2>(ctx, a, fro2_out);
    case LRS_BF16: return three ? run_tc<LRS_BF16, 1, 3>(ctx, a, fro2_out) : run_tc<LRS_BF16, 1, 2>(ctx, a, fro2_out);
    default: return lrs_fail(ctx, LRS_EINVAL, "gemm: bad operand dtype %d", a.adt);
  }
}

}  // namespace lrs
