// The A-pass C = alpha * X^T A_f for a narrow X (paper Alg. 2: B = Q^T A_f,
// the one full read of the snapshot matrix), on the tensor cores with the
// snapshot tiles staged by TMA.
//
// Shapes: A is K x N row-major (K snapshots, N fine dofs, FP32 or BF16), X is
// K x M (M = r <= 256 columns of Q), C is M x N row-major.  One persistent CTA
// per SM walks N in tiles of 128 dofs; each tile is one UMMA with M = 128
// (dofs: TMEM lanes) and N = rN (r rounded up to 16: TMEM columns), K swept
// in slabs of 64 snapshots.
//
// Roles (480 threads):
//   warps 0-3   epilogue: drain a finished accumulator from TMEM and store
//               C (for a fixed r, a warp writes 32 consecutive dofs; or, for
//               C stored n-major, each thread 16 consecutive r-values).
//   warps 4-11  converters: read a raw 64 x 128 slab from shared memory, split
//               it into BF16 pieces (x = x_0 + x_1 [+ x_2]) and write them in
//               the K-major 128-byte-swizzled UMMA layout; fused ||A||_F^2.
//   warp 12     allocates TMEM, issues the MMAs (one thread).
//   warp 13     TMA producer: one 2-D tensor copy per raw slab, RS slabs in
//               flight (up to 96 KB per SM for FP32), zero fill at the edges.
//   warp 14     copies the pre-split X pieces of the slab (L2-resident) with
//               one bulk copy.
// The accumulator is double-buffered in TMEM, so the epilogue of tile t runs
// under the MMAs of tile t+1.  Every wait is bounded (LRS_ETIMEOUT).
//
// Accumulation in K chunks.  The tensor core adds each MMA's products into
// its FP32 accumulator with truncation, so a sum over the whole K sweep (K/16
// MMAs per piece) drifts toward zero by about half an FP32 ulp per MMA: ~4e-6
// relative at K = 2000, a systematic shrink of B that moves the relative
// reconstruction error of a decomposition with eps ~ 2e-4 by ~3e-4.  So the
// MMAs accumulate one chunk of kc slabs at a time (the double buffer now
// alternates per chunk), and the epilogue adds each chunk to a running FP32
// sum kept in a third TMEM region, with round-to-nearest: the drift per
// chunk is then ~4 kc MMAs' worth, unbiased across chunks.  Configurations
// whose TMEM cannot hold the running sum keep the whole-K accumulation.
//
// Shared-memory bandwidth, not HBM, is what limits this loop: per slab the
// raw tile is written (TMA) and read (converters), the pieces are written and
// then read by the MMAs.  To keep the MMA operand reads down, the X pieces sit
// stacked along UMMA N when they fit (max(SA, SX) * rN <= 256): data piece i
// meets [X_0; X_1; ...] in ONE MMA, so each data piece is read once per K
// step, and the epilogue adds the column blocks of the pieces.
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"
#include "bf16_split.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#ifndef LRS_APASS_STACK
#define LRS_APASS_STACK 1
#endif

namespace lrs {

using namespace tc;

namespace {

constexpr int TN = 128;                 // dofs per tile (UMMA M)
constexpr int TK = 64;                  // snapshots per slab (one 128-B swizzle row of BF16)
constexpr int kPieceA = TN * TK * 2;    // 16 KB: one BF16 piece of a data slab
constexpr int kEpiWarps = 4, kConvWarps = 8;
constexpr int kMmaWarp = 12, kRawWarp = 13, kXWarp = 14;
constexpr int kThreads = 15 * 32;
constexpr int kMaxRS = 8, kMaxPS = 4;
constexpr int kMaxR = 256;              // UMMA N limit
constexpr int kChunkSlabs = 2;          // K slabs (of TK snapshots) per accumulation chunk
constexpr size_t kSmemBudget = 227 * 1024 - 2048;   // dynamic bytes (static barriers + slack kept aside)

struct ApParams {
  int64_t M, N, K;
  int64_t Kt, Nt;
  const uint8_t* Xp;          // per slab: SX pieces of rN rows x 128 B (swizzled K-major)
  int rN;                     // UMMA N
  int RS, PS;                 // raw / piece stages
  uint32_t raw_bytes;         // one raw slab: TK x TN x element size
  uint32_t stage_bytes;       // one piece stage: SA data pieces + SX X pieces
  uint32_t acc_cols;          // TMEM columns per accumulator buffer
  uint32_t tmem_cols;         // allocated TMEM columns
  int nacc;                   // accumulator buffers (1 or 2)
  int stacked;                // 1: X pieces stacked along UMMA N (one MMA per data piece)
  int kc;                     // K slabs per accumulation chunk (>= Kt: the whole K at once)
  uint32_t sum_col;           // TMEM column of the running sum (kc < Kt)
  void* C; int c_f64; int c_trans; int vec_ok; int64_t ldc; double alpha;
  int accum;                // C += alpha X^T A instead of C = alpha X^T A
  int* err;
  double* fro2_part;          // per-CTA partial ||A||_F^2 or nullptr
};

// X (K x M, any dtype) -> per slab kt, piece s: rows 0..rN-1 of 64 K values,
// K-major SW128; rows >= M and snapshots >= K are zero.
template <int SX>
__global__ void __launch_bounds__(256) k_prep_xr(const void* __restrict__ X, int32_t xdt, int64_t ldx, int64_t K,
                                                 int64_t M, int64_t Kt, int rN, uint8_t* __restrict__ out) {
  const int64_t total = Kt * (int64_t)rN * 8;
  for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(id % rN);
    const int64_t rest = id / rN;
    const int c = (int)(rest % 8);
    const int64_t kt = rest / 8;
    uint32_t w[SX][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      __nv_bfloat16 p0[SX], p1[SX];
      const int64_t k0 = kt * TK + c * 8 + e;
      split_any<SX>(X, xdt, k0 * ldx + row, (k0 < K && row < M), p0);
      split_any<SX>(X, xdt, (k0 + 1) * ldx + row, (k0 + 1 < K && row < M), p1);
#pragma unroll
      for (int s = 0; s < SX; ++s) w[s][e >> 1] = pack2(p0[s], p1[s]);
    }
    uint8_t* blk = out + kt * (int64_t)SX * rN * 128;
#pragma unroll
    for (int s = 0; s < SX; ++s) {
      uint4* dst = reinterpret_cast<uint4*>(blk + (int64_t)s * rN * 128 + sw128_offset(row, c * 8));
      *dst = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// lane 0 waits, the warp follows its verdict
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, err) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// stage index and phase parity of a ring of n mbarrier-guarded buffers,
// advanced without divisions
struct Ring {
  int idx = 0, n;
  uint32_t phase = 0;
  __device__ explicit Ring(int n_) : n(n_) {}
  __device__ __forceinline__ void next() {
    if (++idx == n) { idx = 0; phase ^= 1u; }
  }
};

template <int RAW, int SA, int SX>
__global__ void __launch_bounds__(kThreads, 1) k_apass(const __grid_constant__ CUtensorMap tmA, ApParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t raw_full[kMaxRS], raw_empty[kMaxRS];
  __shared__ __align__(8) uint64_t a_full[kMaxPS], x_full[kMaxPS], p_empty[kMaxPS];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ double red_f[kConvWarps];

  const uint32_t raw0 = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw0 + 1023u) & ~1023u) - raw0);    // 1024-B aligned
  uint8_t* raw_ring = smem;
  uint8_t* piece_ring = smem + (size_t)P.RS * P.raw_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kP = SA > SX ? SA : SX;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P.RS; ++s) { mbar_init(&raw_full[s], 1); mbar_init(&raw_empty[s], kConvWarps); }
    for (int s = 0; s < P.PS; ++s) {
      mbar_init(&a_full[s], kConvWarps); mbar_init(&x_full[s], 1); mbar_init(&p_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) { mbar_init(&acc_full[a], 1); mbar_init(&acc_empty[a], kEpiWarps); }
    mbar_init(&mma_done, 1);
    fence_mbar_init();
  }
  if (warp == kRawWarp && lane == 0) prefetch_tensormap(&tmA);
  if (warp == kMmaWarp) tmem_alloc(&tmem_base_sh, P.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp < kEpiWarps) {
    // ---------------- epilogue: TMEM -> C ----------------
    Ring ar(P.nacc);
    bool eok = true;
    for (int64_t tile = blockIdx.x; tile < P.Nt && eok; tile += gridDim.x) {
     for (int64_t k0 = 0; k0 < P.Kt; k0 += P.kc, ar.next()) {
      const bool first = k0 == 0, last = k0 + P.kc >= P.Kt;
      const int acc = ar.idx;
      if (!warp_wait(&acc_full[acc], ar.phase, P.err, lane)) { eok = false; break; }
      tc_fence_after();
      const int64_t n = tile * TN + warp * 32 + lane;
      const uint32_t lanes = (uint32_t)(warp * 32) << 16;
      const uint32_t tbase = tmem + (uint32_t)acc * P.acc_cols + lanes;
      const uint32_t sbase = tmem + P.sum_col + lanes;
      for (int c0 = 0; c0 < P.rN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tbase + (uint32_t)c0, v);
        tmem_ld_wait();
        if (P.stacked) {
          // B = sum over the X pieces of the column blocks, in piece order
#pragma unroll
          for (int j = 1; j < SX; ++j) {
            uint32_t u[16];
            tmem_ld16(tbase + (uint32_t)(j * P.rN + c0), u);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = __float_as_uint(__uint_as_float(v[e]) + __uint_as_float(u[e]));
          }
        }
        if (!first) {
          // running sum of the earlier chunks, added with round-to-nearest
          uint32_t u[16];
          tmem_ld16(sbase + (uint32_t)c0, u);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = __float_as_uint(__uint_as_float(u[e]) + __uint_as_float(v[e]));
        }
        if (!last) {
          tmem_st16(sbase + (uint32_t)c0, v);
          continue;
        }
        if (n < P.N) {
          if (P.c_trans) {
            // C stored n-major: this thread's 16 consecutive entries of row n
            const int lim = (int)min((int64_t)16, P.M - c0);
            if (P.c_f64) {
              double* dst = reinterpret_cast<double*>(P.C) + n * P.ldc + c0;
              if (P.accum) {
                double old[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) old[e] = e < lim ? dst[e] : 0.0;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (e < lim) dst[e] = old[e] + P.alpha * (double)__uint_as_float(v[e]);
              } else {
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (e < lim) dst[e] = P.alpha * (double)__uint_as_float(v[e]);
              }
            } else {
              float* dst = reinterpret_cast<float*>(P.C) + n * P.ldc + c0;
              const float fa = (float)P.alpha;
              if (P.accum) {
                // all old values in flight before any store (a store may alias a later load)
                float old[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) old[e] = e < lim ? dst[e] : 0.f;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (e < lim) dst[e] = old[e] + fa * __uint_as_float(v[e]);
              } else if (lim == 16 && P.vec_ok) {
#pragma unroll
                for (int e = 0; e < 16; e += 4)
                  *reinterpret_cast<float4*>(dst + e) =
                      make_float4(fa * __uint_as_float(v[e]), fa * __uint_as_float(v[e + 1]),
                                  fa * __uint_as_float(v[e + 2]), fa * __uint_as_float(v[e + 3]));
              } else {
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (e < lim) dst[e] = fa * __uint_as_float(v[e]);
              }
            }
          } else if (P.c_f64) {
            double* col = reinterpret_cast<double*>(P.C) + n;
            if (P.accum) {
              double old[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) old[e] = c0 + e < P.M ? col[(c0 + e) * P.ldc] : 0.0;
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < P.M) col[(c0 + e) * P.ldc] = old[e] + P.alpha * (double)__uint_as_float(v[e]);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < P.M) col[(c0 + e) * P.ldc] = P.alpha * (double)__uint_as_float(v[e]);
            }
          } else {
            // FP32 output: no FP64 arithmetic (the FP64 pipe is narrow)
            const float fa = (float)P.alpha;
            float* col = reinterpret_cast<float*>(P.C) + n;
            if (P.accum) {
              // all 16 old values in flight before any store (a store may alias a later load)
              float old[16];
#pragma unroll
              for (int e = 0; e < 16; ++e) old[e] = c0 + e < P.M ? col[(c0 + e) * P.ldc] : 0.f;
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < P.M) col[(c0 + e) * P.ldc] = old[e] + fa * __uint_as_float(v[e]);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e)
                if (c0 + e < P.M) col[(c0 + e) * P.ldc] = fa * __uint_as_float(v[e]);
            }
          }
        }
      }
      if (!last) tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
     }
    }
  } else if (warp < kEpiWarps + kConvWarps) {
    // ---------------- converters ----------------
    const int t = threadIdx.x - kEpiWarps * 32;   // 0..255
    const int nl = t & (TN - 1);                  // dof row of the data operand
    const int ch = t >> 7;                        // K chunks {ch, ch+2, ch+4, ch+6}
    double fro2 = 0.0;
    Ring rr(P.RS), pr(P.PS);
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < P.Nt && ok; tile += gridDim.x) {
      float sq = 0.f;     // ||A||_F^2 of this thread's share of the tile: FP32 per tile, FP64 across tiles
      for (int64_t kt = 0; kt < P.Kt; ++kt) {
        const int rs = rr.idx, ps = pr.idx;
        if (!warp_wait(&raw_full[rs], rr.phase, P.err, lane) || !warp_wait(&p_empty[ps], pr.phase ^ 1u, P.err, lane)) {
          ok = false;
          break;
        }
        const uint8_t* src = raw_ring + (size_t)rs * P.raw_bytes;
        uint8_t* dst = piece_ring + (size_t)ps * P.stage_bytes;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = ch + 2 * i;
          uint32_t w[SA][4];
          if constexpr (RAW == LRS_F32) {
            const float* s32 = reinterpret_cast<const float*>(src) + (c * 8) * TN + nl;
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              const float a0 = s32[e * TN], a1 = s32[(e + 1) * TN];
              sq = fmaf(a0, a0, sq);
              sq = fmaf(a1, a1, sq);
              uint32_t u[SA];
              split2_f32<SA>(a0, a1, u);
#pragma unroll
              for (int q = 0; q < SA; ++q) w[q][e >> 1] = u[q];
            }
          } else {
            // BF16 data is its own single piece: move the bits
            const unsigned short* s16 = reinterpret_cast<const unsigned short*>(src) + (c * 8) * TN + nl;
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              const uint32_t b0 = s16[e * TN], b1 = s16[(e + 1) * TN];
              const float a0 = __uint_as_float(b0 << 16), a1 = __uint_as_float(b1 << 16);
              sq = fmaf(a0, a0, sq);
              sq = fmaf(a1, a1, sq);
              w[0][e >> 1] = b0 | (b1 << 16);
            }
          }
#pragma unroll
          for (int q = 0; q < SA; ++q)
            *reinterpret_cast<uint4*>(dst + q * kPieceA + sw128_offset(nl, c * 8)) =
                make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&raw_empty[rs]);
          mbar_arrive(&a_full[ps]);
        }
        rr.next();
        pr.next();
      }
      if (P.fro2_part) fro2 += (double)sq;
    }
    if (P.fro2_part) {
      // per-CTA partial, fixed order (deterministic)
      const double v = warp_sum(fro2);
      if (lane == 0) red_f[warp - kEpiWarps] = v;
      asm volatile("bar.sync 1, %0;" ::"r"(kConvWarps * 32) : "memory");
      if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kConvWarps; ++w) s += red_f[w];
        P.fro2_part[blockIdx.x] = s;
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(TN, P.rN);
      const uint32_t xpiece = (uint32_t)P.rN * 128u;
      Ring pr(P.PS), ar(P.nacc);
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < P.Nt && ok; tile += gridDim.x) {
       for (int64_t k0 = 0; k0 < P.Kt && ok; k0 += P.kc, ar.next()) {
        const int acc = ar.idx;
        if (!mbar_wait(&acc_empty[acc], ar.phase ^ 1u, P.err)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)acc * P.acc_cols;
        const int64_t k1 = k0 + P.kc < P.Kt ? k0 + P.kc : P.Kt;
        for (int64_t kt = k0; kt < k1; ++kt, pr.next()) {
          const int ps = pr.idx;
          const uint32_t ph = pr.phase;
          if (!mbar_wait(&x_full[ps], ph, P.err) || !mbar_wait(&a_full[ps], ph, P.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_u32(piece_ring + (size_t)ps * P.stage_bytes);   // data pieces (UMMA A)
          const uint32_t x0 = a0 + SA * kPieceA;                                     // X pieces (UMMA B)
          if (P.stacked) {
            // data piece i times [X_0; ...; X_{kP-i-1}] in one MMA of N = (kP - i) rN:
            // product a_i x_j lands in TMEM columns [j rN, (j+1) rN)
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
              for (int i = 0; i < SA; ++i) {
                const int nj = (SX < kP - i) ? SX : kP - i;
                const uint64_t ad = sdesc_kmajor_sw128(a0 + i * kPieceA + kk * 32);
                const uint64_t bd = sdesc_kmajor_sw128(x0 + kk * 32);
                const uint32_t accum = (kt == k0 && kk == 0 && i == 0) ? 0u : 1u;
                umma_bf16(d, ad, bd, idesc_bf16_f32(TN, nj * P.rN), accum);
              }
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
#pragma unroll
              for (int i = 0; i < SA; ++i)
#pragma unroll
                for (int j = 0; j < SX; ++j) {
                  if (i + j >= kP) continue;
                  const uint64_t ad = sdesc_kmajor_sw128(a0 + i * kPieceA + kk * 32);
                  const uint64_t bd = sdesc_kmajor_sw128(x0 + j * xpiece + kk * 32);
                  const uint32_t accum = (kt == k0 && kk == 0 && i == 0 && j == 0) ? 0u : 1u;
                  umma_bf16(d, ad, bd, idesc, accum);
                }
            }
          }
          umma_commit(&p_empty[ps]);
        }
        if (!ok) break;
        umma_commit(&acc_full[acc]);
       }
      }
      // every MMA this thread issued has finished before TMEM is released
      umma_commit(&mma_done);
      mbar_wait_quiet(&mma_done, 0);
    }
    __syncwarp();
  } else if (warp == kRawWarp) {
    // ---------------- TMA producer: raw slabs of A ----------------
    if (lane == 0) {
      int64_t it = 0;
      Ring rr(P.RS);
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < P.Nt && ok; tile += gridDim.x) {
        for (int64_t kt = 0; kt < P.Kt; ++kt, ++it, rr.next()) {
          const int s = rr.idx;
          if (!mbar_wait(&raw_empty[s], rr.phase ^ 1u, P.err)) { ok = false; break; }
          mbar_arrive_expect_tx(&raw_full[s], P.raw_bytes);
          tma_load_2d(raw_ring + (size_t)s * P.raw_bytes, &tmA, (int32_t)(tile * TN), (int32_t)(kt * TK),
                      &raw_full[s]);
        }
      }
      if (!ok) {
        // let the copies in flight land before the block exits (bounded)
        for (int b = 0; b < P.RS && it - 1 - b >= 0; ++b) {
          const int64_t j = it - 1 - b;
          mbar_wait_quiet(&raw_full[j % P.RS], (uint32_t)((j / P.RS) & 1));
        }
      }
    }
    __syncwarp();
  } else if (warp == kXWarp) {
    // ---------------- X-piece producer ----------------
    if (lane == 0) {
      const uint32_t xbytes = (uint32_t)SX * (uint32_t)P.rN * 128u;
      int64_t it = 0;
      Ring pr(P.PS);
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < P.Nt && ok; tile += gridDim.x) {
        for (int64_t kt = 0; kt < P.Kt; ++kt, ++it, pr.next()) {
          const int s = pr.idx;
          if (!mbar_wait(&p_empty[s], pr.phase ^ 1u, P.err)) { ok = false; break; }
          mbar_arrive_expect_tx(&x_full[s], xbytes);
          bulk_g2s(piece_ring + (size_t)s * P.stage_bytes + SA * kPieceA, P.Xp + kt * (int64_t)xbytes, xbytes,
                   &x_full[s]);
        }
      }
      if (!ok) {
        for (int b = 0; b < P.PS && it - 1 - b >= 0; ++b) {
          const int64_t j = it - 1 - b;
          mbar_wait_quiet(&x_full[j % P.PS], (uint32_t)((j / P.PS) & 1));
        }
      }
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, P.tmem_cols);
  }
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled encode_fn() {
  static EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

struct ApCfg {
  int rN, RS, PS, stacked;
  uint32_t raw_bytes, stage_bytes, acc_cols, tmem_cols;
  int nacc;
  int kc;             // slabs per accumulation chunk, 0: whole K
  uint32_t sum_col;
  size_t smem;
};

// MMAs a chunk may accumulate before its round-to-nearest add: 16 for two
// pieces of FP32 data, 32 for BF16 data (one exact piece, whose split
// products' own error, 2^-16, is far above a 32-ulp truncation), 48 for
// three pieces
int chunk_mmas(int SA, int SX) { return SX >= 3 ? 48 : (SA == 1 ? 32 : 16); }

bool plan(int64_t M, int64_t Kt, int esize, int SA, int SX, ApCfg* c) {
  if (M < 1 || M > kMaxR) return false;
  c->rN = (int)((M + 15) / 16 * 16);
  c->raw_bytes = (uint32_t)(TK * TN * esize);
  c->stage_bytes = (uint32_t)(SA * kPieceA + SX * c->rN * 128);
  // two piece stages (conversion overlaps the MMAs) unless that leaves fewer
  // than two raw slabs in flight; then one
  c->RS = 0;
  for (int ps = 2; ps >= 1 && c->RS < 2; --ps) {
    c->PS = ps;
    int64_t rs = ((int64_t)kSmemBudget - 1024 - (int64_t)ps * c->stage_bytes) / (int64_t)c->raw_bytes;
    c->RS = (int)(rs > kMaxRS ? kMaxRS : (rs < 0 ? 0 : rs));
  }
  if (c->RS < 2) return false;
  c->smem = 1024 + (size_t)c->RS * c->raw_bytes + (size_t)c->PS * c->stage_bytes;
  // stacking needs the widest MMA, max(SA, SX) pieces of rN, within UMMA N <= 256.
  // Preference: K-chunked accumulation (accuracy) over stacking (fewer operand
  // reads): stacked + chunked, unstacked + chunked, then the whole-K forms.
  // A K sweep no longer than one chunk takes the whole-K form: the same
  // accumulation, without the running-sum region.
  const int kp = SA > SX ? SA : SX;
  const bool can_stack = LRS_APASS_STACK && kp * c->rN <= kMaxR;
  auto pow2 = [](uint32_t need) { uint32_t cols = 32; while (cols < need) cols <<= 1; return cols; };
  const uint32_t sum_cols = (uint32_t)c->rN;
  int npairs = 0;
  for (int i = 0; i < SA; ++i)
    for (int j = 0; j < SX; ++j) npairs += (i + j < kp) ? 1 : 0;
  for (int form = 0; form < 4; ++form) {
    const int stacked = (form == 0 || form == 2) ? 1 : 0;
    const bool chunked = form < 2;
    if (stacked && !can_stack) continue;
    const int per_k = 4 * (stacked ? SA : npairs);              // MMAs per slab into one accumulator
    int kc = chunk_mmas(SA, SX) / per_k;
    if (kc < 1) kc = 1;
    const int width = stacked ? SX * c->rN : c->rN;
    const uint32_t acc_cols = (uint32_t)((width + 63) / 64 * 64);
    if (chunked && Kt > kc) {
      const uint32_t cols = pow2(2 * acc_cols + sum_cols);
      if (cols > 512) continue;
      c->stacked = stacked; c->acc_cols = acc_cols; c->nacc = 2; c->tmem_cols = cols;
      c->sum_col = 2 * acc_cols; c->kc = kc;
      return true;
    }
    c->stacked = stacked; c->acc_cols = acc_cols; c->sum_col = 0; c->kc = 0;
    uint32_t cols = pow2(2 * acc_cols);
    if (cols <= 512) {
      c->nacc = 2;
    } else {
      c->nacc = 1;
      cols = pow2(acc_cols);
    }
    c->tmem_cols = cols;
    return true;
  }
  return false;
}

template <int RAW, int SA, int SX>
lrs_status run_apass(lrs_ctx* ctx, const GemmArgs& a, double* fro2_out) {
  constexpr int esize = RAW == LRS_F32 ? 4 : 2;
  ApCfg cfg;
  if (!plan(a.M, (a.K + TK - 1) / TK, esize, SA, SX, &cfg))
    return lrs_fail(ctx, LRS_EINVAL, "a-pass: r=%lld out of range", (long long)a.M);
  EncodeTiled enc = encode_fn();
  if (!enc) return lrs_fail(ctx, LRS_ECUDA, "a-pass: cuTensorMapEncodeTiled unavailable");
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)a.N, (cuuint64_t)a.K};
  const cuuint64_t gstride[1] = {(cuuint64_t)a.lda * esize};
  const cuuint32_t box[2] = {(cuuint32_t)TN, (cuuint32_t)TK};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult cr = enc(&map, RAW == LRS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          2, const_cast<void*>(a.A), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return lrs_fail(ctx, LRS_ECUDA, "a-pass: tensor map encode failed (%d)", (int)cr);

  ApParams P{};
  P.M = a.M; P.N = a.N; P.K = a.K;
  P.Kt = (a.K + TK - 1) / TK; P.Nt = (a.N + TN - 1) / TN;
  P.rN = cfg.rN; P.RS = cfg.RS; P.PS = cfg.PS;
  P.raw_bytes = cfg.raw_bytes; P.stage_bytes = cfg.stage_bytes;
  P.acc_cols = cfg.acc_cols; P.tmem_cols = cfg.tmem_cols; P.nacc = cfg.nacc; P.stacked = cfg.stacked;
  P.kc = cfg.kc > 0 ? cfg.kc : (int)P.Kt;
  P.sum_col = cfg.sum_col;
  P.C = a.C; P.c_f64 = a.c_f64; P.c_trans = a.c_trans; P.ldc = a.ldc; P.alpha = a.alpha; P.accum = a.accum;
  P.vec_ok = ((reinterpret_cast<uintptr_t>(a.C) & 15u) == 0 && (a.ldc & 3) == 0) ? 1 : 0;

  const size_t xbytes = (size_t)P.Kt * SX * cfg.rN * 128;
  uint8_t* Xp = (uint8_t*)ws_alloc(ctx, xbytes);
  int* err = (int*)ws_alloc(ctx, 256);
  if (!Xp || !err) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (a-pass: %zu B)", xbytes);
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 256, ctx->stream));
  {
    const int64_t total = P.Kt * (int64_t)cfg.rN * 8;
    int64_t nb = (total + 255) / 256;
    if (nb > (int64_t)ctx->num_sms * 32) nb = (int64_t)ctx->num_sms * 32;
    k_prep_xr<SX><<<(unsigned)nb, 256, 0, ctx->stream>>>(a.X, a.xdt, a.ldx, a.K, a.M, P.Kt, cfg.rN, Xp);
    ctx->launches++;
    LRS_CUDA_TRY(ctx, cudaGetLastError());
  }
  P.Xp = Xp;
  P.err = err;
  const unsigned grid = (unsigned)(P.Nt < ctx->num_sms ? P.Nt : ctx->num_sms);
  double* part = nullptr;
  if (fro2_out) {
    part = (double*)ws_alloc(ctx, sizeof(double) * grid);
    if (!part) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (a-pass)");
  }
  P.fro2_part = part;
  auto kern = k_apass<RAW, SA, SX>;
  { const lrs_status _s = raise_dyn_smem(ctx, (const void*)kern, (size_t)(cfg.smem)); if (_s) return _s; }
  const bool timing = ctx->time_kernels && ctx->kev0 && ctx->kev1;
  if (timing) LRS_CUDA_TRY(ctx, cudaEventRecord(ctx->kev0, ctx->stream));
  kern<<<grid, kThreads, cfg.smem, ctx->stream>>>(map, P);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  if (timing) LRS_CUDA_TRY(ctx, cudaEventRecord(ctx->kev1, ctx->stream));
  if (fro2_out) {
    lrs_status st = launch_sum(ctx, part, (int)grid, fro2_out);
    if (st) return st;
  }
  int* h = (int*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {(const int32_t*)err};
    const lrs_status rs = replay_ints(ctx, 1, d, h + 20);
    if (rs) return rs;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 20, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[20] != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "a-pass: a pipeline wait gave up");
  if (timing) {
    float ms = 0.f;
    LRS_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->kev0, ctx->kev1));
    ctx->last_kernel_ms = ms;
  }
  return LRS_OK;
}

}  // namespace

bool apass_eligible(const GemmArgs& a, int prec) {
  if (prec != LRS_PREC_SPLIT_BF16 && prec != LRS_PREC_BF16X3) return false;
  if (a.adt != LRS_F32 && a.adt != LRS_BF16) return false;
  if (a.M < 1 || a.M > kMaxR || a.N < TN || a.K < 1) return false;
  // few column tiles over a long K: the split-K tensor-core kernel fills the SMs, this one cannot
  if (a.N < 64 * TN && a.K >= 8192) return false;
  if (a.N >= (int64_t)1 << 31 || a.K >= (int64_t)1 << 31) return false;
  const int esize = a.adt == LRS_F32 ? 4 : 2;
  if ((reinterpret_cast<uintptr_t>(a.A) & 15u) != 0 || ((a.lda * esize) & 15) != 0) return false;
  if (a.lda >= ((int64_t)1 << 40) / esize) return false;
  const int sa = a.adt == LRS_BF16 ? 1 : (prec == LRS_PREC_BF16X3 ? 3 : 2);
  const int sx = prec == LRS_PREC_BF16X3 ? 3 : 2;
  ApCfg cfg;
  if (!plan(a.M, (a.K + TK - 1) / TK, esize, sa, sx, &cfg)) return false;
  return encode_fn() != nullptr;
}

size_t apass_workspace(int64_t M, int64_t K, int prec) {
  const int64_t rN = (M + 15) / 16 * 16;
  const int sx = prec == LRS_PREC_BF16X3 ? 3 : 2;
  return (size_t)((K + TK - 1) / TK) * sx * rN * 128 + 1024 + 512 + 8 * 1024;
}

lrs_status launch_apass(lrs_ctx* ctx, const GemmArgs& a, int prec, double* fro2_out) {
  const bool three = prec == LRS_PREC_BF16X3;
  if (a.adt == LRS_F32)
    return three ? run_apass<LRS_F32, 3, 3>(ctx, a, fro2_out) : run_apass<LRS_F32, 2, 2>(ctx, a, fro2_out);
  return three ? run_apass<LRS_BF16, 1, 3>(ctx, a, fro2_out) : run_apass<LRS_BF16, 1, 2>(ctx, a, fro2_out);
}

}  // namespace lrs
