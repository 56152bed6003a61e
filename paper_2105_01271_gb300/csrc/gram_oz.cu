// G = B B^T for a wide FP32 B (r x n row-major, r <= 128) on the tensor
// cores, as an exact-slice (Ozaki-type) product: the small SVD of B (Alg. 2)
// needs its Gram to ~2^-46 relative (its tail singular values are ~1e-4 of
// the largest), which FP32-accumulated BF16 products alone cannot give.
//
// Slicing.  Row i is scaled by 2^-(e_i + 1), e_i the exponent with
// max_k |b_ik| < 2^e_i (a pre-pass finds it), so x = b 2^-(e_i+1) has |x| < 1/2
// and the scaling is exact.  x is cut into six pieces
//     x = s_0 + s_1 + ... + s_5 + (|rest| <= 2^-49),
// s_t the round-to-nearest of what is left onto the grid 2^-8(t+1): each
// s_t is an integer of at most 8 significant bits (|.| <= 128) times a power
// of two, so it is exact in BF16 and the FP32 bits of s_t ARE its BF16 bits
// (the low 16 are zero).  The product s_s(i) s_t(j) is an integer times
// 2^-8(s+t+2) ("level" s + t), and every product below level 6 is kept.
//
// Exact accumulation.  A tcgen05.mma (BF16 in, FP32 accumulate) adds
// integer-valued products on one grid exactly as long as every partial sum
// stays below 2^24 units; it truncates otherwise, so a long FP32 sum of
// small terms drifts by ~2^-23 per MMA.  Four TMEM accumulators therefore
// hold one level each, exactly, over a chunk of 256 columns
// (X_st = S_s S_t^T over the chunk):
//     acc_0 = X_00, acc_1 = X_01, acc_2 = X_02 + X_20 + X_11 (<= 2^23.6 units),
//     acc_3 = X_03 + X_12,
// and a fifth takes levels 4 and 5 with their true weights, inexactly (an
// FP32 drift of ~2^-16 of a term ~2^-30 below X_00):
//     acc_4 = X_04 + X_13 + X_22 / 2 + X_05 + X_14 + X_23.
// With S = acc_0/2 + acc_1 + acc_2/2 + acc_3 + acc_4 the sum of all kept
// levels is S + S^T (X_ts = X_st^T; X_00, X_11, X_22 and X_02 + X_20 are
// symmetric): 13 slice products instead of 21.
//
// Column groups.  Five accumulators of N columns fit TMEM's 512 when
// N <= 96: r <= 96 is one group (N = r rounded up to 16); a larger r is two
// groups of 64 columns of G, each on its own CTA (both slice all rows of the
// range: the A operand), the pair adjacent in the grid so the second read of
// the range comes from L2.
//
// Diagonal.  X_33 (level 6) is dropped and acc_4 truncates; off the diagonal
// both errors have random signs, but on it every X_tt term is >= 0, a bias
// of ~2^-44.  So G_ii = sum_k x_ik^2 is summed apart, without bias: over a
// chunk the slicing threads sum their squares error-free in FP32 (x^2 = h + l
// by one FMA, Knuth's two-sum) and fold both words, rounded to 2^-50, into
// int64 (column group 0 only).
//
// Drain.  After each chunk the accumulators are read back (tcgen05.ld) and
// added into one int64 per entry in units of 2^-49: levels 0-3 exactly
// (integers on known grids, converted by magic-number rounding in FP32),
// levels 4-5 rounded to the unit.  A CTA sums at
// most 16384 columns in int64 (|S| <= 2^61 units), then adds the range into
// its FP64 partial S_cta 2^(e_i + e_j + 2); a final kernel forms
// G = sum over CTAs of (S_cta + S_cta^T) in a fixed order (deterministic).
//
// Roles (384 threads, three warps per TMEM lane quarter): every warp slices
// its share of each slab of B (64 columns, read from global memory, written
// as seven K-major 128-byte-swizzled BF16 operands: s_0..s_5 and s_2 / 2) and
// drains its 16-column blocks of its lane quarter; thread 0 also issues the
// MMAs of a slab once all warps have sliced it.  Two slab stages of 112 KB;
// every wait is bounded (LRS_ETIMEOUT).
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace lrs {

using namespace tc;

namespace {

constexpr int kOzK = 64;                        // columns per slab
constexpr int kOzSlabsPerChunk = 4;             // 256 columns per exact accumulation
constexpr int kOzBufs = 7;                      // s_0..s_5, s_2 / 2
constexpr int kOzBuf = 128 * kOzK * 2;          // 16 KB: 128 rows x 64 BF16
constexpr int kOzStage = kOzBufs * kOzBuf;      // 112 KB
constexpr int kOzStages = 2;
constexpr int kOzWarps = 12;                   // slicing + draining (3 per TMEM lane quarter); thread 0 also issues the MMAs
constexpr int kOzThreads = kOzWarps * 32;
constexpr int kOzAccCols = 96;                  // TMEM columns per accumulator (5 x 96 <= 512)
constexpr int64_t kOzRangeMax = 16384;          // columns per int64 range
constexpr size_t kOzSmem = (size_t)kOzStages * kOzStage + 1024;

// slice products: A operand buffer, B operand buffer, accumulator
// (grouped by A operand, so consecutive MMAs share it)
__host__ __device__ constexpr int oz_prod_a(int p) {
  constexpr int t[13] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 2, 2, 6};
  return t[p];
}
__host__ __device__ constexpr int oz_prod_b(int p) {
  constexpr int t[13] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 0, 3, 2};
  return t[p];
}
__host__ __device__ constexpr int oz_prod_acc(int p) {
  constexpr int t[13] = {0, 1, 2, 3, 4, 4, 2, 3, 4, 4, 2, 4, 4};
  return t[p];
}
// the first product of each accumulator in the table (zero-initialises it)
__host__ __device__ constexpr bool oz_first(int p) { return p < 5; }

struct OzParams {
  const float* B;
  int64_t n, ldb;
  int r;
  int cw, ngroups;             // column group width (UMMA N) and count
  int64_t range_cols, nranges;
  int vec;                     // 16-byte loads of B allowed
  const uint32_t* rowmax;      // bits of max_k |b_ik| per row
  double* part;                // per-CTA partial S (r x r, FP64, zeroed)
  double* diag;                // per-CTA partial sum_k b_ik^2 (r, FP64, zeroed)
  int* err;
};

// stage index and phase parity of the slab ring
struct OzRing {
  int idx = 0;
  uint32_t phase = 0;
  __device__ __forceinline__ void next() {
    if (++idx == kOzStages) { idx = 0; phase ^= 1u; }
  }
};

__device__ __forceinline__ bool oz_warp_wait(uint64_t* bar, uint32_t parity, int* err, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, err) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// 32 lanes x 8 columns of 32-bit values: thread t of the warp receives lane
// (quarter*32 + t), columns [col, col+8)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

// round(v 2^50) for |v| < 2^12, from v's significand in integer arithmetic
// (v = m 2^(E-150)); round half up
__device__ __forceinline__ long long oz_ll50(float v) {
  const uint32_t bits = __float_as_uint(v);
  const int E = (int)((bits >> 23) & 0xffu);
  const long long m = (long long)((bits & 0x7fffffu) | (E ? 0x800000u : 0u));
  const int sh = (E ? E : 1) - 100;                 // v 2^50 = m 2^sh
  long long q;
  if (sh >= 0) q = m << sh;
  else if (sh > -63) q = (m + ((1ll << -sh) >> 1)) >> -sh;
  else q = 0;
  return (bits >> 31) ? -q : q;
}

// round-to-nearest integer of v, |v| <= 2^22, by FP32 addition alone: in
// [2^23, 2^24] the float spacing is 1, so v + 1.5 2^23 rounds v and its bits
// count the integers from 1.5 2^23 (no conversion instruction)
__device__ __forceinline__ int oz_rint22(float v) { return __float_as_int(__fadd_rn(v, 12582912.f)) - 0x4B400000; }
// the same for |v| < 2^35: v = a 2^13 + rem, a and rem each rounded by the
// magic add (rem = v - a 2^13 is exact)
__device__ __forceinline__ long long oz_rint35(float v) {
  const float a = __fsub_rn(__fadd_rn(__fmul_rn(v, 1.220703125e-4f), 12582912.f), 12582912.f);
  const float rem = __fmaf_rn(a, -8192.f, v);
  return (long long)oz_rint22(a) * 8192 + oz_rint22(rem);
}

// for the bits of a non-negative float v: the exponent e with v < 2^e, the
// smallest for v > 0 (v = 0 gives 0)
__device__ __forceinline__ int oz_exp(uint32_t bits) {
  if (bits == 0) return 0;
  const int E = (int)(bits >> 23);
  return E > 0 ? E - 126 : -117 - __clz((int)bits);     // subnormal: v = bits 2^-149
}

// 2^k as a float for -126 <= k <= 127
__device__ __forceinline__ float oz_pow2f(int k) { return __int_as_float((127 + k) << 23); }

// cut x (|x| < 1/2) into s_0..s_5 and pack the pair (x0, x1) of each slice
// into one BF16x2 word (x0 in the low half); w[6] gets s_2 / 2
__device__ __forceinline__ void oz_slice_pair(float x0, float x1, uint32_t (&w)[kOzBufs]) {
  // 1.5 * 2^(15 - 8t): adding and subtracting it rounds to the grid 2^-8(t+1)
  const float kM[6] = {49152.f, 192.f, 0.75f, 2.9296875e-3f, 1.1444091796875e-5f, 4.470348358154297e-8f};
  float r0 = x0, r1 = x1;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float s0 = __fsub_rn(__fadd_rn(r0, kM[t]), kM[t]);
    const float s1 = __fsub_rn(__fadd_rn(r1, kM[t]), kM[t]);
    r0 = __fsub_rn(r0, s0);
    r1 = __fsub_rn(r1, s1);
    w[t] = __byte_perm(__float_as_uint(s0), __float_as_uint(s1), 0x7632);
    if (t == 2) w[6] = __byte_perm(__float_as_uint(__fmul_rn(s0, 0.5f)), __float_as_uint(__fmul_rn(s1, 0.5f)), 0x7632);
  }
}

__global__ void __launch_bounds__(kOzThreads, 1) k_gram_oz(OzParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kOzStages], empty[kOzStages], acc_full, acc_empty, mma_done;
  __shared__ uint32_t tmem_base_sh;

  const uint32_t raw0 = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + (((raw0 + 1023u) & ~1023u) - raw0);    // 1024-B aligned stages
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool issuer = threadIdx.x == 0;            // also issues the MMAs

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) { mbar_init(&full[s], kOzWarps); mbar_init(&empty[s], 1); }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, kOzWarps);
    mbar_init(&mma_done, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base_sh, 512);
  // rows >= r of every operand are zero and never sliced
  for (int i = threadIdx.x; i < kOzStages * kOzStage / 16; i += kOzThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  const int tid = threadIdx.x;                     // 0..383
  const int q = warp & 3, part = warp >> 2;        // TMEM lane quarter; 16-column blocks part, part + 3
  const int ri = q * 32 + lane;                    // the G row this thread drains
  const int nblk = P.cw / 16;
  // this CTA's column group is fixed: gridDim.x is a multiple of ngroups
  const int grp = (int)(blockIdx.x % P.ngroups);
  const int gcol0 = grp * P.cw;
  // the exact scale 2^-(e+1) of each task row, as two powers of two in range
  float sa[3], sb[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int row = (tid + kOzThreads * u) >> 3;
    const int re = row < P.r ? oz_exp(P.rowmax[row]) : 0;
    const int rk = -(re + 1), rk1 = (rk >= -126 && rk <= 127) ? rk : rk / 2;
    sa[u] = oz_pow2f(rk1);
    sb[u] = oz_pow2f(rk - rk1);                 // 1 unless 2^rk is out of the normal range
  }
  long long V[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) V[c] = 0;
  // sum of x^2 over this thread's columns of each task row, in int64 units of
  // 2^-50: over a chunk (32 values) the squares are summed error-free in FP32
  // (x^2 = h + l exactly by one FMA, the h by Knuth's two-sum into ph, the
  // rounding errors and the l into pl), then both words are rounded to the
  // unit and added
  long long dq[3] = {0, 0, 0};
  float ph[3] = {0.f, 0.f, 0.f}, pl[3] = {0.f, 0.f, 0.f};
  auto fold = [&]() {
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      dq[u] += oz_ll50(ph[u]) + oz_ll50(pl[u]);
      ph[u] = 0.f;
      pl[u] = 0.f;
    }
  };
  const uint32_t idesc = idesc_bf16_f32(128, P.cw);
  OzRing sr, mr;                                   // slicing ring; MMA ring (issuer)
  uint32_t acc_ph = 0, mma_acc_ph = 0;
  bool ok = true;
  const int64_t nitems = P.nranges * P.ngroups;
  for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
    const int64_t rg = item / P.ngroups;
    const int64_t c0 = rg * P.range_cols;
    const int64_t c1 = c0 + P.range_cols < P.n ? c0 + P.range_cols : P.n;
    const int ns = (int)((c1 - c0 + kOzK - 1) / kOzK);
    for (int s = 0; s <= ns && ok; ++s) {
      if (s < ns) {
        // ---- slice slab s into stage sr.idx ----
        uint8_t* dst = smem + (size_t)sr.idx * kOzStage;
        const int64_t col0 = c0 + (int64_t)s * kOzK;
        // every task's 8 values in flight before any is sliced (and before the
        // wait for the stage)
        float b[3][8];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int t = tid + kOzThreads * u;
          const int row = t >> 3, kc = (t & 7) * 8;
          const int64_t gc = col0 + kc;
          if (t < 128 * 8 && row < P.r && P.vec && gc + 8 <= c1) {
            const float4* p4 = reinterpret_cast<const float4*>(P.B + (int64_t)row * P.ldb + gc);
            const float4 v0 = __ldcs(p4), v1 = __ldcs(p4 + 1);
            b[u][0] = v0.x; b[u][1] = v0.y; b[u][2] = v0.z; b[u][3] = v0.w;
            b[u][4] = v1.x; b[u][5] = v1.y; b[u][6] = v1.z; b[u][7] = v1.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              b[u][e] = (t < 128 * 8 && row < P.r && gc + e < c1) ? P.B[(int64_t)row * P.ldb + gc + e] : 0.f;
          }
        }
        if (!oz_warp_wait(&empty[sr.idx], sr.phase ^ 1u, P.err, lane)) { ok = false; break; }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int t = tid + kOzThreads * u;
          const int row = t >> 3, kc = (t & 7) * 8;
          if (t >= 128 * 8 || row >= P.r) continue;
          uint32_t w[kOzBufs][4];
          float x[8];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            uint32_t wp[kOzBufs];
            x[e] = __fmul_rn(__fmul_rn(b[u][e], sa[u]), sb[u]);
            x[e + 1] = __fmul_rn(__fmul_rn(b[u][e + 1], sa[u]), sb[u]);
            oz_slice_pair(x[e], x[e + 1], wp);
#pragma unroll
            for (int t2 = 0; t2 < kOzBufs; ++t2) w[t2][e >> 1] = wp[t2];
          }
          if (grp == 0) {                                  // the diagonal: one column group
            float sh = ph[u], sl = pl[u];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float h = __fmul_rn(x[e], x[e]);
              const float l = __fmaf_rn(x[e], x[e], -h);
              const float sum = __fadd_rn(sh, h);
              const float bb = __fsub_rn(sum, sh);
              const float er = __fadd_rn(__fsub_rn(sh, __fsub_rn(sum, bb)), __fsub_rn(h, bb));
              sh = sum;
              sl = __fadd_rn(sl, __fadd_rn(er, l));
            }
            ph[u] = sh;
            pl[u] = sl;
          }
          const uint32_t off = sw128_offset((uint32_t)row, (uint32_t)kc);
#pragma unroll
          for (int t2 = 0; t2 < kOzBufs; ++t2)
            *reinterpret_cast<uint4*>(dst + t2 * kOzBuf + off) = make_uint4(w[t2][0], w[t2][1], w[t2][2], w[t2][3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[sr.idx]);
        sr.next();
      }
      // ---- drain the chunk that ended with slab s - 1 ----
      if (s > 0 && (s % kOzSlabsPerChunk == 0 || s == ns)) {
        if (grp == 0) fold();
        if (!oz_warp_wait(&acc_full, acc_ph, P.err, lane)) { ok = false; break; }
        tc_fence_after();
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          const int blk = part + 3 * g;
          if (blk < nblk) {
            const uint32_t tc0 = tmem + lanes + (uint32_t)(blk * 16);
            // a_L = acc_L 2^(16, 24, 32, 40) are exact integers (|a_0|, |a_1| <= 2^22,
            // |a_2| < 2^23.6, |a_3| <= 2^23); in units of 2^-49: acc_0 / 2 = a_0 2^32,
            // acc_1 = a_1 2^25, acc_2 / 2 = a_2 2^16, acc_3 = a_3 2^9; acc_4 is
            // rounded to the unit (|.| < 2^25)
#pragma unroll
            for (int h8 = 0; h8 < 2; ++h8) {
              const uint32_t tc8 = tc0 + (uint32_t)(h8 * 8);
              uint32_t v[8];
              long long acc[8];
              tmem_ld8(tc8, v);
              tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < 8; ++e) acc[e] = (long long)oz_rint22(__uint_as_float(v[e]) * 65536.f) * (1LL << 32);
              tmem_ld8(tc8 + kOzAccCols, v);
              tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < 8; ++e) acc[e] += (long long)oz_rint22(__uint_as_float(v[e]) * 16777216.f) * (1LL << 25);
              tmem_ld8(tc8 + 2 * kOzAccCols, v);
              tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < 8; ++e) acc[e] += oz_rint35(__uint_as_float(v[e]) * 4294967296.f) * (1LL << 16);
              tmem_ld8(tc8 + 3 * kOzAccCols, v);
              tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < 8; ++e) acc[e] += oz_rint35(__uint_as_float(v[e]) * 1099511627776.f) * (1LL << 9);
              tmem_ld8(tc8 + 4 * kOzAccCols, v);
              tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < 8; ++e) V[g * 16 + h8 * 8 + e] += acc[e] + oz_rint35(__uint_as_float(v[e]) * 562949953421312.f);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty);
        acc_ph ^= 1u;
      }
      // ---- issue the MMAs of slab s (one thread) ----
      int mok = 1;
      if (issuer && s < ns) {
        const bool chunk_start = s % kOzSlabsPerChunk == 0;
        // a chunk starts once every warp has drained the previous one
        if (chunk_start && !mbar_wait(&acc_empty, mma_acc_ph ^ 1u, P.err)) mok = 0;
        if (mok && !mbar_wait(&full[mr.idx], mr.phase, P.err)) mok = 0;
        if (mok) {
          tc_fence_after();
          // descriptors of the stage base; an operand is the base plus its
          // byte offset / 16 in the start-address field (no carry: < 256 KB)
          const uint64_t dbase = sdesc_kmajor_sw128(smem_u32(smem + (size_t)mr.idx * kOzStage));
          const uint64_t dboff = dbase + (uint64_t)((uint32_t)gcol0 * 128u >> 4);   // the group's B rows
#pragma unroll
          for (int kk = 0; kk < kOzK / 16; ++kk) {
#pragma unroll
            for (int p = 0; p < 13; ++p) {
              const uint64_t ad = dbase + (uint64_t)((oz_prod_a(p) * kOzBuf + kk * 32) >> 4);
              const uint64_t bd = dboff + (uint64_t)((oz_prod_b(p) * kOzBuf + kk * 32) >> 4);
              const uint32_t accum = (chunk_start && kk == 0 && oz_first(p)) ? 0u : 1u;
              umma_bf16(tmem + (uint32_t)(oz_prod_acc(p) * kOzAccCols), ad, bd, idesc, accum);
            }
          }
          umma_commit(&empty[mr.idx]);
          if (s % kOzSlabsPerChunk == kOzSlabsPerChunk - 1 || s == ns - 1) {
            umma_commit(&acc_full);
            mma_acc_ph ^= 1u;
          }
          mr.next();
        }
      }
      if (__shfl_sync(0xffffffffu, mok, 0) == 0) { ok = false; break; }
    }
    if (!ok) break;
    // ---- range end: S_cta += V 2^-49 2^(e_i + e_j + 2) ----
    if (ri < P.r) {
      const int ei = oz_exp(P.rowmax[ri]);
      double* prow = P.part + (int64_t)blockIdx.x * P.r * P.r + (int64_t)ri * P.r;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int blk = part + 3 * g;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int j = gcol0 + blk * 16 + e;
          if (blk < nblk && j < P.r) {
            const int k = ei + oz_exp(P.rowmax[j]) + 2 - 49;
            // one thread owns the slot: the adds of its ranges land in order
            atomicAdd(prow + j, (double)V[g * 16 + e] * __longlong_as_double((long long)(1023 + k) << 52));
            asm volatile("" ::: "memory");   // one entry at a time (registers)
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) V[c] = 0;
    // ---- range end: the exact diagonal, sum_k b_ik^2 = 2^(2 e_i + 2) sum x^2 ----
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int t = tid + kOzThreads * u;
      if (t >= 128 * 8) break;                       // warp-uniform (whole warps)
      long long dv = dq[u];
      dv += __shfl_xor_sync(0xffffffffu, dv, 1);
      dv += __shfl_xor_sync(0xffffffffu, dv, 2);
      dv += __shfl_xor_sync(0xffffffffu, dv, 4);
      const int row = t >> 3;
      if ((lane & 7) == 0 && row < P.r && grp == 0) {
        const int k = 2 * oz_exp(P.rowmax[row]) + 2 - 50;
        P.diag[(int64_t)blockIdx.x * P.r + row] += (double)dv * __longlong_as_double((long long)(1023 + k) << 52);
      }
      dq[u] = 0;
    }
  }
  if (issuer) {
    // every MMA issued has finished before TMEM is released
    umma_commit(&mma_done);
    mbar_wait_quiet(&mma_done, 0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// max_k |b_ik| per row, as float bits (non-negative floats order as their bits)
__global__ void __launch_bounds__(256) k_row_absmax(const float* __restrict__ B, int64_t n, int64_t ldb, int vec,
                                                    uint32_t* __restrict__ mx) {
  __shared__ float red[8];
  const float* row = B + (int64_t)blockIdx.y * ldb;
  float m = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t done = 0;
  if (vec) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const int64_t n4 = n >> 2;
    for (int64_t c = t0; c < n4; c += stride) {
      const float4 v = __ldcs(r4 + c);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    done = n4 << 2;
  }
  for (int64_t c = done + t0; c < n; c += stride) m = fmaxf(m, fabsf(row[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    atomicMax(mx + blockIdx.y, __float_as_uint(t));
  }
}

// G = sum over CTAs of (S + S^T) off the diagonal and of the exact squares
// on it: a warp per entry, lanes over the partials, fixed shuffle tree
__global__ void k_gram_oz_reduce(const double* __restrict__ part, const double* __restrict__ diag, int np, int r,
                                 double* __restrict__ G) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwt = (gridDim.x * blockDim.x) >> 5;
  const int64_t rr = (int64_t)r * r;
  for (int e = w0; e < r * r; e += nwt) {
    const int i = e / r, j = e - i * r;
    double a = 0.0;
    if (i == j)
      for (int p = lane; p < np; p += 32) a += diag[(int64_t)p * r + i];
    else
      for (int p = lane; p < np; p += 32) a += part[p * rr + (int64_t)i * r + j] + part[p * rr + (int64_t)j * r + i];
    const double s = warp_sum(a);
    if (lane == 0) G[e] = s;
  }
}

}  // namespace

size_t gram_oz_ws(int64_t r, int num_sms) {
  auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  return a256(8 * (size_t)num_sms * (size_t)(r * r)) + a256(8 * (size_t)num_sms * (size_t)r) + a256(4 * (size_t)r) +
         256 + 1024;
}

lrs_status launch_gram_oz(lrs_ctx* ctx, const float* B, int64_t r, int64_t n, int64_t ldb, double* G) {
  if (r < 1 || r > 128 || n < 1 || ldb < n)
    return lrs_fail(ctx, LRS_EINVAL, "gram: r=%lld n=%lld ldb=%lld out of range", (long long)r, (long long)n,
                    (long long)ldb);
  const int ri = (int)r;
  const int rN = (ri + 15) / 16 * 16;
  const int ngroups = rN <= kOzAccCols ? 1 : 2;
  const int cw = ngroups == 1 ? rN : 64;
  // ranges: equal column counts (multiples of 256, at most kOzRangeMax), a
  // whole number of waves of one CTA per SM; the CTAs of a range's column
  // groups are adjacent
  const int64_t sms = ctx->num_sms;
  const int64_t per_wave = sms / ngroups;
  const int64_t waves = (n + per_wave * kOzRangeMax - 1) / (per_wave * kOzRangeMax);
  int64_t range_cols = (n + waves * per_wave - 1) / (waves * per_wave);
  range_cols = (range_cols + 255) / 256 * 256;
  const int64_t nranges = (n + range_cols - 1) / range_cols;
  const int64_t grid = (nranges < per_wave ? nranges : per_wave) * ngroups;

  uint32_t* mx = (uint32_t*)ws_alloc(ctx, 4 * (size_t)r);
  double* part = (double*)ws_alloc(ctx, 8 * (size_t)grid * (size_t)(r * r));
  double* diag = (double*)ws_alloc(ctx, 8 * (size_t)grid * (size_t)r);
  int* err = (int*)ws_alloc(ctx, 256);
  if (!mx || !part || !diag || !err) return lrs_fail(ctx, LRS_ENOMEM, "workspace exhausted (tensor-core gram)");
  const int vec = ((reinterpret_cast<uintptr_t>(B) & 15u) == 0 && (ldb & 3) == 0) ? 1 : 0;
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(mx, 0, 4 * (size_t)r, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 256, ctx->stream));
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(part, 0, 8 * (size_t)grid * (size_t)(r * r), ctx->stream));
  LRS_CUDA_TRY(ctx, cudaMemsetAsync(diag, 0, 8 * (size_t)grid * (size_t)r, ctx->stream));
  {
    int64_t nbx = (4 * sms + r - 1) / r;
    const int64_t cap = (n / 4 + 255) / 256;
    if (nbx > cap) nbx = cap;
    if (nbx < 1) nbx = 1;
    k_row_absmax<<<dim3((unsigned)nbx, (unsigned)r), 256, 0, ctx->stream>>>(B, n, ldb, vec, mx);
    ctx->launches++;
    LRS_CUDA_TRY(ctx, cudaGetLastError());
  }
  OzParams P{};
  P.B = B; P.n = n; P.ldb = ldb; P.r = ri; P.cw = cw; P.ngroups = ngroups;
  P.range_cols = range_cols; P.nranges = nranges; P.vec = vec;
  P.rowmax = mx; P.part = part; P.diag = diag; P.err = err;
  { const lrs_status s = raise_dyn_smem(ctx, (const void*)k_gram_oz, kOzSmem); if (s) return s; }
  k_gram_oz<<<(unsigned)grid, kOzThreads, kOzSmem, ctx->stream>>>(P);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  k_gram_oz_reduce<<<(ri * ri + 7) / 8, 256, 0, ctx->stream>>>(part, diag, (int)grid, ri, G);
  ctx->launches++;
  LRS_CUDA_TRY(ctx, cudaGetLastError());
  int* h = (int*)ctx->host_scratch;
  if (ctx->replay) {
    const int32_t* d[1] = {(const int32_t*)err};
    const lrs_status rs = replay_ints(ctx, 1, d, h + 24);
    if (rs) return rs;
  } else {
    LRS_CUDA_TRY(ctx, cudaMemcpyAsync(h + 24, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LRS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (h[24] != 0) return lrs_fail(ctx, LRS_ETIMEOUT, "tensor-core gram: a pipeline wait gave up");
  return LRS_OK;
}

}  // namespace lrs
