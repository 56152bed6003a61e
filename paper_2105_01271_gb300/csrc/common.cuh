// Shared device/host helpers of the lrs library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/lrs.h"

namespace lrs {

// ---------------------------------------------------------------------------
// element loads of A_f in its storage type, widened to double / float
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ld_f64(const void* p, int32_t dt, int64_t i) {
  if (dt == LRS_F64) return __ldg(reinterpret_cast<const double*>(p) + i);
  if (dt == LRS_F32) return (double)__ldg(reinterpret_cast<const float*>(p) + i);
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
  return (double)__uint_as_float(((unsigned)b) << 16);
}

// FP32 -> FP64 widening on the integer pipe: for a normal number the double
// has the same sign, the exponent rebiased by 1023 - 127 = 896 and the 23
// mantissa bits shifted up by 29 -- exact, the value the conversion
// instruction gives.  +-0 is built the same way; subnormals, infinities and
// NaN take the conversion instruction.  Keeps stencil loads off this part's
// narrow FP64 pipe, which the conversion instruction would otherwise share
// with the accumulation.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (e - 1u < 254u)
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
  return (double)f;
}

// FP64 -> FP32 pair on the integer pipe: hi = x truncated to 24 significant
// bits (exact FP32), lo = the next bits of x rounded to FP32, so hi + lo
// carries x to ~2^-47 relative.  For 2^-74 <= |x| < 2^127 (both parts normal
// FP32); outside it (and for 0, denormals, inf, NaN) the conversion
// instructions.  Keeps the narrow FP64
// pipe (64-cycle issue per warp instruction on this part) for the arithmetic.
__device__ __forceinline__ void split_f64_f2(double x, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7ffu) - 1023;           // unbiased exponent
  if (e >= -74 && e < 127) {                                // hi and lo both normal FP32
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const unsigned long long m = u & 0xfffffffffffffull;     // 52 fraction bits
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    const unsigned rest = (unsigned)(m & 0x1fffffffu);        // the low 29 bits
    // rest * 2^(e - 52): an integer-to-float conversion (rounds 29 to 24
    // bits), then the power of two from its exponent bits
    const float rf = __uint2float_rn(rest);
    lo = rest ? __uint_as_float(sign | __float_as_uint(rf) - ((unsigned)(52 - e) << 23)) : 0.0f;
    return;
  }
  hi = __double2float_rz(x);
  lo = __double2float_rn(x - (double)hi);
}

// Double-float arithmetic on (hi, lo) pairs of FP32 (Knuth's two-sum, the
// FMA two-product): about 2^-46 relative, on the FP32 pipe.  The _rn
// intrinsics keep the compiler from contracting the error-free steps.
struct df32 {
  float hi, lo;
};
__device__ __forceinline__ df32 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}
__device__ __forceinline__ df32 df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  const df32 s = df_two_sum(a.hi, b.hi);
  return df_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  return df_norm(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return df_norm(p, __fmaf_rn(a.lo, b, e));
}
__device__ __forceinline__ df32 df_from_f(float a) { return {a, 0.0f}; }
// a / b: the FP32 quotient and one correction from the double-float remainder
__device__ __forceinline__ df32 df_div(df32 a, df32 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df32 r = df_add(a, df_neg(df_mul_f(b, q1)));
  return df_norm(q1, __fdiv_rn(r.hi, b.hi));
}
// sqrt(a), a > 0: the FP32 root and one correction, (a - s^2) / (2 s)
__device__ __forceinline__ df32 df_sqrt(df32 a) {
  const float s = sqrtf(a.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(a.hi, p), __fsub_rn(a.lo, e));
  return df_norm(s, __fdiv_rn(r, 2.0f * s));
}
__device__ __forceinline__ df32 df_from_f64(double x) {
  df32 r;
  split_f64_f2(x, r.hi, r.lo);
  return r;
}

// element i of A_f widened to double, conversions on the integer pipe
__device__ __forceinline__ double ld_wide(const void* p, int32_t dt, int64_t i) {
  if (dt == LRS_F64) return __ldg(reinterpret_cast<const double*>(p) + i);
  if (dt == LRS_F32) return widen_f32(__ldg(reinterpret_cast<const float*>(p) + i));
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
  return widen_f32(__uint_as_float(((unsigned)b) << 16));
}

__device__ __forceinline__ size_t dtype_size(int32_t dt) {
  return dt == LRS_F64 ? 8 : (dt == LRS_F32 ? 4 : 2);
}

// ---------------------------------------------------------------------------
// pivot comparisons and reciprocal square roots off the FP64 pipe
//
// Pivoting compares non-negative squared norms.  Non-negative doubles order
// exactly as their bit patterns read as integers, so the comparison runs on
// the integer pipe (anything with the sign bit set, and +0, map to key 0).
__device__ __forceinline__ long long norm_key(double a) {
  const long long k = __double_as_longlong(a);
  return k > 0 ? k : 0;
}
// (a, position pa) beats (b, pb): larger value, lower position on ties
__device__ __forceinline__ bool pivot_better(double a, int pa, double b, int pb) {
  const long long ka = norm_key(a), kb = norm_key(b);
  return (ka > kb) || (ka == kb && pa < pb);
}

// 1/sqrt(x) for x > 0 with the short dependency chain this part's FP64 pipe
// wants (each dependent FP64 instruction waits ~64 cycles): the FP32 seed
// comes from the integer-pipe split and widening (no conversion
// instructions), then two Newton-Raphson steps y <- y (3 - x y^2) / 2 in
// FP64 reach FP64 precision.  Outside the seed's range, 1 / sqrt(x).
__device__ __forceinline__ double rsqrt_fast(double x) {
  if (!(x > 1e-22 && x < 1e38)) return 1.0 / sqrt(x);
  float xh, xl;
  split_f64_f2(x, xh, xl);
  double y = widen_f32(rsqrtf(xh));
  const double hx = 0.5 * x;
#pragma unroll
  for (int it = 0; it < 2; ++it) y = y * fma(-hx * y, y, 1.5);
  return y;
}

// A pivot candidate (norm^2, position, physical column) in one 16-byte record,
// written and read with single 16-byte accesses through L2 (ld/st .cg), so a
// block reads another block's candidate in one round trip.
struct __align__(16) PivotCand { double val; int pos; int phys; };

__device__ __forceinline__ void cand_store(PivotCand* p, double v, int pos, int phys) {
  int4 x;
  x.x = __double2loint(v); x.y = __double2hiint(v); x.z = pos; x.w = phys;
  __stcg(reinterpret_cast<int4*>(p), x);
}
__device__ __forceinline__ void cand_load(const PivotCand* p, double& v, int& pos, int& phys) {
  const int4 x = __ldcg(reinterpret_cast<const int4*>(p));
  v = __hiloint2double(x.y, x.x); pos = x.z; phys = x.w;
}

// ---------------------------------------------------------------------------
// warp / block reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; `red` must hold >= 32 elements of shared memory.  All
// threads return the total.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// Grid barrier with a bounded wait.
//
// Used only by kernels launched with cudaLaunchCooperativeKernel, which
// guarantees that all blocks are co-resident.  *count only grows (zeroed
// before the launch): thread 0 of each block arrives with one release-add,
// whose old value tells it which barrier this is (old / gridDim.x), and then
// polls with acquire loads until the count reaches the end of that barrier.
// The release orders every write the block made before the barrier (the
// block barrier before it gathers them to thread 0); the acquire and the
// block barrier after it order every read that follows.  Each wait gives up
// after kSpinLimit polls (about a second), records LRS_ETIMEOUT in *err and
// returns false; every block then leaves the kernel at its next barrier, so a
// lost arrival never hangs the GPU.
// ---------------------------------------------------------------------------
struct GridBarrier {
  unsigned int* count;   // arrivals so far (all barriers of the launch)
  unsigned int* gen;     // unused (kept for the buffer layout)
  int* err;              // 0 = ok, else an lrs_status
};

constexpr long long kSpinLimit = 20000000LL;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_release_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int ld_volatile_s32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

__device__ __forceinline__ bool grid_sync(const GridBarrier& b, long long spin_limit = kSpinLimit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned old = atom_add_release_u32(b.count, 1u);
    const unsigned target = (old / gridDim.x + 1u) * gridDim.x;
    long long it = 0;
    while ((int)(ld_acquire_u32(b.count) - target) < 0) {
      if (((++it) & 63) == 0 && ld_volatile_s32(b.err) != 0) break;
      if (it > spin_limit) { atomicCAS(b.err, 0, (int)LRS_ETIMEOUT); break; }
      if (it > 256) __nanosleep(20);
    }
  }
  __syncthreads();
  return ld_volatile_s32(b.err) == 0;
}

}  // namespace lrs

// ---------------------------------------------------------------------------
// host-side error plumbing
// ---------------------------------------------------------------------------
#define LRS_CUDA_TRY(ctx, expr)                                             \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) {                                                \
      return lrs_fail((ctx), LRS_ECUDA, "%s: %s (%s:%d)", #expr,            \
                      cudaGetErrorString(_e), __FILE__, __LINE__);          \
    }                                                                       \
  } while (0)
