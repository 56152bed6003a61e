// Splitting FP32/FP64 values into BF16 pieces x = x_0 + x_1 (+ x_2) for the
// tensor-core products (each piece is the round-to-nearest BF16 of what the
// previous pieces left over).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include "../../include/lrs.h"

namespace lrs {

template <int S>
__device__ __forceinline__ void split_f32(float a, __nv_bfloat16 (&p)[S]) {
  float r = a;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    p[i] = __float2bfloat16_rn(r);
    r = r - __bfloat162float(p[i]);
  }
}
template <int S>
__device__ __forceinline__ void split_f64(double a, __nv_bfloat16 (&p)[S]) {
  double r = a;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    p[i] = __float2bfloat16_rn((float)r);
    r = r - (double)__bfloat162float(p[i]);
  }
}

template <int S>
__device__ __forceinline__ void split_any(const void* base, int32_t dt, int64_t idx, bool valid,
                                          __nv_bfloat16 (&p)[S]) {
  if (!valid) {
#pragma unroll
    for (int i = 0; i < S; ++i) p[i] = __float2bfloat16_rn(0.f);
    return;
  }
  if (dt == LRS_F64) {
    split_f64<S>(reinterpret_cast<const double*>(base)[idx], p);
  } else if (dt == LRS_F32) {
    split_f32<S>(reinterpret_cast<const float*>(base)[idx], p);
  } else {
    const unsigned short b = reinterpret_cast<const unsigned short*>(base)[idx];
    split_f32<S>(__uint_as_float(((unsigned)b) << 16), p);
  }
}

// Two FP32 values at once: w[i] holds piece i of a (low half) and of b (high
// half).  Bit-identical to split_f32 on each value; one paired conversion per
// piece instead of two.
template <int S>
__device__ __forceinline__ void split2_f32(float a, float b, uint32_t (&w)[S]) {
  float ra = a, rb = b;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(ra, rb);
    uint32_t u;
    memcpy(&u, &h, sizeof(u));
    w[i] = u;
    if (i + 1 < S) {
      ra -= __uint_as_float(u << 16);
      rb -= __uint_as_float(u & 0xffff0000u);
    }
  }
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

}  // namespace lrs
