// Double-float arithmetic on the FP32 pipes.
//
// GB300 executes FP64 at a small fraction of its FP32 rate (a warp-wide FP64
// instruction occupies an SM's FP64 pipe for many cycles), so values that need
// more than FP32 precision inside hot loops are carried as an unevaluated sum
// hi + lo of two floats (~48-bit significand).  The building blocks are the
// classical error-free transformations: Knuth's TwoSum (exact a + b = s + e),
// the FMA-based TwoProd (exact a * b = p + e) and Dekker's FastTwoSum.
#pragma once

#include <cuda_runtime.h>

namespace srw {

struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ dfloat two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const dfloat s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ dfloat df_add(dfloat a, float b) {
  const dfloat s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const dfloat p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
}

__device__ __forceinline__ dfloat df_shfl_xor(dfloat v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ dfloat df_warp_sum(dfloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

// Split a double into hi + lo floats (host or device).
__host__ __device__ __forceinline__ dfloat df_from_double(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

}  // namespace srw
