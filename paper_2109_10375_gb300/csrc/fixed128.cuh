// Exact 128-bit fixed-point cell masses (64 integer, 64 fraction bits).
// Every float >= 2^-41 converts exactly, so sums of masses carry no rounding
// and do not depend on the order in which they are added.
#pragma once

#include "common.cuh"

namespace amber {

typedef unsigned __int128 u128;

// floor(v) for a float v in [0, 2^64) from two 32-bit conversions (the
// 64-bit conversions run on the FP64 pipe, which GB300 keeps narrow).
// hi = trunc(v 2^-32); v - hi 2^32 keeps only the bits of v below 2^32, at
// most 24 of them, so the FMA forms it exactly and lo = its floor.
__device__ __forceinline__ unsigned long long floor_u64(float v) {
  const float hf = truncf(v * 2.3283064365386963e-10f);
  const uint32_t hi = __float2uint_rz(hf);
  const uint32_t lo = __float2uint_rz(fmaf(-hf, 4294967296.0f, v));
  return ((unsigned long long)hi << 32) | lo;
}

// mass -> round-down fixed point; flags negative, NaN/Inf and >= 2^40.
// The largest of three power-of-two scales 2^k (k = 0, 40, 64) that keeps
// m 2^k below 2^64, floor_u64, then a constant shift by 64 - k.  Scaling by
// 2^k is exact, and in each range the float is a whole multiple of 2^-k
// (m >= 2^24: integral; m >= 1: ulp >= 2^-23; m >= 2^-41: ulp >= 2^-64), so
// the result is floor(m 2^64) exactly, from float conversions rather than
// exponent and mantissa bit surgery on the integer ALU.
__device__ __forceinline__ u128 mass_q64(float m, bool& bad) {
  const bool ok = m >= 0.0f && m < 1099511627776.0f;  // [0, 2^40); false for NaN
  bad |= !ok;
  const float v = ok ? m : 0.0f;
  const bool big = v >= 16777216.0f, mid = v >= 1.0f;
  const unsigned long long x = floor_u64(v * (big ? 1.0f : mid ? 1099511627776.0f : 18446744073709551616.0f));
  const unsigned long long lo = big ? 0ull : mid ? (x << 24) : x;
  const unsigned long long hi = big ? x : mid ? (x >> 40) : 0ull;
  return ((u128)hi << 64) | (u128)lo;
}

__device__ __forceinline__ u128 shfl_u128(u128 v, int src) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  return ((u128)__shfl_sync(0xffffffffu, hi, src) << 64) | (u128)__shfl_sync(0xffffffffu, lo, src);
}
__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  return ((u128)__shfl_up_sync(0xffffffffu, hi, d) << 64) | (u128)__shfl_up_sync(0xffffffffu, lo, d);
}
__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  return ((u128)__shfl_down_sync(0xffffffffu, hi, d) << 64) | (u128)__shfl_down_sync(0xffffffffu, lo, d);
}

__device__ __forceinline__ float u128_to_float(u128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return __ull2float_rn(hi) * 18446744073709551616.0f + __ull2float_rn(lo);
}
__device__ __forceinline__ double u128_to_double(u128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return __ull2double_rn(hi) * 18446744073709551616.0 + __ull2double_rn(lo);
}

// total += v for a 128-bit total held as two 64-bit words (exact; order-free).
__device__ __forceinline__ void atomic_add_u128(unsigned long long* total, u128 v) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  const unsigned long long old = atomicAdd(&total[0], lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(&total[1], hi + carry);
}

}  // namespace amber
