// Exact 128-bit fixed-point cell masses (64 integer, 64 fraction bits).
// Every float >= 2^-41 converts exactly, so sums of masses carry no rounding
// and do not depend on the order in which they are added.
#pragma once

#include "common.cuh"

namespace amber {

typedef unsigned __int128 u128;

// mass -> round-down fixed point; flags negative, NaN/Inf and >= 2^40.
__device__ __forceinline__ u128 mass_q64(float m, bool& bad) {
  const uint32_t b = __float_as_uint(m);
  if (b & 0x80000000u) {
    if (b != 0x80000000u) bad = true;  // negative (but -0 is zero)
    return 0;
  }
  const uint32_t e = b >> 23;
  if (e >= 127u + 40u) {  // >= 2^40, Inf or NaN
    bad = true;
    return 0;
  }
  const uint64_t mant = (e == 0) ? (b & 0x7fffffu) : ((b & 0x7fffffu) | 0x800000u);
  const int sh = (int)(e == 0 ? 1u : e) - 150 + 64;  // value = mant 2^(e-150), scaled by 2^64
  if (sh >= 0) return (u128)mant << sh;
  if (sh <= -24) return 0;
  return (u128)(mant >> (-sh));
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
