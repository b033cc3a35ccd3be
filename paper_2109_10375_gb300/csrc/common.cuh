// Device-side helpers shared by the z_re(x) kernels: complex arithmetic,
// in-register DFTs, the device status word and bounded spin-waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include "../../include/amber.h"

namespace amber {

// ---------------------------------------------------------------------------
// Complex numbers (interleaved re, im), float or double.
// ---------------------------------------------------------------------------
template <typename T> struct alignas(2 * sizeof(T)) cpx { T x, y; };

template <typename T> __device__ __forceinline__ cpx<T> mk(T a, T b) { cpx<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {  // a * conj(b)
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return mk(a.x * s, a.y * s); }

// cos(2*pi*r/32) for r in [0, 8]: the first-quadrant values of the 32nd roots
// of unity (mathematical constants).
__device__ __forceinline__ constexpr double q32(int r) {
  return r == 0 ? 1.0
       : r == 1 ? 0.98078528040323044912618223613424
       : r == 2 ? 0.92387953251128675612818318939679
       : r == 3 ? 0.83146961230254523707878837761791
       : r == 4 ? 0.70710678118654752440084436210485
       : r == 5 ? 0.55557023301960222474283081394853
       : r == 6 ? 0.38268343236508977172845998403040
       : r == 7 ? 0.19509032201612826784828486847702
       : 0.0;
}

// Multiply by w^m where w = exp(-2 pi i / 32) (forward) or its conjugate
// (inverse).  m is a compile-time constant after unrolling, so the constants
// fold; quarter turns become swaps.
template <bool INV, typename T>
__device__ __forceinline__ cpx<T> rot32(cpx<T> a, int m) {
  m &= 31;
  const int q = m >> 3, r = m & 7;
  if (r == 0) {
    // exp(-i q pi/2): q=0 -> 1, q=1 -> -i, q=2 -> -1, q=3 -> +i  (forward)
    const int qq = INV ? (4 - q) & 3 : q;
    if (qq == 0) return a;
    if (qq == 1) return mk(a.y, -a.x);
    if (qq == 2) return mk(-a.x, -a.y);
    return mk(-a.y, a.x);
  }
  const T c = (T)q32(r), s = (T)q32(8 - r);   // cos(phi), sin(phi), phi = 2 pi r / 32
  // angle theta = q*pi/2 + phi ; w^m = cos(theta) - i sin(theta) (forward)
  T ct, st;
  if (q == 0) { ct = c; st = s; }
  else if (q == 1) { ct = -s; st = c; }
  else if (q == 2) { ct = -c; st = -s; }
  else { ct = s; st = -c; }
  if (INV) return mk(a.x * ct - a.y * st, a.x * st + a.y * ct);
  return mk(a.x * ct + a.y * st, a.y * ct - a.x * st);
}

constexpr int ilog2c(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Compile-time bit reversal of K over LOG bits.
template <int K, int LOG> struct BitRev {
  static constexpr int value = ((K & 1) << (LOG - 1)) | BitRev<(K >> 1), LOG - 1>::value;
};
template <int K> struct BitRev<K, 0> { static constexpr int value = 0; };

template <int R, typename T, int... K>
__device__ __forceinline__ void bitrev_permute(cpx<T>* v, std::integer_sequence<int, K...>) {
  constexpr int LOG = ilog2c(R);
  const cpx<T> t[R] = {v[BitRev<K, LOG>::value]...};
  ((v[K] = t[K]), ...);
}

// In-register DFT of R points (R = 1..32, power of two), natural order in and
// out: X_k = sum_n v_n exp(-+2 pi i n k / R).  Radix-2 decimation in
// frequency; the bit-reversed output is renamed back at compile time.
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft(cpx<T>* v) {
  if constexpr (R > 1) {
    constexpr int LOG = ilog2c(R);
#pragma unroll
    for (int st = 0; st < LOG; ++st) {
      const int half = R >> (st + 1);
#pragma unroll
      for (int g = 0; g < (1 << st); ++g) {
#pragma unroll
        for (int i = 0; i < half; ++i) {
          const int a0 = g * 2 * half + i;
          const cpx<T> a = v[a0], b = v[a0 + half];
          v[a0] = a + b;
          // twiddle exp(-2 pi i * i / (2 half)) = w32^(i * 32 / (2 half))
          v[a0 + half] = rot32<INV>(a - b, i * (32 / (2 * half)));
        }
      }
    }
    bitrev_permute<R, T>(v, std::make_integer_sequence<int, R>{});
  }
}

// True the first time it is called with a given device current (per flag):
// kernel attributes such as the dynamic shared-memory limit are set per device.
inline bool first_use_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  return (mask.fetch_or(bit) & bit) == 0;
}

// L2 eviction-priority policies for loads and stores that should (evict_last)
// or should not (evict_first) keep their lines in L2.
// Bulk L2 prefetch of the 16-byte-aligned part of [p, p + bytes) (the bulk
// copy engine takes only aligned addresses and sizes).  A hint only; nothing
// waits for it.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  const unsigned long long b = ((unsigned long long)p + 15ull) & ~15ull;
  const unsigned long long e = ((unsigned long long)p + bytes) & ~15ull;
  if (e > b)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"((uint32_t)(e - b)) : "memory");
}

__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void st_hint(float* a, float v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_hint(uint32_t* a, uint32_t v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t* a, unsigned long long pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_hint(const float* a, unsigned long long pol) {
  float v;
  asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}

// Launches that work on several items at once: item i owns blocks
// [prefix[i], prefix[i+1]) of the grid.  The item of block b is the largest i
// with prefix[i] <= b (an item with no blocks is skipped).
__device__ __forceinline__ int find_item(const uint32_t* __restrict__ prefix, int M, uint32_t b) {
  int lo = 0, hi = M - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Status word (device-side errors latch here; no trap, no assert).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(unsigned int* status, unsigned int bit) {
  atomicOr(status, bit);
}

// Bounded spin iterations for every device-side wait (lookback).  With a
// nanosleep backoff this is well under a second of waiting in total.
constexpr unsigned int kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace amber
