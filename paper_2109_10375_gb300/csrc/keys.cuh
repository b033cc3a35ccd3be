// Order-preserving sort keys and the per-sort control block, shared by the
// intensity kernels (which fold the key range in) and the radix sort.
#pragma once

#include "common.cuh"

namespace amber {

constexpr int kMaxHist = 2048;  // digit positions x radix, either key width

// Look-back status word: 2 flag bits over a 30-bit count.  Counts published
// by any tile but the last are < 2^30 because max_cells <= 2^30.
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1u;

// Order-preserving descending keys: ascending key order is descending value.
__device__ __forceinline__ uint32_t enc_desc(float v, bool& bad) {
  bad |= isnan(v);
  v = v + 0.0f;  // -0 -> +0
  const uint32_t b = __float_as_uint(v);
  const uint32_t u = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ~u;
}
__device__ __forceinline__ uint64_t enc_desc(double v, bool& bad) {
  bad |= isnan(v);
  v = v + 0.0;
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const uint64_t u = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  return ~u;
}

template <typename SRC> struct KeyOf;
// FP32 intensities: 9-bit digits over the 32-bit key by default (at most 4
// passes); the sort also has 8-bit instances (see max_passes in sort.cu).
template <> struct KeyOf<float> { using K = uint32_t; static constexpr int RB = 9; };
// FP64 intensities (n <= 256): 8-bit digits over the 64-bit key.
template <> struct KeyOf<double> { using K = uint64_t; static constexpr int RB = 8; };

// Per-sort control block in device memory.
struct SortCtrl {
  unsigned long long kmin, kmax;  // key range
  int npasses;                    // digit passes the range needs
  uint32_t pad;
  uint32_t ticket[8];             // tile tickets, one per pass
  uint32_t hist[kMaxHist];        // [pass][digit] counts of key - kmin
  uint32_t offs[kMaxHist];        // exclusive prefix of hist
};

// Block-wide min/max of this thread's keys folded into ctrl (every thread of
// the block must call it).
template <typename K>
__device__ __forceinline__ void key_range_commit(K lo, K hi, SortCtrl* ctrl) {
  __shared__ K smin[32], smax[32];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const K a = __shfl_down_sync(0xffffffffu, lo, o), b = __shfl_down_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { smin[warp] = lo; smax[warp] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) {
      lo = smin[w] < lo ? smin[w] : lo;
      hi = smax[w] > hi ? smax[w] : hi;
    }
    atomicMin(&ctrl->kmin, (unsigned long long)lo);
    atomicMax(&ctrl->kmax, (unsigned long long)hi);
  }
}

}  // namespace amber
