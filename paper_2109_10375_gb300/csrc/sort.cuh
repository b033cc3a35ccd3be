// Onesweep LSD radix sort: constants, control block and host entry (see sort.cu).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"  // FftProfile, prof_begin/prof_end, ProfKind

namespace amber {

constexpr int kSortThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 4096 keys per tile
constexpr int kLookWindow = 8;                // predecessors read per look-back round trip
constexpr int kMaxRadix = 512;                // 9-bit digits
constexpr int kMaxHist = 2048;                // digit positions x radix, either key width

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
// FP32 intensities: 9-bit digits over the 32-bit key (at most 4 passes).
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

struct SortWork {
  void* keysA;
  void* keysB;
  uint32_t* idxA;
  uint32_t* idxB;
  float* massA;        // mass payload ping-pong (whole-path variant)
  float* massB;
  uint32_t* lookback;  // two regions of sort_lookback_words(max_cells)
  SortCtrl* ctrl;
  int64_t max_cells;
  int num_sms;
};

// Arguments of one digit pass (see k_sort_pass).
struct PassArgs {
  const void* J;        // first pass: intensities (float or double)
  const void* kin;      // later passes: keys - kmin
  const uint32_t* vin;  // later passes: cell indices
  const float* min;     // masses (cell order in the first pass, else ping-pong)
  void* kout;
  uint32_t* vout;
  float* mout;
  uint32_t* vfinal;     // if not null the last needed pass writes the order here,
  float* mfinal;        // and the masses in rank order here; else to its own
                        // parity's vout/mout (pass p writes the A side if p is even)
  int64_t n;
  int pass;
  uint32_t* lb;
  uint32_t* lb_next;
  SortCtrl* ctrl;
  unsigned long long* mass_total;  // first pass with masses: 128-bit sum (lo, hi)
  unsigned int* status;
  unsigned int spin_limit;
};

int64_t sort_tiles(int64_t n);
size_t sort_lookback_words(int64_t n);
cudaError_t sort_ctrl_reset(SortCtrl* ctrl, cudaStream_t s);

// Stable descending rank of J into order.  With mass_in != NULL the masses
// ride along as a payload: mass_out receives them in rank order and
// mass_total (zeroed by the caller) their exact 128-bit sum.  With order (and
// mass_out) NULL the results stay in idxA/massA when the needed pass count
// is odd and in idxB/massB when it is even (read it from ctrl->npasses).  range_ready:
// ctrl was reset and its key range already folded in (by the intensity
// kernel), so the range pass is skipped.
template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in,
                      float* mass_out, unsigned long long* mass_total, bool range_ready, unsigned int* status,
                      cudaStream_t s, FftProfile* prof, unsigned int spin_limit);

cudaError_t wait_timeout_test(uint32_t* zero_word, unsigned int* status, unsigned int spin_limit, cudaStream_t s);

}  // namespace amber
