// Onesweep LSD radix sort: constants and host entry (see sort.cu).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"  // FftProfile, prof_begin/prof_end, ProfKind

namespace amber {

constexpr int kRadix = 256;
constexpr int kSortThreads = 256;  // one thread per digit in the tile epilogue
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 4096 keys per tile
constexpr int kLookWindow = 8;                 // predecessors read per look-back round trip

// Look-back status word: 2 flag bits over a 30-bit count.  Counts published
// by any tile but the last are < 2^30 because max_cells <= 2^30.
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kFlagMask = 3u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1u;

// hist [8][256], offsets [8][256], tickets [8] (uint32), rounded to 256 B
constexpr size_t kSortCtrlBytes = ((16 * kRadix + 8) * 4 + 255) / 256 * 256;

struct SortWork {
  void* keysA;
  void* keysB;
  uint32_t* idxA;
  uint32_t* idxB;
  float* massA;        // mass payload ping-pong (whole-path variant)
  float* massB;
  uint32_t* lookback;  // two regions of sort_tiles(max) * 256 words
  uint32_t* ctrl;      // kSortCtrlBytes
  int num_sms;
};

// Arguments of one digit pass (see k_sort_pass).
struct PassArgs {
  const void* J;           // FIRST: intensities (float or double)
  const void* kin;         // !FIRST: keys
  const uint32_t* vin;     // !FIRST: cell indices
  const float* min;        // MASS: masses (cell order if FIRST, else ping-pong)
  void* kout;              // !LAST
  uint32_t* vout;
  float* mout;             // MASS
  int64_t n;
  int shift;
  const uint32_t* bin_off;
  uint32_t* lb;
  uint32_t* lb_next;
  uint32_t* ticket;
  unsigned long long* mass_total;  // FIRST && MASS: 128-bit sum (lo, hi)
  unsigned int* status;
  unsigned int spin_limit;
};

size_t sort_pass_smem(int key_bytes, bool mass);
int64_t sort_tiles(int64_t n);

// Stable descending rank of J into order.  With mass_in != NULL the masses
// ride along as a payload: mass_out receives them in rank order and
// mass_total (zeroed by the caller) their exact 128-bit sum.
template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in,
                      float* mass_out, unsigned long long* mass_total, unsigned int* status, cudaStream_t s,
                      FftProfile* prof, unsigned int spin_limit);

cudaError_t wait_timeout_test(uint32_t* zero_word, unsigned int* status, unsigned int spin_limit, cudaStream_t s);

}  // namespace amber
