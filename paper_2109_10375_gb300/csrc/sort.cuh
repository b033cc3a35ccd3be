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
  uint32_t* lookback;  // two regions of sort_tiles(max) * 256 words
  uint32_t* ctrl;      // kSortCtrlBytes
  int num_sms;
};

size_t sort_pass_smem(int key_bytes);
int64_t sort_tiles(int64_t n);

template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, unsigned int* status,
                      cudaStream_t s, FftProfile* prof, unsigned int spin_limit);

cudaError_t wait_timeout_test(uint32_t* zero_word, unsigned int* status, unsigned int spin_limit, cudaStream_t s);

}  // namespace amber
