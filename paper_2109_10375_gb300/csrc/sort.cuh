// Onesweep LSD radix sort: constants, control block and host entry (see sort.cu).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"  // FftProfile, prof_begin/prof_end, ProfKind
#include "keys.cuh"

namespace amber {

// Tile geometry (build-time tunables: the defaults were measured best).
#ifndef AMBER_SORT_ITEMS
#define AMBER_SORT_ITEMS 16
#endif
#ifndef AMBER_SORT_MINB
#define AMBER_SORT_MINB 3
#endif
#ifndef AMBER_SORT_THREADS
#define AMBER_SORT_THREADS 256
#endif
constexpr int kSortThreads = AMBER_SORT_THREADS;  // 256 or 512 (divides the radix)
constexpr int kItems = AMBER_SORT_ITEMS;
constexpr int kTile = kSortThreads * kItems;  // 4096 keys per tile
constexpr int kLookWindow = 8;                // predecessors read per look-back round trip
constexpr int kMaxRadix = 512;                // digits of up to 9 bits

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
  unsigned long long* tile_mass;   // first pass with masses: per-tile 128-bit sums (lo, hi)
  unsigned int* status;
  unsigned int spin_limit;
  uint32_t ahead;  // tiles ahead whose inputs are prefetched into L2 (0: none)
};

// Arguments of one sort's histogram and digit-offset kernels.
struct HistArgs {
  const void* J;  // intensities (float or double)
  int64_t n;
  SortCtrl* ctrl;
  uint32_t* lb0;       // look-back region of the first pass (cleared here)
  int64_t lb0_words;
};

// Several sorts run together: one histogram launch, one offset launch (a
// CTA per item) and one launch per digit pass cover every item.  hist_prefix
// and tile_prefix (device, M + 1 entries) give each item's histogram CTAs and
// sort tiles; hist and pass[p] (device, M entries each) the items' arguments.
struct RankMulti {
  int M;
  const HistArgs* hist;
  const uint32_t* hist_prefix;
  uint32_t hist_blocks;
  const PassArgs* pass[4];
  const uint32_t* tile_prefix;
  uint32_t tiles;
};

// Host: the arguments of one sort of J (as rank_impl with the key range
// already folded into w.ctrl) -- its histogram CTAs and the arguments of every
// digit pass; returns the number of passes P (pass[0..P-1] filled).
template <typename SRC>
int rank_args(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in, float* mass_out,
              unsigned long long* tile_mass, unsigned int* status, unsigned int spin_limit, int digit_bits,
              HistArgs* hist, uint32_t* hist_blocks, PassArgs pass[4]);
// Enqueue the histogram, offsets and digit passes of r's sorts (FP32 keys,
// digit_bits 8 or 9, match: digit peers by warp match).
cudaError_t rank_multi(const RankMulti& r, int digit_bits, bool match, cudaStream_t s);

int64_t sort_tiles(int64_t n);
size_t sort_lookback_words(int64_t n);
cudaError_t sort_ctrl_reset(SortCtrl* ctrl, cudaStream_t s);

// Stable descending rank of J into order.  With mass_in != NULL the masses
// ride along as a payload: mass_out receives them in rank order and
// tile_mass[2t], [2t+1] the exact 128-bit sum of tile t's masses (no atomics;
// the abundance matching adds the sort_tiles(n) partials).  With order (and
// mass_out) NULL the results stay in idxA/massA when the needed pass count
// is odd and in idxB/massB when it is even (read it from ctrl->npasses).  range_ready:
// ctrl was reset and its key range already folded in (by the intensity
// kernel), so the range pass is skipped.  digit_bits: 9 or 8 for FP32 keys, 8
// for FP64 (0: the default, 9 / 8); match: 1 digit peers by warp match, 0 by
// ballots (default).  The environment variable AMBER_SORT_RANK=ballot|match
// overrides match.  hist_ready (FP32 keys, 8-bit digits, range_ready): the
// intensity kernel already counted the raw keys' digits into ctrl (hist8 of
// the radiation field), so the sort runs on raw keys without a histogram pass.
template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in,
                      float* mass_out, unsigned long long* tile_mass, bool range_ready, unsigned int* status,
                      cudaStream_t s, FftProfile* prof, unsigned int spin_limit, int digit_bits = 0, int match = 0,
                      bool hist_ready = false);

cudaError_t wait_timeout_test(uint32_t* zero_word, unsigned int* status, unsigned int spin_limit, cudaStream_t s);

}  // namespace amber
