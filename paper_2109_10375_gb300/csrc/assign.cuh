// Abundance matching: workspace layout and host entry (see assign.cu).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"  // FftProfile, prof_begin/prof_end, ProfKind

namespace amber {

typedef unsigned __int128 u128;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kMaxTable = 1 << 16;

// Per-tile look-back record: flag (0 none, 1 aggregate, 2 inclusive) and the
// two 128-bit values; the flag is released after the value is written.
struct __align__(16) ScanTile {
  unsigned int flag;
  unsigned int pad[3];
  unsigned long long agg_lo, agg_hi, inc_lo, inc_hi;
};

// ctrl: total mass (2 x u64) then the tile ticket (u32), zeroed per call
constexpr size_t kAssignCtrlBytes = 256;

struct AssignWork {
  unsigned char* ctrl;
  u128* X;        // [kMaxTable] thresholds
  float* inv_dx;  // [kMaxTable]
  ScanTile* state;
  int num_sms;
};

struct HistoryCoeffs {
  double a, b, c;
  double z_lo, z_hi;  // effective table range (z_lo lowered to a_w if needed)
  int n_table;
};

cudaError_t assign_impl(const AssignWork& w, const uint32_t* order, const float* mass, int64_t n,
                        const HistoryCoeffs& hc, float* zre, double* F, unsigned int* status, cudaStream_t s,
                        FftProfile* prof, unsigned int spin_limit);

}  // namespace amber
