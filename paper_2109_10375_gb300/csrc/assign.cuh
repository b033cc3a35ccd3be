// Abundance matching: workspace layout and host entry (see assign.cu).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "fft.cuh"  // FftProfile, prof_begin/prof_end, ProfKind
#include "fixed128.cuh"

namespace amber {

// Scan tile shape and CTAs per SM (build-time tunables).
#ifndef AMBER_SCAN_THREADS
#define AMBER_SCAN_THREADS 512
#endif
#ifndef AMBER_SCAN_ITEMS
#define AMBER_SCAN_ITEMS 16
#endif
#ifndef AMBER_SCAN_MINB
#define AMBER_SCAN_MINB 2
#endif
constexpr int kScanThreads = AMBER_SCAN_THREADS;
constexpr int kScanItems = AMBER_SCAN_ITEMS;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kMaxTable = 1 << 16;
constexpr int kMaxBuckets = 1024;

constexpr int kBackTilesPerCta = 8;  // scan tiles one scatter-back CTA covers
constexpr int kBucketShift = 23;  // 2^23 cells (32 MB of z_re) per bucket by default

// ctrl: exact total mass (2 x u64) at 0, tile ticket (u32) at 16, scan
// fixed-point shift (int) at 32, scan total (u64) at 40; zeroed per call
constexpr size_t kAssignCtrlBytes = 256;

struct AssignWork {
  unsigned char* ctrl;
  unsigned long long* Xq;  // [kMaxTable] thresholds in the scan's fixed point
  float* inv_dx;           // [kMaxTable]
  float* lin;              // [4][kMaxTable]: P_j, Q_j, alpha_j, beta_j of the linear weightings
  unsigned long long* state;  // per scan tile: look-back word
  uint32_t* bcell;  // per scan tile, (cell, z) pairs grouped by bucket
  float* bz;
  uint16_t* btab;   // [tiles][nbuckets + 1] tile-local bucket starts
  int num_sms;
};

struct HistoryCoeffs {
  double a, b, c;
  double z_lo, z_hi;  // effective table range (z_lo lowered to a_w if needed)
  int n_table;
  int weighting;      // AMBER_WEIGHT_*
  double omega_m;     // growth factor's matter density (AMBER_WEIGHT_MASS_GROWTH)
  double z_mid;       // growth pivot
};

struct ScanArgs {
  const uint32_t* order;
  const float* mass;  // cell order (gathered through order) or rank order
  const uint32_t* order_b;  // with pick: the sort's results sit in (order, mass)
  const float* mass_b;      // for an odd pass count and in (order_b, mass_b) else
  const int* pick;          // &SortCtrl::npasses or null
  int64_t n;
  const unsigned long long* Xq;
  const int* qshift;                // fixed-point shift s of the masses
  const unsigned long long* qtotal;  // total in that fixed point (for F)
  const float* inv_dx;
  int n_table;
  float z_lo, z_hi, dzt;
  double* F;
  unsigned long long* state;
  uint32_t* ticket;
  int nbuckets;
  int bucket_shift;  // bucket of a cell = cell >> bucket_shift
  uint32_t* bcell;
  float* bz;
  uint16_t* btab;
  unsigned int* status;
  unsigned int spin_limit;
  uint32_t ahead;  // tiles ahead whose order and masses are prefetched into L2 (0: none)
  // linear weightings: margin h_j(n) = P_j - alpha_j n - beta_j M_n
  // = Q_j + alpha_j (N - n) + beta_j (T - M_n), P_j = x_j W_N(z_j),
  // Q_j = (x_j - 1) W_N(z_j) (real units)
  const float* linP;
  const float* linQ;
  const float* lina;
  const float* linb;
};

// Arguments of the thresholds kernel (one CTA per matching).
struct ThreshArgs {
  unsigned long long* total;             // exact mass total (2 x u64), formed here from tile_mass if given
  const unsigned long long* tile_mass;   // per-sort-tile partial sums or null
  int64_t ntiles;
  int M;                                 // table points
  double a_w, b_w, c_w, z_lo, z_hi;
  unsigned long long* Xq;
  float* inv_dx;
  int* qshift;
  unsigned long long* qtotal;
  int weighting;
  double omega_m, z_mid;
  int64_t ncells;
  float* lin;
};

// Arguments of the scatter back to cell order.
struct ScatterArgs {
  const uint32_t* bcell;
  const float* bz;
  const uint16_t* btab;
  int nbuckets;
  int64_t tiles;   // scan tiles
  int groups;      // scatter CTAs per bucket
  int wpt;         // warps sharing one tile's run (1, 2, 4, 8); a CTA covers 8 / wpt tiles
  float* zre;
};

// Several matchings run together: one thresholds launch (a CTA per item),
// one scan launch per weighting form (0: mass, 1: linear; items of each form
// contiguous, scan[f] and scan_prefix[f] with Mg[f] entries), one scatter
// launch.  All pointers are device arrays; the matchings' control words and
// scan look-back states must be zeroed beforehand.
struct AssignMulti {
  int M;
  const ThreshArgs* thresh;
  const ScanArgs* scan[2];
  const uint32_t* scan_prefix[2];
  int Mg[2];
  uint32_t scan_tiles[2];
  const ScatterArgs* scatter;
  const uint32_t* scatter_prefix;
  uint32_t scatter_blocks;
};

// Host: the arguments of one matching as assign_impl runs it (the masses in
// rank order and the total from tile_mass, no F).
void assign_args(const AssignWork& w, const uint32_t* order, const float* mass, const unsigned long long* tile_mass,
                 int64_t n, const HistoryCoeffs& hc, float* zre, double* F, unsigned int* status,
                 unsigned int spin_limit, const uint32_t* order_b, const float* mass_b, const int* pick,
                 ThreshArgs* ta, ScanArgs* sa, ScatterArgs* xa);
cudaError_t assign_multi(const AssignMulti& m, cudaStream_t s);

void bucket_plan(int64_t n, int* nbuckets, int* shift);

// Tomographic matching: fill z with NaN (neutral); give cells with a redshift
// intensity +inf (rank first); take the interval's redshift for neutral cells
// at or above z_low (all of them when last).
cudaError_t tomo_fill(float* z, int64_t n, int num_sms, cudaStream_t s);
cudaError_t tomo_mask(float* J, const float* z, int64_t n, SortCtrl* ctrl, int num_sms, cudaStream_t s);
cudaError_t tomo_merge(float* z, const float* ztmp, int64_t n, float z_low, bool last, int num_sms, cudaStream_t s);

// mass_in_rank_order: mass[n] belongs to rank n (sort payload) instead of to
// cell n.  tile_mass: per-tile partial mass sums from the ranking (summed in
// the thresholds kernel); null means one reduction pass over mass.
// order_b/mass_b/pick: see ScanArgs (null for a caller-given order).
cudaError_t assign_impl(const AssignWork& w, const uint32_t* order, const float* mass, bool mass_in_rank_order,
                        const unsigned long long* tile_mass, int64_t n, const HistoryCoeffs& hc, float* zre, double* F,
                        unsigned int* status, cudaStream_t s, FftProfile* prof, unsigned int spin_limit,
                        const uint32_t* order_b = nullptr, const float* mass_b = nullptr, const int* pick = nullptr);

}  // namespace amber
