// Abundance matching (Sec. 3.4.2): the rank-n cell is ionized at z_n where
// the cumulative mass fraction F_n = M_n / M_total equals the history x(z_n)
// (Sec. 3.1.2, Eq. weibull), with x(z) tabulated on uniform redshifts.
//
//   k_mass_reduce   : M_total = sum of all cell masses (order-free, exact)
//   k_thresholds    : table x_j = x(z_j) and integer thresholds
//                     X_j = floor(x_j * M_total) in the scan's fixed point,
//                     so "x_j >= F_n" is the integer test "X_j >= M_n";
//                     plus 1/(X_j - X_j+1)
//   k_scan_assign   : M_n by a decoupled-look-back prefix sum over ranks,
//                     bracket j* by a search in the thresholds amortised over
//                     each thread's run of ranks, interpolate to z_n, and
//                     write (cell, z_n) into buckets of consecutive cells
//   k_scatter_back  : per bucket, z_re[cell] = z_n; a bucket's cells span a
//                     region small enough to stay in L2, so the permuted
//                     writes reach HBM as whole sectors
//
// The total is summed exactly as 128-bit fixed point with 64 fraction bits.
// The running prefix uses 64-bit fixed point whose shift s is chosen from the
// total so it stays below 2^62: each mass is rounded down to a multiple of
// 2^-s, so F_n is off by at most n 2^-60 (1e-9 at 2^30 cells), and no sum
// depends on the order of addition.  Only the interpolation weight is FP32.
#include <cstdlib>

#include "assign.cuh"
#include "fixed128.cuh"
#include "sort.cuh"

namespace amber {

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mass_reduce(const float* __restrict__ mass, int64_t n,
                                                     unsigned long long* __restrict__ total,
                                                     unsigned int* __restrict__ status) {
  u128 acc = 0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // 16-byte loads only from a 16-byte aligned array, else element by element
  const int64_t nvec = (reinterpret_cast<uintptr_t>(mass) & 15) == 0 ? n / 4 : 0;
  for (int64_t v = gtid; v < nvec; v += stride) {
    const float4 m = reinterpret_cast<const float4*>(mass)[v];
    acc += mass_q64(m.x, bad) + mass_q64(m.y, bad) + mass_q64(m.z, bad) + mass_q64(m.w, bad);
  }
  for (int64_t i = nvec * 4 + gtid; i < n; i += stride) acc += mass_q64(mass[i], bad);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc += shfl_down_u128(acc, o);
  __shared__ u128 ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    u128 s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    if (s != 0) atomic_add_u128(total, s);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, AMBER_ERR_INVALID_MASS);
}

// floor(x * T) for x in [0, 1] and T < 2^128, exactly.
__device__ __forceinline__ u128 mul_floor(double x, u128 T) {
  if (!(x > 0.0)) return 0;
  if (x >= 1.0) return T;
  int ex;
  const double f = frexp(x, &ex);                                    // x = f 2^ex, f in [0.5, 1)
  const unsigned long long mant = (unsigned long long)ldexp(f, 53);  // exact 53-bit integer
  const int s = 53 - ex;                                             // x = mant 2^-s, s >= 53
  const unsigned long long tl = (unsigned long long)T, th = (unsigned long long)(T >> 64);
  const unsigned long long p0 = mant * tl, p0h = __umul64hi(mant, tl);
  const unsigned long long p1 = mant * th, p1h = __umul64hi(mant, th);
  const unsigned long long l1 = p0h + p1;
  const unsigned long long c1 = (l1 < p0h) ? 1ull : 0ull;
  const unsigned long long l2 = p1h + c1;
  // 192-bit product (l2:l1:p0) >> s
  if (s >= 192) return 0;
  const u128 top = ((u128)l2 << 64) | (u128)l1;
  if (s >= 64) return top >> (s - 64);
  return (top << (64 - s)) | (u128)(p0 >> s);
}

// Linear growth factor D(a) of flat LCDM (Omega_m = om, Omega_L = 1 - om),
// normalised to D = a early on: D(a) = (5 om / 2) E(a) int_0^a da'/(a' E(a'))^3
// with E(a) = sqrt(om a^-3 + 1 - om).  In closed form D(a) = a 2F1(1/3, 1;
// 11/6; -x) with x = a^3 (1 - om)/om; its power series converges fast for
// x <= 1/2 (every z above ~0.7 at om = 0.3).  Beyond that the integral is
// taken by Simpson's rule after the substitution a' = s^2, which makes the
// integrand 2 s^4 / (om + (1 - om) s^6)^(3/2) smooth at 0.
__device__ double growth_D(double a, double om) {
  const double ol = 1.0 - om;
  const double x = a * a * a * ol / om;
  if (x <= 0.5) {
    double sum = 0.0, term = 1.0;
    for (int k = 0; k < 200 && fabs(term) > 1e-18 * fabs(sum + 1.0); ++k) {
      sum += term;
      term *= -x * (1.0 / 3.0 + k) / (11.0 / 6.0 + k);
    }
    return a * sum;
  }
  const int S = 2048;  // even
  const double s1 = sqrt(a), hs = s1 / S;
  auto f = [&](double sv) {
    const double s2 = sv * sv, s6 = s2 * s2 * s2;
    const double d = om + ol * s6;
    return 2.0 * s2 * s2 / (d * sqrt(d));
  };
  double acc = f(0.0) + f(s1);
  for (int i = 1; i < S; ++i) acc += (i & 1 ? 4.0 : 2.0) * f(i * hs);
  const double I = acc * hs / 3.0;
  const double E = sqrt(om / (a * a * a) + ol);
  return 2.5 * om * E * I;
}

// tile_mass (optional): per-tile partial sums from the ranking; their total
// is formed here (exact, order-free).  From the exact total T (2^-64 units)
// the kernel picks the scan's fixed-point shift s (total below 2^62), and
// tabulates X_j = floor(x_j T 2^(s-64)) so "x_j >= F_n" is the integer test
// "X_j >= M_n", plus 1/(X_j - X_j+1) for the interpolation weight.
__device__ __forceinline__ void thresholds_body(const ThreshArgs& A) {
  unsigned long long* __restrict__ total = A.total;
  const unsigned long long* __restrict__ tile_mass = A.tile_mass;
  const int64_t ntiles = A.ntiles;
  const int M = A.M;
  const double a_w = A.a_w, b_w = A.b_w, c_w = A.c_w, z_lo = A.z_lo, z_hi = A.z_hi;
  unsigned long long* __restrict__ Xq = A.Xq;
  float* __restrict__ inv_dx = A.inv_dx;
  int* __restrict__ qshift = A.qshift;
  unsigned long long* __restrict__ qtotal = A.qtotal;
  const int weighting = A.weighting;
  const double omega_m = A.omega_m, z_mid = A.z_mid;
  const int64_t ncells = A.ncells;
  float* __restrict__ lin = A.lin;
  __shared__ u128 ws[32];
  __shared__ u128 sT;
  __shared__ int s_shift;
  if (tile_mass) {
    u128 acc = 0;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x)
      acc += ((u128)tile_mass[2 * t + 1] << 64) | (u128)tile_mass[2 * t];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += shfl_down_u128(acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      u128 s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
      total[0] = (unsigned long long)s;
      total[1] = (unsigned long long)(s >> 64);
      sT = s;
    }
  } else if (threadIdx.x == 0) {
    sT = ((u128)total[1] << 64) | (u128)total[0];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // bit length L of T; the real total is below 2^(L-64), so s = 126 - L
    // keeps it below 2^62 (s <= 64: no finer than the exact representation)
    int L = 0;
    for (u128 v = sT; v != 0; v >>= 1) ++L;
    int s = 126 - L;
    if (s > 64) s = 64;
    s_shift = s;
    *qshift = s;
    const int sh = 64 - s;
    *qtotal = (unsigned long long)(sh >= 0 ? (sT >> sh) : (sT << (-sh)));
  }
  __syncthreads();
  const u128 T = sT;
  const int sh = 64 - s_shift;  // X in 2^-s units: floor(x T) >> (64 - s)
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const double z = z_lo + (z_hi - z_lo) * (double)j / (double)(M - 1);
    const double u = fmax((z - a_w) / b_w, 0.0);
    const double x = exp(-pow(u, c_w));
    const u128 X = mul_floor(x, T);
    Xq[j] = (unsigned long long)(sh >= 0 ? (X >> sh) : (X << (-sh)));
    if (weighting != AMBER_WEIGHT_MASS) {
      // weight of a cell at z_j: alpha_j + beta_j mass; margin h_j(n) =
      // x_j W_N - W_n.  Two equal forms keep the operands small at either end
      // of the ranking: the head form x_j W_N - alpha_j n - beta_j M_n for the
      // first half of the ranks, and the tail form (x_j - 1) W_N +
      // alpha_j (N - n) + beta_j (T - M_n) for the second, where the weight
      // after rank n (all that is left on the x = 1 plateau) comes from exact
      // differences
      double alpha = 1.0, beta = 0.0;  // volume
      if (weighting == AMBER_WEIGHT_MASS_GROWTH) {
        const double g = growth_D(1.0 / (1.0 + z), omega_m) / growth_D(1.0 / (1.0 + z_mid), omega_m);
        alpha = 1.0 - g;
        beta = g;
      }
      const double Treal = u128_to_double(T) * 5.421010862427522e-20;  // 2^-64
      const double WN = alpha * (double)ncells + beta * Treal;
      lin[j] = (float)(x * WN);
      lin[kMaxTable + j] = (float)((x - 1.0) * WN);
      lin[2 * kMaxTable + j] = (float)alpha;
      lin[3 * kMaxTable + j] = (float)beta;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < M - 1; j += blockDim.x) {
    const unsigned long long d = Xq[j] - Xq[j + 1];
    inv_dx[j] = d > 0 ? 1.0f / __ull2float_rn(d) : 0.0f;
  }
}

__global__ void __launch_bounds__(1024) k_thresholds(const ThreshArgs A) { thresholds_body(A); }

// One CTA per item.
__global__ void __launch_bounds__(1024) k_thresholds_multi(const ThreshArgs* __restrict__ args) {
  thresholds_body(args[blockIdx.x]);
}

// ---------------------------------------------------------------------------
// Cell mass in the scan's 64-bit fixed point: floor(m 2^s), s chosen per call
// by k_thresholds so the total stays below 2^62.  Each cell loses less than
// 2^-s, so over n cells F_n is off by less than n 2^-s / T <= n 2^-62 (2e-10
// relative at 2^30 cells) -- far inside an FP64 running sum's own error.
// scale = 2^s: scaling by a power of two is exact, so this is floor_u64 of
// m 2^s (below 2^62 for every valid mass, since m <= T); masses the total pass
// flagged count as 0.
__device__ __forceinline__ unsigned long long mass_fix(float m, float scale) {
  return (m >= 0.0f && m < 1099511627776.0f) ? floor_u64(m * scale) : 0ull;
}

// u64 -> float from its two 32-bit halves (within two roundings; only the
// interpolation weight uses it)
__device__ __forceinline__ float u64_to_float(unsigned long long x) {
  return fmaf(__uint2float_rn((uint32_t)(x >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)x));
}

// Look-back word of a scan tile: 2 flag bits over a 62-bit prefix.
constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanInc = 2ull << 62;
constexpr unsigned long long kScanMask = 3ull << 62;
constexpr unsigned long long kScanValue = (1ull << 62) - 1ull;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One round of a warp-wide 32-ary search for c = #{j : X_j >= v} (X
// non-increasing), c known to lie in [lo, hi]: lane k probes lo + k step; the
// probes that hold form a prefix, and the range shrinks below step.
__device__ __forceinline__ void count_ge_round(const unsigned long long* __restrict__ X, unsigned long long v,
                                               int& lo, int& hi, int lane) {
  if (lo >= hi) return;  // warp-uniform
  const int step = (hi - lo + 31) >> 5;
  const int q = lo + lane * step;
  const bool t = q < hi && X[q] >= v;
  const int c = __popc(__ballot_sync(0xffffffffu, t));
  const int nlo = c ? lo + (c - 1) * step + 1 : lo;
  const int nhi = min(hi, lo + c * step);
  lo = nlo;
  hi = nhi;
}

constexpr int kScanWin = 64;  // thresholds one tile may span, staged in shared memory

constexpr int kLinCand = 256;  // table points a tile's cells may straddle (linear weightings)

// LIN: a linear weighting (growth or volume).  The exact-integer threshold
// test of the mass weighting is replaced by the margins h_j(n) in FP32: per
// tile, every table point is classified against the box of (n, M_n) the
// tile's cells span -- ionized for all of them, for none, or straddling --
// and each cell takes the largest point that ionizes it among
// max{j : all ionized} and the straddling points above it.
template <bool GATHER, bool WANT_F, bool LIN>
__device__ __forceinline__ void scan_assign_body(const ScanArgs& a) {
  constexpr int NT = kScanThreads, IT = kScanItems, TILE = kScanTile;
  __shared__ int s_jall, s_ncand;
  __shared__ int s_cand[LIN ? kLinCand : 1];
  __shared__ uint32_t sord[TILE + TILE / 32];
  __shared__ float smass[TILE + TILE / 32];
  __shared__ unsigned long long wtot[NT / 32];
  __shared__ unsigned long long s_excl;
  __shared__ uint32_t s_tile;
  __shared__ int s_cx[3];  // c(M_last), c(M_first), first staged threshold (-1: none)
  __shared__ unsigned long long sX[kScanWin];
  __shared__ float sInv[kScanWin];
  __shared__ uint32_t scnt[kMaxBuckets];
  __shared__ uint32_t soff[kMaxBuckets + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(a.ticket, 1u);
    s_jall = -1;
    s_ncand = 0;
  }
  for (int b = tid; b < a.nbuckets; b += NT) scnt[b] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  // n <= 2^30: positions fit 32 bits
  const uint32_t start = tile * (uint32_t)TILE;
  const uint32_t n = (uint32_t)a.n;
  const int cnt = (int)(n - start < (uint32_t)TILE ? n - start : (uint32_t)TILE);
  const bool side_b = a.pick && ((*a.pick - 1) & 1);
  const uint32_t* order = side_b ? a.order_b : a.order;
  const float* mass = side_b ? a.mass_b : a.mass;
  if (tid == 0 && a.ahead) {
    // order and masses of the tile a.ahead tickets later into L2
    const uint32_t fs = (tile + a.ahead) * (uint32_t)TILE;
    if (fs < n) {
      const uint32_t fb = n - fs < (uint32_t)TILE ? n - fs : (uint32_t)TILE;
      prefetch_l2_bulk(order + fs, fb * 4u);
      if constexpr (!GATHER) prefetch_l2_bulk(mass + fs, fb * 4u);
    }
  }
  const float qs = __int_as_float((127 + *a.qshift) << 23);  // 2^s, s in [-2, 64]
  const int M = a.n_table;

  // order (and rank-order masses): coalesced striped loads -> padded shared
  // memory -> a blocked run of IT consecutive ranks per thread
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int p = k * NT + tid;
    sord[p + (p >> 5)] = p < cnt ? order[start + p] : 0u;
    if constexpr (!GATHER) smass[p + (p >> 5)] = p < cnt ? mass[start + p] : 0.0f;
  }
  __syncthreads();
  uint32_t cell[IT];
  float mv[IT];
  unsigned long long run = 0;
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int p = tid * IT + i;
    cell[i] = sord[p + (p >> 5)];
    mv[i] = 0.0f;
    if (p < cnt) mv[i] = GATHER ? mass[cell[i]] : smass[p + (p >> 5)];
    run += mass_fix(mv[i], qs);
  }
  // block exclusive scan of the thread totals
  unsigned long long x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[warp] = x;
  __syncthreads();
  unsigned long long wpre = 0, tile_sum = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    if (w < warp) wpre += wtot[w];
    tile_sum += wtot[w];
  }
  const unsigned long long thr_excl = wpre + x - run;

  // warp 0 publishes the tile's aggregate and starts its look-back load; the
  // bucket slots of every cell (which need no prefix) are taken meanwhile
  unsigned long long lbw = 0;
  int64_t lbt = (int64_t)tile - 1;
  if (warp == 0) {
    if (lane == 0) st_relaxed_u64(a.state + tile, (tile == 0 ? kScanInc : kScanAgg) | tile_sum);
    lbw = (lbt - lane >= 0) ? ld_relaxed_u64(a.state + lbt - lane) : kScanInc;
  }
  uint32_t slot[IT];
  if (a.nbuckets <= 16) {
    // few buckets (small grids: one below 2^23 cells): most lanes share one,
    // and one shared add per lane would serialise on its counter; the lanes
    // of a bucket take their slots with one add for the warp
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const bool ok = tid * IT + i < cnt;
      const unsigned bk = ok ? cell[i] >> a.bucket_shift : 0xffffu;
      const unsigned peers = __match_any_sync(0xffffffffu, bk);
      const int leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (ok && lane == leader) base = atomicAdd(&scnt[bk], (uint32_t)__popc(peers));
      base = __shfl_sync(0xffffffffu, base, leader);
      slot[i] = ok ? base + (uint32_t)__popc(peers & lt) : 0xffffffffu;
    }
  } else {
#pragma unroll
    for (int i = 0; i < IT; ++i)
      slot[i] = (tid * IT + i < cnt) ? atomicAdd(&scnt[cell[i] >> a.bucket_shift], 1u) : 0xffffffffu;
  }
  __syncthreads();

  if (warp == 0) {
    // decoupled look-back: each lane holds one predecessor's word, so a round
    // trip covers 32 tiles; aggregates are summed back to the nearest
    // inclusive prefix
    unsigned long long excl = 0;
    unsigned spins = 0;
    while (true) {
      const unsigned long long f = lbw & kScanMask;
      const unsigned inc_mask = __ballot_sync(0xffffffffu, f == kScanInc);
      const unsigned stop_mask = inc_mask | __ballot_sync(0xffffffffu, f == 0ull);
      const int first = stop_mask ? __ffs(stop_mask) - 1 : 32;
      const bool found = first < 32 && ((inc_mask >> first) & 1u);
      unsigned long long part = (lane < first || (found && lane == first)) ? (lbw & kScanValue) : 0ull;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
      excl += __shfl_sync(0xffffffffu, part, 0);
      if (found) break;
      lbt -= first;
      if (first < 32) {
        if (++spins >= a.spin_limit) {
          if (lane == 0) raise_status(a.status, AMBER_ERR_DEVICE_TIMEOUT);
          break;
        }
        __nanosleep(20);
      }
      lbw = (lbt - lane >= 0) ? ld_relaxed_u64(a.state + lbt - lane) : kScanInc;
    }
    if (lane == 0) {
      if (tile != 0) st_relaxed_u64(a.state + tile, kScanInc | ((excl + tile_sum) & kScanValue));
      s_excl = excl;
    }
    // bracket the whole tile: c(M) = #{j : X_j >= M} at its first and last
    // prefix, both searched at once (three round trips for 2000 thresholds)
    int lo0 = 0, hi0 = LIN ? 0 : M, lo1 = 0, hi1 = LIN ? 0 : M;
    while (lo0 < hi0 || lo1 < hi1) {
      count_ge_round(a.Xq, excl, lo0, hi0, lane);
      count_ge_round(a.Xq, excl + tile_sum, lo1, hi1, lane);
    }
    // thresholds the tile's cells can touch: X_j for j in [c_last - 1, c_first]
    const int base = max(lo1 - 1, 0), L = min(lo0, M - 1) - base + 1;
    const bool stage = !LIN && L <= kScanWin;
    if (stage) {
      for (int i = lane; i < L; i += 32) {
        sX[i] = a.Xq[base + i];
        sInv[i] = (base + i < M - 1) ? a.inv_dx[base + i] : 0.0f;
      }
    }
    if (lane == 0) {
      s_cx[0] = lo1;
      s_cx[1] = lo0;
      s_cx[2] = stage ? base : -1;
    }
  } else if (warp == 1) {
    // tile-local bucket starts (exclusive scan over the buckets) and this
    // tile's row of the offset table
    uint32_t carry = 0;
    uint16_t* row = a.btab + (int64_t)tile * (a.nbuckets + 1);
    for (int b0 = 0; b0 < a.nbuckets; b0 += 32) {
      const int b = b0 + lane;
      const uint32_t c = b < a.nbuckets ? scnt[b] : 0u;
      uint32_t y = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += z;
      }
      if (b < a.nbuckets) {
        soff[b] = carry + y - c;
        row[b] = (uint16_t)(carry + y - c);
      }
      carry += __shfl_sync(0xffffffffu, y, 31);
    }
    if (lane == 0) {
      soff[a.nbuckets] = carry;
      row[a.nbuckets] = (uint16_t)carry;
    }
  }
  __syncthreads();
  unsigned long long Mn = s_excl + thr_excl;
  const double invT = WANT_F ? 1.0 / (double)*a.qtotal : 0.0;
  const float qinv = __int_as_float((127 - *a.qshift) << 23);  // 2^-s: fixed point -> mass units
  const unsigned long long qT = LIN ? *a.qtotal : 0ull;  // total in the prefix's fixed point (>= every M_n)
  // head form (ranks in the first half) or tail form, for the tile's box:
  // h = C_j + sa alpha_j u + sa beta_j v with (C, u, v, sa) = (x W_N, n, M_n, -1)
  // or ((x - 1) W_N, N - n, T - M_n, +1)
  const bool head = start + (uint32_t)cnt / 2u <= n / 2u;
  const float* linC = head ? a.linP : a.linQ;
  const float sa = head ? -1.0f : 1.0f;
  if constexpr (LIN) {
    // (u, v) of the tile's cells lie in the box [u0, u1] x [v0, v1]; a linear
    // margin takes its extremes at the corners
    const float u0 = head ? (float)(start + 1u) : (float)(n - (start + (uint32_t)cnt));
    const float u1 = head ? (float)(start + (uint32_t)cnt) : (float)(n - (start + 1u));
    const float v0 = head ? u64_to_float(s_excl) * qinv : u64_to_float(qT - (s_excl + tile_sum)) * qinv;
    const float v1 = head ? u64_to_float(s_excl + tile_sum) * qinv : u64_to_float(qT - s_excl) * qinv;
    auto classify = [&](int j, float& hmin, float& hmax, float& tol) {
      const float Cj = linC[j], al = sa * a.lina[j], be = sa * a.linb[j];
      const float au0 = al * u0, au1 = al * u1, bv0 = be * v0, bv1 = be * v1;
      hmin = Cj + fminf(au0, au1) + fminf(bv0, bv1);
      hmax = Cj + fmaxf(au0, au1) + fmaxf(bv0, bv1);
      tol = 4e-7f * (fabsf(Cj) + fmaxf(fabsf(au0), fabsf(au1)) + fmaxf(fabsf(bv0), fabsf(bv1)));
    };
    for (int j = tid; j < M; j += NT) {
      float hmin, hmax, tol;
      classify(j, hmin, hmax, tol);
      if (hmin >= tol) atomicMax(&s_jall, j);
    }
    __syncthreads();
    const int jall = s_jall;
    for (int j = jall + 1 + tid; j < M; j += NT) {
      float hmin, hmax, tol;
      classify(j, hmin, hmax, tol);
      if (hmax >= -tol) {
        const int k = atomicAdd(&s_ncand, 1);
        if (k < kLinCand) s_cand[k] = j;
      }
    }
    __syncthreads();
  }
  const int cx_lo = s_cx[0], cx_hi = s_cx[1], wb = s_cx[2];
  // threshold j from the staged window when the tile fits it
  auto Xj = [&](int j) -> unsigned long long { return wb >= 0 ? sX[j - wb] : a.Xq[j]; };
  auto Ij = [&](int j) -> float { return wb >= 0 ? sInv[j - wb] : a.inv_dx[j]; };

  // bracket: cx = #{j : X_j >= M_n}; X is non-increasing in j and M_n grows
  // with rank, so each thread searches the tile's range once, then walks
  // down.  Each (cell, z) goes straight to its bucket-ordered staging slot
  // (order and masses were consumed above, so their shared arrays are free).
  uint32_t* scell = sord;
  float* sz = smass;
  if (LIN && s_ncand == 0) {
    // no table point above max{j : all ionized} can ionize any cell of the
    // tile: every cell takes j* = jall, whose two margin rows are held in
    // registers
    const int js = s_jall;
    const bool mid = js >= 0 && js < M - 1;
    float la0 = 0.f, lb0 = 0.f, P0 = 0.f, Q0 = 0.f, la1 = 0.f, lb1 = 0.f, P1 = 0.f, Q1 = 0.f;
    if (mid) {
      la0 = a.lina[js], lb0 = a.linb[js], P0 = a.linP[js], Q0 = a.linQ[js];
      la1 = a.lina[js + 1], lb1 = a.linb[js + 1], P1 = a.linP[js + 1], Q1 = a.linQ[js + 1];
    }
    const float zc = js < 0 ? a.z_lo : a.z_hi;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int p = tid * IT + i;
      if (p >= cnt) continue;
      Mn += mass_fix(mv[i], qs);
      float z = zc;
      if (mid) {
        const uint32_t rank1 = start + (uint32_t)p + 1u;
        const bool chead = rank1 <= n / 2u;
        const float cs = chead ? -1.0f : 1.0f;
        const float uu = cs * (chead ? (float)rank1 : (float)(n - rank1));
        const float vv = cs * (chead ? u64_to_float(Mn) * qinv : u64_to_float(qT - Mn) * qinv);
        const float h0 = fmaf(lb0, vv, fmaf(la0, uu, chead ? P0 : Q0));
        const float h1 = fmaf(lb1, vv, fmaf(la1, uu, chead ? P1 : Q1));
        float t = h0 / (h0 - h1);
        t = fminf(fmaxf(t, 0.0f), 0.99999994f);
        z = a.z_lo + ((float)js + t) * a.dzt;
      }
      if (WANT_F) a.F[start + p] = (double)Mn * invT;
      const uint32_t q = soff[cell[i] >> a.bucket_shift] + slot[i];
      scell[q + (q >> 5)] = cell[i];
      sz[q + (q >> 5)] = z;
    }
  } else if (!LIN && cx_lo == cx_hi) {
    // the whole tile between two thresholds (all but a few tiles): one
    // interval, its threshold and slope held in registers
    const int j = cx_lo - 1;
    const bool mid = j >= 0 && j < M - 1;
    const unsigned long long Xu = mid ? Xj(j) : 0ull;
    const float Iu = mid ? Ij(j) : 0.0f;
    const float zc = j < 0 ? a.z_lo : a.z_hi;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int p = tid * IT + i;
      if (p >= cnt) continue;
      Mn += mass_fix(mv[i], qs);
      float z = zc;
      if (mid) {
        float t = u64_to_float(Xu - Mn) * Iu;
        t = fminf(fmaxf(t, 0.0f), 0.99999994f);
        z = a.z_lo + ((float)j + t) * a.dzt;
      }
      if (WANT_F) a.F[start + p] = (double)Mn * invT;
      const uint32_t q = soff[cell[i] >> a.bucket_shift] + slot[i];
      scell[q + (q >> 5)] = cell[i];
      sz[q + (q >> 5)] = z;
    }
  } else {
    int cx = -1;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int p = tid * IT + i;
      if (p >= cnt) continue;
      Mn += mass_fix(mv[i], qs);
      if constexpr (LIN) {
        // the cell's own form (a tile can straddle the middle rank; the tile's
        // classification above carries a tolerance for either form)
        const uint32_t rank1 = start + (uint32_t)p + 1u;
        const bool chead = rank1 <= n / 2u;
        const float cs = chead ? -1.0f : 1.0f;
        const float* cC = chead ? a.linP : a.linQ;
        const float uu = cs * (chead ? (float)rank1 : (float)(n - rank1));
        const float vv = cs * (chead ? u64_to_float(Mn) * qinv : u64_to_float(qT - Mn) * qinv);
        auto h = [&](int j) { return fmaf(a.linb[j], vv, fmaf(a.lina[j], uu, cC[j])); };
        int js = s_jall;
        const int nc = s_ncand;
        if (nc <= kLinCand) {
          for (int k = 0; k < nc; ++k) {
            const int c = s_cand[k];
            if (c > js && h(c) >= 0.0f) js = c;
          }
        } else {
          for (int c = M - 1; c > js; --c)
            if (h(c) >= 0.0f) { js = c; break; }
        }
        float z;
        if (js < 0) z = a.z_lo;
        else if (js == M - 1) z = a.z_hi;
        else {
          const float h0 = h(js), h1 = h(js + 1);
          float t = h0 / (h0 - h1);
          t = fminf(fmaxf(t, 0.0f), 0.99999994f);
          z = a.z_lo + ((float)js + t) * a.dzt;
        }
        if (WANT_F) a.F[start + p] = (double)Mn * invT;
        const uint32_t q = soff[cell[i] >> a.bucket_shift] + slot[i];
        scell[q + (q >> 5)] = cell[i];
        sz[q + (q >> 5)] = z;
        continue;
      }
      if (cx < 0) {
        int lo = cx_lo, hi = cx_hi;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (Xj(mid) >= Mn) lo = mid + 1; else hi = mid;
        }
        cx = lo;
      } else {
        while (cx > 0 && Xj(cx - 1) < Mn) --cx;
      }
      const int j = cx - 1;
      float z;
      if (j < 0) z = a.z_lo;
      else if (j == M - 1) z = a.z_hi;
      else {
        float t = u64_to_float(Xj(j) - Mn) * Ij(j);
        t = fminf(fmaxf(t, 0.0f), 0.99999994f);
        z = a.z_lo + ((float)j + t) * a.dzt;
      }
      if (WANT_F) a.F[start + p] = (double)Mn * invT;
      const uint32_t q = soff[cell[i] >> a.bucket_shift] + slot[i];
      scell[q + (q >> 5)] = cell[i];
      sz[q + (q >> 5)] = z;
    }
  }
  __syncthreads();
  // the pairs are read back only after the whole scan: keep them out of L2
  const unsigned long long pol = l2_evict_first();
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int p = k * NT + tid;
    if (p < cnt) {
      st_hint(a.bcell + start + p, scell[p + (p >> 5)], pol);
      st_hint(a.bz + start + p, sz[p + (p >> 5)], pol);
    }
  }
}

template <bool GATHER, bool WANT_F, bool LIN>
__global__ void __launch_bounds__(kScanThreads, AMBER_SCAN_MINB) k_scan_assign(const ScanArgs a) {
  scan_assign_body<GATHER, WANT_F, LIN>(a);
}

// Several matchings at once: CTA b works on item find_item(prefix, M, b) (the
// prefix counts scan tiles), taking its tile from that item's own ticket.
template <bool LIN>
__global__ void __launch_bounds__(kScanThreads, AMBER_SCAN_MINB)
    k_scan_assign_multi(const ScanArgs* __restrict__ args, const uint32_t* __restrict__ prefix, int M) {
  __shared__ ScanArgs sa;
  if (threadIdx.x == 0) sa = args[find_item(prefix, M, blockIdx.x)];
  __syncthreads();
  scan_assign_body<false, false, LIN>(sa);
}

// z_re[cell] = z, bucket after bucket: CTA (bucket b, tile group g) copies
// bucket b's run of every tile in its group (one tile per warp at the
// default group size).  A warp takes its runs in rounds of four 32-pair
// chunks: all the round's loads (lanes read a run coalesced), then its
// stores, so the dependent load -> store chains overlap.  A
// bucket's cells span a bounded region of z_re, so the permuted writes of
// the CTAs working on it stay close together.
// wpt (1, 2, 4 or 8) warps share one tile's run, each taking a contiguous
// part: with few buckets (small grids) a run holds most of a tile's 8192
// pairs, and one warp copying it alone would wait through dozens of rounds.
__device__ __forceinline__ void scatter_back_body(const uint32_t* __restrict__ bcell, const float* __restrict__ bz,
                                                  const uint16_t* __restrict__ btab, int nbuckets, int64_t tiles,
                                                  int groups, int wpt, float* __restrict__ zre, uint32_t blk) {
  constexpr int TPW = 1;  // tiles per warp
  const int b = blk / groups;
  const int64_t g = blk - (int64_t)b * groups;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long stream_pol = l2_evict_first(), keep_pol = l2_evict_last();
  const int tiles_per_cta = kBackTilesPerCta / wpt, part = warp % wpt;
  const int64_t t0 = g * tiles_per_cta + warp / wpt;
  // lane 0 fetches the tile's run bounds and keeps this warp's part of it
  int s_l = 0, e_l = 0;
  if (lane < TPW && t0 + lane < tiles) {
    const uint16_t* row = btab + (t0 + lane) * (nbuckets + 1);
    const int s = row[b], e = row[b + 1];
    s_l = s + ((e - s) * part) / wpt;
    e_l = s + ((e - s) * (part + 1)) / wpt;
  }
  // rounds of 4 x 32 pairs per run: the loads of all the warp's runs, then the stores
  constexpr int G = 4;
  int len = e_l - s_l;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
  int s_k[TPW], e_k[TPW];
#pragma unroll
  for (int k = 0; k < TPW; ++k) {
    s_k[k] = __shfl_sync(0xffffffffu, s_l, k);
    e_k[k] = __shfl_sync(0xffffffffu, e_l, k);
  }
#pragma unroll 1
  for (int j0 = 0; j0 < len; j0 += 32 * G) {
    uint32_t c[TPW * G];
    float zz[TPW * G];
#pragma unroll
    for (int k = 0; k < TPW; ++k) {
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int i = s_k[k] + j0 + 32 * q + lane;
        c[k * G + q] = 0xffffffffu;
        if (i < e_k[k]) {
          const int64_t at = (t0 + k) * kScanTile + i;
          c[k * G + q] = ld_hint(bcell + at, stream_pol);
          zz[k * G + q] = ld_hint(bz + at, stream_pol);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < TPW * G; ++q)
      if (c[q] != 0xffffffffu) st_hint(zre + c[q], zz[q], keep_pol);
  }
}

__global__ void __launch_bounds__(256) k_scatter_back(const uint32_t* __restrict__ bcell,
                                                      const float* __restrict__ bz,
                                                      const uint16_t* __restrict__ btab, int nbuckets,
                                                      int64_t tiles, int groups, int wpt, float* __restrict__ zre) {
  scatter_back_body(bcell, bz, btab, nbuckets, tiles, groups, wpt, zre, blockIdx.x);
}

// Several scatters at once: CTA b works on item find_item(prefix, M, b).
__global__ void __launch_bounds__(256) k_scatter_back_multi(const ScatterArgs* __restrict__ args,
                                                            const uint32_t* __restrict__ prefix, int M) {
  const int it = find_item(prefix, M, blockIdx.x);
  const ScatterArgs& a = args[it];
  scatter_back_body(a.bcell, a.bz, a.btab, a.nbuckets, a.tiles, a.groups, a.wpt, a.zre, blockIdx.x - prefix[it]);
}

// ---------------------------------------------------------------------------
// Tomographic matching helpers: z_re starts as NaN (neutral); before interval
// k's ranking the cells already ionized get intensity +inf so they rank first;
// after its matching a neutral cell takes the interval's redshift when it
// lies at or above the interval's lower bound (always in the last interval).
__global__ void __launch_bounds__(256) k_tomo_fill(float* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = __int_as_float(0x7fc00000);  // quiet NaN
}

// Cells ionized in an earlier interval take the next float above the largest
// intensity of this interval (its key is one below the minimum key): they
// rank first, in cell order, exactly as +inf would, while the key range -- and
// so the number of digit passes -- grows by one key instead of to the top of
// the float range.
__global__ void __launch_bounds__(256) k_tomo_mask(float* __restrict__ J, const float* __restrict__ z, int64_t n,
                                                   const SortCtrl* __restrict__ ctrl) {
  const uint32_t k = (uint32_t)ctrl->kmin - 1u;  // kmin > 0 for finite intensities
  const uint32_t u = ~k;                          // undo the descending flip
  const float first = __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isnan(z[i])) J[i] = first;
}

__global__ void k_tomo_widen(SortCtrl* ctrl) {
  if (ctrl->kmin > 0) ctrl->kmin -= 1;
}

__global__ void __launch_bounds__(256) k_tomo_merge(float* __restrict__ z, const float* __restrict__ ztmp, int64_t n,
                                                    float z_low, bool last) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (isnan(z[i]) && (last || ztmp[i] >= z_low)) z[i] = ztmp[i];
}

static int elem_grid(int64_t n, int num_sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 16));
}

cudaError_t tomo_fill(float* z, int64_t n, int num_sms, cudaStream_t s) {
  k_tomo_fill<<<elem_grid(n, num_sms), 256, 0, s>>>(z, n);
  return cudaGetLastError();
}
cudaError_t tomo_mask(float* J, const float* z, int64_t n, SortCtrl* ctrl, int num_sms, cudaStream_t s) {
  k_tomo_mask<<<elem_grid(n, num_sms), 256, 0, s>>>(J, z, n, ctrl);
  k_tomo_widen<<<1, 1, 0, s>>>(ctrl);
  return cudaGetLastError();
}
cudaError_t tomo_merge(float* z, const float* ztmp, int64_t n, float z_low, bool last, int num_sms, cudaStream_t s) {
  k_tomo_merge<<<elem_grid(n, num_sms), 256, 0, s>>>(z, ztmp, n, z_low, last);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
void bucket_plan(int64_t n, int* nbuckets, int* shift) {
  // buckets of 2^23 consecutive cells: 32 MB of z_re each, so the active
  // bucket stays in L2; at most 128 buckets for 2^30 cells
  *shift = kBucketShift;
  *nbuckets = (int)((n + ((int64_t)1 << kBucketShift) - 1) >> kBucketShift);
}

void assign_args(const AssignWork& w, const uint32_t* order, const float* mass, const unsigned long long* tile_mass,
                 int64_t n, const HistoryCoeffs& hc, float* zre, double* F, unsigned int* status,
                 unsigned int spin_limit, const uint32_t* order_b, const float* mass_b, const int* pick,
                 ThreshArgs* ta, ScanArgs* sa, ScatterArgs* xa) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  unsigned long long* total = reinterpret_cast<unsigned long long*>(w.ctrl);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(w.ctrl + 16);
  int* qshift = reinterpret_cast<int*>(w.ctrl + 32);
  unsigned long long* qtotal = reinterpret_cast<unsigned long long*>(w.ctrl + 40);
  ThreshArgs& t = *ta;
  t.total = total;
  t.tile_mass = tile_mass;
  t.ntiles = tile_mass ? sort_tiles(n) : 0;
  t.M = hc.n_table;
  t.a_w = hc.a;
  t.b_w = hc.b;
  t.c_w = hc.c;
  t.z_lo = hc.z_lo;
  t.z_hi = hc.z_hi;
  t.Xq = w.Xq;
  t.inv_dx = w.inv_dx;
  t.qshift = qshift;
  t.qtotal = qtotal;
  t.weighting = hc.weighting;
  t.omega_m = hc.omega_m;
  t.z_mid = hc.z_mid;
  t.ncells = n;
  t.lin = w.lin;

  ScanArgs& a = *sa;
  a.order = order;
  a.mass = mass;
  a.order_b = order_b;
  a.mass_b = mass_b;
  a.pick = pick;
  a.n = n;
  a.Xq = w.Xq;
  a.qshift = qshift;
  a.qtotal = qtotal;
  a.inv_dx = w.inv_dx;
  a.n_table = hc.n_table;
  a.z_lo = (float)hc.z_lo;
  a.z_hi = (float)hc.z_hi;
  a.dzt = (float)((hc.z_hi - hc.z_lo) / (double)(hc.n_table - 1));
  a.F = F;
  a.state = w.state;
  a.ticket = ticket;
  bucket_plan(n, &a.nbuckets, &a.bucket_shift);
  a.bcell = w.bcell;
  a.bz = w.bz;
  a.btab = w.btab;
  a.status = status;
  a.spin_limit = spin_limit;
  a.ahead = (uint32_t)w.num_sms;  // half the resident wave (2 CTAs per SM): measured best
  a.linP = w.lin;
  a.linQ = w.lin + kMaxTable;
  a.lina = w.lin + 2 * kMaxTable;
  a.linb = w.lin + 3 * kMaxTable;

  ScatterArgs& x = *xa;
  x.bcell = w.bcell;
  x.bz = w.bz;
  x.btab = w.btab;
  x.nbuckets = a.nbuckets;
  x.tiles = tiles;
  // warps per tile run: about 128 pairs each on average (a tile's 8192 pairs
  // spread over the buckets)
  x.wpt = 1;
  while (x.wpt < 8 && kScanTile / a.nbuckets >= 256 * x.wpt) x.wpt *= 2;
  const int tiles_per_cta = kBackTilesPerCta / x.wpt;
  x.groups = (int)((tiles + tiles_per_cta - 1) / tiles_per_cta);
  x.zre = zre;
}

cudaError_t assign_impl(const AssignWork& w, const uint32_t* order, const float* mass, bool mass_in_rank_order,
                        const unsigned long long* tile_mass, int64_t n, const HistoryCoeffs& hc, float* zre, double* F,
                        unsigned int* status, cudaStream_t s, FftProfile* prof, unsigned int spin_limit,
                        const uint32_t* order_b, const float* mass_b, const int* pick) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  ThreshArgs ta;
  ScanArgs a;
  ScatterArgs xa;
  assign_args(w, order, mass, tile_mass, n, hc, zre, F, status, spin_limit, order_b, mass_b, pick, &ta, &a, &xa);
  cudaError_t e = cudaMemsetAsync(w.ctrl, 0, kAssignCtrlBytes, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.state, 0, (size_t)tiles * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;

  if (!tile_mass) {  // masses in cell order: one exact reduction pass
    prof_begin(prof, PK_MASS_REDUCE, s);
    int grid = (int)std::min<int64_t>((n / 4 + 255) / 256, (int64_t)w.num_sms * 8);
    if (grid < 1) grid = 1;
    k_mass_reduce<<<grid, 256, 0, s>>>(mass, n, ta.total, status);
    prof_end(prof, PK_MASS_REDUCE, s);
  }

  prof_begin(prof, PK_THRESHOLDS, s);
  k_thresholds<<<1, 1024, 0, s>>>(ta);
  prof_end(prof, PK_THRESHOLDS, s);

  prof_begin(prof, PK_SCAN_ASSIGN, s);
  const unsigned g = (unsigned)tiles;
  const bool gather = !mass_in_rank_order, lin = hc.weighting != AMBER_WEIGHT_MASS;
  const int v = (gather ? 4 : 0) | (F ? 2 : 0) | (lin ? 1 : 0);
  switch (v) {
    case 0: k_scan_assign<false, false, false><<<g, kScanThreads, 0, s>>>(a); break;
    case 1: k_scan_assign<false, false, true><<<g, kScanThreads, 0, s>>>(a); break;
    case 2: k_scan_assign<false, true, false><<<g, kScanThreads, 0, s>>>(a); break;
    case 3: k_scan_assign<false, true, true><<<g, kScanThreads, 0, s>>>(a); break;
    case 4: k_scan_assign<true, false, false><<<g, kScanThreads, 0, s>>>(a); break;
    case 5: k_scan_assign<true, false, true><<<g, kScanThreads, 0, s>>>(a); break;
    case 6: k_scan_assign<true, true, false><<<g, kScanThreads, 0, s>>>(a); break;
    default: k_scan_assign<true, true, true><<<g, kScanThreads, 0, s>>>(a); break;
  }
  prof_end(prof, PK_SCAN_ASSIGN, s);
  prof_begin(prof, PK_SCATTER_BACK, s);
  k_scatter_back<<<(unsigned)(xa.groups * xa.nbuckets), 256, 0, s>>>(xa.bcell, xa.bz, xa.btab, xa.nbuckets, xa.tiles,
                                                                     xa.groups, xa.wpt, xa.zre);
  prof_end(prof, PK_SCATTER_BACK, s);
  return cudaGetLastError();
}

cudaError_t assign_multi(const AssignMulti& m, cudaStream_t s) {
  k_thresholds_multi<<<m.M, 1024, 0, s>>>(m.thresh);
  if (m.scan_tiles[0]) k_scan_assign_multi<false><<<m.scan_tiles[0], kScanThreads, 0, s>>>(m.scan[0], m.scan_prefix[0], m.Mg[0]);
  if (m.scan_tiles[1]) k_scan_assign_multi<true><<<m.scan_tiles[1], kScanThreads, 0, s>>>(m.scan[1], m.scan_prefix[1], m.Mg[1]);
  k_scatter_back_multi<<<m.scatter_blocks, 256, 0, s>>>(m.scatter, m.scatter_prefix, m.M);
  return cudaGetLastError();
}

}  // namespace amber
