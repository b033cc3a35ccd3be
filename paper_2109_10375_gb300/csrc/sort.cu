// Ranking of cells by intensity (Sec. 3.4.2): a stable least-significant-
// digit radix sort of order-preserving keys with the cell index as payload,
// so order[r] is the cell of rank r in descending intensity with ties in
// ascending cell index.  The paper ranks with a parallel quicksort; here the
// sort is a onesweep LSD radix sort with 8-bit digits:
//
//   k_sort_histogram : one read of the intensities; digit counts for every
//                      digit position at once (shared-memory counters, with
//                      one add per warp when all 32 lanes share a digit)
//   k_sort_offsets   : exclusive scan of each digit histogram
//   k_sort_pass      : per digit position, tiles claim ids from an atomic
//                      ticket, rank keys locally (8 warp ballots give each
//                      lane its peers of equal digit; per-warp digit
//                      counters), publish per-digit tile counts, resolve
//                      their global offset by decoupled look-back over
//                      predecessor tiles, and scatter through shared memory
//                      so each digit run is written contiguously.
//
// The whole-path variant carries the cell mass as a second payload, so the
// abundance matching reads masses in rank order without a random gather; its
// first pass also sums the masses (exact 128-bit fixed point).
//
// Keys: descending float order maps to ascending uint32 (uint64 for double)
// by flipping; -0.0 is folded into +0.0 and NaN latches AMBER_ERR_NONFINITE.
#include <cstring>

#include "fixed128.cuh"
#include "sort.cuh"

namespace amber {

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
template <> struct KeyOf<float> { using K = uint32_t; };
template <> struct KeyOf<double> { using K = uint64_t; };

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Count digit d of this lane into h[d]: a single add when the whole warp
// agrees (the high key bytes of a narrow intensity range), else one per lane.
__device__ __forceinline__ void hist_add(uint32_t* h, unsigned d) {
  const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
  if (__all_sync(0xffffffffu, d == d0)) {
    if ((threadIdx.x & 31) == 0) atomicAdd(&h[d0], 32u);
  } else {
    atomicAdd(&h[d], 1u);
  }
}

// ---------------------------------------------------------------------------
template <typename SRC>
__global__ void __launch_bounds__(256) k_sort_histogram(const SRC* __restrict__ J, int64_t n,
                                                        uint32_t* __restrict__ hist,
                                                        uint32_t* __restrict__ lb0, int64_t lb0_words,
                                                        unsigned int* __restrict__ status) {
  using K = typename KeyOf<SRC>::K;
  constexpr int P = sizeof(K);         // digit positions
  constexpr int V = 16 / sizeof(SRC);  // elements per 16-byte load
  __shared__ uint32_t h[P][kRadix];
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  bool bad = false;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // full 16-byte vectors; every lane of a warp runs the same trip count
  const int64_t nvec = n / V;
  const int64_t vec_iters = (nvec + nthreads - 1) / nthreads;
  for (int64_t it = 0; it < vec_iters; ++it) {
    const int64_t v = it * nthreads + gtid;
    const bool ok = v < nvec;
    SRC x[V];
    if (ok) {
      const uint4 raw = reinterpret_cast<const uint4*>(J)[v];
      memcpy(x, &raw, 16);
    }
    const bool all_ok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const K key = ok ? enc_desc(x[e], bad) : K(0);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const unsigned d = (unsigned)(key >> (8 * p)) & 0xffu;
        if (all_ok) hist_add(h[p], d);
        else if (ok) atomicAdd(&h[p][d], 1u);
      }
    }
  }
  // ragged tail (< V elements)
  for (int64_t i = nvec * V + gtid; i < n; i += nthreads) {
    const K key = enc_desc(J[i], bad);
#pragma unroll
    for (int p = 0; p < P; ++p) atomicAdd(&h[p][(unsigned)(key >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
  // clear the look-back area of the first digit pass
  for (int64_t w = gtid; w < lb0_words; w += nthreads) lb0[w] = 0;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(status, AMBER_ERR_NONFINITE);
}

// One CTA: exclusive scan of each of the P digit histograms -> bin offsets.
__global__ void __launch_bounds__(kRadix) k_sort_offsets(const uint32_t* __restrict__ hist,
                                                         uint32_t* __restrict__ offs, int P) {
  __shared__ uint32_t s[kRadix];
  for (int p = 0; p < P; ++p) {
    const uint32_t c = hist[p * kRadix + threadIdx.x];
    s[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < kRadix; o <<= 1) {
      const uint32_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    offs[p * kRadix + threadIdx.x] = s[threadIdx.x] - c;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// One digit pass.  FIRST: keys come from the intensities (encoded on load),
// payload = cell index, and (MASS) masses are read in cell order, summed into
// mass_total and checked.  LAST: only the payloads are written.
// ---------------------------------------------------------------------------
template <typename SRC, bool FIRST, bool LAST, bool MASS>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_pass(const PassArgs a) {
  using K = typename KeyOf<SRC>::K;
  constexpr int NW = kSortThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* skey = reinterpret_cast<K*>(smem_raw);                                  // [kTile]
  uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kTile);               // [kTile]
  float* smass = reinterpret_cast<float*>(sval + kTile);                     // [kTile] if MASS
  uint32_t* whist = reinterpret_cast<uint32_t*>(smass + (MASS ? kTile : 0)); // [NW][256]
  uint32_t* dstart = whist + NW * kRadix;                                    // [256]
  uint32_t* gbase = dstart + kRadix;                                         // [256]
  __shared__ uint32_t s_tile;
  __shared__ uint32_t wsum[NW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
  for (int i = tid; i < NW * kRadix; i += kSortThreads) whist[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t start = (int64_t)tile * kTile;
  const int64_t n = a.n;
  const int shift = a.shift;
  if (a.lb_next) a.lb_next[(int64_t)tile * kRadix + tid] = 0;  // kSortThreads == kRadix
  const int64_t wbase = start + warp * kItems * 32 + lane;       // item it at wbase + 32 it

  // ---- keys (warp-striped) and their local ranks, packed rank | digit << 16
  K key[kItems];
  uint32_t rd[kItems];
  bool bad = false;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t g = wbase + 32 * it;
    const bool ok = g < n;
    if constexpr (FIRST) key[it] = ok ? enc_desc(reinterpret_cast<const SRC*>(a.J)[g], bad) : K(0);
    else key[it] = ok ? reinterpret_cast<const K*>(a.kin)[g] : K(0);
  }
  uint32_t* wh = whist + warp * kRadix;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const bool ok = wbase + 32 * it < n;
    const unsigned d = (unsigned)(key[it] >> shift) & 0xffu;
    unsigned peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? bb : ~bb;
    }
    uint32_t base = 0;
    if (ok) base = wh[d];
    __syncwarp();
    if (ok && (peers & lt) == 0u) wh[d] = base + __popc(peers);
    __syncwarp();
    rd[it] = ok ? ((base + __popc(peers & lt)) | (d << 16)) : 0xffffffffu;
  }
  __syncthreads();

  // ---- per digit (thread = digit): warp prefixes and the tile count
  const int d = tid;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t c = whist[w * kRadix + d];
    whist[w * kRadix + d] = cnt;
    cnt += c;
  }
  uint32_t* my = a.lb + (int64_t)tile * kRadix + d;
  st_relaxed_u32(my, (tile == 0 ? kFlagInc : kFlagAgg) | cnt);
  {
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) wpre += (w < warp) ? wsum[w] : 0u;
    dstart[d] = wpre + x - cnt;
  }
  __syncthreads();

  // ---- keys and payloads into shared memory in tile-sorted order; payloads
  // are loaded here so they never occupy registers during the ranking
  u128 msum = 0;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    if (rd[it] == 0xffffffffu) continue;
    const unsigned dd = rd[it] >> 16;
    const uint32_t p = dstart[dd] + whist[warp * kRadix + dd] + (rd[it] & 0xffffu);
    const int64_t g = wbase + 32 * it;
    skey[p] = key[it];
    sval[p] = FIRST ? (uint32_t)g : a.vin[g];
    if constexpr (MASS) {
      const float mv = a.min[g];
      smass[p] = mv;
      if constexpr (FIRST) msum += mass_q64(mv, bad);
    }
  }
  if constexpr (FIRST && MASS) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) msum += shfl_down_u128(msum, o);
    if (lane == 0 && msum != 0) atomic_add_u128(a.mass_total, msum);
  }

  // ---- decoupled look-back for digit d, kLookWindow predecessors per round
  // trip: sum aggregates back to the nearest inclusive prefix
  uint32_t excl = 0;
  if (tile > 0) {
    int64_t t = (int64_t)tile - 1;
    unsigned spins = 0;
    while (true) {
      uint32_t w[kLookWindow];
#pragma unroll
      for (int k = 0; k < kLookWindow; ++k)
        w[k] = (t - k >= 0) ? ld_relaxed_u32(a.lb + (t - k) * kRadix + d) : kFlagInc;
      bool stop = false, done = false;
      int adv = 0;
#pragma unroll
      for (int k = 0; k < kLookWindow; ++k) {
        if (!stop) {
          const uint32_t f = w[k] & kFlagMask;
          if (f == 0u) {
            stop = true;
          } else {
            excl += w[k] & kValueMask;
            ++adv;
            if (f == kFlagInc) stop = done = true;
          }
        }
      }
      if (done) break;
      t -= adv;
      if (adv < kLookWindow) {  // the tile at t has published nothing yet
        if (++spins >= a.spin_limit) { raise_status(a.status, AMBER_ERR_DEVICE_TIMEOUT); break; }
        __nanosleep(20);
      }
    }
    st_relaxed_u32(my, kFlagInc | ((excl + cnt) & kValueMask));
  }
  gbase[d] = a.bin_off[d] + excl - dstart[d];
  __syncthreads();

  // ---- write out: consecutive positions of one digit go to consecutive addresses
  const int cnt_tile = (int)(n - start < (int64_t)kTile ? n - start : (int64_t)kTile);
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int p = it * kSortThreads + tid;
    if (p < cnt_tile) {
      const K kk = skey[p];
      const uint32_t g = gbase[(unsigned)(kk >> shift) & 0xffu] + p;
      if constexpr (!LAST) reinterpret_cast<K*>(a.kout)[g] = kk;
      a.vout[g] = sval[p];
      if constexpr (MASS) a.mout[g] = smass[p];
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0)
    raise_status(a.status, (FIRST && MASS) ? (AMBER_ERR_NONFINITE | AMBER_ERR_INVALID_MASS) : AMBER_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
size_t sort_pass_smem(int key_bytes, bool mass) {
  return (size_t)kTile * key_bytes + (size_t)kTile * 4 * (mass ? 2 : 1) + (size_t)(kSortThreads / 32) * kRadix * 4 +
         2 * kRadix * 4;
}

int64_t sort_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

template <typename SRC, bool FIRST, bool LAST, bool MASS>
static void launch_pass(const PassArgs& a, int64_t tiles, cudaStream_t s) {
  const size_t smem = sort_pass_smem(sizeof(typename KeyOf<SRC>::K), MASS);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sort_pass<SRC, FIRST, LAST, MASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_sort_pass<SRC, FIRST, LAST, MASS><<<(unsigned)tiles, kSortThreads, smem, s>>>(a);
}

template <typename SRC, bool MASS>
static void launch_pass_rt(bool first, bool last, const PassArgs& a, int64_t tiles, cudaStream_t s) {
  if (first && last) launch_pass<SRC, true, true, MASS>(a, tiles, s);
  else if (first) launch_pass<SRC, true, false, MASS>(a, tiles, s);
  else if (last) launch_pass<SRC, false, true, MASS>(a, tiles, s);
  else launch_pass<SRC, false, false, MASS>(a, tiles, s);
}

template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in,
                      float* mass_out, unsigned long long* mass_total, unsigned int* status, cudaStream_t s,
                      FftProfile* prof, unsigned int spin_limit) {
  using K = typename KeyOf<SRC>::K;
  constexpr int P = sizeof(K);
  const bool with_mass = mass_in != nullptr;
  const int64_t tiles = sort_tiles(n);
  const int64_t lbw = tiles * kRadix;  // words per look-back region
  cudaError_t e = cudaMemsetAsync(w.ctrl, 0, kSortCtrlBytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* hist = w.ctrl;                   // [8][256]
  uint32_t* offs = w.ctrl + 8 * kRadix;      // [8][256]
  uint32_t* tickets = w.ctrl + 16 * kRadix;  // [8]
  uint32_t* lbA = w.lookback;
  uint32_t* lbB = w.lookback + lbw;

  prof_begin(prof, PK_SORT_HIST, s);
  {
    int grid = (int)std::min<int64_t>((n / (16 / (int)sizeof(SRC)) + 255) / 256, (int64_t)w.num_sms * 8);
    if (grid < 1) grid = 1;
    k_sort_histogram<SRC><<<grid, 256, 0, s>>>(J, n, hist, lbA, lbw, status);
    k_sort_offsets<<<1, kRadix, 0, s>>>(hist, offs, P);
  }
  prof_end(prof, PK_SORT_HIST, s);

  K* kA = reinterpret_cast<K*>(w.keysA);
  K* kB = reinterpret_cast<K*>(w.keysB);
  const void* kin = nullptr;
  const uint32_t* vin = nullptr;
  const float* mcur = mass_in;
  for (int p = 0; p < P; ++p) {
    const bool first = p == 0, last = p == P - 1;
    PassArgs a;
    a.J = J;
    a.kin = kin;
    a.vin = vin;
    a.min = mcur;
    a.kout = (p & 1) ? (void*)kB : (void*)kA;
    a.vout = last ? order : ((p & 1) ? w.idxB : w.idxA);
    a.mout = with_mass ? (last ? mass_out : ((p & 1) ? w.massB : w.massA)) : nullptr;
    a.n = n;
    a.shift = 8 * p;
    a.bin_off = offs + p * kRadix;
    a.lb = (p & 1) ? lbB : lbA;
    a.lb_next = last ? nullptr : ((p & 1) ? lbA : lbB);
    a.ticket = tickets + p;
    a.mass_total = mass_total;
    a.status = status;
    a.spin_limit = spin_limit;
    prof_begin(prof, PK_SORT_PASS, s);
    if (with_mass) launch_pass_rt<SRC, true>(first, last, a, tiles, s);
    else launch_pass_rt<SRC, false>(first, last, a, tiles, s);
    prof_end(prof, PK_SORT_PASS, s);
    kin = a.kout;
    vin = a.vout;
    mcur = a.mout;
  }
  return cudaGetLastError();
}

template cudaError_t rank_impl<float>(const SortWork&, const float*, int64_t, uint32_t*, const float*, float*,
                                      unsigned long long*, unsigned int*, cudaStream_t, FftProfile*, unsigned int);
template cudaError_t rank_impl<double>(const SortWork&, const double*, int64_t, uint32_t*, const float*, float*,
                                       unsigned long long*, unsigned int*, cudaStream_t, FftProfile*, unsigned int);

// Failure-detection hook: the look-back wait on a word nothing publishes.
__global__ void k_wait_never(const uint32_t* __restrict__ word, unsigned int* __restrict__ status,
                             unsigned int spin_limit) {
  unsigned spins = 0;
  while (true) {
    const uint32_t s = ld_relaxed_u32(word);
    if ((s & kFlagMask) != 0u) break;
    if (++spins >= spin_limit) { raise_status(status, AMBER_ERR_DEVICE_TIMEOUT); break; }
    __nanosleep(32);
  }
}

cudaError_t wait_timeout_test(uint32_t* zero_word, unsigned int* status, unsigned int spin_limit, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(zero_word, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  k_wait_never<<<1, 1, 0, s>>>(zero_word, status, spin_limit);
  return cudaGetLastError();
}

}  // namespace amber
