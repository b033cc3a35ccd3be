// Ranking of cells by intensity (Sec. 3.4.2): a stable least-significant-
// digit radix sort of order-preserving keys with the cell index as payload,
// so order[r] is the cell of rank r in descending intensity with ties in
// ascending cell index.  The paper ranks with a parallel quicksort; here the
// sort is a onesweep LSD radix sort with 8-bit digits:
//
//   k_sort_histogram : one read of the intensities; digit counts for every
//                      digit position at once (warp-aggregated shared atomics)
//   k_sort_offsets   : exclusive scan of each digit histogram
//   k_sort_pass      : per digit position, tiles claim ids from an atomic
//                      ticket, rank keys locally (warp match + per-warp digit
//                      counters), publish per-digit tile counts, resolve
//                      their global offset by decoupled look-back over
//                      predecessor tiles, and scatter through shared memory
//                      so each digit run is written contiguously.
//
// Keys: descending float order maps to ascending uint32 (uint64 for double)
// by flipping; -0.0 is folded into +0.0 and NaN latches AMBER_ERR_NONFINITE.
#include "sort.cuh"

namespace amber {

template <typename K> __device__ __forceinline__ K enc_desc(float v, bool& bad);
template <> __device__ __forceinline__ uint32_t enc_desc<uint32_t>(float v, bool& bad) {
  bad |= isnan(v);
  v = v + 0.0f;  // -0 -> +0
  const uint32_t b = __float_as_uint(v);
  const uint32_t u = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ~u;
}
template <typename K> __device__ __forceinline__ K enc_desc_d(double v, bool& bad);
template <> __device__ __forceinline__ uint64_t enc_desc_d<uint64_t>(double v, bool& bad) {
  bad |= isnan(v);
  v = v + 0.0;
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const uint64_t u = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  return ~u;
}

template <typename SRC> struct KeyOf;
template <> struct KeyOf<float> {
  using K = uint32_t;
  static __device__ __forceinline__ K enc(float v, bool& bad) { return enc_desc<uint32_t>(v, bad); }
};
template <> struct KeyOf<double> {
  using K = uint64_t;
  static __device__ __forceinline__ K enc(double v, bool& bad) { return enc_desc_d<uint64_t>(v, bad); }
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
template <typename SRC>
__global__ void __launch_bounds__(256) k_sort_histogram(const SRC* __restrict__ J, int64_t n,
                                                        uint32_t* __restrict__ hist,
                                                        uint32_t* __restrict__ lb0, int64_t lb0_words,
                                                        unsigned int* __restrict__ status) {
  using K = typename KeyOf<SRC>::K;
  constexpr int P = sizeof(K);  // digit positions
  __shared__ uint32_t h[P][kRadix];
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of iterations so the warp
  // match below always sees all 32 lanes
  const int64_t warp_base = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31));
  for (int64_t i0 = warp_base; i0 < n; i0 += stride) {
    const int64_t i = i0 + (threadIdx.x & 31);
    const bool ok = i < n;
    const K key = ok ? KeyOf<SRC>::enc(J[i], bad) : K(0);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const unsigned d = ok ? (unsigned)(key >> (8 * p)) & 0xffu : 0x100u;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (ok && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * kRadix; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
  // clear the look-back area of the first digit pass
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < lb0_words; w += stride) lb0[w] = 0;
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
// payload = cell index.  LAST: only the payload (the rank order) is written.
// ---------------------------------------------------------------------------
template <typename SRC, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const SRC* __restrict__ J, const typename KeyOf<SRC>::K* __restrict__ kin, const uint32_t* __restrict__ vin,
    typename KeyOf<SRC>::K* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
    const uint32_t* __restrict__ bin_off, uint32_t* __restrict__ lb, uint32_t* __restrict__ lb_next,
    uint32_t* __restrict__ ticket, unsigned int* __restrict__ status, unsigned int spin_limit) {
  using K = typename KeyOf<SRC>::K;
  constexpr int NW = kSortThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* skey = reinterpret_cast<K*>(smem_raw);                                  // [kTile]
  uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kTile);               // [kTile]
  uint32_t* whist = sval + kTile;                                            // [NW][256]
  uint32_t* dstart = whist + NW * kRadix;                                    // [256] tile digit start
  uint32_t* gbase = dstart + kRadix;                                         // [256] global base - dstart
  __shared__ uint32_t s_tile;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  for (int i = tid; i < NW * kRadix; i += kSortThreads) whist[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t start = (int64_t)tile * kTile;
  if (lb_next) lb_next[(int64_t)tile * kRadix + tid] = 0;  // kSortThreads == kRadix

  // ---- load (warp-striped) and rank locally
  K key[kItems];
  uint32_t val[kItems];
  unsigned dig[kItems];
  bool bad = false;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int pos = warp * kItems * 32 + it * 32 + lane;
    const int64_t g = start + pos;
    const bool ok = g < n;
    if (FIRST) {
      key[it] = ok ? KeyOf<SRC>::enc(J[g], bad) : K(0);
      val[it] = (uint32_t)g;
    } else {
      key[it] = ok ? kin[g] : K(0);
      val[it] = ok ? vin[g] : 0u;
    }
    dig[it] = ok ? (unsigned)(key[it] >> shift) & 0xffu : 0x100u;
  }
  uint32_t rank[kItems];
  uint32_t* wh = whist + warp * kRadix;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const unsigned d = dig[it];
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t base = 0;
    if (d < 0x100u) base = wh[d];
    rank[it] = base + __popc(peers & lanemask_lt());
    __syncwarp();
    if (d < 0x100u && (__ffs(peers) - 1) == lane) wh[d] = base + __popc(peers);
    __syncwarp();
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
  // publish this tile's count for digit d (tile 0 publishes its inclusive value)
  uint32_t* my = lb + (int64_t)tile * kRadix + d;
  if (tile == 0) st_relaxed_u32(my, kFlagInc | cnt);
  else st_relaxed_u32(my, kFlagAgg | cnt);

  // tile-local digit starts: exclusive scan of cnt over the 256 digits
  {
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    __shared__ uint32_t wsum[NW];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) wpre += (w < warp) ? wsum[w] : 0u;
    dstart[d] = wpre + x - cnt;
  }

  // ---- decoupled look-back for digit d
  uint32_t excl = 0;
  if (tile > 0) {
    int64_t t = (int64_t)tile - 1;
    unsigned spins = 0;
    while (t >= 0) {
      const uint32_t s = ld_relaxed_u32(lb + t * kRadix + d);
      const uint32_t flag = s & kFlagMask;
      if (flag == 0u) {
        if (++spins >= spin_limit) { raise_status(status, AMBER_ERR_DEVICE_TIMEOUT); break; }
        __nanosleep(32);
        continue;
      }
      excl += s & kValueMask;
      if (flag == kFlagInc) break;
      --t;
    }
    const uint32_t inc = excl + cnt;
    st_relaxed_u32(my, kFlagInc | (inc & kValueMask));
  }
  __syncthreads();  // dstart, whist prefixes visible
  gbase[d] = bin_off[d] + excl - dstart[d];

  // ---- scatter into shared memory in tile-sorted order
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const unsigned dd = dig[it];
    if (dd < 0x100u) {
      const uint32_t p = dstart[dd] + whist[warp * kRadix + dd] + rank[it];
      skey[p] = key[it];
      sval[p] = val[it];
    }
  }
  __syncthreads();
  // ---- write out: consecutive positions of one digit go to consecutive addresses
  const int cnt_tile = (int)(n - start < (int64_t)kTile ? n - start : (int64_t)kTile);
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int p = it * kSortThreads + tid;
    if (p < cnt_tile) {
      const K kk = skey[p];
      const uint32_t g = gbase[(unsigned)(kk >> shift) & 0xffu] + p;
      if (!LAST) kout[g] = kk;
      vout[g] = sval[p];
    }
  }
  if (FIRST && __any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, AMBER_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
size_t sort_pass_smem(int key_bytes) {
  return (size_t)kTile * key_bytes + (size_t)kTile * 4 + (size_t)(kSortThreads / 32) * kRadix * 4 + 2 * kRadix * 4;
}

int64_t sort_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, unsigned int* status,
                      cudaStream_t s, FftProfile* prof, unsigned int spin_limit) {
  using K = typename KeyOf<SRC>::K;
  constexpr int P = sizeof(K);
  const int64_t tiles = sort_tiles(n);
  const int64_t lbw = tiles * kRadix;  // words per look-back region
  static bool attr = false;
  const size_t smem = sort_pass_smem(sizeof(K));
  if (!attr) {
    cudaFuncSetAttribute(k_sort_pass<SRC, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_sort_pass<SRC, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_sort_pass<SRC, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_sort_pass<SRC, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  cudaError_t e = cudaMemsetAsync(w.ctrl, 0, kSortCtrlBytes, s);
  if (e != cudaSuccess) return e;
  uint32_t* hist = w.ctrl;                       // [8][256]
  uint32_t* offs = w.ctrl + 8 * kRadix;          // [8][256]
  uint32_t* tickets = w.ctrl + 16 * kRadix;      // [8]
  uint32_t* lbA = w.lookback;
  uint32_t* lbB = w.lookback + lbw;

  prof_begin(prof, PK_SORT_HIST, s);
  {
    int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)w.num_sms * 8);
    if (grid < 1) grid = 1;
    k_sort_histogram<SRC><<<grid, 256, 0, s>>>(J, n, hist, lbA, lbw, status);
    k_sort_offsets<<<1, kRadix, 0, s>>>(hist, offs, P);
  }
  prof_end(prof, PK_SORT_HIST, s);

  K* kA = reinterpret_cast<K*>(w.keysA);
  K* kB = reinterpret_cast<K*>(w.keysB);
  const K* kin = nullptr;
  const uint32_t* vin = nullptr;
  for (int p = 0; p < P; ++p) {
    const bool first = p == 0, last = p == P - 1;
    uint32_t* lb = (p & 1) ? lbB : lbA;
    uint32_t* lbn = last ? nullptr : ((p & 1) ? lbA : lbB);
    K* kout = (p & 1) ? kB : kA;
    uint32_t* vout = last ? order : ((p & 1) ? w.idxB : w.idxA);
    prof_begin(prof, PK_SORT_PASS, s);
    if (first && last)
      k_sort_pass<SRC, true, true><<<(unsigned)tiles, kSortThreads, smem, s>>>(J, kin, vin, kout, vout, n, 8 * p,
          offs + p * kRadix, lb, lbn, tickets + p, status, spin_limit);
    else if (first)
      k_sort_pass<SRC, true, false><<<(unsigned)tiles, kSortThreads, smem, s>>>(J, kin, vin, kout, vout, n, 8 * p,
          offs + p * kRadix, lb, lbn, tickets + p, status, spin_limit);
    else if (last)
      k_sort_pass<SRC, false, true><<<(unsigned)tiles, kSortThreads, smem, s>>>(J, kin, vin, kout, vout, n, 8 * p,
          offs + p * kRadix, lb, lbn, tickets + p, status, spin_limit);
    else
      k_sort_pass<SRC, false, false><<<(unsigned)tiles, kSortThreads, smem, s>>>(J, kin, vin, kout, vout, n, 8 * p,
          offs + p * kRadix, lb, lbn, tickets + p, status, spin_limit);
    prof_end(prof, PK_SORT_PASS, s);
    kin = kout;
    vin = vout;
  }
  return cudaGetLastError();
}

template cudaError_t rank_impl<float>(const SortWork&, const float*, int64_t, uint32_t*, unsigned int*,
                                      cudaStream_t, FftProfile*, unsigned int);
template cudaError_t rank_impl<double>(const SortWork&, const double*, int64_t, uint32_t*, unsigned int*,
                                       cudaStream_t, FftProfile*, unsigned int);

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
