// Ranking of cells by intensity (Sec. 3.4.2): a stable least-significant-
// digit radix sort of order-preserving keys with the cell index as payload,
// so order[r] is the cell of rank r in descending intensity with ties in
// ascending cell index.  The paper ranks with a parallel quicksort; here the
// sort is a onesweep LSD radix sort:
//
//   k_key_range      : min and max key (the sort runs on key - min, so a
//                      field whose intensities span a few octaves needs
//                      27 bits: three 9-bit digits or four 8-bit ones
//                      instead of four or more)
//   k_sort_histogram : one read of the intensities; counts of every digit
//                      position at once (shared-memory counters, one add per
//                      warp when all 32 lanes share a digit)
//   k_sort_offsets   : exclusive scan of each digit histogram and the number
//                      of passes the key range needs
//   k_sort_pass      : per digit position, tiles claim ids from an atomic
//                      ticket, rank keys locally (one warp ballot per digit
//                      bit gives each lane its peers of equal digit; per-warp
//                      digit counters), publish per-digit tile counts,
//                      resolve their global offset by decoupled look-back
//                      over predecessor tiles, and scatter through shared
//                      memory so each digit run is written contiguously.
//                      Passes beyond the needed count return at once; the
//                      last needed pass writes only the payloads.
//
// The whole-path variant carries the cell mass as a second payload, so the
// abundance matching reads masses in rank order without a random gather; its
// first pass also sums each tile's masses (exact 128-bit fixed point).
//
// Keys: descending float order maps to ascending uint32 (uint64 for double)
// by flipping; -0.0 is folded into +0.0 and NaN latches AMBER_ERR_NONFINITE.
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "fixed128.cuh"
#include "sort.cuh"

namespace amber {

// RB: digit width in bits (KeyOf<SRC>::RB by default; FP32 keys also have an
// 8-bit instantiation the autotuner can choose).
template <typename SRC, int RB = KeyOf<SRC>::RB> constexpr int max_passes() {
  return (8 * (int)sizeof(typename KeyOf<SRC>::K) + RB - 1) / RB;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Count digit d of this lane into h[d]: a single add when the whole warp
// agrees (the top digit of a spatially smooth intensity field often does),
// else one per lane.
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
__global__ void __launch_bounds__(256) k_key_range(const SRC* __restrict__ J, int64_t n,
                                                   SortCtrl* __restrict__ ctrl, unsigned int* __restrict__ status) {
  using K = typename KeyOf<SRC>::K;
  bool bad = false;
  K lo = ~K(0), hi = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const K k = enc_desc(J[i], bad);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  key_range_commit(lo, hi, ctrl);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(status, AMBER_ERR_NONFINITE);
}

// The histogram of one sort, run by CTA blk of nblk.
template <typename SRC, int RB>
__device__ __forceinline__ void sort_histogram_body(const SRC* __restrict__ J, int64_t n, SortCtrl* __restrict__ ctrl,
                                                    uint32_t* __restrict__ lb0, int64_t lb0_words, int64_t blk,
                                                    int64_t nblk) {
  using K = typename KeyOf<SRC>::K;
  constexpr int R = 1 << RB, P = max_passes<SRC, RB>();
  constexpr int V = 16 / sizeof(SRC);  // elements per 16-byte load
  __shared__ uint32_t h[P][R];
  for (int i = threadIdx.x; i < P * R; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const K kmin = (K)ctrl->kmin;
  // digit positions the key range needs (the rest stay zero and are never read)
  int np = 0;
  {
    const K range = (K)ctrl->kmax - kmin;
    while (np < P && (RB * np >= (int)(8 * sizeof(K)) || (range >> (RB * np)) != 0)) ++np;
    if (np < 1) np = 1;
  }
  bool bad = false;
  const int64_t nthreads = nblk * blockDim.x;
  const int64_t gtid = blk * blockDim.x + threadIdx.x;
  // 16-byte loads only from a 16-byte aligned array (a caller's view may start
  // anywhere on its element size); otherwise every element takes the tail loop
  const bool vec = (reinterpret_cast<uintptr_t>(J) & 15) == 0;
  const int64_t nvec = vec ? n / V : 0;
  // two 16-byte loads in flight per thread and round
  constexpr int U = 2;
  const int64_t rounds = (nvec + U * nthreads - 1) / (U * nthreads);
  for (int64_t it = 0; it < rounds; ++it) {  // the same trip count on every lane
    K key[U][V];
    bool ok[U];
    {
      SRC x[U][V];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t v = (it * U + u) * nthreads + gtid;
        ok[u] = v < nvec;
        if (ok[u]) {
          const uint4 raw = reinterpret_cast<const uint4*>(J)[v];
          memcpy(x[u], &raw, 16);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int e = 0; e < V; ++e) key[u][e] = ok[u] ? K(enc_desc(x[u][e], bad) - kmin) : K(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool all_ok = __all_sync(0xffffffffu, ok[u]);
      // digit position by digit position (warp-uniform tests, once per V
      // keys): one shared add per key below the top digit; the top digit of
      // a smooth field tends to agree across a warp, which then adds once
#pragma unroll
      for (int p = 0; p < P; ++p) {
        if (p < np - 1) {
          if (ok[u]) {
#pragma unroll
            for (int e = 0; e < V; ++e) atomicAdd(&h[p][(unsigned)(key[u][e] >> (RB * p)) & (R - 1)], 1u);
          }
        } else if (p == np - 1) {
#pragma unroll
          for (int e = 0; e < V; ++e) {
            const unsigned d = (unsigned)(key[u][e] >> (RB * p)) & (R - 1);
            if (all_ok) hist_add(h[p], d);
            else if (ok[u]) atomicAdd(&h[p][d], 1u);
          }
        }
      }
    }
  }
  for (int64_t i = nvec * V + gtid; i < n; i += nthreads) {  // ragged tail
    const K key = K(enc_desc(J[i], bad) - kmin);
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (p < np) atomicAdd(&h[p][(unsigned)(key >> (RB * p)) & (R - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P * R; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(&ctrl->hist[i], c);
  }
  for (int64_t w = gtid; w < lb0_words; w += nthreads) lb0[w] = 0;  // look-back of the first pass
}

template <typename SRC, int RB>
__global__ void __launch_bounds__(256) k_sort_histogram(const SRC* __restrict__ J, int64_t n,
                                                        SortCtrl* __restrict__ ctrl,
                                                        uint32_t* __restrict__ lb0, int64_t lb0_words) {
  sort_histogram_body<SRC, RB>(J, n, ctrl, lb0, lb0_words, blockIdx.x, gridDim.x);
}

// Several sorts at once: CTA b works on item find_item(prefix, M, b).
template <typename SRC, int RB>
__global__ void __launch_bounds__(256) k_sort_histogram_multi(const HistArgs* __restrict__ args,
                                                              const uint32_t* __restrict__ prefix, int M) {
  const int it = find_item(prefix, M, blockIdx.x);
  const HistArgs& a = args[it];
  sort_histogram_body<SRC, RB>(reinterpret_cast<const SRC*>(a.J), a.n, a.ctrl, a.lb0, a.lb0_words,
                               blockIdx.x - prefix[it], prefix[it + 1] - prefix[it]);
}

// One CTA: exclusive scan of each digit histogram, and the pass count.
// raw: the histogram counted raw keys (the intensity kernel's digit counts):
// the sort then runs on key - 0, so the key minimum is reset to 0.
template <typename SRC, int RB>
__device__ __forceinline__ void sort_offsets_body(SortCtrl* __restrict__ ctrl, bool raw = false) {
  using K = typename KeyOf<SRC>::K;
  constexpr int R = 1 << RB, P = max_passes<SRC, RB>();
  __shared__ uint32_t wsum[8];
  __shared__ uint32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int p = 0; p < P; ++p) {
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int d0 = 0; d0 < R; d0 += 256) {
      const int d = d0 + threadIdx.x;
      const uint32_t c = ctrl->hist[p * R + d];
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncthreads();
      uint32_t pre = carry, tot = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        pre += (w < warp) ? wsum[w] : 0u;
        tot += wsum[w];
      }
      ctrl->offs[p * R + d] = pre + x - c;
      __syncthreads();
      if (threadIdx.x == 0) carry += tot;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    if (raw) ctrl->kmin = 0;
    const K range = (K)ctrl->kmax - (K)ctrl->kmin;
    int bits = 0;
    while (bits < (int)(8 * sizeof(K)) && (range >> bits) != 0) ++bits;
    const int np = (bits + RB - 1) / RB;
    ctrl->npasses = np < 1 ? 1 : np;
  }
}

template <typename SRC, int RB>
__global__ void __launch_bounds__(256) k_sort_offsets(SortCtrl* __restrict__ ctrl, bool raw) {
  sort_offsets_body<SRC, RB>(ctrl, raw);
}

// One CTA per item.
template <typename SRC, int RB>
__global__ void __launch_bounds__(256) k_sort_offsets_multi(const HistArgs* __restrict__ args) {
  sort_offsets_body<SRC, RB>(args[blockIdx.x].ctrl);
}

// ---------------------------------------------------------------------------
// One digit pass.  FIRST: keys come from the intensities (encoded, minus the
// minimum key), payload = cell index, and (MASS) masses are read in cell
// order, summed per tile into tile_mass and checked.  The last needed pass writes
// only the payloads (to the final arrays).
// ---------------------------------------------------------------------------
template <typename SRC, int RB, bool FIRST, bool MASS, bool MATCH>
__device__ __forceinline__ void sort_pass_body(const PassArgs& a) {
  using K = typename KeyOf<SRC>::K;
  constexpr int R = 1 << RB, DPT = R / kSortThreads;  // digits per thread
  static_assert(DPT >= 1 && R <= kMaxRadix, "digit width");
  constexpr int NW = kSortThreads / 32;
  const int npasses = a.ctrl->npasses;
  if (a.pass >= npasses) return;  // the key range needs fewer digits
  const bool last = a.pass == npasses - 1;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* skey = reinterpret_cast<K*>(smem_raw);                                  // [kTile]
  uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kTile);               // [kTile]
  float* smass = reinterpret_cast<float*>(sval + kTile);                     // [kTile] if MASS
  uint32_t* whist = reinterpret_cast<uint32_t*>(smass + (MASS ? kTile : 0)); // [NW][R]
  uint32_t* dstart = whist + NW * R;                                         // [R]
  uint32_t* gbase = dstart + R;                                              // [R]
  __shared__ uint32_t s_tile;
  __shared__ uint32_t wsum[NW];
  __shared__ u128 wmass[NW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(&a.ctrl->ticket[a.pass], 1u);
  for (int i = tid; i < NW * R; i += kSortThreads) whist[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  // n <= 2^30, so every cell index and tile position fits 32 bits
  const uint32_t start = tile * (uint32_t)kTile;
  const uint32_t n = (uint32_t)a.n;
  const int shift = RB * a.pass;
  if (tid == 0) {
    // the payloads are read only after the ranking: start pulling them into L2
    const uint32_t bytes = (n - start < (uint32_t)kTile ? n - start : (uint32_t)kTile) * 4u;
    if constexpr (MASS) prefetch_l2_bulk(a.min + start, bytes);
    if constexpr (!FIRST) prefetch_l2_bulk(a.vin + start, bytes);
    // and all inputs of the tile a.ahead tickets later, which a CTA starting
    // soon will take (tiles go out in ticket order)
    const uint32_t fs = (tile + a.ahead) * (uint32_t)kTile;
    if (a.ahead && fs < n) {
      const uint32_t fb = n - fs < (uint32_t)kTile ? n - fs : (uint32_t)kTile;
      if constexpr (FIRST) prefetch_l2_bulk(reinterpret_cast<const SRC*>(a.J) + fs, fb * (uint32_t)sizeof(SRC));
      else prefetch_l2_bulk(reinterpret_cast<const K*>(a.kin) + fs, fb * (uint32_t)sizeof(K));
      if constexpr (MASS) prefetch_l2_bulk(a.min + fs, fb * 4u);
      if constexpr (!FIRST) prefetch_l2_bulk(a.vin + fs, fb * 4u);
    }
  }
  if (a.lb_next) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) a.lb_next[(int64_t)tile * R + j * kSortThreads + tid] = 0;
  }
  const uint32_t wbase = start + warp * kItems * 32 + lane;  // item it at wbase + 32 it
  const K kmin = FIRST ? (K)a.ctrl->kmin : K(0);

  // ---- keys (warp-striped) and their local ranks, packed rank | digit << 16
  K key[kItems];
  uint32_t rd[kItems];
  bool bad = false;
  uint32_t* wh = whist + warp * R;
  const unsigned lt = lanemask_lt();
  // Full tiles (all but the last) take a copy of the ranking without the
  // bounds guards and the ballot of in-range lanes.
  auto rank_items = [&](auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const uint32_t g = wbase + 32 * it;
      const bool ok = FULL || g < n;
      if constexpr (FIRST) key[it] = ok ? K(enc_desc(reinterpret_cast<const SRC*>(a.J)[g], bad) - kmin) : K(0);
      else key[it] = ok ? reinterpret_cast<const K*>(a.kin)[g] : K(0);
    }
#pragma unroll
    for (int it = 0; it < kItems; ++it) {
      const bool ok = FULL || wbase + 32 * it < n;
      const unsigned d = (unsigned)(key[it] >> shift) & (R - 1);
      unsigned peers;
      if constexpr (MATCH) {
        // lanes holding the same digit (out-of-range lanes group apart)
        peers = __match_any_sync(0xffffffffu, ok ? d : 0x10000u);
      } else {
        // the same set from one ballot per digit bit: keep the lanes whose bit
        // agrees.  m is the bit sign-extended (all ones when set), so the lanes
        // that agree with this one are ~(ballot ^ m)
        peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int b = 0; b < RB; ++b) {
          const unsigned m = (unsigned)((int)(d << (31 - b)) >> 31);
          peers &= ~(__ballot_sync(0xffffffffu, m != 0u) ^ m);
        }
      }
      uint32_t base = 0;
      if (ok) base = wh[d];
      __syncwarp();
      if (ok && (peers & lt) == 0u) wh[d] = base + __popc(peers);
      __syncwarp();
      rd[it] = ok ? ((base + __popc(peers & lt)) | (d << 16)) : 0xffffffffu;
    }
  };
  if (start + (uint32_t)kTile <= n) rank_items(std::true_type{});
  else rank_items(std::false_type{});
  __syncthreads();

  // ---- per digit (thread tid owns digits tid + 256 j): warp prefixes, the
  // tile count, and its publication for successors
  uint32_t cnt[DPT];
#pragma unroll
  for (int j = 0; j < DPT; ++j) {
    const int d = j * kSortThreads + tid;
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t x = whist[w * R + d];
      whist[w * R + d] = c;
      c += x;
    }
    cnt[j] = c;
    st_relaxed_u32(a.lb + (int64_t)tile * R + d, (tile == 0 ? kFlagInc : kFlagAgg) | c);
  }
  {
    // tile-local digit starts: exclusive scan over the R digits
    uint32_t carry = 0;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      uint32_t x = cnt[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncthreads();
      uint32_t wpre = 0, tot = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        wpre += (w < warp) ? wsum[w] : 0u;
        tot += wsum[w];
      }
      const uint32_t ds = carry + wpre + x - cnt[j];
      dstart[j * kSortThreads + tid] = ds;
#pragma unroll
      for (int w = 0; w < NW; ++w) whist[w * R + j * kSortThreads + tid] += ds;
      carry += tot;
      __syncthreads();
    }
  }

  // ---- keys, then payloads, into shared memory in tile-sorted order.  The
  // payloads are loaded only now (their L2 prefetch was issued at the start),
  // all kItems at once into the registers the keys just freed.
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    if (rd[it] == 0xffffffffu) continue;
    const unsigned dd = rd[it] >> 16;
    rd[it] = whist[warp * R + dd] + (rd[it] & 0xffffu);  // tile position
    skey[rd[it]] = key[it];
  }
  uint32_t pv[kItems];
  float pm[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const uint32_t g = wbase + 32 * it;
    const bool ok = rd[it] != 0xffffffffu;
    pv[it] = FIRST ? g : (ok ? a.vin[g] : 0u);
    if constexpr (MASS) pm[it] = ok ? a.min[g] : 0.0f;
  }
  u128 msum = 0;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    if (rd[it] == 0xffffffffu) continue;
    sval[rd[it]] = pv[it];
    if constexpr (MASS) {
      smass[rd[it]] = pm[it];
      if constexpr (FIRST) msum += mass_q64(pm[it], bad);
    }
  }
  if constexpr (FIRST && MASS) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) msum += shfl_down_u128(msum, o);
    if (lane == 0) wmass[warp] = msum;  // summed per tile after the next barrier
  }

  // ---- decoupled look-back per digit, kLookWindow predecessors per round
  // trip: sum aggregates back to the nearest inclusive prefix
#pragma unroll
  for (int j = 0; j < DPT; ++j) {
    const int d = j * kSortThreads + tid;
    uint32_t excl = 0;
    if (tile > 0) {
      int64_t t = (int64_t)tile - 1;
      unsigned spins = 0;
      while (true) {
        uint32_t w[kLookWindow];
#pragma unroll
        for (int k = 0; k < kLookWindow; ++k)
          w[k] = (t - k >= 0) ? ld_relaxed_u32(a.lb + (t - k) * R + d) : kFlagInc;
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
      st_relaxed_u32(a.lb + (int64_t)tile * R + d, kFlagInc | ((excl + cnt[j]) & kValueMask));
    }
    gbase[d] = a.ctrl->offs[a.pass * R + d] + excl - dstart[d];
  }
  __syncthreads();
  if constexpr (FIRST && MASS) {
    if (tid == 0) {
      u128 t = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) t += wmass[w];
      a.tile_mass[2 * (int64_t)tile] = (unsigned long long)t;
      a.tile_mass[2 * (int64_t)tile + 1] = (unsigned long long)(t >> 64);
    }
  }

  // ---- write out: consecutive positions of one digit go to consecutive addresses
  const int cnt_tile = (int)(n - start < (uint32_t)kTile ? n - start : (uint32_t)kTile);
  K* kout = reinterpret_cast<K*>(a.kout);
  // the last needed pass writes the order to vfinal when given, else to its
  // own parity's buffers (which it does not read)
  uint32_t* vout = (last && a.vfinal) ? a.vfinal : a.vout;
  float* mout = (last && a.mfinal) ? a.mfinal : a.mout;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int p = it * kSortThreads + tid;
    if (p < cnt_tile) {
      const K kk = skey[p];
      const uint32_t g = gbase[(unsigned)(kk >> shift) & (R - 1)] + p;
      if (!last) kout[g] = kk;
      vout[g] = sval[p];
      if constexpr (MASS) mout[g] = smass[p];
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0)
    raise_status(a.status, (FIRST && MASS) ? (AMBER_ERR_NONFINITE | AMBER_ERR_INVALID_MASS) : AMBER_ERR_NONFINITE);
}

template <typename SRC, int RB, bool FIRST, bool MASS, bool MATCH>
__global__ void __launch_bounds__(kSortThreads, AMBER_SORT_MINB) k_sort_pass(const PassArgs a) {
  sort_pass_body<SRC, RB, FIRST, MASS, MATCH>(a);
}

// Several sorts at once: CTA b works on item find_item(prefix, M, b) (the
// prefix counts tiles), taking its tile from that item's own ticket.
template <typename SRC, int RB, bool FIRST, bool MASS, bool MATCH>
__global__ void __launch_bounds__(kSortThreads, AMBER_SORT_MINB)
    k_sort_pass_multi(const PassArgs* __restrict__ args, const uint32_t* __restrict__ prefix, int M) {
  __shared__ PassArgs sa;
  if (threadIdx.x == 0) sa = args[find_item(prefix, M, blockIdx.x)];
  __syncthreads();
  sort_pass_body<SRC, RB, FIRST, MASS, MATCH>(sa);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
template <typename SRC, int RB> static size_t pass_smem(bool mass) {
  constexpr int R = 1 << RB;
  return (size_t)kTile * sizeof(typename KeyOf<SRC>::K) + (size_t)kTile * 4 * (mass ? 2 : 1) +
         (size_t)(kSortThreads / 32) * R * 4 + 2 * R * 4;
}

int64_t sort_tiles(int64_t n) { return (n + kTile - 1) / kTile; }
size_t sort_lookback_words(int64_t n) { return (size_t)sort_tiles(n) * kMaxRadix; }

template <typename SRC, int RB, bool FIRST, bool MASS, bool MATCH>
static void launch_pass_v(const PassArgs& a, int64_t tiles, cudaStream_t s) {
  const size_t smem = pass_smem<SRC, RB>(MASS);
  static std::atomic<unsigned long long> attr{0};  // per instantiation and device
  if (first_use_on_device(attr))
    cudaFuncSetAttribute(k_sort_pass<SRC, RB, FIRST, MASS, MATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  k_sort_pass<SRC, RB, FIRST, MASS, MATCH><<<(unsigned)tiles, kSortThreads, smem, s>>>(a);
}

// Digit peers by ballots (one per digit bit) or by warp match; measured on
// GB300 the ballots are faster (35.2 vs 37.7 ms for the three passes at
// 1024^3).  The caller (the context's tuning) picks; AMBER_SORT_RANK=
// ballot|match overrides it.
static int rank_env() {
  static const int m = [] {
    const char* v = getenv("AMBER_SORT_RANK");
    return !v ? -1 : strcmp(v, "match") == 0 ? 1 : strcmp(v, "ballot") == 0 ? 0 : -1;
  }();
  return m;
}

template <typename SRC, int RB, bool FIRST, bool MASS>
static void launch_pass(const PassArgs& a, int64_t tiles, cudaStream_t s, bool match) {
  if (match) launch_pass_v<SRC, RB, FIRST, MASS, true>(a, tiles, s);
  else launch_pass_v<SRC, RB, FIRST, MASS, false>(a, tiles, s);
}

cudaError_t sort_ctrl_reset(SortCtrl* ctrl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(SortCtrl), s);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(&ctrl->kmin, 0xff, sizeof(ctrl->kmin), s);
}

template <typename SRC, int RB>
static cudaError_t rank_impl_rb(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in,
                                float* mass_out, unsigned long long* tile_mass, bool range_ready,
                                unsigned int* status, cudaStream_t s, FftProfile* prof, unsigned int spin_limit,
                                bool match, bool hist_ready) {
  using K = typename KeyOf<SRC>::K;
  constexpr int R = 1 << RB, P = max_passes<SRC, RB>();
  const bool with_mass = mass_in != nullptr;
  const int64_t tiles = sort_tiles(n);
  const int64_t lbw = tiles * R;  // words per look-back region used
  SortCtrl* ctrl = w.ctrl;
  cudaError_t e;
  if (!range_ready) {
    e = sort_ctrl_reset(ctrl, s);
    if (e != cudaSuccess) return e;
  }
  uint32_t* lbA = w.lookback;
  uint32_t* lbB = w.lookback + sort_lookback_words(w.max_cells);

  prof_begin(prof, PK_SORT_HIST, s);
  if (hist_ready && range_ready && sizeof(SRC) == 4 && RB == 8) {
    // the intensity kernel counted the raw keys' digits: clear the first
    // pass's look-back and form the offsets of a raw-key sort
    e = cudaMemsetAsync(lbA, 0, (size_t)lbw * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_sort_offsets<SRC, RB><<<1, 256, 0, s>>>(ctrl, true);
  } else {
    int grid = (int)std::min<int64_t>((n / (16 / (int)sizeof(SRC)) + 255) / 256, (int64_t)w.num_sms * 8);
    if (grid < 1) grid = 1;
    if (!range_ready) k_key_range<SRC><<<grid, 256, 0, s>>>(J, n, ctrl, status);
    k_sort_histogram<SRC, RB><<<grid, 256, 0, s>>>(J, n, ctrl, lbA, lbw);
    k_sort_offsets<SRC, RB><<<1, 256, 0, s>>>(ctrl, false);
  }
  prof_end(prof, PK_SORT_HIST, s);

  K* kA = reinterpret_cast<K*>(w.keysA);
  K* kB = reinterpret_cast<K*>(w.keysB);
  const void* kin = nullptr;
  const uint32_t* vin = nullptr;
  const float* mcur = mass_in;
  for (int p = 0; p < P; ++p) {
    PassArgs a;
    a.J = J;
    a.kin = kin;
    a.vin = vin;
    a.min = mcur;
    a.kout = (p & 1) ? (void*)kB : (void*)kA;
    a.vout = (p & 1) ? w.idxB : w.idxA;
    a.mout = with_mass ? ((p & 1) ? w.massB : w.massA) : nullptr;
    a.vfinal = order;
    a.mfinal = mass_out;
    a.n = n;
    a.pass = p;
    a.lb = (p & 1) ? lbB : lbA;
    a.lb_next = (p == P - 1) ? nullptr : ((p & 1) ? lbA : lbB);
    a.ctrl = ctrl;
    a.tile_mass = tile_mass;
    a.status = status;
    a.spin_limit = spin_limit;
    a.ahead = (uint32_t)w.num_sms;  // a third of the resident wave: measured best
    prof_begin(prof, PK_SORT_PASS, s);
    if (p == 0) {
      if (with_mass) launch_pass<SRC, RB, true, true>(a, tiles, s, match);
      else launch_pass<SRC, RB, true, false>(a, tiles, s, match);
    } else {
      if (with_mass) launch_pass<SRC, RB, false, true>(a, tiles, s, match);
      else launch_pass<SRC, RB, false, false>(a, tiles, s, match);
    }
    prof_end(prof, PK_SORT_PASS, s);
    kin = a.kout;
    vin = a.vout;
    mcur = a.mout;
  }
  return cudaGetLastError();
}

template <typename SRC>
cudaError_t rank_impl(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in,
                      float* mass_out, unsigned long long* tile_mass, bool range_ready, unsigned int* status,
                      cudaStream_t s, FftProfile* prof, unsigned int spin_limit, int digit_bits, int match,
                      bool hist_ready) {
  const int env = rank_env();
  const bool m = env >= 0 ? env == 1 : match == 1;
  if (digit_bits == 0) digit_bits = KeyOf<SRC>::RB;
  if constexpr (sizeof(SRC) == 4) {
    if (digit_bits == 8)
      return rank_impl_rb<SRC, 8>(w, J, n, order, mass_in, mass_out, tile_mass, range_ready, status, s, prof,
                                  spin_limit, m, hist_ready);
    if (digit_bits == 9)
      return rank_impl_rb<SRC, 9>(w, J, n, order, mass_in, mass_out, tile_mass, range_ready, status, s, prof,
                                  spin_limit, m, hist_ready);
  } else {
    if (digit_bits == 8)
      return rank_impl_rb<SRC, 8>(w, J, n, order, mass_in, mass_out, tile_mass, range_ready, status, s, prof,
                                  spin_limit, m, hist_ready);
  }
  return cudaErrorInvalidValue;
}

template <typename SRC>
int rank_args(const SortWork& w, const SRC* J, int64_t n, uint32_t* order, const float* mass_in, float* mass_out,
              unsigned long long* tile_mass, unsigned int* status, unsigned int spin_limit, int digit_bits,
              HistArgs* hist, uint32_t* hist_blocks, PassArgs pass[4]) {
  using K = typename KeyOf<SRC>::K;
  const int RB = digit_bits ? digit_bits : KeyOf<SRC>::RB;
  const int P = (8 * (int)sizeof(K) + RB - 1) / RB;
  const int R = 1 << RB;
  const int64_t tiles = sort_tiles(n);
  uint32_t* lbA = w.lookback;
  uint32_t* lbB = w.lookback + sort_lookback_words(w.max_cells);
  hist->J = J;
  hist->n = n;
  hist->ctrl = w.ctrl;
  hist->lb0 = lbA;
  hist->lb0_words = tiles * R;
  int grid = (int)std::min<int64_t>((n / (16 / (int)sizeof(SRC)) + 255) / 256, (int64_t)w.num_sms * 8);
  *hist_blocks = (uint32_t)std::max(grid, 1);
  K* kA = reinterpret_cast<K*>(w.keysA);
  K* kB = reinterpret_cast<K*>(w.keysB);
  const void* kin = nullptr;
  const uint32_t* vin = nullptr;
  const float* mcur = mass_in;
  for (int p = 0; p < P; ++p) {
    PassArgs& a = pass[p];
    a.J = J;
    a.kin = kin;
    a.vin = vin;
    a.min = mcur;
    a.kout = (p & 1) ? (void*)kB : (void*)kA;
    a.vout = (p & 1) ? w.idxB : w.idxA;
    a.mout = mass_in ? ((p & 1) ? w.massB : w.massA) : nullptr;
    a.vfinal = order;
    a.mfinal = mass_out;
    a.n = n;
    a.pass = p;
    a.lb = (p & 1) ? lbB : lbA;
    a.lb_next = (p == P - 1) ? nullptr : ((p & 1) ? lbA : lbB);
    a.ctrl = w.ctrl;
    a.tile_mass = tile_mass;
    a.status = status;
    a.spin_limit = spin_limit;
    a.ahead = (uint32_t)w.num_sms;
    kin = a.kout;
    vin = a.vout;
    mcur = a.mout;
  }
  return P;
}

template <int RB, bool FIRST, bool MATCH>
static void launch_pass_multi(const RankMulti& r, int p, cudaStream_t s) {
  const size_t smem = pass_smem<float, RB>(true);
  static std::atomic<unsigned long long> attr{0};  // per instantiation and device
  if (first_use_on_device(attr))
    cudaFuncSetAttribute(k_sort_pass_multi<float, RB, FIRST, true, MATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  k_sort_pass_multi<float, RB, FIRST, true, MATCH><<<r.tiles, kSortThreads, smem, s>>>(r.pass[p], r.tile_prefix, r.M);
}

template <int RB>
static cudaError_t rank_multi_rb(const RankMulti& r, bool match, cudaStream_t s) {
  constexpr int P = max_passes<float, RB>();
  k_sort_histogram_multi<float, RB><<<r.hist_blocks, 256, 0, s>>>(r.hist, r.hist_prefix, r.M);
  k_sort_offsets_multi<float, RB><<<r.M, 256, 0, s>>>(r.hist);
  for (int p = 0; p < P; ++p) {
    if (p == 0) {
      if (match) launch_pass_multi<RB, true, true>(r, p, s);
      else launch_pass_multi<RB, true, false>(r, p, s);
    } else {
      if (match) launch_pass_multi<RB, false, true>(r, p, s);
      else launch_pass_multi<RB, false, false>(r, p, s);
    }
  }
  return cudaGetLastError();
}

cudaError_t rank_multi(const RankMulti& r, int digit_bits, bool match, cudaStream_t s) {
  const int env = rank_env();
  const bool m = env >= 0 ? env == 1 : match;
  if (digit_bits == 8) return rank_multi_rb<8>(r, m, s);
  if (digit_bits == 9) return rank_multi_rb<9>(r, m, s);
  return cudaErrorInvalidValue;
}

template int rank_args<float>(const SortWork&, const float*, int64_t, uint32_t*, const float*, float*,
                              unsigned long long*, unsigned int*, unsigned int, int, HistArgs*, uint32_t*,
                              PassArgs[4]);

template cudaError_t rank_impl<float>(const SortWork&, const float*, int64_t, uint32_t*, const float*, float*,
                                      unsigned long long*, bool, unsigned int*, cudaStream_t, FftProfile*,
                                      unsigned int, int, int, bool);
template cudaError_t rank_impl<double>(const SortWork&, const double*, int64_t, uint32_t*, const float*, float*,
                                       unsigned long long*, bool, unsigned int*, cudaStream_t, FftProfile*,
                                       unsigned int, int, int, bool);

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
