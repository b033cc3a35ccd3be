// Abundance matching (Sec. 3.4.2): the rank-n cell is ionized at z_n where
// the cumulative mass fraction F_n = M_n / M_total equals the history x(z_n)
// (Sec. 3.1.2, Eq. weibull), with x(z) tabulated on uniform redshifts.
//
//   k_mass_reduce   : M_total = sum of all cell masses (order-free)
//   k_thresholds    : table x_j = x(z_j) and the exact integer thresholds
//                     X_j = floor(x_j * M_total), so "x_j >= F_n" is the
//                     integer test "X_j >= M_n"; plus 1/(X_j - X_j+1)
//   k_scan_assign   : M_n by a decoupled-look-back prefix sum over ranks
//                     (gathering mass[order[n]]), bracket j* by a search in
//                     the thresholds amortised over each thread's run of
//                     ranks, interpolate, scatter z_re[order[n]] = z_n.
//
// Masses are summed exactly as 128-bit fixed point with 64 fraction bits
// (every float >= 2^-41 is represented exactly), so the prefix sums carry no
// rounding at all and do not depend on summation order; only the final
// interpolation weight is rounded (FP32).
#include "assign.cuh"

namespace amber {

__device__ __forceinline__ u128 mass_q64(float m, bool& bad) {
  const uint32_t b = __float_as_uint(m);
  if (b & 0x80000000u) {
    if (b != 0x80000000u) bad = true;  // negative (but -0 is zero)
    return 0;
  }
  const uint32_t e = b >> 23;
  if (e >= 127u + 40u) {  // >= 2^40, Inf or NaN
    bad = true;
    return 0;
  }
  const uint64_t mant = (e == 0) ? (b & 0x7fffffu) : ((b & 0x7fffffu) | 0x800000u);
  const int sh = (int)(e == 0 ? 1u : e) - 150 + 64;  // value = mant * 2^(e-150), scaled by 2^64
  if (sh >= 0) return (u128)mant << sh;
  if (sh <= -24) return 0;
  return (u128)(mant >> (-sh));
}

__device__ __forceinline__ u128 shfl_u128(u128 v, int src) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  return ((u128)__shfl_sync(0xffffffffu, hi, src) << 64) | (u128)__shfl_sync(0xffffffffu, lo, src);
}
__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  return ((u128)__shfl_up_sync(0xffffffffu, hi, d) << 64) | (u128)__shfl_up_sync(0xffffffffu, lo, d);
}
__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  return ((u128)__shfl_down_sync(0xffffffffu, hi, d) << 64) | (u128)__shfl_down_sync(0xffffffffu, lo, d);
}

__device__ __forceinline__ float u128_to_float(u128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return __ull2float_rn(hi) * 18446744073709551616.0f + __ull2float_rn(lo);
}
__device__ __forceinline__ double u128_to_double(u128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return __ull2double_rn(hi) * 18446744073709551616.0 + __ull2double_rn(lo);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mass_reduce(const float* __restrict__ mass, int64_t n,
                                                     unsigned long long* __restrict__ total,
                                                     unsigned int* __restrict__ status) {
  u128 acc = 0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc += mass_q64(mass[i], bad);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc += shfl_down_u128(acc, o);
  __shared__ u128 ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    u128 s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    const unsigned long long lo = (unsigned long long)s, hi = (unsigned long long)(s >> 64);
    const unsigned long long old = atomicAdd(&total[0], lo);
    const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&total[1], hi + carry);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, AMBER_ERR_INVALID_MASS);
}

// floor(x * T) for x in [0, 1] and T < 2^128, exactly.
__device__ __forceinline__ u128 mul_floor(double x, u128 T) {
  if (!(x > 0.0)) return 0;
  if (x >= 1.0) return T;
  int ex;
  const double f = frexp(x, &ex);                        // x = f 2^ex, f in [0.5, 1)
  const unsigned long long mant = (unsigned long long)ldexp(f, 53);  // exact 53-bit integer
  const int s = 53 - ex;                                 // x = mant 2^-s, s >= 53
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

__global__ void __launch_bounds__(256) k_thresholds(const unsigned long long* __restrict__ total, int M,
                                                    double a_w, double b_w, double c_w, double z_lo, double z_hi,
                                                    u128* __restrict__ X, float* __restrict__ inv_dx) {
  const u128 T = ((u128)total[1] << 64) | (u128)total[0];
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const double z = z_lo + (z_hi - z_lo) * (double)j / (double)(M - 1);
    const double u = fmax((z - a_w) / b_w, 0.0);
    const double x = exp(-pow(u, c_w));
    X[j] = mul_floor(x, T);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < M - 1; j += blockDim.x) {
    const u128 d = X[j] - X[j + 1];
    inv_dx[j] = d > 0 ? 1.0f / u128_to_float(d) : 0.0f;
  }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void publish(ScanTile* st, u128 v, unsigned int flag) {
  volatile unsigned long long* p = (flag == 1u) ? &st->agg_lo : &st->inc_lo;
  p[0] = (unsigned long long)v;
  p[1] = (unsigned long long)(v >> 64);
  __threadfence();
  st_release_u32(&st->flag, flag);
}

template <bool WANT_F>
__global__ void __launch_bounds__(kScanThreads) k_scan_assign(
    const uint32_t* __restrict__ order, const float* __restrict__ mass, int64_t n,
    const unsigned long long* __restrict__ total, const u128* __restrict__ X, const float* __restrict__ inv_dx,
    int M, float z_lo, float z_hi, float dzt, float* __restrict__ zre, double* __restrict__ Fout,
    ScanTile* __restrict__ state, uint32_t* __restrict__ ticket, unsigned int* __restrict__ status,
    unsigned int spin_limit) {
  constexpr int NT = kScanThreads, IT = kScanItems, TILE = kScanTile;
  __shared__ uint32_t sord[TILE + TILE / 32];
  __shared__ u128 wtot[NT / 32];
  __shared__ u128 s_excl;
  __shared__ uint32_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t start = (int64_t)tile * TILE;
  const int cnt = (int)(n - start < (int64_t)TILE ? n - start : (int64_t)TILE);

  // order: coalesced striped load -> padded shared -> blocked per thread
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int p = k * NT + tid;
    sord[p + (p >> 5)] = p < cnt ? order[start + p] : 0u;
  }
  __syncthreads();
  uint32_t cell[IT];
  u128 loc[IT];
  bool bad = false;
  u128 run = 0;
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int p = tid * IT + i;
    cell[i] = sord[p + (p >> 5)];
    const u128 q = (p < cnt) ? mass_q64(mass[cell[i]], bad) : (u128)0;
    run += q;
    loc[i] = run;
  }
  // block exclusive scan of the thread totals
  u128 x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u128 y = shfl_up_u128(x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[warp] = x;
  __syncthreads();
  u128 wpre = 0, tile_sum = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    if (w < warp) wpre += wtot[w];
    tile_sum += wtot[w];
  }
  const u128 thr_excl = wpre + x - run;

  if (tid == 0) {
    ScanTile* me = state + tile;
    u128 excl = 0;
    if (tile == 0) {
      publish(me, tile_sum, 2u);
    } else {
      publish(me, tile_sum, 1u);
      int64_t t = (int64_t)tile - 1;
      unsigned spins = 0;
      while (t >= 0) {
        ScanTile* o = state + t;
        const unsigned int f = ld_acquire_u32(&o->flag);
        if (f == 0u) {
          if (++spins >= spin_limit) { raise_status(status, AMBER_ERR_DEVICE_TIMEOUT); break; }
          __nanosleep(32);
          continue;
        }
        const volatile unsigned long long* v = (f == 2u) ? &o->inc_lo : &o->agg_lo;
        excl += ((u128)v[1] << 64) | (u128)v[0];
        if (f == 2u) break;
        --t;
      }
      publish(me, excl + tile_sum, 2u);
    }
    s_excl = excl;
  }
  __syncthreads();
  const u128 base = s_excl + thr_excl;
  const u128 T = ((u128)total[1] << 64) | (u128)total[0];
  const double invT = WANT_F ? 1.0 / u128_to_double(T) : 0.0;

  // bracket: cntX = #{j : X_j >= M_n}; X is non-increasing in j and M_n grows
  // along the thread's ranks, so one binary search then a short walk down.
  int cx = -1;
#pragma unroll
  for (int i = 0; i < IT; ++i) {
    const int p = tid * IT + i;
    if (p >= cnt) break;
    const u128 Mn = base + loc[i];
    if (cx < 0) {
      int lo = 0, hi = M;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (X[mid] >= Mn) lo = mid + 1; else hi = mid;
      }
      cx = lo;
    } else {
      while (cx > 0 && X[cx - 1] < Mn) --cx;
    }
    const int j = cx - 1;
    float z;
    if (j < 0) z = z_lo;
    else if (j == M - 1) z = z_hi;
    else {
      float t = u128_to_float(X[j] - Mn) * inv_dx[j];
      t = fminf(fmaxf(t, 0.0f), 0.99999994f);
      z = z_lo + ((float)j + t) * dzt;
    }
    zre[cell[i]] = z;
    if (WANT_F) Fout[start + p] = u128_to_double(Mn) * invT;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, AMBER_ERR_INVALID_MASS);
}

// ---------------------------------------------------------------------------
cudaError_t assign_impl(const AssignWork& w, const uint32_t* order, const float* mass, int64_t n,
                        const HistoryCoeffs& hc, float* zre, double* F, unsigned int* status, cudaStream_t s,
                        FftProfile* prof, unsigned int spin_limit) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaMemsetAsync(w.ctrl, 0, kAssignCtrlBytes, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.state, 0, (size_t)tiles * sizeof(ScanTile), s);
  if (e != cudaSuccess) return e;
  unsigned long long* total = reinterpret_cast<unsigned long long*>(w.ctrl);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(w.ctrl + 16);

  prof_begin(prof, PK_MASS_REDUCE, s);
  int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)w.num_sms * 8);
  if (grid < 1) grid = 1;
  k_mass_reduce<<<grid, 256, 0, s>>>(mass, n, total, status);
  prof_end(prof, PK_MASS_REDUCE, s);

  prof_begin(prof, PK_THRESHOLDS, s);
  k_thresholds<<<1, 256, 0, s>>>(total, hc.n_table, hc.a, hc.b, hc.c, hc.z_lo, hc.z_hi, w.X, w.inv_dx);
  prof_end(prof, PK_THRESHOLDS, s);

  const float dzt = (float)((hc.z_hi - hc.z_lo) / (double)(hc.n_table - 1));
  prof_begin(prof, PK_SCAN_ASSIGN, s);
  if (F)
    k_scan_assign<true><<<(unsigned)tiles, kScanThreads, 0, s>>>(order, mass, n, total, w.X, w.inv_dx, hc.n_table,
        (float)hc.z_lo, (float)hc.z_hi, dzt, zre, F, w.state, ticket, status, spin_limit);
  else
    k_scan_assign<false><<<(unsigned)tiles, kScanThreads, 0, s>>>(order, mass, n, total, w.X, w.inv_dx, hc.n_table,
        (float)hc.z_lo, (float)hc.z_hi, dzt, zre, F, w.state, ticket, status, spin_limit);
  prof_end(prof, PK_SCAN_ASSIGN, s);
  return cudaGetLastError();
}

}  // namespace amber
