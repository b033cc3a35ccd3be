// Radiation field J = IDFT(DFT(S) * K(|k|)) on an n^3 periodic grid
// (Sec. 3.4.1, Eq. intensity), as five HBM passes over a half spectrum:
//
//   x-pass  R2C   S[z][y][x]      -> H[z][y][kx]      (two real rows per complex FFT)
//   y-pass  fwd   H along y, in place
//   z-pass  fwd along z, multiply by K(|k|)/n^3, inverse along z (one round trip)
//   y-pass  inv   H along y, in place
//   x-pass  C2R   H -> J[z][y][x]
//
// H is [n][n][RS] complex with RS = n/2 + 2 (rows 16-byte aligned); columns
// kx in [0, n/2] are live.  Each CTA transforms a batch of lines held in
// registers and shared memory with a two-stage Stockham decomposition
// n = R0 * R1 (R0 = n for n <= 32): stage A reads its inputs straight from
// global memory, stage B writes its outputs straight back, so every 1D
// transform costs one read and one write of the line and one shared-memory
// exchange.  In the z-pass the forward stage B and the inverse stage A touch
// the same register set, so the kernel multiply happens in registers.
#pragma once

#include <cuda.h>  // CUtensorMap (the z pass's TMA descriptor)

#include "common.cuh"
#include "keys.cuh"

namespace amber {

// Per size N, variant V: the radix split N = R0 R1, elements per thread E
// (a multiple of both radices), lines per strided tile SB and row pairs per
// x-pass tile XP.  Variant 0 is the default; variant 1 (N >= 128) is the
// alternative split or tile the autotuner times against it.
template <int N, int V = 0> struct FftCfg;
//                                           R0  R1   E  strided-lines  x-pairs
template <> struct FftCfg<1024, 0> { static constexpr int R0 = 32, R1 = 32, E = 32, SB = 8,  XP = 8;  };
template <> struct FftCfg<512, 0>  { static constexpr int R0 = 32, R1 = 16, E = 32, SB = 16, XP = 16; };
template <> struct FftCfg<256, 0>  { static constexpr int R0 = 16, R1 = 16, E = 16, SB = 16, XP = 16; };
template <> struct FftCfg<128, 0>  { static constexpr int R0 = 16, R1 = 8,  E = 16, SB = 32, XP = 32; };
template <> struct FftCfg<64, 0>   { static constexpr int R0 = 8,  R1 = 8,  E = 8,  SB = 32, XP = 32; };
template <> struct FftCfg<32, 0>   { static constexpr int R0 = 32, R1 = 1,  E = 32, SB = 32, XP = 32; };
template <> struct FftCfg<16, 0>   { static constexpr int R0 = 16, R1 = 1,  E = 16, SB = 32, XP = 32; };
template <> struct FftCfg<8, 0>    { static constexpr int R0 = 8,  R1 = 1,  E = 8,  SB = 32, XP = 32; };
template <> struct FftCfg<4, 0>    { static constexpr int R0 = 4,  R1 = 1,  E = 4,  SB = 32, XP = 32; };
template <> struct FftCfg<1024, 1> { static constexpr int R0 = 32, R1 = 32, E = 32, SB = 4,  XP = 4;  };
template <> struct FftCfg<512, 1>  { static constexpr int R0 = 16, R1 = 32, E = 32, SB = 8,  XP = 8;  };
template <> struct FftCfg<256, 1>  { static constexpr int R0 = 32, R1 = 8,  E = 32, SB = 8,  XP = 8;  };
template <> struct FftCfg<128, 1>  { static constexpr int R0 = 8,  R1 = 16, E = 16, SB = 16, XP = 16; };

template <int N, int V = 0> constexpr int strided_threads() { return FftCfg<N, V>::SB * N / FftCfg<N, V>::E; }
template <int N, int V = 0> constexpr int xpass_threads() { return FftCfg<N, V>::XP * N / FftCfg<N, V>::E; }

// Shared-memory layout of a strided tile: element (n, b) of line b.  With
// 8 float2 lines a row is 64 bytes; the pad per 32 rows puts the row groups
// a stage-A butterfly writes (n = 32 j + r) on alternating bank halves.
template <typename T, int N, int V = 0> struct StridedSmem {
  static constexpr int SB = FftCfg<N, V>::SB;
  static constexpr int PAD = (SB * (int)sizeof(cpx<T>) == 64) ? 8 : 0;
  static constexpr int elems = N * SB + (N / 32) * PAD;
  static __device__ __forceinline__ int pos(int n, int b) { return n * SB + b + (n >> 5) * PAD; }
};

// Shared-memory layout of x-pass lines: line p, element n.  One pad element
// per R0 keeps stage-A writes (n = R0 j + r, lanes along j) conflict-free.
template <typename T, int N, int V = 0> struct XSmem {
  static constexpr int R0 = FftCfg<N, V>::R0;
  static constexpr int LS = N + N / R0;
  static constexpr int elems = FftCfg<N, V>::XP * LS;
  static __device__ __forceinline__ int pos(int p, int n) { return p * LS + n + n / R0; }
};

// K(|k|)/C at lattice |k|^2 = k2 (an exact integer), |k| = kf sqrt(k2):
// arctan(|k| l)/|k|, and l at k = 0.  FP32 uses one reciprocal square root
// instead of a square root and a division.
template <typename T> __device__ __forceinline__ T kernel_K(T k2, T l_mfp, T kf, T norm);
template <> __device__ __forceinline__ float kernel_K<float>(float k2, float l, float kf, float norm) {
  if (k2 == 0.f) return l * norm;
  const float r = rsqrtf(k2);          // 1/sqrt(k2)
  return atanf(kf * l * (k2 * r)) * (r * (norm / kf));
}
template <> __device__ __forceinline__ double kernel_K<double>(double k2, double l, double kf, double norm) {
  if (k2 == 0.0) return l * norm;
  const double k = kf * sqrt(k2);
  return atan(k * l) / k * norm;
}

// Number of SM ids: with CTAs per SM, the launch index distance of one resident wave
__device__ __forceinline__ int sm_count() {
  unsigned n;
  asm("mov.u32 %0, %%nsmid;" : "=r"(n));
  return (int)n;
}

__device__ __forceinline__ int signed_freq(int m, int n) { return m < n / 2 ? m : m - n; }

// K(|k|)/n^3 of one tile's columns kx0 .. kx0 + SB - 1 at ky for |kz| = 0..n/2
// into Kt (row |kz|, column b).  Evaluated per tile while the tile's loads
// are in flight: a table over |k|^2 read from L2 was measured slower.
template <typename T, int N, int SB, int NT>
__device__ __forceinline__ void tile_kernel(T* Kt, int kx0, int ky, int tid, T kf, T l_mfp, T norm) {
#pragma unroll 1
  for (int i = tid; i < (N / 2 + 1) * SB; i += NT) {
    const int kza = i / SB, kx = kx0 + (i - kza * SB);
    Kt[i] = kernel_K<T>((T)(kx * kx + ky * ky + kza * kza), l_mfp, kf, norm);
  }
}

// ---------------------------------------------------------------------------
// Strided passes (y forward, y inverse, z convolution).  A CTA owns SB
// consecutive kx columns of one line family; lane mapping is column-fastest
// so each row of the tile is one contiguous global segment.
// ---------------------------------------------------------------------------
enum { PASS_FWD = 0, PASS_INV = 1, PASS_CONV = 2 };

// OOP (z-pass only): the tile is read from Hin, a spectrum kept by the
// caller, and the result written to H; otherwise H is read and written in place.
// MULTI (z-pass only): several transforms of size N back to back, item_stride
// elements apart; line family `outer` of the launch is line y = outer % N of
// item outer / N, whose box and l_mfp give kp[2 item] = kf, kp[2 item + 1] = l.
// CTAs per SM the strided passes are compiled for (build-time tunables): two
// keep 128 registers per thread at 256 threads.
#ifndef AMBER_ZPASS_MINB
#define AMBER_ZPASS_MINB 2
#endif
#ifndef AMBER_YPASS_MINB
#define AMBER_YPASS_MINB 2
#endif
template <typename T, int N, int MODE, int V = 0, bool OOP = false, bool MULTI = false>
__global__ void __launch_bounds__(strided_threads<N, V>(), MODE == PASS_CONV ? AMBER_ZPASS_MINB : AMBER_YPASS_MINB)
k_fft_strided(cpx<T>* __restrict__ H, int64_t elem_stride, int64_t outer_stride, int ncol,
              int ntx, const cpx<T>* __restrict__ tw, T kf, T l_mfp, T norm,
              const cpx<T>* __restrict__ Hin = nullptr, int64_t item_stride = 0,
              const T* __restrict__ kp = nullptr) {
  using C = FftCfg<N, V>;
  using L = StridedSmem<T, N, V>;
  constexpr int R0 = C::R0, R1 = C::R1, E = C::E, SB = C::SB, NT = strided_threads<N, V>();
  constexpr int QA = E / R0, QB = (R1 > 1) ? E / R1 : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);

  const int tid = threadIdx.x;
  int outer = blockIdx.x / ntx;
  const int kx0 = (blockIdx.x - outer * ntx) * SB;
  int64_t item_off = 0;
  if constexpr (MULTI) {
    const int item = outer / N;
    outer -= item * N;
    item_off = (int64_t)item * item_stride;
    kf = kp[2 * item];
    l_mfp = kp[2 * item + 1];
  }
  cpx<T>* base = H + item_off + (int64_t)outer * outer_stride + kx0;
  const cpx<T>* ibase = OOP ? Hin + (int64_t)outer * outer_stride + kx0 : base;

  cpx<T> v[E];
  // ---- forward stage A: radix R0 over n = j + r N/R0, read from global
#pragma unroll
  for (int q = 0; q < QA; ++q) {
    const int id = tid + q * NT;
    const int b = id % SB, j = id / SB;
    const bool ok = kx0 + b < ncol;
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int n = j + r * (N / R0);
      v[q * R0 + r] = ok ? ibase[(int64_t)n * elem_stride + b] : mk<T>(0, 0);
    }
  }
  if constexpr (MODE == PASS_CONV) {
    // K(|k|)/n^3 of this tile's columns for |kz| = 0..N/2, into shared memory
    // after the tile, while the loads are in flight
    tile_kernel<T, N, SB, NT>(reinterpret_cast<T*>(sm + L::elems), kx0, signed_freq(outer, N), tid, kf, l_mfp,
                              norm);
    if constexpr (R1 == 1) __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < QA; ++q) dft<R0, MODE == PASS_INV>(v + q * R0);
  if constexpr (R1 == 1) {
    // single stage (n <= 32): v already holds natural order n = r for j = 0
  } else {
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R0; ++r) sm[L::pos(j * R0 + r, b)] = v[q * R0 + r];
    }
    __syncthreads();
    // ---- forward stage B: radix R1 over n = j + r R0, twiddle w_N^(j r)
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        cpx<T> x = sm[L::pos(j + r * R0, b)];
        if (r > 0) {
          const cpx<T> w = tw[j * r];
          x = (MODE == PASS_INV) ? cmulc(x, w) : cmul(x, w);
        }
        v[q * R1 + r] = x;
      }
      dft<R1, MODE == PASS_INV>(v + q * R1);
    }
  }

  if constexpr (MODE != PASS_CONV) {
    // ---- write natural order n = j + r R0 (or n = r when single stage)
    constexpr int QO = (R1 > 1) ? QB : QA;
    constexpr int RO = (R1 > 1) ? R1 : R0;
#pragma unroll
    for (int q = 0; q < QO; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
      if (kx0 + b < ncol) {
#pragma unroll
        for (int r = 0; r < RO; ++r) {
          const int n = (R1 > 1) ? j + r * R0 : r;
          base[(int64_t)n * elem_stride + b] = v[q * RO + r];
        }
      }
    }
  } else {
    // ---- z-pass: multiply by K(|k|)/n^3 at kz = n, ky = outer, kx = kx0 + b
    constexpr int QO = (R1 > 1) ? QB : QA;
    constexpr int RO = (R1 > 1) ? R1 : R0;
    const T* Kt = reinterpret_cast<const T*>(sm + L::elems);
#pragma unroll
    for (int q = 0; q < QO; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < RO; ++r) {
        const int n = (R1 > 1) ? j + r * R0 : r;
        const int kza = n <= N / 2 ? n : N - n;
        v[q * RO + r] = scale(v[q * RO + r], Kt[kza * SB + b]);
      }
      // inverse stage A (radix RO) on the same elements: n = j + r N/RO
      dft<RO, true>(v + q * RO);
    }
    if constexpr (R1 > 1) {
      // inverse plan is (R1, R0): stage A wrote n = j R1 + r
      __syncthreads();  // all forward stage-B reads of sm are done
#pragma unroll
      for (int q = 0; q < QB; ++q) {
        const int id = tid + q * NT;
        const int b = id % SB, j = id / SB;
#pragma unroll
        for (int r = 0; r < R1; ++r) sm[L::pos(j * R1 + r, b)] = v[q * R1 + r];
      }
      __syncthreads();
      // inverse stage B: radix R0 over n = j + r R1, twiddle conj(w_N^(j r))
#pragma unroll
      for (int q = 0; q < QA; ++q) {
        const int id = tid + q * NT;
        const int b = id % SB, j = id / SB;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          cpx<T> x = sm[L::pos(j + r * R1, b)];
          if (r > 0) x = cmulc(x, tw[j * r]);
          v[q * R0 + r] = x;
        }
        dft<R0, true>(v + q * R0);
        if (kx0 + b < ncol) {
          // the store addresses are recomputed here: kept live from the
          // loads, they would spill
          cpx<T>* ob;
          int64_t es;
          asm volatile("mov.b64 %0, %1;" : "=l"(ob) : "l"(base));
          asm volatile("mov.b64 %0, %1;" : "=l"(es) : "l"(elem_stride));
#pragma unroll
          for (int r = 0; r < R0; ++r) ob[(int64_t)(j + r * R1) * es + b] = v[q * R0 + r];
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < QA; ++q) {
        const int id = tid + q * NT;
        const int b = id % SB;
        if (kx0 + b < ncol) {
#pragma unroll
          for (int r = 0; r < R0; ++r) base[(int64_t)r * elem_stride + b] = v[q * R0 + r];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// z pass with TMA-staged tiles (FP32, two-stage sizes): a persistent CTA
// walks tiles (outer = ky line, SB columns); each tile -- N rows of SB
// complex values, one 8*SB-byte segment per row -- arrives in shared memory
// by cp.async.bulk.tensor (N/ZBOX boxes of SB x 1 x ZBOX elements of a 3D
// tensor map over H: x = kx, y, z), completion counted by an mbarrier.  The
// arithmetic is the z pass's (forward stage A from the staged tile, forward
// stage B, K multiply, inverse stages), so the results equal it bit for bit.
// The next tile's copy is issued once the current tile's shared-memory reads
// are done, overlapping its global stores and the other CTA's work.  Every
// mbarrier wait is bounded: a wait that runs out latches
// AMBER_ERR_DEVICE_TIMEOUT, waits once more (bounded) for the copy in flight
// and ends the kernel.
// ---------------------------------------------------------------------------
constexpr int kZBox = 256;  // rows per TMA box (a box dimension is at most 256)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// true when the phase with this parity has completed; up to `limit` tries
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// bytes of k_fft_zconv_tma's dynamic shared memory before its mbarrier, and in all
template <int N, int V>
constexpr size_t zpass_tma_mbar_offset() {
  return ((size_t)StridedSmem<float, N, V>::elems * 8 + (size_t)(N / 2 + 1) * FftCfg<N, V>::SB * 4 + 7) & ~(size_t)7;
}
template <int N, int V>
constexpr size_t zpass_tma_smem() { return zpass_tma_mbar_offset<N, V>() + 8; }

template <int N, int V>
__device__ __forceinline__ void zpass_tma_issue(const CUtensorMap* tmap, uint32_t dst, uint32_t mbar, int kx0,
                                                int y) {
  constexpr int SB = FftCfg<N, V>::SB;
  constexpr int ZB = N < kZBox ? N : kZBox;
  constexpr uint32_t bytes = (uint32_t)N * SB * 8u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
#pragma unroll
  for (int k = 0; k < N / ZB; ++k) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst + (uint32_t)(k * ZB * SB * 8)), "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(kx0), "r"(y),
          "r"(k * ZB), "r"(mbar)
        : "memory");
  }
}

template <int N, int V = 0>
__global__ void __launch_bounds__(strided_threads<N, V>(), 2)
k_fft_zconv_tma(const __grid_constant__ CUtensorMap tmap, cpx<float>* __restrict__ H, int ncol, int ntx, int ntiles,
                const cpx<float>* __restrict__ tw, float kf, float l_mfp, float norm,
                unsigned int* __restrict__ status) {
  using T = float;
  using C = FftCfg<N, V>;
  using L = StridedSmem<T, N, V>;
  constexpr int R0 = C::R0, R1 = C::R1, E = C::E, SB = C::SB, NT = strided_threads<N, V>();
  constexpr int QA = E / R0, QB = E / R1;
  static_assert(R1 > 1, "two-stage sizes only");
  const int64_t elem_stride = (int64_t)N * (N / 2 + 2), outer_stride = N / 2 + 2;
  // dynamic shared memory only (its base is 1024-byte aligned): the staged
  // tile / exchange area, the K table, the mbarrier
  extern __shared__ __align__(1024) unsigned char smem_tma[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_tma);
  T* Kt = reinterpret_cast<T*>(sm + L::elems);  // K over |kz| = 0..N/2 for the tile's columns
  const uint32_t buf = smem_u32(sm), mbar = buf + (uint32_t)zpass_tma_mbar_offset<N, V>();
  const int tid = threadIdx.x;
  constexpr unsigned kLimit = 1u << 22;

  int tile = blockIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tile < ntiles) zpass_tma_issue<N, V>(&tmap, buf, mbar, (tile % ntx) * SB, tile / ntx);
  }
  __syncthreads();
  uint32_t parity = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    {
      // K(|k|)/n^3 for this tile while its rows are in flight
      const int outer = tile / ntx;
      tile_kernel<T, N, SB, NT>(Kt, (tile - outer * ntx) * SB, signed_freq(outer, N), tid, kf, l_mfp, norm);
    }
    const bool ok = mbar_wait_bounded(mbar, parity, kLimit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        raise_status(status, AMBER_ERR_DEVICE_TIMEOUT);
        mbar_wait_bounded(mbar, parity, kLimit);  // let the copy in flight land before leaving
      }
      return;
    }
    parity ^= 1u;
    cpx<T> v[E];
    // ---- forward stage A from the staged tile (row n, column b at n SB + b)
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R0; ++r) v[q * R0 + r] = sm[(j + r * (N / R0)) * SB + b];
    }
#pragma unroll
    for (int q = 0; q < QA; ++q) dft<R0, false>(v + q * R0);
    __syncthreads();  // the staged tile is read: its space becomes the exchange area
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R0; ++r) sm[L::pos(j * R0 + r, b)] = v[q * R0 + r];
    }
    __syncthreads();
    // ---- forward stage B, the kernel multiply, inverse stage A (registers)
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        cpx<T> x = sm[L::pos(j + r * R0, b)];
        if (r > 0) x = cmul(x, tw[j * r]);
        v[q * R1 + r] = x;
      }
      dft<R1, false>(v + q * R1);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int n = j + r * R0;
        const int kza = n <= N / 2 ? n : N - n;
        v[q * R1 + r] = scale(v[q * R1 + r], Kt[kza * SB + b]);
      }
      dft<R1, true>(v + q * R1);
    }
    __syncthreads();  // all forward stage-B reads of the exchange area are done
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R1; ++r) sm[L::pos(j * R1 + r, b)] = v[q * R1 + r];
    }
    __syncthreads();
    // ---- inverse stage B: radix R0 over n = j + r R1, twiddle conj(w_N^(j r))
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
#pragma unroll
      for (int r = 0; r < R0; ++r) {
        cpx<T> x = sm[L::pos(j + r * R1, b)];
        if (r > 0) x = cmulc(x, tw[j * r]);
        v[q * R0 + r] = x;
      }
      dft<R0, true>(v + q * R0);
    }
    __syncthreads();  // the exchange area is read: the next tile may land in it
    if (tid == 0 && tile + (int)gridDim.x < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int nt = tile + (int)gridDim.x;
      zpass_tma_issue<N, V>(&tmap, buf, mbar, (nt % ntx) * SB, nt / ntx);
    }
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int b = id % SB, j = id / SB;
      // the store base is recomputed here from the tile index: kept live
      // across the stages it would spill
      int t;
      asm volatile("mov.b32 %0, %1;" : "=r"(t) : "r"(tile));
      const int o = t / ntx, c0 = (t - o * ntx) * SB;
      if (c0 + b < ncol) {
        cpx<T>* ob = H + (int64_t)o * outer_stride + c0 + b;
#pragma unroll
        for (int r = 0; r < R0; ++r) ob[(int64_t)(j + r * R1) * elem_stride] = v[q * R0 + r];
      }
    }
  }
}

// Host: the 3D tensor map of the half spectrum H (x = kx over n/2 + 2
// columns of which the first n/2 + 1 are read, y, z; 8-byte elements) with boxes of SB x 1 x min(n, 256), for
// k_fft_zconv_tma.  False when the driver's encoder is unavailable or refuses.
bool zpass_tensor_map(CUtensorMap* map, const void* H, int n, int SB);

// ---------------------------------------------------------------------------
// x-pass R2C: rows 2p and 2p+1 form z = a + i b; after the complex FFT
// A_k = (Z_k + conj Z_{N-k})/2 and B_k = (Z_k - conj Z_{N-k})/(2i), k <= N/2.
// ---------------------------------------------------------------------------
// MULTI: several transforms of size N back to back in H; the rows of item i
// (rows [i rpi, (i+1) rpi), rpi = N^2) come from srcs[i].  A CTA's rows never
// straddle two items (rpi is a multiple of 2 XP).
template <typename T, int N, int V = 0, bool MULTI = false>
// FP32: three CTAs per SM (measured faster for the forward x pass only)
__global__ void __launch_bounds__(xpass_threads<N, V>(), sizeof(T) == 4 ? 3 : 1)
k_fft_r2c_x(const T* __restrict__ src, cpx<T>* __restrict__ H, int64_t nrows, int RS,
            const cpx<T>* __restrict__ tw, const T* const* __restrict__ srcs = nullptr, int64_t rpi = 0) {
  using C = FftCfg<N, V>;
  using L = XSmem<T, N, V>;
  constexpr int R0 = C::R0, R1 = C::R1, E = C::E, XP = C::XP, NT = xpass_threads<N, V>();
  constexpr int QA = E / R0, QB = (R1 > 1) ? E / R1 : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * 2 * XP;
  // first element of row ra of the launch
  auto row_ptr = [&](int64_t ra) -> const T* {
    if constexpr (MULTI) {
      const int64_t it = ra / rpi;
      return srcs[it] + (ra - it * rpi) * N;
    } else {
      return src + ra * N;
    }
  };
  if (tid == 0) {
    // the rows of the CTA one SM count ahead into L2 (a third of the resident
    // wave: measured faster than a whole wave ahead, 1.63 vs 1.95 ms at 1024^3)
    const int64_t r2 = ((int64_t)blockIdx.x + sm_count()) * 2 * XP;
    if (r2 < nrows) prefetch_l2_bulk(row_ptr(r2), (uint32_t)(min((int64_t)2 * XP, nrows - r2) * N * sizeof(T)));
  }
  const T* rbase = row_ptr(row0);  // this CTA's rows, all of one item

  cpx<T> v[E];
#pragma unroll
  for (int q = 0; q < QA; ++q) {
    const int id = tid + q * NT;
    const int j = id % (N / R0), p = id / (N / R0);
    const int64_t ra = row0 + 2 * p;
    const bool ok = ra + 1 < nrows;
    const T* a = rbase + (int64_t)(2 * p) * N;
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int n = j + r * (N / R0);
      v[q * R0 + r] = ok ? mk<T>(a[n], a[N + n]) : mk<T>(0, 0);
    }
    dft<R0, false>(v + q * R0);
    if constexpr (R1 == 1) {
#pragma unroll
      for (int r = 0; r < R0; ++r) sm[L::pos(p, r)] = v[q * R0 + r];
    } else {
#pragma unroll
      for (int r = 0; r < R0; ++r) sm[L::pos(p, j * R0 + r)] = v[q * R0 + r];
    }
  }
  __syncthreads();
  if constexpr (R1 > 1) {
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int id = tid + q * NT;
      const int j = id % R0, p = id / R0;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        cpx<T> x = sm[L::pos(p, j + r * R0)];
        if (r > 0) x = cmul(x, tw[j * r]);
        v[q * R1 + r] = x;
      }
      dft<R1, false>(v + q * R1);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int id = tid + q * NT;
      const int j = id % R0, p = id / R0;
#pragma unroll
      for (int r = 0; r < R1; ++r) sm[L::pos(p, j + r * R0)] = v[q * R1 + r];
    }
    __syncthreads();
  }
  // split the two real transforms, write k in [0, N/2]
  constexpr int NK = N / 2 + 1;
  for (int idx = tid; idx < XP * NK; idx += NT) {
    const int p = idx / NK, k = idx - p * NK;
    const int64_t ra = row0 + 2 * p;
    if (ra + 1 >= nrows) continue;
    const cpx<T> zk = sm[L::pos(p, k)];
    const cpx<T> zn = sm[L::pos(p, (N - k) & (N - 1))];
    const T h = (T)0.5;
    const cpx<T> A = mk<T>(h * (zk.x + zn.x), h * (zk.y - zn.y));
    const cpx<T> B = mk<T>(h * (zk.y + zn.y), h * (zn.x - zk.x));
    H[ra * RS + k] = A;
    H[(ra + 1) * RS + k] = B;
  }
}

// ---------------------------------------------------------------------------
// x-pass C2R: Z_k = A_k + i B_k (k <= N/2), Z_{N-k} = conj A_k + i conj B_k;
// DC and Nyquist use the real parts only.  Re z -> row 2p, Im z -> row 2p+1.
// The 1/n^3 normalisation was applied with the kernel in the z-pass.
// ---------------------------------------------------------------------------
// MULTI: several transforms of size N back to back; the key range of item
// row0 / rpi folds into krange[item] (one control block per item).
// HIST (FP32): the intensities' raw 32-bit sort keys are also counted into
// krange's histogram, four 8-bit digit positions, so a sort of raw keys with
// 8-bit digits needs no histogram pass of its own.
template <typename T, int N, int V = 0, bool MULTI = false, bool HIST = false>
__global__ void __launch_bounds__(xpass_threads<N, V>())
k_fft_c2r_x(const cpx<T>* __restrict__ H, T* __restrict__ J, int64_t nrows, int RS,
            const cpx<T>* __restrict__ tw, unsigned int* __restrict__ status, SortCtrl* __restrict__ krange,
            int64_t rpi = 0) {
  using C = FftCfg<N, V>;
  using L = XSmem<T, N, V>;
  using K = typename KeyOf<T>::K;
  constexpr int R0 = C::R0, R1 = C::R1, E = C::E, XP = C::XP, NT = xpass_threads<N, V>();
  constexpr int QA = E / R0, QB = (R1 > 1) ? E / R1 : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * 2 * XP;
  if (tid == 0) {
    // the rows of the CTA one resident wave ahead (two per SM) into L2
    const int64_t r2 = ((int64_t)blockIdx.x + 2 * sm_count()) * 2 * XP;
    if (r2 < nrows) prefetch_l2_bulk(H + r2 * RS, (uint32_t)(min((int64_t)2 * XP, nrows - r2) * RS * sizeof(cpx<T>)));
  }

  // columns k < N/2 of both rows of each pair: E/2 per thread, all loads
  // issued before any shared-memory store
  constexpr int LPT = (XP * (N / 2)) / NT;
  static_assert(LPT * NT == XP * (N / 2), "x-pass tile must split evenly");
  cpx<T> A[LPT], Bv[LPT];
#pragma unroll
  for (int u = 0; u < LPT; ++u) {
    const int idx = tid + u * NT;
    const int p = idx / (N / 2), k = idx - p * (N / 2);
    const int64_t ra = row0 + 2 * p;
    const bool ok = ra + 1 < nrows;
    A[u] = ok ? H[ra * RS + k] : mk<T>(0, 0);
    Bv[u] = ok ? H[(ra + 1) * RS + k] : mk<T>(0, 0);
  }
#pragma unroll
  for (int u = 0; u < LPT; ++u) {
    const int idx = tid + u * NT;
    const int p = idx / (N / 2), k = idx - p * (N / 2);
    if (k == 0) {
      sm[L::pos(p, 0)] = mk<T>(A[u].x, Bv[u].x);
    } else {
      sm[L::pos(p, k)] = mk<T>(A[u].x - Bv[u].y, A[u].y + Bv[u].x);
      sm[L::pos(p, N - k)] = mk<T>(A[u].x + Bv[u].y, Bv[u].x - A[u].y);
    }
  }
  if (tid < XP) {  // Nyquist column k = N/2 (real parts only)
    const int64_t ra = row0 + 2 * tid;
    T ax = 0, bx = 0;
    if (ra + 1 < nrows) { ax = H[ra * RS + N / 2].x; bx = H[(ra + 1) * RS + N / 2].x; }
    sm[L::pos(tid, N / 2)] = mk<T>(ax, bx);
  }
  __syncthreads();

  cpx<T> v[E];
#pragma unroll
  for (int q = 0; q < QA; ++q) {
    const int id = tid + q * NT;
    const int j = id % (N / R0), p = id / (N / R0);
#pragma unroll
    for (int r = 0; r < R0; ++r) v[q * R0 + r] = sm[L::pos(p, j + r * (N / R0))];
    dft<R0, true>(v + q * R0);
  }
  bool bad = false, nan = false;
  K klo = ~K(0), khi = 0;
  static_assert(!HIST || sizeof(K) == 4, "digit counts of 32-bit keys");
  __shared__ uint32_t shist[HIST ? 4 * 256 : 1];
  if constexpr (HIST) {
    for (int i = tid; i < 4 * 256; i += NT) shist[i] = 0;
    __syncthreads();
  }
  auto track = [&](T x) {
    bad |= !isfinite(x);
    const K kk = enc_desc(x, nan);
    klo = kk < klo ? kk : klo;
    khi = kk > khi ? kk : khi;
    if constexpr (HIST) {
      // the two low digits: one add per key
      atomicAdd(&shist[kk & 255u], 1u);
      atomicAdd(&shist[256 + ((kk >> 8) & 255u)], 1u);
      // neighbouring cells of a smooth field often share the upper digits:
      // one add for the active lanes when they all agree
      const unsigned am = __activemask();
      const int leader = __ffs(am) - 1;
#pragma unroll
      for (int p = 2; p < 4; ++p) {
        const unsigned d = (unsigned)(kk >> (8 * p)) & 255u;
        const unsigned d0 = __shfl_sync(am, d, leader);
        if (__all_sync(am, d == d0)) {
          if ((int)(threadIdx.x & 31) == leader) atomicAdd(&shist[p * 256 + d0], (uint32_t)__popc(am));
        } else {
          atomicAdd(&shist[p * 256 + d], 1u);
        }
      }
    }
  };
  if constexpr (R1 == 1) {
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int p = id / (N / R0);
      const int64_t ra = row0 + 2 * p;
      if (ra + 1 < nrows) {
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          J[ra * N + r] = v[q * R0 + r].x;
          J[(ra + 1) * N + r] = v[q * R0 + r].y;
          track(v[q * R0 + r].x);
          track(v[q * R0 + r].y);
        }
      }
    }
  } else {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < QA; ++q) {
      const int id = tid + q * NT;
      const int j = id % (N / R0), p = id / (N / R0);
#pragma unroll
      for (int r = 0; r < R0; ++r) sm[L::pos(p, j * R0 + r)] = v[q * R0 + r];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      const int id = tid + q * NT;
      const int j = id % R0, p = id / R0;
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        cpx<T> x = sm[L::pos(p, j + r * R0)];
        if (r > 0) x = cmulc(x, tw[j * r]);
        v[q * R1 + r] = x;
      }
      dft<R1, true>(v + q * R1);
      const int64_t ra = row0 + 2 * p;
      if (ra + 1 < nrows) {
#pragma unroll
        for (int r = 0; r < R1; ++r) {
          const int n = j + r * R0;
          J[ra * N + n] = v[q * R1 + r].x;
          J[(ra + 1) * N + n] = v[q * R1 + r].y;
          track(v[q * R1 + r].x);
          track(v[q * R1 + r].y);
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(status, AMBER_ERR_NONFINITE);
  // fold the intensities' key range into the sort's control block
  if constexpr (MULTI) key_range_commit(klo, khi, krange + row0 / rpi);
  else if (krange) key_range_commit(klo, khi, krange);
  if constexpr (HIST) {
    __syncthreads();
    for (int i = tid; i < 4 * 256; i += NT) {
      const uint32_t c = shist[i];
      if (c) atomicAdd(&krange->hist[i], c);
    }
  }
}

// ---------------------------------------------------------------------------
// Host launcher for one radiation field of size N.
// ---------------------------------------------------------------------------
struct FftProfile;  // opaque; see host runtime
void prof_begin(FftProfile* p, int kind, cudaStream_t s);
void prof_end(FftProfile* p, int kind, cudaStream_t s);

enum ProfKind {
  PK_R2C_X = 0, PK_FFT_Y_FWD, PK_FFT_Z_CONV, PK_FFT_Y_INV, PK_C2R_X,
  PK_SORT_HIST, PK_SORT_PASS, PK_MASS_REDUCE, PK_THRESHOLDS, PK_SCAN_ASSIGN, PK_SCATTER_BACK, PK_COUNT
};

// spec_in (optional): the x- and y-transformed source kept by the caller
// (source_spectrum_n's output); the first two passes are skipped and the z
// pass reads it, leaving it unchanged.
// hist8 (FP32, krange given): the inverse x pass also counts the raw keys'
// four 8-bit digits into krange's histogram.
template <typename T, int N, int V = 0>
cudaError_t radiation_field_n(const T* src, T* J, cpx<T>* H, const cpx<T>* tw, double box, double l_mfp,
                              unsigned int* status, cudaStream_t s, FftProfile* prof, SortCtrl* krange,
                              const cpx<T>* spec_in = nullptr, bool hist8 = false, bool tma = false) {
  using C = FftCfg<N, V>;
  const int RS = N / 2 + 2;
  const int ncol = N / 2 + 1;
  const int64_t nrows = (int64_t)N * N;
  const T kf = (T)(2.0 * 3.14159265358979323846 / box);
  const T norm = (T)(1.0 / ((double)N * N * N));
  const size_t xs = XSmem<T, N, V>::elems * sizeof(cpx<T>);
  const size_t ss = StridedSmem<T, N, V>::elems * sizeof(cpx<T>);
  // the z pass adds its table of K over |kz| = 0..N/2 for the tile's columns
  const size_t sc = ss + (size_t)(N / 2 + 1) * C::SB * sizeof(T);
  static std::atomic<unsigned long long> attr_done{0};  // per instantiation and device
  if (first_use_on_device(attr_done)) {
    cudaFuncSetAttribute(k_fft_r2c_x<T, N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_c2r_x<T, N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_FWD, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_INV, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_CONV, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_CONV, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sc);
    if constexpr (sizeof(T) == 4)
      cudaFuncSetAttribute(k_fft_c2r_x<T, N, V, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
  }
  const int xgrid = (int)((nrows / 2 + C::XP - 1) / C::XP);
  const int ntx = (ncol + C::SB - 1) / C::SB;
  const int sgrid = N * ntx;

  if (!spec_in) {
    prof_begin(prof, PK_R2C_X, s);
    k_fft_r2c_x<T, N, V><<<xgrid, xpass_threads<N, V>(), xs, s>>>(src, H, nrows, RS, tw);
    prof_end(prof, PK_R2C_X, s);
    // y-pass: lines (z, kx); element stride RS; outer (z) stride N*RS
    prof_begin(prof, PK_FFT_Y_FWD, s);
    k_fft_strided<T, N, PASS_FWD, V><<<sgrid, strided_threads<N, V>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx,
                                                                             tw, kf, (T)l_mfp, norm);
    prof_end(prof, PK_FFT_Y_FWD, s);
  }
  // z-pass: lines (y, kx); element stride N*RS; outer (y) stride RS
  prof_begin(prof, PK_FFT_Z_CONV, s);
  bool z_done = false;
  if constexpr (sizeof(T) == 4 && C::R1 > 1) {
    CUtensorMap map;
    if (tma && zpass_tensor_map(&map, spec_in ? (const void*)spec_in : (const void*)H, N, C::SB)) {
      static std::atomic<unsigned long long> tma_attr{0};
      if (first_use_on_device(tma_attr))
        cudaFuncSetAttribute(k_fft_zconv_tma<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)zpass_tma_smem<N, V>());
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int grid = sgrid < 2 * sms ? sgrid : 2 * sms;
      k_fft_zconv_tma<N, V><<<grid, strided_threads<N, V>(), zpass_tma_smem<N, V>(), s>>>(
          map, H, ncol, ntx, sgrid, tw, kf, (T)l_mfp, norm, status);
      z_done = true;
    }
  }
  if (z_done) {
  } else if (spec_in)
    k_fft_strided<T, N, PASS_CONV, V, true><<<sgrid, strided_threads<N, V>(), sc, s>>>(
        H, (int64_t)N * RS, RS, ncol, ntx, tw, kf, (T)l_mfp, norm, spec_in);
  else
    k_fft_strided<T, N, PASS_CONV, V><<<sgrid, strided_threads<N, V>(), sc, s>>>(
        H, (int64_t)N * RS, RS, ncol, ntx, tw, kf, (T)l_mfp, norm);
  prof_end(prof, PK_FFT_Z_CONV, s);
  prof_begin(prof, PK_FFT_Y_INV, s);
  k_fft_strided<T, N, PASS_INV, V><<<sgrid, strided_threads<N, V>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx, tw,
                                                                       kf, (T)l_mfp, norm);
  prof_end(prof, PK_FFT_Y_INV, s);
  prof_begin(prof, PK_C2R_X, s);
  if constexpr (sizeof(T) == 4) {
    if (hist8 && krange)
      k_fft_c2r_x<T, N, V, false, true><<<xgrid, xpass_threads<N, V>(), xs, s>>>(H, J, nrows, RS, tw, status, krange);
    else
      k_fft_c2r_x<T, N, V><<<xgrid, xpass_threads<N, V>(), xs, s>>>(H, J, nrows, RS, tw, status, krange);
  } else {
    k_fft_c2r_x<T, N, V><<<xgrid, xpass_threads<N, V>(), xs, s>>>(H, J, nrows, RS, tw, status, krange);
  }
  prof_end(prof, PK_C2R_X, s);
  return cudaGetLastError();
}

// Radiation fields of M same-size items in one launch per pass.  The items'
// half spectra lie back to back in H (M n^2 (n/2 + 2) elements) and their
// intensities back to back in J (M n^3); srcs (device array of M pointers)
// holds the sources, kp (device, 2 M values) each item's kf = 2 pi / box and
// l_mfp, kranges (device, M control blocks) the blocks the items' key ranges
// fold into.  Requires n^2 to be a multiple of the x-pass tile (n >= 8).
template <typename T, int N, int V = 0>
cudaError_t radiation_field_multi_n(const T* const* srcs, int M, T* J, cpx<T>* H, const cpx<T>* tw, const T* kp,
                                    unsigned int* status, cudaStream_t s, SortCtrl* kranges) {
  using C = FftCfg<N, V>;
  static_assert((N * N) % (2 * C::XP) == 0, "an x-pass tile must not straddle two items");
  const int RS = N / 2 + 2;
  const int ncol = N / 2 + 1;
  const int64_t rpi = (int64_t)N * N;
  const int64_t nrows = rpi * M;
  const int64_t item_stride = rpi * RS;
  const T norm = (T)(1.0 / ((double)N * N * N));
  const size_t xs = XSmem<T, N, V>::elems * sizeof(cpx<T>);
  const size_t ss = StridedSmem<T, N, V>::elems * sizeof(cpx<T>);
  const size_t sc = ss + (size_t)(N / 2 + 1) * C::SB * sizeof(T);
  static std::atomic<unsigned long long> attr_done{0};  // per instantiation and device
  if (first_use_on_device(attr_done)) {
    cudaFuncSetAttribute(k_fft_r2c_x<T, N, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_c2r_x<T, N, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_FWD, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_INV, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_CONV, V, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sc);
  }
  const int xgrid = (int)((nrows / 2 + C::XP - 1) / C::XP);
  const int ntx = (ncol + C::SB - 1) / C::SB;
  const int sgrid = M * N * ntx;
  const T zero = (T)0;
  k_fft_r2c_x<T, N, V, true><<<xgrid, xpass_threads<N, V>(), xs, s>>>(nullptr, H, nrows, RS, tw, srcs, rpi);
  // y passes: the z planes of all items are one run of M N planes
  k_fft_strided<T, N, PASS_FWD, V><<<sgrid, strided_threads<N, V>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx, tw,
                                                                           zero, zero, zero);
  k_fft_strided<T, N, PASS_CONV, V, false, true><<<sgrid, strided_threads<N, V>(), sc, s>>>(
      H, (int64_t)N * RS, RS, ncol, ntx, tw, zero, zero, norm, nullptr, item_stride, kp);
  k_fft_strided<T, N, PASS_INV, V><<<sgrid, strided_threads<N, V>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx, tw,
                                                                           zero, zero, zero);
  k_fft_c2r_x<T, N, V, true><<<xgrid, xpass_threads<N, V>(), xs, s>>>(H, J, nrows, RS, tw, status, kranges, rpi);
  return cudaGetLastError();
}

// Forward transform only: H = DFT(src) as the half spectrum [n][n][n/2+2]
// (x-pass R2C, then forward y and z passes, unnormalised), for the analysis
// of fields (power spectra).
template <typename T, int N>
cudaError_t forward_spectrum_n(const T* src, cpx<T>* H, const cpx<T>* tw, cudaStream_t s) {
  using C = FftCfg<N>;
  const int RS = N / 2 + 2;
  const int ncol = N / 2 + 1;
  const int64_t nrows = (int64_t)N * N;
  const size_t xs = XSmem<T, N>::elems * sizeof(cpx<T>);
  const size_t ss = StridedSmem<T, N>::elems * sizeof(cpx<T>);
  static std::atomic<unsigned long long> attr_done{0};  // per instantiation and device
  if (first_use_on_device(attr_done)) {
    cudaFuncSetAttribute(k_fft_r2c_x<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
  }
  const int xgrid = (int)((nrows / 2 + C::XP - 1) / C::XP);
  const int ntx = (ncol + C::SB - 1) / C::SB;
  const int sgrid = N * ntx;
  const T zero = (T)0;
  k_fft_r2c_x<T, N><<<xgrid, xpass_threads<N>(), xs, s>>>(src, H, nrows, RS, tw);
  k_fft_strided<T, N, PASS_FWD><<<sgrid, strided_threads<N>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx, tw,
                                                                       zero, zero, zero);
  k_fft_strided<T, N, PASS_FWD><<<sgrid, strided_threads<N>(), ss, s>>>(H, (int64_t)N * RS, RS, ncol, ntx, tw,
                                                                       zero, zero, zero);
  return cudaGetLastError();
}

// The first two passes of the radiation field: H = the x R2C and forward y
// transforms of src (z not yet transformed), the spectrum radiation_field_n
// takes as spec_in.  The tile variant must match the one that later consumes
// it for bit-identical results (any variant gives the same layout).
template <typename T, int N, int V = 0>
cudaError_t source_spectrum_n(const T* src, cpx<T>* H, const cpx<T>* tw, cudaStream_t s, FftProfile* prof) {
  using C = FftCfg<N, V>;
  const int RS = N / 2 + 2;
  const int ncol = N / 2 + 1;
  const int64_t nrows = (int64_t)N * N;
  const size_t xs = XSmem<T, N, V>::elems * sizeof(cpx<T>);
  const size_t ss = StridedSmem<T, N, V>::elems * sizeof(cpx<T>);
  static std::atomic<unsigned long long> attr_done{0};  // per instantiation and device
  if (first_use_on_device(attr_done)) {
    cudaFuncSetAttribute(k_fft_r2c_x<T, N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_FWD, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
  }
  const int xgrid = (int)((nrows / 2 + C::XP - 1) / C::XP);
  const int ntx = (ncol + C::SB - 1) / C::SB;
  const int sgrid = N * ntx;
  const T zero = (T)0;
  prof_begin(prof, PK_R2C_X, s);
  k_fft_r2c_x<T, N, V><<<xgrid, xpass_threads<N, V>(), xs, s>>>(src, H, nrows, RS, tw);
  prof_end(prof, PK_R2C_X, s);
  prof_begin(prof, PK_FFT_Y_FWD, s);
  k_fft_strided<T, N, PASS_FWD, V><<<sgrid, strided_threads<N, V>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx, tw,
                                                                           zero, zero, zero);
  prof_end(prof, PK_FFT_Y_FWD, s);
  return cudaGetLastError();
}

// Inverse transform only: out = unnormalised inverse DFT of the half spectrum
// H (z and y passes in place, then the C2R x-pass into out); the caller folds
// 1/n^3 into the spectrum.  A non-finite output latches AMBER_ERR_NONFINITE.
template <typename T, int N>
cudaError_t inverse_spectrum_n(cpx<T>* H, T* out, const cpx<T>* tw, unsigned int* status, cudaStream_t s) {
  using C = FftCfg<N>;
  const int RS = N / 2 + 2;
  const int ncol = N / 2 + 1;
  const int64_t nrows = (int64_t)N * N;
  const size_t xs = XSmem<T, N>::elems * sizeof(cpx<T>);
  const size_t ss = StridedSmem<T, N>::elems * sizeof(cpx<T>);
  static std::atomic<unsigned long long> attr_done{0};  // per instantiation and device
  if (first_use_on_device(attr_done)) {
    cudaFuncSetAttribute(k_fft_c2r_x<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs);
    cudaFuncSetAttribute(k_fft_strided<T, N, PASS_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
  }
  const int xgrid = (int)((nrows / 2 + C::XP - 1) / C::XP);
  const int ntx = (ncol + C::SB - 1) / C::SB;
  const int sgrid = N * ntx;
  const T zero = (T)0;
  k_fft_strided<T, N, PASS_INV><<<sgrid, strided_threads<N>(), ss, s>>>(H, (int64_t)N * RS, RS, ncol, ntx, tw,
                                                                       zero, zero, zero);
  k_fft_strided<T, N, PASS_INV><<<sgrid, strided_threads<N>(), ss, s>>>(H, RS, (int64_t)N * RS, ncol, ntx, tw,
                                                                       zero, zero, zero);
  k_fft_c2r_x<T, N><<<xgrid, xpass_threads<N>(), xs, s>>>(H, out, nrows, RS, tw, status, nullptr);
  return cudaGetLastError();
}

}  // namespace amber
