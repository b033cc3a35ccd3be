// Analysis of reionization-redshift fields (Sec. 2.3, Eqs. deltaz, epsz, Pk,
// Dk, bias, rcc).
//
//   k_sum_f64     : cell mean of z (FP64 accumulation)
//   k_delta_z     : delta_z = ((1 + z) - (1 + zbar)) / (1 + zbar)
//   k_eps_pdf     : histogram and moments of epsilon = (z - zref)/(1 + zref)
//   k_power_bins  : shell sums of |A|^2, |B|^2, Re(A B*) over the half
//                   spectrum; mode weights 2 for 0 < kx < n/2 (the conjugate
//                   mode is not stored), else 1
//   k_power_final : shell averages in the continuum normalisation
//
// Shell b holds the integer wave vectors m with round(|m|) = b, decided
// exactly in integers: b is the one integer with b^2 - b < |m|^2 <= b^2 + b.
#include <cmath>

#include "fft.cuh"
#include "spectra.cuh"

namespace amber {

int power_bins(int n) { return (int)std::llround(std::sqrt(3.0) * n / 2.0) + 1; }

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one double per thread into *out (one atomic per block).
__device__ __forceinline__ void block_add_f64(double v, double* out) {
  __shared__ double ws[32];
  v = warp_sum_f64(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    atomicAdd(out, s);
  }
}

__global__ void __launch_bounds__(256) k_sum_f64(const float* __restrict__ z, int64_t n, double* __restrict__ acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  const bool vec = (reinterpret_cast<uintptr_t>(z) & 15) == 0;
  const int64_t nv = vec ? n / 4 : 0;
  for (int64_t v = gtid; v < nv; v += stride) {
    const float4 q = reinterpret_cast<const float4*>(z)[v];
    s += ((double)q.x + (double)q.y) + ((double)q.z + (double)q.w);  // pairs of floats add exactly
  }
  for (int64_t i = nv * 4 + gtid; i < n; i += stride) s += (double)z[i];
  block_add_f64(s, acc);
}

__global__ void __launch_bounds__(256) k_delta_z(const float* __restrict__ z, int64_t n,
                                                 const double* __restrict__ acc, float* __restrict__ out,
                                                 double* __restrict__ zbar_out) {
  const double zbar = *acc / (double)n;
  const float zb = (float)zbar, inv = (float)(1.0 / (1.0 + zbar));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gtid == 0 && zbar_out) *zbar_out = zbar;
  for (int64_t i = gtid; i < n; i += stride) out[i] = (z[i] - zb) * inv;
}

__global__ void __launch_bounds__(256) k_eps_pdf(const float* __restrict__ z, const float* __restrict__ zref,
                                                 int64_t n, float lo, float hi, float scale, int nbins,
                                                 unsigned long long* __restrict__ counts,
                                                 double* __restrict__ moments) {
  extern __shared__ unsigned int hist[];  // nbins + 2
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = gtid; i < n; i += stride) {
    const float e = (z[i] - zref[i]) / (1.0f + zref[i]);
    int b;
    if (!(e >= lo)) b = 0;  // below (or NaN)
    else if (e >= hi) b = nbins + 1;
    else b = 1 + min((int)((e - lo) * scale), nbins - 1);
    atomicAdd(&hist[b], 1u);
    s1 += (double)e;
    s2 += (double)e * (double)e;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x)
    if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
  if (moments) {
    block_add_f64(s1, moments);
    __syncthreads();
    block_add_f64(s2, moments + 1);
  }
}

// One warp per row (kz, ky) of the half spectrum; lane l takes a contiguous
// run of kx, along which |m| and so the shell never decrease, and adds each
// shell's run into shared memory when the shell changes.
template <bool CROSS>
__global__ void __launch_bounds__(256) k_power_bins(const float2* __restrict__ Ha, const float2* __restrict__ Hb,
                                                    int n, int nb, double* __restrict__ acc) {
  extern __shared__ double sacc[];  // [kPowerAcc][nb]
  for (int i = threadIdx.x; i < kPowerAcc * nb; i += blockDim.x) sacc[i] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int RS = n / 2 + 2, ncol = n / 2 + 1;
  const int chunk = (ncol + 31) / 32;
  const int c0 = lane * chunk, c1 = min(c0 + chunk, ncol);
  const int64_t rows = (int64_t)n * n;
  for (int64_t row = (int64_t)blockIdx.x * nw + warp; row < rows; row += (int64_t)gridDim.x * nw) {
    const int zi = (int)(row / n), yi = (int)(row - (int64_t)zi * n);
    const int mz = zi < n / 2 ? zi : zi - n, my = yi < n / 2 ? yi : yi - n;
    const int r2 = my * my + mz * mz;
    const float2* pa = Ha + row * RS;
    const float2* pb = CROSS ? Hb + row * RS : nullptr;
    int cur = -1;
    float sw = 0.f, sk = 0.f, saa = 0.f, sbb = 0.f, sab = 0.f;
    auto flush = [&]() {
      if (cur >= 0) {
        atomicAdd(&sacc[cur], (double)sw);
        atomicAdd(&sacc[nb + cur], (double)sk);
        atomicAdd(&sacc[2 * nb + cur], (double)saa);
        if (CROSS) {
          atomicAdd(&sacc[3 * nb + cur], (double)sbb);
          atomicAdd(&sacc[4 * nb + cur], (double)sab);
        }
      }
    };
    for (int mx = c0; mx < c1; ++mx) {
      const int m2 = r2 + mx * mx;
      int b = (int)(sqrtf((float)m2) + 0.5f);
      while (b > 0 && b * b - b >= m2) --b;  // exact: b^2 - b < m2 <= b^2 + b
      while (b * b + b < m2) ++b;
      if (b != cur) {
        flush();
        cur = b;
        sw = sk = saa = sbb = sab = 0.f;
      }
      const float w = (mx == 0 || mx == n / 2) ? 1.f : 2.f;
      const float2 a = pa[mx];
      sw += w;
      sk += w * sqrtf((float)m2);
      saa += w * fmaf(a.x, a.x, a.y * a.y);
      if constexpr (CROSS) {
        const float2 q = pb[mx];
        sbb += w * fmaf(q.x, q.x, q.y * q.y);
        sab += w * fmaf(a.x, q.x, a.y * q.y);
      }
    }
    flush();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPowerAcc * nb; i += blockDim.x)
    if (sacc[i] != 0.0) atomicAdd(&acc[i], sacc[i]);
}

__global__ void k_power_final(const double* __restrict__ acc, int nb, double kf, double norm, bool cross,
                              double* __restrict__ k, double* __restrict__ Paa, double* __restrict__ Pbb,
                              double* __restrict__ Pab, double* __restrict__ modes) {
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double m = acc[b];
    const double inv = m > 0.0 ? 1.0 / m : 0.0;
    modes[b] = m;
    k[b] = kf * acc[nb + b] * inv;
    Paa[b] = norm * acc[2 * nb + b] * inv;
    if (Pbb) Pbb[b] = cross ? norm * acc[3 * nb + b] * inv : 0.0;
    if (Pab) Pab[b] = cross ? norm * acc[4 * nb + b] * inv : 0.0;
  }
}

// Derived shell statistics (Eqs. Dk, bias, rcc), FP64 per shell:
// Delta^2 = k^3 P / (2 pi^2), b = sqrt(P_aa / P_bb), r = P_ab / sqrt(P_aa P_bb).
// A shell without modes has P = 0 and gets Delta^2 = 0 and NaN ratios (0/0).
__global__ void k_power_derived(const double* __restrict__ k, const double* __restrict__ Paa,
                                const double* __restrict__ Pbb, const double* __restrict__ Pab, int nb,
                                double* __restrict__ D2aa, double* __restrict__ D2bb, double* __restrict__ bias,
                                double* __restrict__ r) {
  const double inv2pi2 = 1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const double kb = k[b], k3 = kb * kb * kb, a = Paa[b];
    D2aa[b] = k3 * a * inv2pi2;
    if (Pbb) {
      const double q = Pbb[b];
      if (D2bb) D2bb[b] = k3 * q * inv2pi2;
      if (bias) bias[b] = sqrt(a / q);
      if (r && Pab) r[b] = Pab[b] / sqrt(a * q);
    }
  }
}

cudaError_t power_derived_impl(const double* k, const double* Paa, const double* Pbb, const double* Pab, int nb,
                               double* D2aa, double* D2bb, double* bias, double* r, cudaStream_t s) {
  k_power_derived<<<(nb + 255) / 256, 256, 0, s>>>(k, Paa, Pbb, Pab, nb, D2aa, D2bb, bias, r);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int num_sms) {
  int64_t g = (n + 1023) / 1024;
  g = std::min<int64_t>(g, (int64_t)num_sms * 8);
  return (int)std::max<int64_t>(g, 1);
}

cudaError_t sum_f64_impl(const float* x, int64_t n, double* acc, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  k_sum_f64<<<grid_for(n, num_sms), 256, 0, s>>>(x, n, acc);
  return cudaGetLastError();
}

cudaError_t delta_z_impl(const float* z, int64_t n, float* out, double* acc, double* zbar_out, int num_sms,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  const int g = grid_for(n, num_sms);
  k_sum_f64<<<g, 256, 0, s>>>(z, n, acc);
  k_delta_z<<<g, 256, 0, s>>>(z, n, acc, out, zbar_out);
  return cudaGetLastError();
}

cudaError_t epsilon_pdf_impl(const float* z, const float* zref, int64_t n, double lo, double hi, int nbins,
                             unsigned long long* counts, double* moments, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)(nbins + 2) * sizeof(unsigned long long), s);
  if (e == cudaSuccess && moments) e = cudaMemsetAsync(moments, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)(nbins + 2) * sizeof(unsigned int);
  static std::atomic<unsigned long long> attr{0};
  if (first_use_on_device(attr))
    cudaFuncSetAttribute(k_eps_pdf, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  k_eps_pdf<<<grid_for(n, num_sms), 256, smem, s>>>(z, zref, n, (float)lo, (float)hi, (float)(nbins / (hi - lo)),
                                                    nbins, counts, moments);
  return cudaGetLastError();
}

cudaError_t power_impl(const void* Ha, const void* Hb, int n, double box, double* acc, double* k, double* Paa,
                       double* Pbb, double* Pab, double* modes, int num_sms, cudaStream_t s) {
  const int nb = power_bins(n);
  if (nb > kMaxPowerBins) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)kPowerAcc * nb * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)kPowerAcc * nb * sizeof(double);
  static std::atomic<unsigned long long> attr{0};
  if (first_use_on_device(attr)) {
    cudaFuncSetAttribute(k_power_bins<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kPowerAcc * kMaxPowerBins * 8));
    cudaFuncSetAttribute(k_power_bins<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kPowerAcc * kMaxPowerBins * 8));
  }
  const int64_t rows = (int64_t)n * n;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, (int64_t)num_sms * 4));
  const auto* a = reinterpret_cast<const float2*>(Ha);
  const auto* b = reinterpret_cast<const float2*>(Hb);
  if (Hb) k_power_bins<true><<<g, 256, smem, s>>>(a, b, n, nb, acc);
  else k_power_bins<false><<<g, 256, smem, s>>>(a, nullptr, n, nb, acc);
  const double kf = 2.0 * 3.14159265358979323846 / box;
  const double norm = box * box * box / ((double)n * n * n * (double)n * n * n);
  k_power_final<<<1, 1024, 0, s>>>(acc, nb, kf, norm, Hb != nullptr, k, Paa, Pbb, Pab, modes);
  return cudaGetLastError();
}

}  // namespace amber
