// Source field for the serving path (step a0): the excursion-set collapsed
// fraction analogue of Sec. 3.3 (Eq. fcoll with the ESF-E halo density,
// rho_h = f_coll rho (1 + delta)), applied to a density field:
//
//   mass = 1 + max(delta, -0.99)
//   S    = mass * erfc((delta_c - delta) / (sqrt(2) sigma_f)),  S /= mean(S)
//
// sigma_f stands in for sqrt(sigma^2(M_min) - sigma^2(M_s)).  The mean is an
// exact 128-bit fixed-point sum, so the normalisation does not depend on the
// order of summation.  The source normalisation does not change z_re
// (abundance matching is normalisation-free, Sec. 3.4.1); it is kept so S
// matches the recipe.
#include "fixed128.cuh"
#include "source.cuh"

namespace amber {

__global__ void __launch_bounds__(256) k_source_raw(const float* __restrict__ delta, int64_t n, float delta_c,
                                                    float inv_s2, float* __restrict__ S, float* __restrict__ mass,
                                                    unsigned long long* __restrict__ total,
                                                    unsigned int* __restrict__ status) {
  u128 acc = 0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float d = delta[i];
    // 1 + max(d, -0.99) rounded once to float: 1 + d is exact before the
    // rounding, and below the floor the value is 0.01 itself
    const float m = fmaxf(1.0f + d, 0.01f);
    const float s = m * erfcf((delta_c - d) * inv_s2);
    S[i] = s;
    if (mass) mass[i] = m;
    acc += mass_q64(s, bad);
    bad |= isnan(d);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc += shfl_down_u128(acc, o);
  __shared__ u128 ws[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    u128 t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    if (t != 0) atomic_add_u128(total, t);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, AMBER_ERR_NONFINITE);
}

__global__ void __launch_bounds__(256) k_source_scale(float* __restrict__ S, int64_t n,
                                                      const unsigned long long* __restrict__ total) {
  const u128 T = ((u128)total[1] << 64) | (u128)total[0];  // 2^-64 units
  const float f = (float)((double)n / (u128_to_double(T) * 5.42101086242752217e-20));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) S[i] *= f;
}

cudaError_t source_field_impl(const float* delta, int64_t n, double delta_c, double sigma_f, float* S, float* mass,
                              unsigned long long* total, int num_sms, unsigned int* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(total, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
  if (grid < 1) grid = 1;
  k_source_raw<<<grid, 256, 0, s>>>(delta, n, (float)delta_c, (float)(1.0 / (1.4142135623730951 * sigma_f)), S,
                                     mass, total, status);
  k_source_scale<<<grid, 256, 0, s>>>(S, n, total);
  return cudaGetLastError();
}

}  // namespace amber
