// Source-field pipeline on the GPU (Sec. 3.2, Eq. xlpt; Sec. 3.2.1, Eqs.
// interlace and Wofk; Sec. 3.3, Eq. fcoll).
//
//   k_spec_op     : one operator on the half spectrum: Hessian k_a k_b / k^2,
//                   gradient of the inverse Laplacian -i k_a / k^2 (of a
//                   linear combination of two spectra), sharp-k or top-hat
//                   filter; with the inverse transform's 1/n^3
//   k_s2_diag/sub : the second-order source sum_{i<j} phi,ii phi,jj - phi,ij^2
//   k_assign<P>   : NGP / CIC / TSC assignment of one particle per lattice
//                   point (FP32 atomics on the mesh)
//   k_interlace   : [A + e^{i k.dX} B] / 2 / W(k)^p, Nyquist modes zeroed
//   k_scale, k_fcoll : elementwise
//
// An odd derivative along an axis whose wave number is the Nyquist one has
// no real counterpart and is set to 0 (for the mixed Hessian terms too).
#include <cmath>

#include "fft.cuh"
#include "lpt.cuh"

namespace amber {

enum SpecOp { OP_HESS = 0, OP_GRADINV = 1, OP_SHARPK = 2, OP_TOPHAT = 3 };

struct SpecOpArgs {
  const float2* A;
  const float2* B;  // optional second spectrum (OP_GRADINV)
  float2* out;      // may alias A
  int n;
  int op, a, b;     // axes 0 = x, 1 = y, 2 = z
  float c1, c2;     // out = op (c1 A + c2 B) scale
  float kf;         // 2 pi / box
  float R;          // filter radius (box units)
  double m2max;     // sharp-k: keep m^2 <= m2max, i.e. k R <= 1
  float scale;
};

__device__ __forceinline__ float tophat_w(float x) {
  if (x < 0.5f) {  // series: the closed form cancels for small x
    const float x2 = x * x;
    return 1.0f - x2 * (0.1f - x2 * (1.0f / 280.0f - x2 * (1.0f / 15120.0f)));
  }
  float sn, cs;
  sincosf(x, &sn, &cs);
  return 3.0f * (sn - x * cs) / (x * x * x);
}

__global__ void __launch_bounds__(256) k_spec_op(const SpecOpArgs p) {
  const int n = p.n, ncol = n / 2 + 1, RS = n / 2 + 2;
  const int64_t total = (int64_t)n * n * ncol;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % ncol);
    const int64_t row = e / ncol;
    const int y = (int)(row % n), z = (int)(row / n);
    const int m[3] = {x, y < n / 2 ? y : y - n, z < n / 2 ? z : z - n};
    const bool nyq[3] = {x == n / 2, y == n / 2, z == n / 2};
    const int64_t at = row * RS + x;
    float2 v = p.A[at];
    v.x *= p.c1;
    v.y *= p.c1;
    if (p.B) {
      const float2 w = p.B[at];
      v.x = fmaf(p.c2, w.x, v.x);
      v.y = fmaf(p.c2, w.y, v.y);
    }
    const int m2i = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
    float2 r = make_float2(0.f, 0.f);
    if (p.op == OP_HESS) {
      const bool zero = m2i == 0 || (p.a != p.b && (nyq[p.a] || nyq[p.b]));
      const float f = zero ? 0.f : (float)(m[p.a] * m[p.b]) / (float)m2i;  // k_a k_b / k^2
      r = make_float2(v.x * f, v.y * f);
    } else if (p.op == OP_GRADINV) {
      // -i k_a / k^2 times v
      const float c = (m2i == 0 || nyq[p.a]) ? 0.f : (float)m[p.a] / ((float)m2i * p.kf);
      r = make_float2(c * v.y, -c * v.x);
    } else if (p.op == OP_SHARPK) {
      const float f = (double)m2i <= p.m2max ? 1.f : 0.f;
      r = make_float2(v.x * f, v.y * f);
    } else {
      const float f = tophat_w(p.kf * sqrtf((float)m2i) * p.R);
      r = make_float2(v.x * f, v.y * f);
    }
    p.out[at] = make_float2(r.x * p.scale, r.y * p.scale);
  }
}

__global__ void __launch_bounds__(256) k_s2_diag(const float* __restrict__ xx, const float* __restrict__ yy,
                                                 const float* __restrict__ zz, float* __restrict__ s2, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s2[i] = fmaf(xx[i], yy[i], fmaf(xx[i], zz[i], yy[i] * zz[i]));
}

__global__ void __launch_bounds__(256) k_s2_sub(const float* __restrict__ ab, float* __restrict__ s2, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s2[i] = fmaf(-ab[i], ab[i], s2[i]);
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// One particle per thread: lattice point (ix, iy, iz) displaced by psi
// (box units, inv_dx cells per unit) plus `shift` cells on every axis; the
// nearest mesh point is floor(pos + 1/2), d = pos - that point in [-1/2, 1/2).
template <int P>
__global__ void __launch_bounds__(256) k_assign(const float* __restrict__ px, const float* __restrict__ py,
                                                const float* __restrict__ pz, const float* __restrict__ mass, int n,
                                                float inv_dx, float shift, float* __restrict__ mesh) {
  const int64_t np = (int64_t)n * n * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % n), iy = (int)((i / n) % n), iz = (int)(i / ((int64_t)n * n));
    const float pos[3] = {ix + px[i] * inv_dx + shift, iy + py[i] * inv_dx + shift, iz + pz[i] * inv_dx + shift};
    int base[3];
    float w[3][3];  // offsets -1, 0, +1
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float b = floorf(pos[a] + 0.5f);
      const float d = pos[a] - b;
      base[a] = (int)b;
      if (P == 1) {
        w[a][0] = 0.f; w[a][1] = 1.f; w[a][2] = 0.f;
      } else if (P == 2) {
        const float ad = fabsf(d);
        w[a][1] = 1.f - ad;
        w[a][0] = d < 0.f ? ad : 0.f;
        w[a][2] = d >= 0.f ? ad : 0.f;
      } else {
        w[a][0] = 0.5f * (0.5f - d) * (0.5f - d);
        w[a][1] = 0.75f - d * d;
        w[a][2] = 0.5f * (0.5f + d) * (0.5f + d);
      }
    }
    const float m = mass ? mass[i] : 1.0f;
#pragma unroll
    for (int oz = 0; oz < 3; ++oz) {
      if (w[2][oz] == 0.f) continue;
      const int64_t zo = (int64_t)wrap(base[2] + oz - 1, n) * n * n;
#pragma unroll
      for (int oy = 0; oy < 3; ++oy) {
        if (w[1][oy] == 0.f) continue;
        const int64_t yo = zo + (int64_t)wrap(base[1] + oy - 1, n) * n;
        const float wzy = m * w[2][oz] * w[1][oy];
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
          if (w[0][ox] == 0.f) continue;
          atomicAdd(&mesh[yo + wrap(base[0] + ox - 1, n)], wzy * w[0][ox]);
        }
      }
    }
  }
}

// [A + e^{i k.dX} B] / 2 / W(k)^p * scale into A, dX = (dx/2)(1,1,1):
// k_a dx / 2 = pi m_a / n.  scale = 1/sum(mass) (mean 1 and the inverse
// transform's 1/n^3 together); *total holds sum(mass).
__global__ void __launch_bounds__(256) k_interlace(float2* __restrict__ A, const float2* __restrict__ B, int n, int p,
                                                   const double* __restrict__ total) {
  const int ncol = n / 2 + 1, RS = n / 2 + 2;
  const float scale = (float)(1.0 / *total);
  const int64_t cnt = (int64_t)n * n * ncol;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(e % ncol);
    const int64_t row = e / ncol;
    const int y = (int)(row % n), z = (int)(row / n);
    const int64_t at = row * RS + x;
    if (x == n / 2 || y == n / 2 || z == n / 2) {
      A[at] = make_float2(0.f, 0.f);
      continue;
    }
    const int my = y < n / 2 ? y : y - n, mz = z < n / 2 ? z : z - n;
    const int mm[3] = {x, my, mz};
    float W = 1.f;
    for (int a = 0; a < 3; ++a) {
      if (mm[a] == 0) continue;
      const float t = (float)mm[a] / (float)n;  // k dx / 2 in units of pi
      W *= sinpif(t) / (3.14159265358979f * t);
    }
    float Wp = 1.f;
    for (int q = 0; q < p; ++q) Wp *= W;
    float sn, cs;
    sincospif((float)(mm[0] + mm[1] + mm[2]) / (float)n, &sn, &cs);
    const float2 a = A[at], b = B[at];
    const float f = 0.5f * scale / Wp;
    A[at] = make_float2(f * (a.x + cs * b.x - sn * b.y), f * (a.y + cs * b.y + sn * b.x));
  }
}

__global__ void __launch_bounds__(256) k_scale_mesh(float* __restrict__ rho, int64_t n3, const double* __restrict__ total) {
  const float f = (float)((double)n3 / *total);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    rho[i] *= f;
}

__global__ void __launch_bounds__(256) k_set_total(double* __restrict__ total, double v) { *total = v; }

__global__ void __launch_bounds__(256) k_fcoll(const float* __restrict__ df, int64_t n, float dc, float inv,
                                               float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = erfcf((dc - df[i]) * inv);
}

// ---------------------------------------------------------------------------
static int grid_of(int64_t work, int num_sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)num_sms * 16));
}

static cudaError_t spec_op(const LptWork& w, const SpecOpArgs& p, cudaStream_t s) {
  const int64_t cnt = (int64_t)p.n * p.n * (p.n / 2 + 1);
  k_spec_op<<<grid_of(cnt, w.num_sms), 256, 0, s>>>(p);
  return cudaGetLastError();
}

static SpecOpArgs op_args(int n, double box, int op, const void* A, const void* B, void* out) {
  SpecOpArgs p{};
  p.A = reinterpret_cast<const float2*>(A);
  p.B = reinterpret_cast<const float2*>(B);
  p.out = reinterpret_cast<float2*>(out);
  p.n = n;
  p.op = op;
  p.c1 = 1.f;
  p.c2 = 0.f;
  p.kf = (float)(2.0 * 3.14159265358979323846 / box);
  p.scale = (float)(1.0 / ((double)n * n * n));
  return p;
}

cudaError_t lpt_impl(const LptWork& w, int n, double box, double D1, double D2, const float* delta, float* psi_x,
                     float* psi_y, float* psi_z, cudaStream_t s) {
  const int64_t n3 = (int64_t)n * n * n;
  const int g = grid_of(n3, w.num_sms);
  cudaError_t e = forward_spectrum_f32(n, delta, w.H0, w.tw, s);
  // diagonal second derivatives of phi1 (k_a k_b delta / k^2) into psi as scratch
  float* diag[3] = {psi_x, psi_y, psi_z};
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    SpecOpArgs p = op_args(n, box, OP_HESS, w.H0, nullptr, w.H2);
    p.a = p.b = a;
    e = spec_op(w, p, s);
    if (e == cudaSuccess) e = inverse_spectrum_f32(n, w.H2, diag[a], w.tw, w.status, s);
  }
  if (e == cudaSuccess) {
    k_s2_diag<<<g, 256, 0, s>>>(psi_x, psi_y, psi_z, w.F0, n3);
    e = cudaGetLastError();
  }
  const int off[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
    SpecOpArgs p = op_args(n, box, OP_HESS, w.H0, nullptr, w.H2);
    p.a = off[q][0];
    p.b = off[q][1];
    e = spec_op(w, p, s);
    if (e == cudaSuccess) e = inverse_spectrum_f32(n, w.H2, w.F1, w.tw, w.status, s);
    if (e == cudaSuccess) {
      k_s2_sub<<<g, 256, 0, s>>>(w.F1, w.F0, n3);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = forward_spectrum_f32(n, w.F0, w.H1, w.tw, s);
  // psi_a = -D1 grad_a phi1 + D2 grad_a phi2 = (-i k_a / k^2)(-D1 delta + D2 S2)
  float* out[3] = {psi_x, psi_y, psi_z};
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    SpecOpArgs p = op_args(n, box, OP_GRADINV, w.H0, w.H1, w.H2);
    p.a = a;
    p.c1 = (float)(-D1);
    p.c2 = (float)D2;
    e = spec_op(w, p, s);
    if (e == cudaSuccess) e = inverse_spectrum_f32(n, w.H2, out[a], w.tw, w.status, s);
  }
  return e;
}

static cudaError_t assign(int order, int n, double box, float shift, const float* px, const float* py,
                          const float* pz, const float* mass, float* mesh, int num_sms, cudaStream_t s) {
  const int64_t n3 = (int64_t)n * n * n;
  cudaError_t e = cudaMemsetAsync(mesh, 0, (size_t)n3 * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const float inv_dx = (float)(n / box);
  const int g = grid_of(n3, num_sms);
  if (order == 1) k_assign<1><<<g, 256, 0, s>>>(px, py, pz, mass, n, inv_dx, shift, mesh);
  else if (order == 2) k_assign<2><<<g, 256, 0, s>>>(px, py, pz, mass, n, inv_dx, shift, mesh);
  else k_assign<3><<<g, 256, 0, s>>>(px, py, pz, mass, n, inv_dx, shift, mesh);
  return cudaGetLastError();
}

cudaError_t mesh_impl(const LptWork& w, int n, double box, int order, bool interlace, const float* psi_x,
                      const float* psi_y, const float* psi_z, const float* mass, float* rho, cudaStream_t s) {
  const int64_t n3 = (int64_t)n * n * n;
  cudaError_t e;
  if (mass) {
    e = sum_f64_impl(mass, n3, w.acc, w.num_sms, s);
  } else {
    k_set_total<<<1, 1, 0, s>>>(w.acc, (double)n3);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = assign(order, n, box, 0.f, psi_x, psi_y, psi_z, mass, rho, w.num_sms, s);
  if (e != cudaSuccess) return e;
  if (!interlace) {
    k_scale_mesh<<<grid_of(n3, w.num_sms), 256, 0, s>>>(rho, n3, w.acc);
    return cudaGetLastError();
  }
  e = assign(order, n, box, 0.5f, psi_x, psi_y, psi_z, mass, w.F0, w.num_sms, s);
  if (e == cudaSuccess) e = forward_spectrum_f32(n, rho, w.H0, w.tw, s);
  if (e == cudaSuccess) e = forward_spectrum_f32(n, w.F0, w.H1, w.tw, s);
  if (e == cudaSuccess) {
    const int64_t cnt = (int64_t)n * n * (n / 2 + 1);
    k_interlace<<<grid_of(cnt, w.num_sms), 256, 0, s>>>(reinterpret_cast<float2*>(w.H0),
                                                         reinterpret_cast<const float2*>(w.H1), n, order, w.acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = inverse_spectrum_f32(n, w.H0, rho, w.tw, w.status, s);
  return e;
}

cudaError_t fcoll_impl(const LptWork& w, int n, double box, double R, int filter, double delta_c, double dsigma2,
                       const float* delta, float* out, cudaStream_t s) {
  const int64_t n3 = (int64_t)n * n * n;
  cudaError_t e = forward_spectrum_f32(n, delta, w.H0, w.tw, s);
  if (e == cudaSuccess) {
    SpecOpArgs p = op_args(n, box, filter == 0 ? OP_SHARPK : OP_TOPHAT, w.H0, nullptr, w.H0);
    p.R = (float)R;
    const double kfR = 2.0 * 3.14159265358979323846 / box * R;
    p.m2max = 1.0 / (kfR * kfR);
    e = spec_op(w, p, s);
  }
  if (e == cudaSuccess) e = inverse_spectrum_f32(n, w.H0, out, w.tw, w.status, s);
  if (e == cudaSuccess) {
    k_fcoll<<<grid_of(n3, w.num_sms), 256, 0, s>>>(out, n3, (float)delta_c, (float)(1.0 / std::sqrt(2.0 * dsigma2)),
                                                   out);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace amber
