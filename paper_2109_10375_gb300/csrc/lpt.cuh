// Source-field pipeline (Sec. 3.2, 3.2.1, 3.3): second-order Lagrangian
// displacements, mesh assignment with interlacing and deconvolution, and the
// ESF collapsed fraction.  See lpt.cu.
#pragma once

#include "common.cuh"

namespace amber {

// Buffers a call may use: three half spectra (H0..H2, each n^2 (n/2 + 2)
// complex floats) and two real n^3 float fields (F0, F1), plus one double.
struct LptWork {
  void* H0;
  void* H1;
  void* H2;
  float* F0;
  float* F1;
  double* acc;
  const void* tw;  // FP32 twiddles of this n
  unsigned int* status;
  int num_sms;
};

cudaError_t inverse_spectrum_f32(int n, void* H, float* out, const void* tw, unsigned int* status, cudaStream_t s);
cudaError_t forward_spectrum_f32(int n, const float* src, void* H, const void* tw, cudaStream_t s);
cudaError_t sum_f64_impl(const float* x, int64_t n, double* acc, int num_sms, cudaStream_t s);

// psi = x - q = -D1 grad phi1 + D2 grad phi2 (box units), lap phi1 = delta_lin,
// lap phi2 = sum_{i<j} (phi1,ii phi1,jj - phi1,ij^2).  psi_x/y/z: n^3 floats
// out (also used as scratch).
cudaError_t lpt_impl(const LptWork& w, int n, double box, double D1, double D2, const float* delta, float* psi_x,
                     float* psi_y, float* psi_z, cudaStream_t s);

// rho / mean on the n^3 mesh from particles at q + psi with masses `mass`
// (NULL: all equal), window order 1..3; with interlace the second mesh's
// particles move by half a cell and the two are combined and deconvolved.
cudaError_t mesh_impl(const LptWork& w, int n, double box, int order, bool interlace, const float* psi_x,
                      const float* psi_y, const float* psi_z, const float* mass, float* rho, cudaStream_t s);

// f_coll = erfc((delta_c - delta_f) / sqrt(2 dsigma2)) of delta_lin filtered
// with a sharp k-space (filter 0) or top-hat (filter 1) window of radius R.
cudaError_t fcoll_impl(const LptWork& w, int n, double box, double R, int filter, double delta_c, double dsigma2,
                       const float* delta, float* out, cudaStream_t s);

}  // namespace amber
