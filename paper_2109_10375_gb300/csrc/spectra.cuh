// Analysis of reionization-redshift fields (Sec. 2.3): normalised redshift
// field, fractional-difference PDF and spherical-shell power spectra.
#pragma once

#include "common.cuh"

namespace amber {

constexpr int kMaxPowerBins = 1024;  // round(sqrt(3) n / 2) + 1 <= 888 for n <= 1024
constexpr int kPowerAcc = 5;         // per shell: modes, sum |m|, aa, bb, ab

int power_bins(int n);

// Forward R2C transform of an n^3 float field into the half spectrum H.
cudaError_t forward_spectrum_f32(int n, const float* src, void* H, const void* tw, cudaStream_t s);

// delta_z = ((1 + z) - (1 + zbar)) / (1 + zbar), zbar the cell mean (FP64 sum);
// acc: one double of device scratch; zbar_out (device, optional).
cudaError_t delta_z_impl(const float* z, int64_t n, float* out, double* acc, double* zbar_out, int num_sms,
                         cudaStream_t s);

// Histogram of epsilon = ((1 + z) - (1 + zref)) / (1 + zref) over [lo, hi) in
// nbins equal bins; counts[0] and counts[nbins + 1] take the values below and
// above.  moments (optional): sum of epsilon and of epsilon^2.
cudaError_t epsilon_pdf_impl(const float* z, const float* zref, int64_t n, double lo, double hi, int nbins,
                             unsigned long long* counts, double* moments, int num_sms, cudaStream_t s);

// Shell sums of the half spectra Ha (and Hb, may be null) of an n^3 grid
// into acc[kPowerAcc][nb] (zeroed here), then the shell averages in the
// continuum normalisation P = box^3 / n^6 <|A|^2>: k (mean |k|), Paa, Pbb,
// Pab, modes (device, caller-owned, nb each; Pbb/Pab may be null).
cudaError_t power_impl(const void* Ha, const void* Hb, int n, double box, double* acc, double* k, double* Paa,
                       double* Pbb, double* Pab, double* modes, int num_sms, cudaStream_t s);

// Delta^2 of a (and b) (Eq. Dk), bias (Eq. bias) and cross-correlation (Eq. rcc)
// per shell from power_impl's outputs; Pbb/Pab and every output but D2aa may be
// null (the ratios need Pbb).
cudaError_t power_derived_impl(const double* k, const double* Paa, const double* Pbb, const double* Pab, int nb,
                               double* D2aa, double* D2bb, double* bias, double* r, cudaStream_t s);

}  // namespace amber
