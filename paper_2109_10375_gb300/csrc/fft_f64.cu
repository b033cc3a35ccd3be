// Instantiations of the radiation-field FFT passes for double (see fft.cuh).
#include "fft.cuh"

namespace amber {

cudaError_t radiation_field_f64(int n, const double* src, double* J, void* H, const void* tw, double box, double l_mfp,
                               unsigned int* status, cudaStream_t s, FftProfile* prof,
                               SortCtrl* krange) {
  auto* h = reinterpret_cast<cpx<double>*>(H);
  auto* w = reinterpret_cast<const cpx<double>*>(tw);
  switch (n) {
    case 4: return radiation_field_n<double, 4>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    case 8: return radiation_field_n<double, 8>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    case 16: return radiation_field_n<double, 16>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    case 32: return radiation_field_n<double, 32>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    case 64: return radiation_field_n<double, 64>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    case 128: return radiation_field_n<double, 128>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    case 256: return radiation_field_n<double, 256>(src, J, h, w, box, l_mfp, status, s, prof, krange);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace amber
