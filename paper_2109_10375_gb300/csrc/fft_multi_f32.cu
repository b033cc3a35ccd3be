// Instantiations of the multi-item radiation field for float: several
// realisations of one grid size in one launch per pass (see fft.cuh).
#include "fft.cuh"

namespace amber {

cudaError_t radiation_field_multi_f32(int n, int variant, const float* const* srcs, int M, float* J, void* H,
                                      const void* tw, const float* kp, unsigned int* status, cudaStream_t s,
                                      SortCtrl* kranges) {
  auto* h = reinterpret_cast<cpx<float>*>(H);
  auto* w = reinterpret_cast<const cpx<float>*>(tw);
  if (variant == 1) {
    switch (n) {
      case 128: return radiation_field_multi_n<float, 128, 1>(srcs, M, J, h, w, kp, status, s, kranges);
      case 256: return radiation_field_multi_n<float, 256, 1>(srcs, M, J, h, w, kp, status, s, kranges);
      case 512: return radiation_field_multi_n<float, 512, 1>(srcs, M, J, h, w, kp, status, s, kranges);
      case 1024: return radiation_field_multi_n<float, 1024, 1>(srcs, M, J, h, w, kp, status, s, kranges);
      default: return cudaErrorInvalidValue;
    }
  }
  if (variant != 0) return cudaErrorInvalidValue;
  switch (n) {
    case 8: return radiation_field_multi_n<float, 8>(srcs, M, J, h, w, kp, status, s, kranges);
    case 16: return radiation_field_multi_n<float, 16>(srcs, M, J, h, w, kp, status, s, kranges);
    case 32: return radiation_field_multi_n<float, 32>(srcs, M, J, h, w, kp, status, s, kranges);
    case 64: return radiation_field_multi_n<float, 64>(srcs, M, J, h, w, kp, status, s, kranges);
    case 128: return radiation_field_multi_n<float, 128>(srcs, M, J, h, w, kp, status, s, kranges);
    case 256: return radiation_field_multi_n<float, 256>(srcs, M, J, h, w, kp, status, s, kranges);
    case 512: return radiation_field_multi_n<float, 512>(srcs, M, J, h, w, kp, status, s, kranges);
    case 1024: return radiation_field_multi_n<float, 1024>(srcs, M, J, h, w, kp, status, s, kranges);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace amber
