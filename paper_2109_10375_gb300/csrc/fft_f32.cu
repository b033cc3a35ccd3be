// Instantiations of the radiation-field FFT passes for float (see fft.cuh).
#include <cstdint>

#include "fft.cuh"

namespace amber {

namespace {
// cuTensorMapEncodeTiled, fetched from the driver at run time (the library
// links only the CUDA runtime)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiled) nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}
}  // namespace

bool zpass_tensor_map(CUtensorMap* map, const void* H, int n, int SB) {
  EncodeTiled enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(H) & 15u)) return false;
  const cuuint64_t rs = (cuuint64_t)(n / 2 + 2);
  const cuuint64_t dims[3] = {(cuuint64_t)(n / 2 + 1), (cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[2] = {rs * 8, (cuuint64_t)n * rs * 8};  // bytes, y then z
  const cuuint32_t box[3] = {(cuuint32_t)SB, 1u, (cuuint32_t)(n < kZBox ? n : kZBox)};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  // L2 promotion of the 64-byte rows to 128 or 256 bytes was measured no faster
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(H), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t radiation_field_f32(int n, const float* src, float* J, void* H, const void* tw, double box, double l_mfp,
                               unsigned int* status, cudaStream_t s, FftProfile* prof,
                               SortCtrl* krange, int variant, const void* spec_in, bool hist8, bool tma) {
  auto* h = reinterpret_cast<cpx<float>*>(H);
  auto* w = reinterpret_cast<const cpx<float>*>(tw);
  auto* si = reinterpret_cast<const cpx<float>*>(spec_in);
  if (variant == 1) {
    switch (n) {
      case 128: return radiation_field_n<float, 128, 1>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
      case 256: return radiation_field_n<float, 256, 1>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
      case 512: return radiation_field_n<float, 512, 1>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
      case 1024: return radiation_field_n<float, 1024, 1>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
      default: return cudaErrorInvalidValue;
    }
  }
  if (variant != 0) return cudaErrorInvalidValue;
  switch (n) {
    case 4: return radiation_field_n<float, 4>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 8: return radiation_field_n<float, 8>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 16: return radiation_field_n<float, 16>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 32: return radiation_field_n<float, 32>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 64: return radiation_field_n<float, 64>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 128: return radiation_field_n<float, 128>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 256: return radiation_field_n<float, 256>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 512: return radiation_field_n<float, 512>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    case 1024: return radiation_field_n<float, 1024>(src, J, h, w, box, l_mfp, status, s, prof, krange, si, hist8, tma);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t source_spectrum_f32(int n, const float* src, void* H, const void* tw, cudaStream_t s, FftProfile* prof,
                               int variant) {
  auto* h = reinterpret_cast<cpx<float>*>(H);
  auto* w = reinterpret_cast<const cpx<float>*>(tw);
  if (variant == 1) {
    switch (n) {
      case 128: return source_spectrum_n<float, 128, 1>(src, h, w, s, prof);
      case 256: return source_spectrum_n<float, 256, 1>(src, h, w, s, prof);
      case 512: return source_spectrum_n<float, 512, 1>(src, h, w, s, prof);
      case 1024: return source_spectrum_n<float, 1024, 1>(src, h, w, s, prof);
      default: return cudaErrorInvalidValue;
    }
  }
  if (variant != 0) return cudaErrorInvalidValue;
  switch (n) {
    case 4: return source_spectrum_n<float, 4>(src, h, w, s, prof);
    case 8: return source_spectrum_n<float, 8>(src, h, w, s, prof);
    case 16: return source_spectrum_n<float, 16>(src, h, w, s, prof);
    case 32: return source_spectrum_n<float, 32>(src, h, w, s, prof);
    case 64: return source_spectrum_n<float, 64>(src, h, w, s, prof);
    case 128: return source_spectrum_n<float, 128>(src, h, w, s, prof);
    case 256: return source_spectrum_n<float, 256>(src, h, w, s, prof);
    case 512: return source_spectrum_n<float, 512>(src, h, w, s, prof);
    case 1024: return source_spectrum_n<float, 1024>(src, h, w, s, prof);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t forward_spectrum_f32(int n, const float* src, void* H, const void* tw, cudaStream_t s) {
  auto* h = reinterpret_cast<cpx<float>*>(H);
  auto* w = reinterpret_cast<const cpx<float>*>(tw);
  switch (n) {
    case 4: return forward_spectrum_n<float, 4>(src, h, w, s);
    case 8: return forward_spectrum_n<float, 8>(src, h, w, s);
    case 16: return forward_spectrum_n<float, 16>(src, h, w, s);
    case 32: return forward_spectrum_n<float, 32>(src, h, w, s);
    case 64: return forward_spectrum_n<float, 64>(src, h, w, s);
    case 128: return forward_spectrum_n<float, 128>(src, h, w, s);
    case 256: return forward_spectrum_n<float, 256>(src, h, w, s);
    case 512: return forward_spectrum_n<float, 512>(src, h, w, s);
    case 1024: return forward_spectrum_n<float, 1024>(src, h, w, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t inverse_spectrum_f32(int n, void* H, float* out, const void* tw, unsigned int* status, cudaStream_t s) {
  auto* h = reinterpret_cast<cpx<float>*>(H);
  auto* w = reinterpret_cast<const cpx<float>*>(tw);
  switch (n) {
    case 4: return inverse_spectrum_n<float, 4>(h, out, w, status, s);
    case 8: return inverse_spectrum_n<float, 8>(h, out, w, status, s);
    case 16: return inverse_spectrum_n<float, 16>(h, out, w, status, s);
    case 32: return inverse_spectrum_n<float, 32>(h, out, w, status, s);
    case 64: return inverse_spectrum_n<float, 64>(h, out, w, status, s);
    case 128: return inverse_spectrum_n<float, 128>(h, out, w, status, s);
    case 256: return inverse_spectrum_n<float, 256>(h, out, w, status, s);
    case 512: return inverse_spectrum_n<float, 512>(h, out, w, status, s);
    case 1024: return inverse_spectrum_n<float, 1024>(h, out, w, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace amber
