// Source field from a density field (step a0), see source.cu.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace amber {

cudaError_t source_field_impl(const float* delta, int64_t n, double delta_c, double sigma_f, float* S, float* mass,
                              unsigned long long* total, int num_sms, unsigned int* status, cudaStream_t s);

}  // namespace amber
