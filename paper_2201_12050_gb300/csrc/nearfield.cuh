// Near-field product (nearfield.cu).
#pragma once
#include "common.cuh"

namespace fmpb {

// y (+)= sum_delta S_delta p_{c - delta}; offs_dev: n_near x 3 int offsets on
// the device, S: n_near x n x n float-float, p float-float, y complex double.
fmpb_status near_apply(const float4* S, const int* offs_dev, int n_near, int n, const int M[3], int R, const float4* p,
                       cd* y, bool accumulate, cudaStream_t st);

// FP32 operators: S and p complex FP32.
fmpb_status near_apply_f32(const float2* S, const int* offs_dev, int n_near, int n, const int M[3], int R,
                           const float2* p, cd* y, bool accumulate, cudaStream_t st);

}  // namespace fmpb
