// Packed FP32 helpers: two independent lanes per float2 (two targets per
// thread in the P2P kernels), one FADD2/FMUL2/FFMA2 instruction per operation.
#pragma once
#include <cuda_runtime.h>

namespace pfmm {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

}  // namespace pfmm
