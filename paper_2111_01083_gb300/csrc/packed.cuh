// Packed FP32 helpers: two independent lanes per float2 (two targets per
// thread in the P2P kernels), one FADD2/FMUL2/FFMA2 instruction per operation.
#pragma once
#include <cuda_runtime.h>

namespace pfmm {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
#if defined(PFMM_P2P_SCALAR)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
#elif defined(PFMM_P2P_FMA_ONLY)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __ffma2_rn(a, make_float2(1.f, 1.f), b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __ffma2_rn(a, b, make_float2(0.f, 0.f)); }
#else
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
#endif
#if defined(PFMM_P2P_SCALAR)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#else
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#endif


}  // namespace pfmm
