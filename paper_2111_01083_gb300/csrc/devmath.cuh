// Small device math helpers shared by the library's kernels (float and
// double overloads of the CUDA math functions used on the hot path).
#pragma once
#include <cuda_runtime.h>

namespace pfmm {
namespace dm {

__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sincospi_(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ float em1(float x) { return expm1f(x); }
__device__ __forceinline__ double em1(double x) { return expm1(x); }

// e^{2 pi i m u} for a fixed-point fraction u = U / 2^32 (turns).  The product
// m * U wraps modulo 2^32, which is exact range reduction of the phase.
__device__ __forceinline__ void phase_fixed(int m, int U, float* s, float* c) {
  unsigned ph = (unsigned)m * (unsigned)U;
  float turns = (float)(int)ph * 2.3283064365386963e-10f;  // 2^-32
  sincospif(2.0f * turns, s, c);
}

// e^{a + i b} - 1 without cancellation for small |a|, |b|:
//   re = expm1(a) (1 - 2 sin^2(b/2)) - 2 sin^2(b/2),  im = e^a sin b
template <typename T>
__device__ __forceinline__ void expm1c(T a, T b, T* re, T* im) {
  T em = em1(a);
  T sh, ch;
  sincos_(T(0.5) * b, &sh, &ch);
  T s2 = T(2) * sh * sh;
  *re = em * (T(1) - s2) - s2;
  *im = (em + T(1)) * (T(2) * sh * ch);
}

// Exact FP32 -> FP64 conversion by bit operations on the integer pipes.  On
// this GPU the conversion instruction runs on the FP64 unit (about 1/64 of
// the FP32 rate), so FP32 kernels that hand many partial sums to FP64
// outputs convert this way: sign | (exponent + 1023 - 127) << 52 |
// mantissa << 29 for normal numbers, infinities and NaNs kept, zero and FP32
// subnormals to a signed zero (the FP32 kernels flush subnormals anyway).
__device__ __forceinline__ double f2d(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
  const unsigned hi = (u & 0x80000000u) | (e ? ((ed << 20) | ((u >> 3) & 0xfffffu)) : 0u);
  const unsigned lo = e ? (u << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// Running sum of many terms.  FP32: Kahan compensation (the error stays at a
// few ulp of the result instead of growing with the number of terms); FP64:
// plain sum.
template <typename T>
struct KSum {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    if constexpr (sizeof(T) == 4) {
      const T y = v - c;
      const T t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += v;
    }
  }
  __device__ __forceinline__ double value() const {
    if constexpr (sizeof(T) == 4)
      return f2d(s) - f2d(c);
    else
      return (double)s - (double)c;
  }
};

}  // namespace dm
}  // namespace pfmm
