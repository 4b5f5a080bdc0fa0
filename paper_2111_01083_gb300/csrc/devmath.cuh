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

// FP32 sine and cosine on the FMA pipe.  On |x| <= pi/4 the Taylor series
// about 0 truncated after the x^9 (sine) and x^10 (cosine) terms is exact to
// 2e-9, below FP32 rounding; the argument is first reduced exactly by
// quarter turns, and the quadrant applied by swaps and sign changes.
__device__ __forceinline__ void sincos_quarter(float x, float* s, float* c) {
  const float x2 = x * x;
  float ps = fmaf(x2, 2.75573192e-6f, -1.98412698e-4f);  // 1/9!, -1/7!
  ps = fmaf(x2, ps, 8.33333333e-3f);                     // 1/5!
  ps = fmaf(x2, ps, -1.66666667e-1f);                    // -1/3!
  *s = fmaf(x * x2, ps, x);
  float pc = fmaf(x2, -2.75573192e-7f, 2.48015873e-5f);  // -1/10!, 1/8!
  pc = fmaf(x2, pc, -1.38888889e-3f);                    // -1/6!
  pc = fmaf(x2, pc, 4.16666667e-2f);                     // 1/4!
  pc = fmaf(x2, pc, -0.5f);
  *c = fmaf(x2, pc, 1.0f);
}
// (sin, cos)(x + q pi/2) from (sin, cos)(x)
__device__ __forceinline__ void quadrant(int q, float s0, float c0, float* s, float* c) {
  const bool sw = (q & 1) != 0;
  const float ss = sw ? c0 : s0, cc = sw ? s0 : c0;
  *s = (q & 2) ? -ss : ss;
  *c = ((q + 1) & 2) ? -cc : cc;
}
// sin and cos of 2 pi ph / 2^32 (a fixed-point phase in turns, wrapping
// modulo 2^32): the quadrant is the rounded top two bits, the remainder is
// exact in [-2^29, 2^29).
__device__ __forceinline__ void sincos_turns(unsigned ph, float* s, float* c) {
  const unsigned q = ((ph + 0x20000000u) >> 30) & 3u;
  const int r = (int)(ph - (q << 30));
  float s0, c0;
  sincos_quarter((float)r * 1.46291808e-9f, &s0, &c0);  // 2 pi / 2^32
  quadrant((int)q, s0, c0, s, c);
}
// sin and cos of a moderate FP32 argument (|x| < ~1e3): two-constant
// reduction by pi/2 (Cody and Waite), then the quarter-turn polynomials.
__device__ __forceinline__ void sincos_red(float x, float* s, float* c) {
  const float q = rintf(x * 0.636619772f);
  float r = fmaf(-q, 1.57079637f, x);
  r = fmaf(-q, -4.37113900e-8f, r);
  float s0, c0;
  sincos_quarter(r, &s0, &c0);
  quadrant((int)q & 3, s0, c0, s, c);
}
// e^x through the MUFU base-2 exponential (relative error ~1e-7 (1 + |x|))
__device__ __forceinline__ float ex_fast(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x * 1.44269504f));
  return r;
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

// FP32 expm1c with the FMA-pipe sine and cosine
__device__ __forceinline__ void expm1c_fast(float a, float b, float* re, float* im) {
  const float em = expm1f(a);
  float sh, ch;
  sincos_red(0.5f * b, &sh, &ch);
  const float s2 = 2.0f * sh * sh;
  *re = em * (1.0f - s2) - s2;
  *im = (em + 1.0f) * (2.0f * sh * ch);
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
