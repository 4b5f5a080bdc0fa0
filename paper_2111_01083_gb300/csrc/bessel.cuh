// Modified Bessel functions K0, K1 of real argument x > 0 for the modified
// Helmholtz Green's function (1/2pi) K0(beta r) and its gradient
// -(beta/2pi) K1(beta r) r_hat.  CUDA has no K0/K1; these are written from
// the published methods named below.
#pragma once
#include <cuda_runtime.h>

namespace pfmm {
namespace bes {

// FP32: rational/polynomial fits of Abramowitz & Stegun 9.8.1, 9.8.3 (I0, I1
// for |x| <= 3.75) and 9.8.5-9.8.8 (K0, K1); relative error below 2.2e-7.
__device__ __forceinline__ void k01f(float x, float* k0, float* k1) {
  if (x <= 2.0f) {
    float t = x * (1.0f / 3.75f);
    float t2 = t * t;
    float i0 = 1.0f + t2 * (3.5156229f + t2 * (3.0899424f + t2 * (1.2067492f + t2 * (0.2659732f + t2 * (0.0360768f + t2 * 0.0045813f)))));
    float i1 = x * (0.5f + t2 * (0.87890594f + t2 * (0.51498869f + t2 * (0.15084934f + t2 * (0.02658733f + t2 * (0.00301532f + t2 * 0.00032411f))))));
    float y = 0.25f * x * x;
    float lg = __logf(0.5f * x);
    *k0 = -lg * i0 + (-0.57721566f + y * (0.42278420f + y * (0.23069756f + y * (0.03488590f + y * (0.00262698f + y * (0.00010750f + y * 0.0000074f))))));
    *k1 = (x * lg * i1 + (1.0f + y * (0.15443144f + y * (-0.67278579f + y * (-0.18156897f + y * (-0.01919402f + y * (-0.00110404f + y * (-0.00004686f))))))) ) / x;
  } else {
    float y = 2.0f / x;
    float e = __expf(-x) * rsqrtf(x);
    *k0 = e * (1.25331414f + y * (-0.07832358f + y * (0.02189568f + y * (-0.01062446f + y * (0.00587872f + y * (-0.00251540f + y * 0.00053208f))))));
    *k1 = e * (1.25331414f + y * (0.23498619f + y * (-0.03655620f + y * (0.01504268f + y * (-0.00780353f + y * (0.00325614f + y * (-0.00068245f)))))));
  }
}

// FP32 K0 only (same fits as k01f).
__device__ __forceinline__ float k0f(float x) {
  if (x <= 2.0f) {
    float t = x * (1.0f / 3.75f);
    float t2 = t * t;
    float i0 = 1.0f + t2 * (3.5156229f + t2 * (3.0899424f + t2 * (1.2067492f + t2 * (0.2659732f + t2 * (0.0360768f + t2 * 0.0045813f)))));
    float y = 0.25f * x * x;
    return -__logf(0.5f * x) * i0 + (-0.57721566f + y * (0.42278420f + y * (0.23069756f + y * (0.03488590f + y * (0.00262698f + y * (0.00010750f + y * 0.0000074f))))));
  }
  float y = 2.0f / x;
  return __expf(-x) * rsqrtf(x) * (1.25331414f + y * (-0.07832358f + y * (0.02189568f + y * (-0.01062446f + y * (0.00587872f + y * (-0.00251540f + y * 0.00053208f))))));
}

// FP32 from x^2 (x = beta r), no division, MUFU approximations: the same
// A&S 9.8 fits written in x^2 so that the small-argument branch needs no
// square root and the large-argument branch gets 1/x, x and x^-1/2 from two
// rsqrt: ix = rsqrt(x^2), x = x^2 ix, rx = rsqrt(x).
namespace mufu {
__device__ __forceinline__ float rsqrt(float x) { float r; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float rcp(float x) { float r; asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float ex2(float x) { float r; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
__device__ __forceinline__ float lg2(float x) { float r; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x)); return r; }
}  // namespace mufu

__device__ __forceinline__ float k0f_x2(float x2) {
  if (x2 <= 4.0f) {
    const float t2 = x2 * (1.0f / 14.0625f);  // (x / 3.75)^2
    const float i0 = 1.0f + t2 * (3.5156229f + t2 * (3.0899424f + t2 * (1.2067492f + t2 * (0.2659732f + t2 * (0.0360768f + t2 * 0.0045813f)))));
    const float y = 0.25f * x2;
    const float lg = 0.34657359027997264f * mufu::lg2(y);  // ln(x / 2) = (ln 2 / 2) log2(x^2 / 4)
    return -lg * i0 + (-0.57721566f + y * (0.42278420f + y * (0.23069756f + y * (0.03488590f + y * (0.00262698f + y * (0.00010750f + y * 0.0000074f))))));
  }
  const float ix = mufu::rsqrt(x2);
  const float x = x2 * ix;
  const float rx = mufu::rsqrt(x);
  const float e = mufu::ex2(-1.4426950408889634f * x);
  const float y = 2.0f * ix;
  return e * rx * (1.25331414f + y * (-0.07832358f + y * (0.02189568f + y * (-0.01062446f + y * (0.00587872f + y * (-0.00251540f + y * 0.00053208f))))));
}

// K0(x) and K1(x) / x from x^2.
__device__ __forceinline__ void k01f_x2(float x2, float* k0, float* k1ix) {
  if (x2 <= 4.0f) {
    const float t2 = x2 * (1.0f / 14.0625f);
    const float i0 = 1.0f + t2 * (3.5156229f + t2 * (3.0899424f + t2 * (1.2067492f + t2 * (0.2659732f + t2 * (0.0360768f + t2 * 0.0045813f)))));
    // I1(x) = x p1(t2)
    const float p1 = 0.5f + t2 * (0.87890594f + t2 * (0.51498869f + t2 * (0.15084934f + t2 * (0.02658733f + t2 * (0.00301532f + t2 * 0.00032411f)))));
    const float y = 0.25f * x2;
    const float lg = 0.34657359027997264f * mufu::lg2(y);
    *k0 = -lg * i0 + (-0.57721566f + y * (0.42278420f + y * (0.23069756f + y * (0.03488590f + y * (0.00262698f + y * (0.00010750f + y * 0.0000074f))))));
    // K1(x) = (x^2 ln(x/2) p1 + q1(y)) / x  ->  K1 / x = ln(x/2) p1 + q1(y) / x^2
    const float q1 = 1.0f + y * (0.15443144f + y * (-0.67278579f + y * (-0.18156897f + y * (-0.01919402f + y * (-0.00110404f + y * (-0.00004686f))))));
    *k1ix = lg * p1 + q1 * mufu::rcp(x2);
    return;
  }
  const float ix = mufu::rsqrt(x2);
  const float x = x2 * ix;
  const float rx = mufu::rsqrt(x);
  const float e = mufu::ex2(-1.4426950408889634f * x) * rx;
  const float y = 2.0f * ix;
  *k0 = e * (1.25331414f + y * (-0.07832358f + y * (0.02189568f + y * (-0.01062446f + y * (0.00587872f + y * (-0.00251540f + y * 0.00053208f))))));
  *k1ix = e * ix * (1.25331414f + y * (0.23498619f + y * (-0.03655620f + y * (0.01504268f + y * (-0.00780353f + y * (0.00325614f + y * (-0.00068245f)))))));
}

// FP64.  x <= 2: the ascending series (DLMF 10.31.1-10.31.2),
//   K0 = -(ln(x/2) + gamma) I0(x) + sum_{k>=1} H_k (x^2/4)^k / (k!)^2,
//   K1 = 1/x + ln(x/2) I1(x) - (x/4) sum_{k>=0} (psi(k+1) + psi(k+2)) (x^2/4)^k / (k! (k+1)!).
// x > 2: the integral K_nu(x) = int_0^inf e^{-x cosh t} cosh(nu t) dt (DLMF 10.32.9) with
// u = 2 sqrt(x) sinh(t/2), which gives
//   K0 = e^{-x} int_0^inf e^{-u^2/2} / sqrt(x + u^2/4) du,
//   K1 = e^{-x} int_0^inf e^{-u^2/2} (1 + u^2/(2x)) / sqrt(x + u^2/4) du,
// by the trapezoidal rule (step 0.45, 22 nodes), which converges
// geometrically for these analytic, Gaussian-decaying integrands.
__device__ __forceinline__ void k01d(double x, double* k0, double* k1) {
  const double eg = 0.57721566490153286061;
  if (x <= 2.0) {
    double z = 0.25 * x * x;
    double tk = 1.0, t1 = 1.0, H = 0.0;
    double I0 = 0.0, S0 = 0.0, I1 = 0.0, S1 = 0.0;
    for (int k = 0; k < 30; ++k) {
      if (k > 0) {
        tk *= z / ((double)k * k);
        t1 *= z / ((double)k * (k + 1));
        H += 1.0 / k;
      }
      I0 += tk;
      S0 += H * tk;
      I1 += t1;
      S1 += (-2.0 * eg + 2.0 * H + 1.0 / (k + 1)) * t1;
    }
    I1 *= 0.5 * x;
    double lg = log(0.5 * x);
    *k0 = -(lg + eg) * I0 + S0;
    *k1 = 1.0 / x + lg * I1 - 0.25 * x * S1;
  } else {
    const double h = 0.45;
    double s0 = 0.5 / sqrt(x), s1 = s0;
    for (int k = 1; k < 22; ++k) {
      double u = k * h, u2 = u * u;
      double e = exp(-0.5 * u2);
      double r = 1.0 / sqrt(x + 0.25 * u2);
      s0 += e * r;
      s1 += e * (1.0 + u2 / (2.0 * x)) * r;
    }
    double e = exp(-x) * h;
    *k0 = e * s0;
    *k1 = e * s1;
  }
}

}  // namespace bes
}  // namespace pfmm
