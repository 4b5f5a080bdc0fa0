// Modified Bessel functions K0, K1 of real argument x > 0 for the modified
// Helmholtz Green's function (1/2pi) K0(beta r) and its gradient
// -(beta/2pi) K1(beta r) r_hat, and the combination K1(x)/x - 1/x^2 of the
// modified Stokeslet.  CUDA has no K0/K1; these are written from
// the published methods named below.
#pragma once
#include <cuda_runtime.h>
#include "packed.cuh"

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

// K0(x) and E(x) = K1(x)/x - 1/x^2 from x^2 (the modified Stokeslet).  For
// x <= 2 the A&S 9.8.7 form x K1 = x^2 ln(x/2) p1 + q1(y), q1 = 1 + y q1'(y),
// gives E = ln(x/2) p1 + q1'(y) / 4 (y / x^2 = 1/4) with no cancellation; for
// x > 2, E = K1/x - 1/x^2 directly (|1/x^2| <= 1/4, no cancellation either).
__device__ __forceinline__ void k0ef_x2(float x2, float* k0, float* e) {
  if (x2 <= 4.0f) {
    const float t2 = x2 * (1.0f / 14.0625f);
    const float i0 = 1.0f + t2 * (3.5156229f + t2 * (3.0899424f + t2 * (1.2067492f + t2 * (0.2659732f + t2 * (0.0360768f + t2 * 0.0045813f)))));
    const float p1 = 0.5f + t2 * (0.87890594f + t2 * (0.51498869f + t2 * (0.15084934f + t2 * (0.02658733f + t2 * (0.00301532f + t2 * 0.00032411f)))));
    const float y = 0.25f * x2;
    const float lg = 0.34657359027997264f * mufu::lg2(y);
    *k0 = -lg * i0 + (-0.57721566f + y * (0.42278420f + y * (0.23069756f + y * (0.03488590f + y * (0.00262698f + y * (0.00010750f + y * 0.0000074f))))));
    const float q1p = 0.15443144f + y * (-0.67278579f + y * (-0.18156897f + y * (-0.01919402f + y * (-0.00110404f + y * (-0.00004686f)))));
    *e = lg * p1 + 0.25f * q1p;
    return;
  }
  const float ix = mufu::rsqrt(x2);
  const float x = x2 * ix;
  const float rx = mufu::rsqrt(x);
  const float ex = mufu::ex2(-1.4426950408889634f * x) * rx;
  const float y = 2.0f * ix;
  *k0 = ex * (1.25331414f + y * (-0.07832358f + y * (0.02189568f + y * (-0.01062446f + y * (0.00587872f + y * (-0.00251540f + y * 0.00053208f))))));
  const float k1ix = ex * ix * (1.25331414f + y * (0.23498619f + y * (-0.03655620f + y * (0.01504268f + y * (-0.00780353f + y * (0.00325614f + y * (-0.00068245f)))))));
  *e = k1ix - ix * ix;
}

// Packed (two lanes) versions of k0f_x2 / k01f_x2, one branch per formula:
// a lane pair whose lanes fall on different sides of x = 2 evaluates both
// formulas and selects per lane.
namespace pk {
__device__ __forceinline__ float2 poly6(float2 t, float c0, float c1, float c2, float c3, float c4, float c5, float c6) {
  float2 p = fma2(t, f2(c6), f2(c5));
  p = fma2(t, p, f2(c4));
  p = fma2(t, p, f2(c3));
  p = fma2(t, p, f2(c2));
  p = fma2(t, p, f2(c1));
  return fma2(t, p, f2(c0));
}
__device__ __forceinline__ float2 lnhalf(float2 y) {  // ln(x/2) from y = x^2/4
  return mul2(make_float2(mufu::lg2(y.x), mufu::lg2(y.y)), f2(0.34657359027997264f));
}
__device__ __forceinline__ float2 k0_small(float2 x2) {
  const float2 t2 = mul2(x2, f2(1.0f / 14.0625f));
  const float2 i0 = poly6(t2, 1.0f, 3.5156229f, 3.0899424f, 1.2067492f, 0.2659732f, 0.0360768f, 0.0045813f);
  const float2 y = mul2(x2, f2(0.25f));
  const float2 lg = lnhalf(y);
  const float2 p = poly6(y, -0.57721566f, 0.42278420f, 0.23069756f, 0.03488590f, 0.00262698f, 0.00010750f, 0.0000074f);
  return fma2(make_float2(-lg.x, -lg.y), i0, p);
}
// e^-x x^-1/2 and 1/x from x^2
__device__ __forceinline__ void large_common(float2 x2, float2* e, float2* ix) {
  *ix = make_float2(mufu::rsqrt(x2.x), mufu::rsqrt(x2.y));
  const float2 x = mul2(x2, *ix);
  const float2 rx = make_float2(mufu::rsqrt(x.x), mufu::rsqrt(x.y));
  const float2 a = mul2(x, f2(-1.4426950408889634f));
  *e = mul2(make_float2(mufu::ex2(a.x), mufu::ex2(a.y)), rx);
}
__device__ __forceinline__ float2 k0_large(float2 x2) {
  float2 e, ix;
  large_common(x2, &e, &ix);
  const float2 y = add2(ix, ix);
  return mul2(e, poly6(y, 1.25331414f, -0.07832358f, 0.02189568f, -0.01062446f, 0.00587872f, -0.00251540f, 0.00053208f));
}
__device__ __forceinline__ float2 k0(float2 x2) {
  const bool sx = x2.x <= 4.0f, sy = x2.y <= 4.0f;
  if (sx && sy) return k0_small(x2);
  if (!sx && !sy) return k0_large(x2);
  const float2 a = k0_small(x2), b = k0_large(x2);
  return make_float2(sx ? a.x : b.x, sy ? a.y : b.y);
}
// K0 and K1/x
__device__ __forceinline__ void k01_small(float2 x2, float2* k0v, float2* k1ix) {
  const float2 t2 = mul2(x2, f2(1.0f / 14.0625f));
  const float2 i0 = poly6(t2, 1.0f, 3.5156229f, 3.0899424f, 1.2067492f, 0.2659732f, 0.0360768f, 0.0045813f);
  const float2 p1 = poly6(t2, 0.5f, 0.87890594f, 0.51498869f, 0.15084934f, 0.02658733f, 0.00301532f, 0.00032411f);
  const float2 y = mul2(x2, f2(0.25f));
  const float2 lg = lnhalf(y);
  const float2 p = poly6(y, -0.57721566f, 0.42278420f, 0.23069756f, 0.03488590f, 0.00262698f, 0.00010750f, 0.0000074f);
  *k0v = fma2(make_float2(-lg.x, -lg.y), i0, p);
  const float2 q1 = poly6(y, 1.0f, 0.15443144f, -0.67278579f, -0.18156897f, -0.01919402f, -0.00110404f, -0.00004686f);
  *k1ix = fma2(lg, p1, mul2(q1, make_float2(mufu::rcp(x2.x), mufu::rcp(x2.y))));
}
__device__ __forceinline__ void k01_large(float2 x2, float2* k0v, float2* k1ix) {
  float2 e, ix;
  large_common(x2, &e, &ix);
  const float2 y = add2(ix, ix);
  *k0v = mul2(e, poly6(y, 1.25331414f, -0.07832358f, 0.02189568f, -0.01062446f, 0.00587872f, -0.00251540f, 0.00053208f));
  *k1ix = mul2(mul2(e, ix),
               poly6(y, 1.25331414f, 0.23498619f, -0.03655620f, 0.01504268f, -0.00780353f, 0.00325614f, -0.00068245f));
}
__device__ __forceinline__ void k01(float2 x2, float2* k0v, float2* k1ix) {
  const bool sx = x2.x <= 4.0f, sy = x2.y <= 4.0f;
  if (sx && sy) { k01_small(x2, k0v, k1ix); return; }
  if (!sx && !sy) { k01_large(x2, k0v, k1ix); return; }
  float2 a0, a1, b0, b1;
  k01_small(x2, &a0, &a1);
  k01_large(x2, &b0, &b1);
  *k0v = make_float2(sx ? a0.x : b0.x, sy ? a0.y : b0.y);
  *k1ix = make_float2(sx ? a1.x : b1.x, sy ? a1.y : b1.y);
}
}  // namespace pk

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

// FP64 K0(x) and E(x) = K1(x)/x - 1/x^2: for x <= 2 from the series of k01d
// with the 1/x term of K1 left out (E = ln(x/2) I1(x)/x - S1/4), otherwise
// from k01d.
__device__ __forceinline__ void k0ed(double x, double* k0, double* e) {
  const double eg = 0.57721566490153286061;
  if (x <= 2.0) {
    double z = 0.25 * x * x;
    double tk = 1.0, t1 = 1.0, H = 0.0;
    double I0 = 0.0, S0 = 0.0, I1x = 0.0, S1 = 0.0;
    for (int k = 0; k < 30; ++k) {
      if (k > 0) {
        tk *= z / ((double)k * k);
        t1 *= z / ((double)k * (k + 1));
        H += 1.0 / k;
      }
      I0 += tk;
      S0 += H * tk;
      I1x += t1;
      S1 += (-2.0 * eg + 2.0 * H + 1.0 / (k + 1)) * t1;
    }
    I1x *= 0.5;  // I1(x) / x
    double lg = log(0.5 * x);
    *k0 = -(lg + eg) * I0 + S0;
    *e = lg * I1x - 0.25 * S1;
  } else {
    double k1;
    k01d(x, k0, &k1);
    *e = k1 / x - 1.0 / (x * x);
  }
}

}  // namespace bes
}  // namespace pfmm
