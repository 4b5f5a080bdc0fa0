// Point preparation and the direct far-field path (Sec. 6: P q = L (D (R q))).
//
//   k_prep_points : wrap + rotate points into the canonical cell (Sec. 1),
//                   FP64 and FP32 copies, fixed-point x/d phase
//   k_prep_q      : strengths in the canonical frame, FP64 compatibility
//                   moments sum q, sum |q|, sum q y' (Eq. chargeneutral,
//                   Eq. phis2 / Eq. pss0)
//   k_far_form    : coefficients c = R q for the south/north modes and the
//                   west/east quadrature nodes (Theorems south_thm, west_thm,
//                   south_thm_lap, west_thm_lap, south_thm_s, west_thm_s)
//   k_far_weights : lattice weights D (FP64), w = D c
//   k_far_eval    : u = Re(L w) at the targets (+ gradient / Stokes velocity)
//
// Modified Stokes (Theorems south_thm_ms, west_thm_ms) runs the three far
// kernels twice, once per plane-wave family (Far::msfam): the beta family
// (decay chi_m, kappa) and the Laplace family (|alpha_m|, |lambda|), each with
// two force channels and 2 x 2 blocks; the second pass adds to the first.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include "pfmm_impl.h"
#include "devmath.cuh"
#include "lattice_weights.cuh"
#include "multi.cuh"

namespace pfmm {

// ----------------------------------------------------------------------------
// K0: points
// ----------------------------------------------------------------------------
struct PtsArgs {
  Geom g;
  int64_t n, istride;
  const double* pts;
  double* c64;
  float* cf;
  int* U;
  int* status;
  int* V;
  double invY, xid;
};

__device__ __forceinline__ void k_prep_points_body(uint3 bid, const PtsArgs& A) {
  const Geom& g = A.g;
  const int64_t n = A.n, istride = A.istride;
  const double* __restrict__ pts = A.pts;
  double* __restrict__ c64 = A.c64;
  float* __restrict__ cf = A.cf;
  int* __restrict__ U = A.U;
  int* __restrict__ status = A.status;
  int* __restrict__ V = A.V;
  const double invY = A.invY, xid = A.xid;
  int64_t i = bid.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = pts[i], y = pts[istride + i];
  if (!isfinite(x) || !isfinite(y)) {
    atomicOr(status, ST_NONFINITE);
    x = 0.0;
    y = 0.0;
  }
  double xc = g.rot[0] * x + g.rot[1] * y, yc = g.rot[2] * x + g.rot[3] * y;
  double u1 = g.ainv[0] * xc + g.ainv[1] * yc, u2 = g.ainv[3] * yc;
  u1 -= floor(u1 + 0.5);
  if (!g.p1) {
    u2 -= floor(u2 + 0.5);
  } else if (!(u2 >= -0.5 && u2 < 0.5)) {
    // singly periodic: no wrap across the strip; the point is outside it
    atomicOr(status, ST_OUTSIDE);
    u2 = 0.0;
  }
  xc = u1 * g.d + u2 * g.xi;
  yc = u2 * g.eta;
  c64[i] = xc;
  c64[n + i] = yc;
  cf[i] = (float)xc;
  cf[n + i] = (float)yc;
  // x / d = u1 + u2 xi / d (no FP64 division)
  double v = fma(u2, xid, u1);
  v -= floor(v + 0.5);
  U[i] = (int)(unsigned)(long long)llrint(v * 4294967296.0);
  // singly periodic NUFFT: fixed-point phase 2^32 y / Y of the transform in y
  // (|y| < eta/2 = Y/4, so the signed value is exact to 2^-32 Y)
  if (V) V[i] = (int)llrint(yc * invY * 4294967296.0);
}
PFMM_CELL_KERNELS(k_prep_points, PtsArgs, )

// Optional projection to zero net charge / force: net sums per rhs and
// component (input frame) into mom[r*8 + 5 + c]; k_prep_q then subtracts the
// mean before using the strengths.
// part != NULL (deterministic mode): each warp writes its sums to
// part[warp][r * ncomp + c] instead of adding them to mom; k_ordered_sum adds
// them up in warp order afterwards.
struct NetArgs {
  int ncomp, nrhs;
  int64_t ns, qs;
  const double* q;
  double* mom;
  double* part;
};

__device__ __forceinline__ void k_net_body(uint3 bid, const NetArgs& A) {
  const int ncomp = A.ncomp, nrhs = A.nrhs;
  const int64_t ns = A.ns, qs = A.qs;
  const double* __restrict__ q = A.q;
  double* __restrict__ mom = A.mom;
  double* __restrict__ part = A.part;
  int64_t i = bid.x * (int64_t)blockDim.x + threadIdx.x;
  int lane = threadIdx.x & 31;
  const int64_t warp = i >> 5;
  for (int r = 0; r < nrhs; ++r)
    for (int c = 0; c < ncomp; ++c) {
      double v = (i < ns) ? q[((size_t)r * ncomp + c) * qs + i] : 0.0;
      if (!isfinite(v)) v = 0.0;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        if (part) part[(size_t)warp * nrhs * ncomp + r * ncomp + c] = v;
        else atomicAdd(mom + r * 8 + 5 + c, v);
      }
    }
}
PFMM_CELL_KERNELS(k_net, NetArgs, )

// out[(i / g) * ostride + i % g] += sum_{b < nb} part[b * m + i], i < m, in
// the order b = 0, 1, ... (the deterministic mode's fixed-order reduction of
// per-warp or per-block partial sums)
__global__ void k_ordered_sum(const double* __restrict__ part, int nb, int m, int g, int ostride,
                              double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * m + i];
  out[(size_t)(i / g) * ostride + i % g] += s;
}

// K0: strengths (canonical frame) and the moments per rhs:
//   mom[r*8+0] = sum q (Stokes: sum f_x), [1] = sum f_y, [2] = sum |q| (all comps), [3] = sum q y' (f_x y')
// The cancelling sums 0, 1 and 3 are FP64; sum |q| (only the scale of the
// neutrality test) is FP32.  Each thread sums kPrepPts points (a block covers
// kPrepPts * blockDim.x consecutive points, coalesced per step), so the warp
// reductions in FP64 (slow on this GPU) are amortised over several points.
constexpr int kPrepPts = 8;

__device__ __forceinline__ bool finite64(double v) {
  return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}

struct QArgs {
  Geom g;
  int ncomp, nrhs;
  int64_t ns, qs;
  const double* q;
  const double* src64;
  double* qc;
  float* qf;
  double* mom;
  int* status;
  int project;
  double* part;
};

__device__ __forceinline__ void k_prep_q_body(uint3 bid, const QArgs& A) {
  const Geom& g = A.g;
  const int ncomp = A.ncomp, nrhs = A.nrhs, project = A.project;
  const int64_t ns = A.ns, qs = A.qs;
  const double* __restrict__ q = A.q;
  const double* __restrict__ src64 = A.src64;
  double* __restrict__ qc = A.qc;
  float* __restrict__ qf = A.qf;
  double* __restrict__ mom = A.mom;
  int* __restrict__ status = A.status;
  double* __restrict__ part = A.part;
  const int64_t base = (int64_t)bid.x * blockDim.x * kPrepPts + threadIdx.x;
  const int64_t warp = ((int64_t)bid.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const double inv_ns = project ? 1.0 / (double)ns : 0.0;
  bool bad = false;
  for (int r = 0; r < nrhs; ++r) {
    const double mx = project ? mom[r * 8 + 5] * inv_ns : 0.0;
    const double my = (project && ncomp == 2) ? mom[r * 8 + 6] * inv_ns : 0.0;
    double v0 = 0.0, v1 = 0.0, v3 = 0.0;
    float v2 = 0.f;
#pragma unroll 2
    for (int k = 0; k < kPrepPts; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x;
      if (i >= ns) break;
      double a, b = 0.0;
      if (ncomp == 1) {
        a = q[(size_t)r * qs + i] - mx;
      } else {
        const double fx = q[((size_t)r * 2) * qs + i] - mx, fy = q[((size_t)r * 2 + 1) * qs + i] - my;
        a = g.rot[0] * fx + g.rot[1] * fy;
        b = g.rot[2] * fx + g.rot[3] * fy;
      }
      if (!finite64(a) || !finite64(b)) {
        bad = true;
        a = 0.0;
        b = 0.0;
      }
      const float af = (float)a, bf = (float)b;
      if (ncomp == 1) {
        if (qc) qc[(size_t)r * ns + i] = a;
        qf[(size_t)r * ns + i] = af;
      } else {
        qc[((size_t)r * 2) * ns + i] = a;
        qc[((size_t)r * 2 + 1) * ns + i] = b;
        qf[((size_t)r * 2) * ns + i] = af;
        qf[((size_t)r * 2 + 1) * ns + i] = bf;
        v1 += b;
      }
      v0 += a;
      v3 = fma(a, src64[ns + i], v3);
      v2 += fabsf(af) + fabsf(bf);
    }
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_down_sync(0xffffffffu, v0, o);
      if (ncomp == 2) v1 += __shfl_down_sync(0xffffffffu, v1, o);
      v2 += __shfl_down_sync(0xffffffffu, v2, o);
      v3 += __shfl_down_sync(0xffffffffu, v3, o);
    }
    if (lane == 0) {
      if (part) {  // deterministic mode: part[warp][r * 4 + k]
        double* w = part + ((size_t)warp * nrhs + r) * 4;
        w[0] = v0;
        w[1] = v1;
        w[2] = (double)v2;
        w[3] = v3;
      } else {
        atomicAdd(mom + r * 8 + 0, v0);
        if (ncomp == 2) atomicAdd(mom + r * 8 + 1, v1);
        atomicAdd(mom + r * 8 + 2, (double)v2);
        atomicAdd(mom + r * 8 + 3, v3);
      }
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}
PFMM_CELL_KERNELS(k_prep_q, QArgs, )

// ----------------------------------------------------------------------------
// term decoding.  Term list: [south m_lo..M | north m_lo..M | west 0..Nq-1 | east 0..Nq-1]
// part: 0 S, 1 N, 2 W, 3 E.  For S/N: a = alpha_m, b = chi_m, m.  W/E: a = lambda, b = kappa.
// ----------------------------------------------------------------------------
struct Term {
  int part, m;
  double a, b, w;
};

// plane waves with decay sqrt(a^2 + beta^2) (modified Helmholtz, the modified
// Stokes beta family) or |a| (Laplace, Stokes, the modified Stokes Laplace family)
__device__ __forceinline__ bool decays_beta(const Far& f) {
  return f.kernel == PFMM_MODHELM || (f.kernel == PFMM_MSTOKES && f.msfam == 0);
}

__device__ __forceinline__ Term decode_term(const Far& f, const Geom& g, int t) {
  Term T;
  int mlo = f.mode0 ? 0 : 1;
  if (t < 2 * f.nsn) {
    T.part = t < f.nsn ? 0 : 1;
    T.m = (t < f.nsn ? t : t - f.nsn) + mlo;
    T.a = 2.0 * M_PI * T.m / g.d;
    T.b = decays_beta(f) ? sqrt(T.a * T.a + f.beta * f.beta) : fabs(T.a);
    T.w = 0;
  } else {
    int n = t - 2 * f.nsn;
    T.part = n < f.Nq ? 2 : 3;
    if (n >= f.Nq) n -= f.Nq;
    T.m = n;
    T.a = f.nodes[2 * n];
    T.w = f.nodes[2 * n + 1];
    T.b = decays_beta(f) ? sqrt(T.a * T.a + f.beta * f.beta) : T.a;
  }
  return T;
}

// The same decoding in FP32 for the mixed kernels (no FP64 division or
// square root per term): alpha_m = m (2 pi / d), decays from an FP32 square
// root.  The south/north phases of the mixed path come from the fixed-point
// phase, so alpha_m enters only the gradient factors.
struct TermF {
  int part, m;
  float a, b;
};
__device__ __forceinline__ TermF decode_term_f(const Far& f, int t) {
  TermF T;
  const int mlo = f.mode0 ? 0 : 1;
  const float b2 = f.beta_f * f.beta_f;
  if (t < 2 * f.nsn) {
    T.part = t < f.nsn ? 0 : 1;
    T.m = (t < f.nsn ? t : t - f.nsn) + mlo;
    T.a = (float)T.m * f.alpha1f;
    T.b = decays_beta(f) ? sqrtf(fmaf(T.a, T.a, b2)) : fabsf(T.a);
  } else {
    int n = t - 2 * f.nsn;
    T.part = n < f.Nq ? 2 : 3;
    if (n >= f.Nq) n -= f.Nq;
    T.m = n;
    T.a = __double2float_rn(f.nodes[2 * n]);
    T.b = decays_beta(f) ? sqrtf(fmaf(T.a, T.a, b2)) : T.a;
  }
  return T;
}

// FP64 value of a kernel-precision number (FP32: the integer-pipe conversion)
__device__ __forceinline__ double to_d(float v) { return dm::f2d(v); }
__device__ __forceinline__ double to_d(double v) { return v; }

// ----------------------------------------------------------------------------
// K1: coefficient formation.  grid (chunks, term blocks, rhs groups).
// coef layout [nrhs][nch][nterm] complex double; Stokes channels:
//   0,1: c_a = sum R f (x, y comps)    (W/E: R - 1)
//   2,3: c_b = sum R coord f           (coord = y' for S/N, x~' for W/E: the west/east frame)
// ----------------------------------------------------------------------------
constexpr int kFormThreads = 128;
constexpr int kFormSub = 64;
constexpr int kRB = 4;  // rhs per block (FP64 path, Stokes kernels)
// rhs per block: 8 for the FP32 scalar kernels (one plane wave serves all 8)
template <typename T, int KER>
constexpr int rb_of() {
  return (sizeof(T) == 4 && (KER == PFMM_LAPLACE || KER == PFMM_MODHELM)) ? 8 : kRB;
}

template <typename T>
struct FormArgs {
  Far f;
  Geom g;
  int ns, chunk;
  const T* sx;
  const T* sy;
  const int* sU;
  const T* qv;
  double* coef;
  double* part;
};

template <typename T, int KER>
__device__ __forceinline__ void k_far_form_body(uint3 bid, const FormArgs<T>& A) {
  const Far& f = A.f;
  const Geom& g = A.g;
  const int ns = A.ns, chunk = A.chunk;
  const T* __restrict__ sx = A.sx;
  const T* __restrict__ sy = A.sy;
  const int* __restrict__ sU = A.sU;
  const T* __restrict__ qv = A.qv;
  double* __restrict__ coef = A.coef;
  double* __restrict__ part = A.part;
  constexpr int NC = (KER == PFMM_STOKES || KER == PFMM_MSTOKES) ? 2 : 1;
  constexpr int NCH = (KER == PFMM_STOKES) ? 4 : NC;
  __shared__ T s_x[kFormSub], s_y[kFormSub];
  __shared__ T s_xw[kFormSub], s_yw[kFormSub];  // west/east frame coordinates
  __shared__ int s_U[kFormSub];
  constexpr int RB = rb_of<T, KER>();
  __shared__ T s_q[RB][NC][kFormSub];

  const int t = bid.y * kFormThreads + threadIdx.x;
  const bool active = t < f.nterm;
  const int r0 = bid.z * RB;
  const int nr = min(RB, f.nrhs - r0);
  int tpart, tmm;
  T a, b;
  double inv_d = 0.0;
  if constexpr (sizeof(T) == 4) {
    const TermF tf = decode_term_f(f, active ? t : 0);
    tpart = tf.part;
    tmm = tf.m;
    a = tf.a;
    b = tf.b;
  } else {
    const Term tm = decode_term(f, g, active ? t : 0);
    tpart = tm.part;
    tmm = tm.m;
    a = (T)tm.a;
    b = (T)tm.b;
    inv_d = 1.0 / g.d;
  }
  const T sgn = (tpart == 0 || tpart == 2) ? T(1) : T(-1);
  const bool sn = tpart < 2;
  const bool we_m1 = !sn && (KER == PFMM_LAPLACE || KER == PFMM_STOKES);

  double acc[RB][NCH][2];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int c = 0; c < NCH; ++c) acc[r][c][0] = acc[r][c][1] = 0.0;

  const int j0 = bid.x * chunk;
  const int j1 = min(ns, j0 + chunk);
  for (int jb = j0; jb < j1; jb += kFormSub) {
    const int nb = min(kFormSub, j1 - jb);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += kFormThreads) {
      const T x = sx[jb + k], y = sy[jb + k];
      s_x[k] = x;
      s_y[k] = y;
      s_xw[k] = T(g.wc) * x - T(g.ws) * y;
      s_yw[k] = T(g.ws) * x + T(g.wc) * y;
      s_U[k] = sU ? sU[jb + k] : 0;
    }
    for (int k = threadIdx.x; k < RB * NC * kFormSub; k += kFormThreads) {
      int r = k / (NC * kFormSub), rem = k % (NC * kFormSub), c = rem / kFormSub, jj = rem % kFormSub;
      s_q[r][c][jj] = (r < nr && jj < nb) ? qv[((size_t)(r0 + r) * NC + c) * ns + jb + jj] : T(0);
    }
    __syncthreads();
    if (!active) continue;
    T sub[RB][NCH][2];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < NCH; ++c) sub[r][c][0] = sub[r][c][1] = T(0);
    for (int jj = 0; jj < nb; ++jj) {
      // south/north: canonical (x, y); west/east: the west/east frame
      const T x = sn ? s_x[jj] : s_xw[jj], y = sn ? s_y[jj] : s_yw[jj];
      T Rr, Ri, Qr, Qi;  // R (for c_b / plain) and Q (for c_a: R or R - 1)
      if (sn) {
        T e, sp, cp;
        if constexpr (sizeof(T) == 4) {
          e = dm::ex_fast(sgn * b * y);
          dm::sincos_turns((unsigned)tmm * (unsigned)s_U[jj], &sp, &cp);
        } else {
          e = dm::ex(sgn * b * y);
          dm::sincospi_(T(2.0 * tmm * ((double)x * inv_d)), &sp, &cp);
        }
        Rr = e * cp;
        Ri = -e * sp;
        Qr = Rr;
        Qi = Ri;
      } else {
        if (we_m1) {
          if constexpr (sizeof(T) == 4)
            dm::expm1c_fast(sgn * b * x, -a * y, &Qr, &Qi);
          else
            dm::expm1c(sgn * b * x, -a * y, &Qr, &Qi);
          Rr = Qr + T(1);
          Ri = Qi;
        } else {
          T e, sp, cp;
          if constexpr (sizeof(T) == 4) {
            e = dm::ex_fast(sgn * b * x);
            dm::sincos_red(a * y, &sp, &cp);
          } else {
            e = dm::ex(sgn * b * x);
            dm::sincos_(a * y, &sp, &cp);
          }
          Rr = e * cp;
          Ri = -e * sp;
          Qr = Rr;
          Qi = Ri;
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (NC == 1) {
          const T s = s_q[r][0][jj];
          sub[r][0][0] += Qr * s;
          sub[r][0][1] += Qi * s;
        } else if (KER == PFMM_MSTOKES) {
          const T fx = s_q[r][0][jj], fy = s_q[r][1][jj];
          sub[r][0][0] += Qr * fx;
          sub[r][0][1] += Qi * fx;
          sub[r][NCH - 1][0] += Qr * fy;
          sub[r][NCH - 1][1] += Qi * fy;
        } else {
          const T fx = s_q[r][0][jj], fy = s_q[r][1][jj];
          const T cd = sn ? y : x;
          const T Br = Rr * cd, Bi = Ri * cd;
          sub[r][0][0] += Qr * fx;
          sub[r][0][1] += Qi * fx;
          sub[r][1][0] += Qr * fy;
          sub[r][1][1] += Qi * fy;
          sub[r][NCH - 2][0] += Br * fx;
          sub[r][NCH - 2][1] += Bi * fx;
          sub[r][NCH - 1][0] += Br * fy;
          sub[r][NCH - 1][1] += Bi * fy;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        acc[r][c][0] += to_d(sub[r][c][0]);
        acc[r][c][1] += to_d(sub[r][c][1]);
      }
  }
  if (!active) return;
  // deterministic mode: this source chunk's sums go to part[chunk][...] (same
  // layout as coef), added in chunk order by k_ordered_sum
  double* base = part ? part + (size_t)bid.x * f.nrhs * NCH * f.nterm * 2 : coef;
  for (int r = 0; r < nr; ++r)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      double* dst = base + (((size_t)(r0 + r) * NCH + c) * f.nterm + t) * 2;
      if (part) {
        dst[0] = acc[r][c][0];
        dst[1] = acc[r][c][1];
      } else {
        atomicAdd(dst, acc[r][c][0]);
        atomicAdd(dst + 1, acc[r][c][1]);
      }
    }
}

template <typename T, int KER>
__global__ void __launch_bounds__(kFormThreads) k_far_form(const __grid_constant__ FormArgs<T> A) {
  k_far_form_body<T, KER>(blockIdx, A);
}
template <typename T, int KER>
__global__ void __launch_bounds__(kFormThreads) k_far_form_multi(const FormArgs<T>* __restrict__ cells,
                                                                 const int* __restrict__ off,
                                                                 const uint3* __restrict__ dims, int n) {
  const SubBlock s = sub_block(off, dims, n);
  k_far_form_body<T, KER>(s.bid, cells[s.cell]);
}

// ----------------------------------------------------------------------------
// K2: weights.  One thread per (term, rhs).  FP64.
//   scalar: W (1 complex)          u += Re(L W)   (Laplace W/E: Re((L-1) W))
//   Stokes: Wa[2], Wb[2]           u_k += Re(L Wa_k) + coord Re(L Wb_k)   (W/E: (L-1) Wa)
// mom[r*8+4] = c0: Laplace: -(1/(d eta)) sum q y' (m = 0 of south + north, Eq. phis3),
//        Stokes: -(1/(d eta)) sum f_x y' (Eq. pss0); added as c0 * y.
// ----------------------------------------------------------------------------
template <typename T2>
__device__ __forceinline__ void store_w(T2* p, dcx v) {
  p->x = v.r;
  p->y = v.i;
}

template <typename T2>
struct WArgs {
  Far f;
  Geom g;
  const double* coef;
  double* mom;
  T2* wts;
  int* status;
};

template <typename T2>
__device__ __forceinline__ void k_far_weights_body(uint3 bid, const WArgs<T2>& A) {
  const Far& f = A.f;
  const Geom& g = A.g;
  const double* __restrict__ coef = A.coef;
  double* __restrict__ mom = A.mom;
  T2* __restrict__ wts = A.wts;
  int* __restrict__ status = A.status;
  int t = bid.x * blockDim.x + threadIdx.x;
  int r = bid.y;
  const int K = f.kernel;
  if (t == 0) {
    double mq = mom[r * 8 + 0], mfy = mom[r * 8 + 1], mabs = mom[r * 8 + 2], my = mom[r * 8 + 3];
    if (K == PFMM_LAPLACE || K == PFMM_STOKES) {
      double net = (K == PFMM_STOKES) ? fmax(fabs(mq), fabs(mfy)) : fabs(mq);
      if (net > 1e-8 * mabs + 1e-300) atomicOr(status, ST_NOT_NEUTRAL);
      // the m = 0 mode of the south/north parts; none in the singly periodic case
      mom[r * 8 + 4] = f.rows3 ? -my / (g.d * g.eta) : 0.0;
    } else {
      mom[r * 8 + 4] = 0.0;
    }
  }
  if (t >= f.nterm) return;
  Term tm = decode_term(f, g, t);
  const double d = g.d, xi = g.xi, eta = g.eta;
  const lw::WeFrame fr{g.wdx, g.wdy, g.wxr, g.wyr};
  const int nch = f.nch;
  auto C = [&](int c) {
    const double* p = coef + (((size_t)r * nch + c) * f.nterm + t) * 2;
    return dcx{p[0], p[1]};
  };
  const bool north = tm.part == 1, east = tm.part == 3;
  if (K == PFMM_MSTOKES) {
    dcx D[2][2];
    double fac = 1.0;
    if (tm.part < 2) {
      lw::ms_sn(d, xi, eta, tm.a, tm.b, f.beta, f.msfam, north, D);
      fac = (tm.m == 0) ? 1.0 : 2.0;  // +-m pairs
    } else {
      lw::ms_we(fr, g.wc, g.ws, g.m0, tm.a, tm.b, tm.w, f.beta, f.msfam, east, D);
    }
    const dcx c[2] = {C(0), C(1)};
    for (int i = 0; i < 2; ++i)
      store_w(wts + (((size_t)r * 2 + i) * f.nterm + t), cscale(cadd(cmul(D[i][0], c[0]), cmul(D[i][1], c[1])), fac));
    return;
  }
  if (K != PFMM_STOKES) {
    dcx D;
    double fac = 1.0;
    if (tm.part < 2) {
      D = lw::sn_scalar(d, xi, eta, tm.a, tm.b, north);
      fac = (tm.m == 0) ? 1.0 : 2.0;  // +-m pairs
    } else {
      D = lw::we_scalar(fr, g.m0, tm.a, tm.b, tm.w, east, f.rows3 != 0);
    }
    store_w(wts + (size_t)r * f.nterm + t, cscale(cmul(D, C(0)), fac));
    return;
  }
  dcx Da[2][2], Db[2][2];
  if (tm.part < 2)
    lw::sn_stokes(d, xi, eta, tm.a, north, Da, Db);
  else
    lw::we_stokes(fr, g.wc, g.ws, g.m0, tm.a, tm.w, east, Da, Db, f.rows3 != 0);
  const dcx ca[2] = {C(0), C(1)}, cb[2] = {C(2), C(3)};
  dcx wa[2], wb[2];
  lw::stokes_apply(Da, Db, ca, cb, north || east, (tm.part < 2) ? 2.0 : 1.0, wa, wb);
  for (int i = 0; i < 2; ++i) {
    store_w(wts + (((size_t)r * 4 + i) * f.nterm + t), wa[i]);
    store_w(wts + (((size_t)r * 4 + 2 + i) * f.nterm + t), wb[i]);
  }
}

template <typename T2>
__global__ void k_far_weights(const __grid_constant__ WArgs<T2> A) {
  k_far_weights_body<T2>(blockIdx, A);
}
template <typename T2>
__global__ void k_far_weights_multi(const WArgs<T2>* __restrict__ cells, const int* __restrict__ off,
                                    const uint3* __restrict__ dims, int n) {
  const SubBlock s = sub_block(off, dims, n);
  k_far_weights_body<T2>(s.bid, cells[s.cell]);
}

// ----------------------------------------------------------------------------
// K3: evaluation at targets.  grid (target blocks, rhs groups); terms staged
// in shared memory in chunks.
// ----------------------------------------------------------------------------
constexpr int kEvalThreads = 128;
constexpr int kEvalChunk = 64;

template <typename T, typename T2>
struct EvalArgs {
  Far f;
  Geom g;
  int nt;
  const T* tx;
  const T* ty;
  const int* tU;
  const T2* wts;
  const double* mom;
  int64_t os;
  double* pot;
  double* grad;
  int accum;
};

template <typename T, typename T2, int KER>
__device__ __forceinline__ void k_far_eval_body64(uint3 bid, const EvalArgs<T, T2>& A) {
  const Far& f = A.f;
  const Geom& g = A.g;
  const int nt = A.nt, accum = A.accum;
  const T* __restrict__ tx = A.tx;
  const T* __restrict__ ty = A.ty;
  const int* __restrict__ tU = A.tU;
  const T2* __restrict__ wts = A.wts;
  const double* __restrict__ mom = A.mom;
  const int64_t os = A.os;
  double* __restrict__ pot = A.pot;
  double* __restrict__ grad = A.grad;
  constexpr bool VEC = KER == PFMM_STOKES || KER == PFMM_MSTOKES;
  constexpr int NW = (KER == PFMM_STOKES) ? 4 : (KER == PFMM_MSTOKES ? 2 : 1);
  __shared__ T s_a[kEvalChunk], s_b[kEvalChunk];
  __shared__ int s_m[kEvalChunk], s_part[kEvalChunk];
  __shared__ T2 s_w[kRB][NW][kEvalChunk];
  const int l = bid.x * kEvalThreads + threadIdx.x;
  const bool in = l < nt;
  const int r0 = bid.y * kRB;
  const int nr = min(kRB, f.nrhs - r0);
  const T x = in ? tx[l] : T(0), y = in ? ty[l] : T(0);
  // west/east frame coordinates; its gradient is rotated back per term
  const T wc = T(g.wc), ws = T(g.ws);
  const T xw = wc * x - ws * y, yw = ws * x + wc * y;
  const int U = (in && tU) ? tU[l] : 0;
  const double xd = (sizeof(T) == 8 && in) ? (double)x / g.d : 0.0;  // FP64 path's phase
  // accumulators: scalar [pot, gx, gy]; Stokes [ux, uy].  Compensated in FP32:
  // a few hundred terms of the size of the result are summed per target.
  constexpr int NA = VEC ? 2 : 3;
  dm::KSum<T> acc[kRB][NA];

  for (int t0 = 0; t0 < f.nterm; t0 += kEvalChunk) {
    const int nc = min(kEvalChunk, f.nterm - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += kEvalThreads) {
      if constexpr (sizeof(T) == 4) {
        const TermF tm = decode_term_f(f, t0 + k);
        s_a[k] = tm.a;
        s_b[k] = tm.b;
        s_m[k] = tm.m;
        s_part[k] = tm.part;
      } else {
        const Term tm = decode_term(f, g, t0 + k);
        s_a[k] = (T)tm.a;
        s_b[k] = (T)tm.b;
        s_m[k] = tm.m;
        s_part[k] = tm.part;
      }
    }
    for (int k = threadIdx.x; k < kRB * NW * kEvalChunk; k += kEvalThreads) {
      int r = k / (NW * kEvalChunk), rem = k % (NW * kEvalChunk), c = rem / kEvalChunk, tt = rem % kEvalChunk;
      T2 v;
      v.x = T(0);
      v.y = T(0);
      if (r < nr && tt < nc) v = wts[((size_t)(r0 + r) * NW + c) * f.nterm + t0 + tt];
      s_w[r][c][tt] = v;
    }
    __syncthreads();
    if (!in) continue;
    for (int k = 0; k < nc; ++k) {
      const int part = s_part[k];
      const T a = s_a[k], b = s_b[k];
      T Lr, Li, Mr, Mi;  // L and the potential factor (L - 1 for Laplace/Stokes W/E)
      if (part < 2) {
        const T sy = part == 0 ? T(1) : T(-1);
        T e = dm::ex(-sy * b * y);
        T sp, cp;
        if constexpr (sizeof(T) == 4)
          dm::phase_fixed(s_m[k], U, &sp, &cp);
        else
          dm::sincospi_(T(2.0 * s_m[k] * xd), &sp, &cp);
        Lr = e * cp;
        Li = e * sp;
        Mr = Lr;
        Mi = Li;
      } else {
        const T sx = part == 2 ? T(1) : T(-1);
        if (KER == PFMM_LAPLACE || KER == PFMM_STOKES) {
          dm::expm1c(-sx * b * xw, a * yw, &Mr, &Mi);
          Lr = Mr + T(1);
          Li = Mi;
        } else {
          T e = dm::ex(-sx * b * xw);
          T sp, cp;
          dm::sincos_(a * yw, &sp, &cp);
          Lr = e * cp;
          Li = e * sp;
          Mr = Lr;
          Mi = Li;
        }
      }
#pragma unroll
      for (int r = 0; r < kRB; ++r) {
        if (KER == PFMM_MSTOKES) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const T2 w = s_w[r][c][k];
            acc[r][c].add(Lr * w.x - Li * w.y);
          }
        } else if (KER != PFMM_STOKES) {
          const T2 w = s_w[r][0][k];
          const T Pr = Lr * w.x - Li * w.y, Pi = Lr * w.y + Li * w.x;
          acc[r][0].add(Mr * w.x - Mi * w.y);
          if (part < 2) {
            acc[r][1].add(-a * Pi);
            acc[r][2].add(-(part == 0 ? b : -b) * Pr);
          } else {
            const T gx = -(part == 2 ? b : -b) * Pr, gy = -a * Pi;  // in the west/east frame
            acc[r][1].add(wc * gx + ws * gy);
            acc[r][2].add(wc * gy - ws * gx);
          }
        } else {
          const T cd = part < 2 ? y : xw;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const T2 wa = s_w[r][c][k], wb = s_w[r][2 + c][k];
            acc[r][c].add((Mr * wa.x - Mi * wa.y) + cd * (Lr * wb.x - Li * wb.y));
          }
        }
      }
    }
  }
  if (!in) return;
  const double* R = g.rot;  // input = rot^T canonical
  const double yd = to_d(y);
  for (int r = 0; r < nr; ++r) {
    const double cc = mom[(r0 + r) * 8 + 4];
    if (VEC) {
      double ux = acc[r][0].value() + cc * yd, uy = acc[r][1].value();
      double* px = pot + ((size_t)(r0 + r) * 2) * os + l;
      double* py = pot + ((size_t)(r0 + r) * 2 + 1) * os + l;
      *px = (accum ? *px : 0.0) + R[0] * ux + R[2] * uy;
      *py = (accum ? *py : 0.0) + R[1] * ux + R[3] * uy;
    } else {
      double p = acc[r][0].value();
      if (cc != 0.0) p += cc * yd;
      if (pot) pot[(size_t)(r0 + r) * os + l] = p;
      if (grad) {
        const double gx = acc[r][1].value(), gy = acc[r][2].value() + cc;
        grad[((size_t)(r0 + r) * 2) * os + l] = R[0] * gx + R[2] * gy;
        grad[((size_t)(r0 + r) * 2 + 1) * os + l] = R[1] * gx + R[3] * gy;
      }
    }
  }
}

// FP32 evaluation (mixed path).  Per (target, term): the plane wave from one
// MUFU exponential and the FMA-pipe sine/cosine (the south/north phase from
// the fixed-point coordinate, exact range reduction), then per rhs the real
// part of L w; RB right-hand sides per block (8 for the scalar kernels, so
// that each plane wave serves all of them), the gradient only when asked
// for (GRAD).  Terms are summed in FP32 over groups of kEvalGroup and the
// group sums added with Kahan compensation.  Term data are staged once per
// chunk as (a, b, m, part) in shared memory.
constexpr int kEvalGroup = 16;

template <typename T2, int KER, bool GRAD>
__device__ __forceinline__ void k_far_eval_body32(uint3 bid, const EvalArgs<float, T2>& A) {
  using T = float;
  const Far& f = A.f;
  const Geom& g = A.g;
  const int nt = A.nt, accum = A.accum;
  const int64_t os = A.os;
  constexpr bool VEC = KER == PFMM_STOKES || KER == PFMM_MSTOKES;
  constexpr int NW = (KER == PFMM_STOKES) ? 4 : (KER == PFMM_MSTOKES ? 2 : 1);
  constexpr int RB = rb_of<T, KER>();
  // accumulators: scalar [pot, gx, gy] (gradient only with GRAD); Stokes [ux, uy]
  constexpr int NA = VEC ? 2 : (GRAD ? 3 : 1);
  __shared__ float4 s_t[kEvalChunk];  // a, b, m (int bits), part (int bits)
  __shared__ T2 s_w[RB][NW][kEvalChunk];
  const int l = bid.x * kEvalThreads + threadIdx.x;
  const bool in = l < nt;
  const int r0 = bid.y * RB;
  const int nr = min(RB, f.nrhs - r0);
  const T x = in ? A.tx[l] : T(0), y = in ? A.ty[l] : T(0);
  const T wc = T(g.wc), ws = T(g.ws);
  const T xw = wc * x - ws * y, yw = ws * x + wc * y;
  const unsigned U = (in && A.tU) ? (unsigned)A.tU[l] : 0u;
  dm::KSum<T> acc[RB][NA];
  T sum[RB][NA];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int c = 0; c < NA; ++c) sum[r][c] = T(0);

  for (int t0 = 0; t0 < f.nterm; t0 += kEvalChunk) {
    const int nc = min(kEvalChunk, f.nterm - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += kEvalThreads) {
      const TermF tm = decode_term_f(f, t0 + k);
      s_t[k] = make_float4(tm.a, tm.b, __int_as_float(tm.m), __int_as_float(tm.part));
    }
    for (int k = threadIdx.x; k < RB * NW * kEvalChunk; k += kEvalThreads) {
      const int r = k / (NW * kEvalChunk), rem = k % (NW * kEvalChunk), c = rem / kEvalChunk, tt = rem % kEvalChunk;
      T2 v;
      v.x = T(0);
      v.y = T(0);
      if (r < nr && tt < nc) v = A.wts[((size_t)(r0 + r) * NW + c) * f.nterm + t0 + tt];
      s_w[r][c][tt] = v;
    }
    __syncthreads();
    if (!in) continue;
    for (int k = 0; k < nc; ++k) {
      const float4 tm = s_t[k];
      const int part = __float_as_int(tm.w);
      const T a = tm.x, b = tm.y;
      T Lr, Li, Mr, Mi;  // L and the potential factor (L - 1 for Laplace/Stokes W/E)
      if (part < 2) {
        const T e = dm::ex_fast(part == 0 ? -b * y : b * y);
        T sp, cp;
        dm::sincos_turns((unsigned)__float_as_int(tm.z) * U, &sp, &cp);
        Lr = e * cp;
        Li = e * sp;
        Mr = Lr;
        Mi = Li;
      } else {
        const T sx = part == 2 ? T(1) : T(-1);
        if (KER == PFMM_LAPLACE || KER == PFMM_STOKES) {
          // e^{-sx b xw + i a yw} - 1 without cancellation
          const T em = expm1f(-sx * b * xw);
          T sh, ch;
          dm::sincos_red(T(0.5) * a * yw, &sh, &ch);
          const T s2 = T(2) * sh * sh;
          Mr = em * (T(1) - s2) - s2;
          Mi = (em + T(1)) * (T(2) * sh * ch);
          Lr = Mr + T(1);
          Li = Mi;
        } else {
          const T e = dm::ex_fast(-sx * b * xw);
          T sp, cp;
          dm::sincos_red(a * yw, &sp, &cp);
          Lr = e * cp;
          Li = e * sp;
          Mr = Lr;
          Mi = Li;
        }
      }
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (KER == PFMM_MSTOKES) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const T2 w = s_w[r][c][k];
            sum[r][c] = fmaf(Lr, w.x, fmaf(-Li, w.y, sum[r][c]));
          }
        } else if (KER != PFMM_STOKES) {
          const T2 w = s_w[r][0][k];
          sum[r][0] = fmaf(Mr, w.x, fmaf(-Mi, w.y, sum[r][0]));
          if (GRAD) {
            const T Pr = Lr * w.x - Li * w.y, Pi = Lr * w.y + Li * w.x;
            if (part < 2) {
              sum[r][1 % NA] = fmaf(-a, Pi, sum[r][1 % NA]);
              sum[r][2 % NA] = fmaf(-(part == 0 ? b : -b), Pr, sum[r][2 % NA]);
            } else {
              const T gx = -(part == 2 ? b : -b) * Pr, gy = -a * Pi;  // in the west/east frame
              sum[r][1 % NA] += wc * gx + ws * gy;
              sum[r][2 % NA] += wc * gy - ws * gx;
            }
          }
        } else {
          const T cd = part < 2 ? y : xw;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const T2 wa = s_w[r][c][k], wb = s_w[r][2 + c][k];
            sum[r][c] += (Mr * wa.x - Mi * wa.y) + cd * (Lr * wb.x - Li * wb.y);
          }
        }
      }
      if ((k & (kEvalGroup - 1)) == kEvalGroup - 1 || k == nc - 1) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int c = 0; c < NA; ++c) {
            acc[r][c].add(sum[r][c]);
            sum[r][c] = T(0);
          }
      }
    }
  }
  if (!in) return;
  const double* R = g.rot;  // input = rot^T canonical
  const double yd = dm::f2d(y);
  for (int r = 0; r < nr; ++r) {
    const double cc = A.mom[(r0 + r) * 8 + 4];
    if (VEC) {
      double ux = acc[r][0].value(), uy = acc[r][1 % NA].value();
      if (cc != 0.0) ux += cc * yd;
      double* px = A.pot + ((size_t)(r0 + r) * 2) * os + l;
      double* py = A.pot + ((size_t)(r0 + r) * 2 + 1) * os + l;
      *px = (accum ? *px : 0.0) + R[0] * ux + R[2] * uy;
      *py = (accum ? *py : 0.0) + R[1] * ux + R[3] * uy;
    } else {
      double p = acc[r][0].value();
      if (cc != 0.0) p += cc * yd;
      if (A.pot) A.pot[(size_t)(r0 + r) * os + l] = p;
      if (GRAD && A.grad) {
        const double gx = acc[r][1 % NA].value(), gy = acc[r][2 % NA].value() + cc;
        A.grad[((size_t)(r0 + r) * 2) * os + l] = R[0] * gx + R[2] * gy;
        A.grad[((size_t)(r0 + r) * 2 + 1) * os + l] = R[1] * gx + R[3] * gy;
      }
    }
  }
}

template <typename T, typename T2, int KER, bool GRAD>
__device__ __forceinline__ void k_far_eval_body(uint3 bid, const EvalArgs<T, T2>& A) {
  if constexpr (sizeof(T) == 4)
    k_far_eval_body32<T2, KER, GRAD>(bid, A);
  else
    k_far_eval_body64<T, T2, KER>(bid, A);
}

template <typename T, typename T2, int KER, bool GRAD>
__global__ void __launch_bounds__(kEvalThreads) k_far_eval(const __grid_constant__ EvalArgs<T, T2> A) {
  k_far_eval_body<T, T2, KER, GRAD>(blockIdx, A);
}
template <typename T, typename T2, int KER, bool GRAD>
__global__ void __launch_bounds__(kEvalThreads) k_far_eval_multi(const EvalArgs<T, T2>* __restrict__ cells,
                                                                 const int* __restrict__ off,
                                                                 const uint3* __restrict__ dims, int n) {
  const SubBlock s = sub_block(off, dims, n);
  k_far_eval_body<T, T2, KER, GRAD>(s.bid, cells[s.cell]);
}

// memsets of 8-byte words (multi-cell zeroing)
__device__ __forceinline__ void k_zero_body(uint3 bid, const ZeroArgs& A) {
  const long long i = (long long)bid.x * 256 + threadIdx.x;
  if (i < A.n) A.p[i] = 0ull;
}
PFMM_CELL_KERNELS(k_zero, ZeroArgs, __launch_bounds__(256))

cudaError_t zero_or_record(void* p, size_t bytes, cudaStream_t st) {
  if (!g_rec) return bytes ? cudaMemsetAsync(p, 0, bytes, st) : cudaSuccess;
  if ((bytes & 7) || (reinterpret_cast<uintptr_t>(p) & 7)) return cudaErrorInvalidValue;
  const ZeroArgs a{(unsigned long long*)p, (long long)(bytes / 8)};
  return launch_or_record(k_zero, k_zero_multi, PH_ZERO, dim3((unsigned)((a.n + 255) / 256)), 256, 0, st, a);
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
static inline int cdiv_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

cudaError_t launch_prep(const pfmm_plan* p, char* ws, int64_t ns, const double* src, const double* q, int64_t nt,
                        const double* trg, bool self, cudaStream_t st) {
  const Layout& L = p->lay;
  int* status = (int*)(ws + L.status);
  const bool wantV = p->p1_nu && p->path == PFMM_PATH_NUFFT;
  const double invY = p->p1_nu ? 1.0 / p->p1_Y : 0.0;
  const double xid = p->geom.xi / p->geom.d;
  cudaError_t e;
  {
    const PtsArgs a{p->geom, ns, p->s_stride, src, (double*)(ws + L.src64), (float*)(ws + L.srcf),
                    (int*)(ws + L.srcU), status, wantV ? (int*)(ws + L.srcV) : nullptr, invY, xid};
    e = launch_or_record(k_prep_points, k_prep_points_multi, PH_PTS, dim3(cdiv_i(ns, 256)), 256, 0, st, a);
    if (e != cudaSuccess) return e;
  }
  if (!self && nt > 0) {
    const PtsArgs a{p->geom, nt, p->t_stride, trg, (double*)(ws + L.trg64), (float*)(ws + L.trgf),
                    (int*)(ws + L.trgU), status, wantV ? (int*)(ws + L.trgV) : nullptr, invY, xid};
    e = launch_or_record(k_prep_points, k_prep_points_multi, PH_PTS, dim3(cdiv_i(nt, 256)), 256, 0, st, a);
    if (e != cudaSuccess) return e;
  }
  g_launches = (!self && nt > 0) ? 3 : 2;
  const int project = (p->opts.flags & PFMM_PROJECT_NEUTRAL) &&
                      (p->opts.kernel == PFMM_LAPLACE || p->opts.kernel == PFMM_STOKES);
  // deterministic mode: per-warp partial sums, added in warp order
  double* part = (p->opts.flags & PFMM_DETERMINISTIC) ? (double*)(ws + L.det) : nullptr;
  if (part && g_rec) return cudaErrorNotSupported;
  const int nwarp = cdiv_i(ns, 32), nrhs = p->opts.nrhs;
  // k_prep_q: kPrepPts points per thread, every warp of its grid writes a partial
  const int qblocks = cdiv_i(ns, 256 * kPrepPts), qwarps = qblocks * 8;
  double* mom = (double*)(ws + L.moments);
  if (project) {
    const NetArgs a{p->ncomp, nrhs, ns, p->s_stride, q, mom, part};
    e = launch_or_record(k_net, k_net_multi, PH_NET, dim3(cdiv_i(ns, 256)), 256, 0, st, a);
    if (e != cudaSuccess) return e;
    ++g_launches;
    if (part) {
      const int m = nrhs * p->ncomp;
      k_ordered_sum<<<cdiv_i(m, 128), 128, 0, st>>>(part, nwarp, m, p->ncomp, 8, mom + 5);
      ++g_launches;
    }
  }
  {
    const QArgs a{p->geom, p->ncomp, nrhs, ns, p->s_stride, q, (const double*)(ws + L.src64),
                  (double*)(ws + L.qc), (float*)(ws + L.qf), mom, status, project, part};
    e = launch_or_record(k_prep_q, k_prep_q_multi, PH_Q, dim3(qblocks), 256, 0, st, a);
    if (e != cudaSuccess) return e;
  }
  if (part) {
    k_ordered_sum<<<cdiv_i(4 * nrhs, 128), 128, 0, st>>>(part, qwarps, 4 * nrhs, 4, 8, mom);
    ++g_launches;
  }
  return launch_status();
}

// One pass of formation, weights and evaluation for the terms of `f`.  The
// modified Stokes Laplace family (second = true) takes its nodes after the
// beta family's, its coefficients and weights after the beta family's, and
// adds to the velocity the first pass wrote.
template <typename T, typename T2, int KER>
static cudaError_t run_far_direct(const pfmm_plan* p, Far f, bool second, char* ws, int64_t ns, int64_t nt,
                                  bool self, double* pot, double* grad, cudaStream_t st) {
  const Layout& L = p->lay;
  const int nw = (KER == PFMM_STOKES) ? 4 : (KER == PFMM_MSTOKES ? 2 : 1);  // weight rows per rhs
  f.nodes = (const double*)(ws + L.nodes) + (second ? 2 * p->far.Nq : 0);
  const Geom& g = p->geom;
  f.alpha1f = (float)(2.0 * M_PI / g.d);
  f.beta_f = (float)f.beta;
  const bool mixed = sizeof(T) == 4;
  const T* sx = mixed ? (const T*)(ws + L.srcf) : (const T*)(ws + L.src64);
  const T* sy = sx + ns;
  const int* sU = (const int*)(ws + L.srcU);
  const T* qv = mixed ? (const T*)(ws + L.qf) : (const T*)(ws + L.qc);
  double* coef = (double*)(ws + L.coef) + (second ? (size_t)f.nrhs * p->far.nch * p->far.nterm * 2 : 0);
  double* mom = (double*)(ws + L.moments);
  const int ph = second ? PH_FORM2 : PH_FORM;
  int nrg = cdiv_i(f.nrhs, rb_of<T, KER>());
  g_launches = (f.nterm > 0) ? 3 : 2;
  cudaError_t e;
  if (f.nterm > 0) {
    const bool det = (p->opts.flags & PFMM_DETERMINISTIC) != 0;
    if (det && g_rec) return cudaErrorNotSupported;
    int ny = cdiv_i(f.nterm, kFormThreads);
    // single cell: enough blocks to fill every SM several times; one of many
    // cells of a batch: source chunks of at least 2048 (the cells together
    // fill the GPU)
    int want = g_rec ? std::max(1, cdiv_i(ns, 2048) * ny * nrg) : 4 * 152 * 4;
    int nchunk = std::max(1, std::min(cdiv_i(ns, kFormSub), want / std::max(1, ny * nrg)));
    if (det) nchunk = std::min(nchunk, kDetChunks);
    int chunk = cdiv_i(cdiv_i(ns, nchunk), kFormSub) * kFormSub;
    nchunk = cdiv_i(ns, chunk);
    dim3 grid(nchunk, ny, nrg);
    double* part = det ? (double*)(ws + L.det) : nullptr;
    const FormArgs<T> a{f, g, (int)ns, chunk, sx, sy, sU, qv, coef, part};
    e = launch_or_record(k_far_form<T, KER>, k_far_form_multi<T, KER>, ph, grid, kFormThreads, 0, st, a);
    if (e != cudaSuccess) return e;
    if (det) {
      // every (rhs, channel, term) of every chunk is written (inactive terms as 0)
      const int m = f.nrhs * f.nch * f.nterm * 2;
      k_ordered_sum<<<cdiv_i(m, 128), 128, 0, st>>>(part, nchunk, m, m, 0, coef);
      ++g_launches;
    }
  }
  T2* w = (T2*)(ws + L.wts) + (second ? (size_t)f.nrhs * nw * p->far.nterm : 0);
  {
    const dim3 gw(cdiv_i(std::max(1, f.nterm), 128), f.nrhs);
    const WArgs<T2> a{f, g, coef, mom, w, (int*)(ws + L.status)};
    e = launch_or_record(k_far_weights<T2>, k_far_weights_multi<T2>, ph + 1, gw, 128, 0, st, a);
    if (e != cudaSuccess) return e;
  }
  const T* tx = self ? sx : (mixed ? (const T*)(ws + L.trgf) : (const T*)(ws + L.trg64));
  const T* ty = tx + nt;
  const int* tU = self ? sU : (const int*)(ws + L.trgU);
  {
    const dim3 ge(cdiv_i(nt, kEvalThreads), cdiv_i(f.nrhs, rb_of<T, KER>()));
    const EvalArgs<T, T2> a{f, g, (int)nt, tx, ty, tU, w, mom, p->o_stride, pot, grad, second ? 1 : 0};
    constexpr bool SC = KER == PFMM_LAPLACE || KER == PFMM_MODHELM;
    if (SC && grad)
      e = launch_or_record(k_far_eval<T, T2, KER, SC>, k_far_eval_multi<T, T2, KER, SC>, ph + 2, ge, kEvalThreads, 0,
                           st, a);
    else
      e = launch_or_record(k_far_eval<T, T2, KER, false>, k_far_eval_multi<T, T2, KER, false>, ph + 2, ge,
                           kEvalThreads, 0, st, a);
    if (e != cudaSuccess) return e;
  }
  return launch_status();
}

cudaError_t launch_far_direct(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot,
                              double* grad, cudaStream_t st) {
  const bool mixed = p->opts.precision == PFMM_MIXED;
  switch (p->opts.kernel) {
    case PFMM_LAPLACE:
      return mixed ? run_far_direct<float, float2, PFMM_LAPLACE>(p, p->far, false, ws, ns, nt, self, pot, grad, st)
                   : run_far_direct<double, double2, PFMM_LAPLACE>(p, p->far, false, ws, ns, nt, self, pot, grad, st);
    case PFMM_MODHELM:
      return mixed ? run_far_direct<float, float2, PFMM_MODHELM>(p, p->far, false, ws, ns, nt, self, pot, grad, st)
                   : run_far_direct<double, double2, PFMM_MODHELM>(p, p->far, false, ws, ns, nt, self, pot, grad, st);
    case PFMM_MSTOKES: {
      cudaError_t e = mixed
          ? run_far_direct<float, float2, PFMM_MSTOKES>(p, p->far, false, ws, ns, nt, self, pot, grad, st)
          : run_far_direct<double, double2, PFMM_MSTOKES>(p, p->far, false, ws, ns, nt, self, pot, grad, st);
      const int n1 = g_launches;
      if (e != cudaSuccess) return e;
      e = mixed ? run_far_direct<float, float2, PFMM_MSTOKES>(p, p->far2, true, ws, ns, nt, self, pot, grad, st)
                : run_far_direct<double, double2, PFMM_MSTOKES>(p, p->far2, true, ws, ns, nt, self, pot, grad, st);
      g_launches += n1;
      return e;
    }
    default:
      return mixed ? run_far_direct<float, float2, PFMM_STOKES>(p, p->far, false, ws, ns, nt, self, pot, grad, st)
                   : run_far_direct<double, double2, PFMM_STOKES>(p, p->far, false, ws, ns, nt, self, pot, grad, st);
  }
}

// Adjoint contractions:  out[k][j] = sum_r a[r][j] * b[r][k][j]  (k = 0, 1), with
// row strides sa for a and sb for b; used for dL/ds_j = sum_r q_rj grad psi_r(s_j)
// and dL/dt_l = sum_r g_rl grad u_r(t_l).
// A second pair (c, d) is added when c != NULL (targets = sources: both the
// source and the target role of a point contribute to one derivative).
__global__ void k_contract(int nrhs, int64_t n, const double* __restrict__ a, int64_t sa,
                           const double* __restrict__ b, int64_t sb, const double* __restrict__ c,
                           const double* __restrict__ d, double* __restrict__ out) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  double x = 0.0, y = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    const double w = a[(size_t)r * sa + j];
    x += w * b[((size_t)r * 2) * sb + j];
    y += w * b[((size_t)r * 2 + 1) * sb + j];
    if (c) {
      const double v = c[(size_t)r * sa + j];
      x += v * d[((size_t)r * 2) * sb + j];
      y += v * d[((size_t)r * 2 + 1) * sb + j];
    }
  }
  out[j] = x;
  out[n + j] = y;
}

cudaError_t launch_contract(int nrhs, int64_t n, const double* a, int64_t sa, const double* b, int64_t sb,
                            const double* c, const double* d, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_contract<<<cdiv_i(n, 256), 256, 0, st>>>(nrhs, n, a, sa, b, sb, c, d, out);
  return cudaGetLastError();
}

__global__ void k_pressure(int nrhs, int64_t nt, const double* __restrict__ g, double* __restrict__ pres) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nt) return;
  for (int r = 0; r < nrhs; ++r)
    pres[(size_t)r * nt + l] = -(g[((size_t)(2 * r) * 2) * nt + l] + g[((size_t)(2 * r + 1) * 2 + 1) * nt + l]);
}

cudaError_t launch_pressure(int nrhs, int64_t nt, const double* g, double* pres, cudaStream_t st) {
  if (nt == 0) return cudaSuccess;
  k_pressure<<<cdiv_i(nt, 256), 256, 0, st>>>(nrhs, nt, g, pres);
  return cudaGetLastError();
}

cudaError_t launch_zero_out(const pfmm_plan* p, int64_t nt, double* pot, double* grad, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  size_t nr = p->opts.nrhs;
  if (pot) e = zero_or_record(pot, nr * p->nout * nt * sizeof(double), st);
  if (e == cudaSuccess && grad) e = zero_or_record(grad, nr * 2 * nt * sizeof(double), st);
  return e;
}

}  // namespace pfmm
