// NUFFT far-field path for the south/north parts (Sec. 6, Eqs. fastanterp,
// fastinterp; Fig. nufftgrids) of the Laplace, modified Helmholtz and Stokes
// kernels.
//
// Formation (Eq. fastanterp):  c^S_m = sum_n e^{ chi_m ybar_n} F_n(m),
//                              c^N_m = sum_n e^{-chi_m ybar_n} F_n(m),
//   F_n(m) = sum_j gamma(y'_j, n) q_j e^{-i alpha_m x'_j}   (type-1 NUFFT per GL line n)
// with gamma the barycentric Gauss-Legendre interpolation weights on
// ybar_n in [-eta/2, eta/2] (Sec. 2.4, Eq. baryweights), chi_m = |alpha_m|
// (Laplace, Stokes) or sqrt(alpha_m^2 + beta^2) (modified Helmholtz, m = 0
// included).  Stokes spreads four charge channels per right-hand side,
// f_x, f_y, y' f_x, y' f_y: the first two give c_a, the last two c_b of
// Theorem south_thm_s.
// Evaluation (Eq. fastinterp):  u(t) = sum_n gamma(y, n) G_n(x),
//   G_n(x) = Re sum_m e^{i alpha_m x} v_n(m),
//   v_n(m) = w^S_m e^{-chi_m ybar_n} + w^N_m e^{chi_m ybar_n}  (type-2 NUFFT per line)
// and the y-derivative through v^y_n(m) = -chi_m w^S_m e^{-chi ybar} + chi_m w^N_m e^{chi ybar}.
// Stokes: u_k(t) = sum_n gamma(y, n) (Ga_{k,n}(x) + y Gb_{k,n}(x)), with the
// lines of the weights Wa and Wb of Theorem south_thm_s.
// Modified Stokes (Theorem south_thm_ms): the two force channels are spread
// once; both plane-wave families (decay chi_m and |alpha_m|) are formed from
// the same line spectra F_n(m) with their own line factors e^{+-decay ybar_n},
// weighted by their 2 x 2 blocks, and summed into one evaluation line per GL
// line (u_x + i u_y).
//
// Type-1/type-2 transforms: exponential-of-semicircle kernel
// phi(z) = exp(b (sqrt(1 - z^2) - 1)) of width w grid points, b = 2.30 w,
// fine grid of nf >= 2 (2M + 1) points (power of two) on theta = 2 pi x / d,
// a radix-2 FFT in shared memory, deconvolution by the kernel's Fourier
// transform.  With h = 2 pi / nf and alpha = w h / 2:
//   type 1:  F(k) = (2/w) B(k) / phihat(alpha k),  B = FFT(spread grid)
//   type 2:  G(theta) = (2/w) sum_l b_l phi((theta - theta_l)/alpha),
//            b = IFFT(v(k) / phihat(alpha k)).
// Two real lines share one complex FFT (real + i imag).
#include <algorithm>
#include <climits>
#include <mutex>
#include <cmath>
#include "pfmm_impl.h"
#include "devmath.cuh"
#include "lattice_weights.cuh"
#include "multi.cuh"

namespace pfmm {

struct NufftArgs {
  int nf, logn, w, M, n_gl, nrhs, ns, nt;
  int kernel, nch, npk, mlo;  // pfmm_kernel, charge channels per rhs, spectrum lines per rhs, first mode
  int64_t os;                 // output row stride
  double es_beta, d, eta, xi, beta;
  const double* gl;      // [n_gl][2] (ybar_n, sigma_n)
  const double* phihat;  // [M+1] phihat(alpha k), k = 0..M
  const double* tw;      // [nf/2][2] (cos, sin)(2 pi k / nf)
  // singly periodic west/east: Chebyshev coefficients [kRhoCheb] of 1/Psi(y)
  // in t = rho_c y (NULL otherwise), applied to the GL weights of every point
  const double* rho;
  double rho_c;
  float glf[64];  // (ybar_n, sigma_n) in FP32 for the mixed kernels (n_gl <= 32)
};

// FP64 value of a kernel-precision number (FP32: the integer-pipe conversion)
__device__ __forceinline__ double to_d(float v) { return dm::f2d(v); }
__device__ __forceinline__ double to_d(double v) { return v; }

// Transform coordinate in FP64: the FP32 path reads it from the signed
// fixed-point phase U = 2^32 y / Y (singly periodic transforms only, |y| < Y/4).
template <typename T>
__device__ __forceinline__ double spread_coord(T x, int U, const NufftArgs& a) {
  if constexpr (sizeof(T) == 4)
    return (double)U * (a.d * 2.3283064365386963e-10);
  else
    return (double)x;
}

// 1/Psi(y) by Clenshaw's recurrence on the plan's Chebyshev series.
__device__ __forceinline__ double rho_at(const NufftArgs& a, double y) {
  const double t = y * a.rho_c, t2 = 2.0 * t;
  double b1 = 0.0, b2 = 0.0;
  for (int k = kRhoCheb - 1; k >= 1; --k) {
    const double b0 = fma(t2, b1, a.rho[k] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(t, b1, a.rho[0] - b2);
}

// Position on the fine grid, u = theta / h = nf x / d (mod nf), split as
// u = i + f with i an integer and 0 <= f <= 1.  FP32 path: from the 32-bit
// fixed-point phase U = 2^32 x / d (mod 2^32) written by the point
// preparation, so that f is exact to 2^-24 whatever the cell width (an FP32
// product x nf / d would lose ~ulp(nf/2) grid units at the cell edge).  FP64
// path: from x.
template <typename T>
__device__ __forceinline__ void grid_pos(T x, int U, const NufftArgs& a, int* i, T* f) {
  if constexpr (sizeof(T) == 4) {
    const unsigned v = (unsigned)U;
    *i = (int)(v >> (32 - a.logn));
    *f = (float)(v << a.logn) * 2.3283064365386963e-10f;  // 2^-32
  } else {
    T u = x * (T)(a.nf / a.d);
    u -= (T)a.nf * floor(u / (T)a.nf);
    const T fl = floor(u);
    *i = (int)fl;
    *f = u - fl;
  }
}

// ES kernel values at the w grid points around u = i + f (grid units); WA is
// the array length (a compile-time bound >= w).  Returns l0, the first grid
// index (not reduced mod nf); z_k = (u - (l0 + k)) / (w/2).
template <typename T, int WA>
__device__ __forceinline__ int es_weights(int i, T f, int w, T beta, T* ker) {
  const T half = T(0.5) * w;
  const int c = (int)ceil(f - half);
#pragma unroll
  for (int k = 0; k < WA; ++k) {
    if (k < w) {
      const T z = (f - (T)(c + k)) / half;
      const T s = T(1) - z * z;
      ker[k] = s > T(0) ? dm::ex(beta * (sqrt(s) - T(1))) : T(0);
    }
  }
  return i + c;
}

// Barycentric interpolation weights gamma(y, n) (second form); GA is the
// array length (a compile-time bound >= n_gl).
template <typename T, int GA>
__device__ __forceinline__ void bary(T y, const NufftArgs& a, int n_gl, T* g) {
  T sum = T(0);
  int hit = -1;
#pragma unroll
  for (int n = 0; n < GA; ++n) {
    if (n < n_gl) {
      // the mixed kernels read the FP32 copy of the nodes (no FP64 conversions)
      const T yb = sizeof(T) == 4 ? (T)a.glf[2 * n] : (T)a.gl[2 * n];
      const T sg = sizeof(T) == 4 ? (T)a.glf[2 * n + 1] : (T)a.gl[2 * n + 1];
      const T dy = y - yb;
      if (dy == T(0)) hit = n;
      g[n] = sg / (dy == T(0) ? T(1) : dy);
      sum += g[n];
    }
  }
  const T inv = T(1) / sum;
#pragma unroll
  for (int n = 0; n < GA; ++n)
    if (n < n_gl) g[n] = hit >= 0 ? (n == hit ? T(1) : T(0)) : g[n] * inv;
}

// ---------------------------------------------------------------------------
// K4: anterpolation + spreading.  One block per source chunk.  The charge
// vectors v = (rhs r, channel c) are spread in groups of `vg` that share one
// shared-memory grid each ([vg][n_gl][nf] FP32 on the mixed path): per point
// the grid position, the w ES values and the n_gl barycentric weights are
// computed once per group and serve every vector of it; each group is then
// added to the global FP64 grid [nrhs][nch][n_gl][nf].  Channels: scalar q;
// Stokes f_x, f_y, y' f_x, y' f_y; modified Stokes f_x, f_y.  W and NGL are
// the ES width and the number of GL lines when known at compile time (the
// weight arrays then stay in registers), 0 for the general case.
// ---------------------------------------------------------------------------
constexpr int kSpreadThreads = 256;

template <typename T>
struct SpreadArgs {
  NufftArgs a;
  int chunk;
  const T* sx;
  const T* sy;
  const int* sU;
  const T* qv;
  double* grid;
  int use_smem, vg;
};

template <typename T, int W, int NGL>
__device__ __forceinline__ void k_nufft_spread_body(uint3 bid, const SpreadArgs<T>& A) {
  const NufftArgs& a = A.a;
  const int chunk = A.chunk, use_smem = A.use_smem, vg = A.vg;
  const T* __restrict__ sx = A.sx;
  const T* __restrict__ sy = A.sy;
  const int* __restrict__ sU = A.sU;
  const T* __restrict__ qv = A.qv;
  double* __restrict__ grid = A.grid;
  extern __shared__ unsigned char smem_raw[];
  T* sg = reinterpret_cast<T*>(smem_raw);  // [vg][n_gl][nf] when use_smem
  __shared__ int s_lo, s_hi;
  constexpr int WA = W ? W : 16, GA = NGL ? NGL : 32;
  const int w = W ? W : a.w, ngl = NGL ? NGL : a.n_gl;
  const int ngrid = ngl * a.nf;
  const int j0 = bid.x * chunk, j1 = min(a.ns, j0 + chunk);
  const T beta = (T)a.es_beta;
  const int ncomp = a.nch >= 2 ? 2 : 1;  // Stokes (4 channels) and modified Stokes (2) spread forces
  const int nv = a.nrhs * a.nch;
  // The grid columns this block touches: the sources are spatially sorted,
  // so a block's chunk covers a short range of columns in a long cell; only
  // that range (modulo nf) is cleared and added to the global grid.
  int cl = 0, span = a.nf;
  if (use_smem) {
    if (threadIdx.x == 0) {
      s_lo = INT_MAX;
      s_hi = INT_MIN;
    }
    __syncthreads();
    int lo = INT_MAX, hi = INT_MIN;
    const T half = T(0.5) * w;
    for (int j = j0 + threadIdx.x; j < j1; j += kSpreadThreads) {
      int gi;
      T gf;
      grid_pos(sx[j], sU[j], a, &gi, &gf);
      const int l0 = gi + (int)ceil(gf - half);
      lo = min(lo, l0);
      hi = max(hi, l0 + w - 1);
    }
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
    __syncthreads();
    if (s_hi >= s_lo && s_hi - s_lo + 1 < a.nf) {
      cl = s_lo;
      span = s_hi - s_lo + 1;
    }
  }
  for (int v0 = 0; v0 < nv; v0 += vg) {
    const int nvg = min(vg, nv - v0);
    if (use_smem)
      for (int k = threadIdx.x; k < nvg * ngl * span; k += kSpreadThreads) {
        const int row = k / span, col = (cl + k % span) & (a.nf - 1);
        sg[(size_t)row * a.nf + col] = T(0);
      }
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += kSpreadThreads) {
      const T x = sx[j], y = sy[j];
      int gi;
      T gf, ker[WA], gam[GA];
      grid_pos(x, sU[j], a, &gi, &gf);
      const int l0 = es_weights<T, WA>(gi, gf, w, beta, ker);
      bary<T, GA>(y, a, ngl, gam);
      if (a.rho) {
        const T rh = (T)rho_at(a, spread_coord(x, sU[j], a));
#pragma unroll
        for (int n = 0; n < GA; ++n) gam[n] *= rh;
      }
      for (int vv = 0; vv < nvg; ++vv) {
        const int v = v0 + vv, r = v / a.nch, c = v % a.nch;
        const T q0 = qv[((size_t)r * ncomp + (c & 1)) * a.ns + j];
        const T q = c >= 2 ? q0 * y : q0;
        T* sgv = sg + (size_t)vv * ngrid;
        double* gr = grid + (size_t)v * ngrid;
#pragma unroll
        for (int n = 0; n < GA; ++n) {
          if (n < ngl) {
            const T gq = gam[n] * q;
#pragma unroll
            for (int k = 0; k < WA; ++k) {
              if (k < w) {
                const int l = (l0 + k) & (a.nf - 1);
                if (use_smem)
                  atomicAdd(sgv + n * a.nf + l, gq * ker[k]);
                else
                  atomicAdd(gr + n * a.nf + l, to_d(gq * ker[k]));
              }
            }
          }
        }
      }
    }
    __syncthreads();
    if (use_smem) {
      double* g = grid + (size_t)v0 * ngrid;
      for (int k = threadIdx.x; k < nvg * ngl * span; k += kSpreadThreads) {
        const int row = k / span, col = (cl + k % span) & (a.nf - 1);
        const size_t o = (size_t)row * a.nf + col;
        const T val = sg[o];
        if (val != T(0)) atomicAdd(g + o, to_d(val));
      }
      __syncthreads();
    }
  }
}

template <typename T, int W, int NGL>
__global__ void __launch_bounds__(kSpreadThreads) k_nufft_spread(const __grid_constant__ SpreadArgs<T> A) {
  k_nufft_spread_body<T, W, NGL>(blockIdx, A);
}
template <typename T, int W, int NGL>
__global__ void __launch_bounds__(kSpreadThreads) k_nufft_spread_multi(const SpreadArgs<T>* __restrict__ cells,
                                                                       const int* __restrict__ off,
                                                                       const uint3* __restrict__ dims, int n) {
  const SubBlock s = sub_block(off, dims, n);
  k_nufft_spread_body<T, W, NGL>(s.bid, cells[s.cell]);
}

// ---------------------------------------------------------------------------
// K5: radix-2 complex FFT in shared memory (iterative, decimation in time,
// bit-reversed load), FP64 with twiddles from the plan's FP64 table.  One
// block per transform.  sign = -1 forward, +1 inverse.
// ---------------------------------------------------------------------------
__device__ void fft_smem(double2* s, int n, const double* __restrict__ tw, int sign) {
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len >> 1, step = n / len;
    for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
      const int grp = b / half, k = b % half;
      const int i0 = grp * len + k, i1 = i0 + half;
      const double cs = __ldg(tw + 2 * k * step), sn = sign * __ldg(tw + 2 * k * step + 1);
      const double2 x1 = s[i1];
      const double2 t = {x1.x * cs - x1.y * sn, x1.x * sn + x1.y * cs};
      const double2 x0 = s[i0];
      s[i0] = {x0.x + t.x, x0.y + t.y};
      s[i1] = {x0.x - t.x, x0.y - t.y};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int i, int logn) { return __brev(i) >> (32 - logn); }

// Forward transforms of the spread grids, two real lines per FFT, then
// deconvolution: F(k) for k = 0..M of every line (charge vector, GL line)
// written to Fk [nrhs][nch][n_gl][M+1] (double2).
struct FwdArgs {
  NufftArgs a;
  const double* grid;
  double2* Fk;
};

__device__ __forceinline__ void k_nufft_fwd_body(uint3 bid, const FwdArgs& A) {
  const NufftArgs& a = A.a;
  const double* __restrict__ grid = A.grid;
  double2* __restrict__ Fk = A.Fk;
  extern __shared__ unsigned char smem_raw[];
  double2* s = reinterpret_cast<double2*>(smem_raw);
  const int nline = a.nrhs * a.nch * a.n_gl;
  const int n0 = 2 * bid.x, n1 = 2 * bid.x + 1;
  const double* g0 = grid + (size_t)n0 * a.nf;
  const double* g1 = (n1 < nline) ? grid + (size_t)n1 * a.nf : nullptr;
  for (int i = threadIdx.x; i < a.nf; i += blockDim.x) {
    const int j = bitrev(i, a.logn);
    s[j] = {g0[i], g1 ? g1[i] : 0.0};
  }
  __syncthreads();
  fft_smem(s, a.nf, a.tw, -1);
  const double scale = 2.0 / a.w;
  for (int k = threadIdx.x; k <= a.M; k += blockDim.x) {
    const double2 zk = s[k], zm = s[(a.nf - k) & (a.nf - 1)];
    // X = (Z_k + conj Z_-k)/2, Y = (Z_k - conj Z_-k)/(2i)
    const double xr = 0.5 * (zk.x + zm.x), xi = 0.5 * (zk.y - zm.y);
    const double yr = 0.5 * (zk.y + zm.y), yi = -0.5 * (zk.x - zm.x);
    const double dec = scale / a.phihat[k];
    Fk[(size_t)n0 * (a.M + 1) + k] = make_double2(xr * dec, xi * dec);
    if (n1 < nline) Fk[(size_t)n1 * (a.M + 1) + k] = make_double2(yr * dec, yi * dec);
  }
}
PFMM_CELL_KERNELS(k_nufft_fwd, FwdArgs, )

// Mode combination, lattice weights and evaluation-line spectra (FP64).
// One thread per (rhs, mode m = mlo..M).  Writes the type-2 input spectra,
// layout spec [nrhs][npk][nf] (double2), zero elsewhere (cleared before):
//   scalar: line n: pot_n + i gy_n;  line n_gl + p: gx_{2p} + i gx_{2p+1}
//   Stokes: line n: Ga_{x,n} + i Ga_{y,n};  line n_gl + n: Gb_{x,n} + i Gb_{y,n}
// A real output line Re sum_m e^{i m theta} a_m packed with a second one
// (b_m) into a complex line has H_m = (a_m + i b_m)/2, H_-m = (conj a_m + i conj b_m)/2
// for m >= 1, and H_0 = a_0 + i b_0 (a_0, b_0 real).
struct ModesArgs {
  NufftArgs a;
  const double2* Fk;
  double2* spec;
  int want_grad;
};

template <int KER>
__device__ __forceinline__ void k_nufft_modes_body(uint3 bid, const ModesArgs& A) {
  const NufftArgs& a = A.a;
  const double2* __restrict__ Fk = A.Fk;
  double2* __restrict__ spec = A.spec;
  const int want_grad = A.want_grad;
  const int m = bid.x * blockDim.x + threadIdx.x + a.mlo;
  const int r = bid.y;
  if (m > a.M) return;
  const double al = 2.0 * M_PI * m / a.d;
  const double chi = (KER == PFMM_MODHELM) ? sqrt(al * al + a.beta * a.beta) : fabs(al);
  const double pre = (2.0 / a.w) / a.phihat[m];
  double2* base = spec + (size_t)r * a.npk * a.nf;
  auto put = [&](int line, dcx va, dcx vb) {
    double2* row = base + (size_t)line * a.nf;
    if (m == 0) {
      row[0] = {pre * (va.r - vb.i), pre * (va.i + vb.r)};
      return;
    }
    row[m] = {0.5 * pre * (va.r - vb.i), 0.5 * pre * (va.i + vb.r)};
    row[a.nf - m] = {0.5 * pre * (va.r + vb.i), 0.5 * pre * (-va.i + vb.r)};
  };
  auto F = [&](int c, int n) {
    const double2 v = Fk[(((size_t)r * a.nch + c) * a.n_gl + n) * (a.M + 1) + m];
    return dcx{v.x, v.y};
  };
  if (KER == PFMM_MSTOKES) {
    dcx v[32][2];
    for (int n = 0; n < a.n_gl; ++n) v[n][0] = v[n][1] = dcx{0, 0};
    const double fac = (m == 0) ? 1.0 : 2.0;  // the +-m pair
    for (int fam = 0; fam < 2; ++fam) {
      if (fam == 1 && m == 0) break;  // the Laplace family has no m = 0 term
      const double dec = fam == 0 ? sqrt(al * al + a.beta * a.beta) : fabs(al);
      dcx cS[2] = {{0, 0}, {0, 0}}, cN[2] = {{0, 0}, {0, 0}};
      for (int n = 0; n < a.n_gl; ++n) {
        const double yb = a.gl[2 * n];
        const double ep = exp(dec * yb), em = exp(-dec * yb);
        for (int k = 0; k < 2; ++k) {
          const dcx f = F(k, n);
          cS[k] = cadd(cS[k], cscale(f, ep));
          cN[k] = cadd(cN[k], cscale(f, em));
        }
      }
      dcx DS[2][2], DN[2][2], wS[2], wN[2];
      lw::ms_sn(a.d, a.xi, a.eta, al, dec, a.beta, fam, false, DS);
      lw::ms_sn(a.d, a.xi, a.eta, al, dec, a.beta, fam, true, DN);
      for (int i = 0; i < 2; ++i) {
        wS[i] = cscale(cadd(cmul(DS[i][0], cS[0]), cmul(DS[i][1], cS[1])), fac);
        wN[i] = cscale(cadd(cmul(DN[i][0], cN[0]), cmul(DN[i][1], cN[1])), fac);
      }
      for (int n = 0; n < a.n_gl; ++n) {
        const double yb = a.gl[2 * n];
        const double es = exp(-dec * yb), en = exp(dec * yb);
        for (int i = 0; i < 2; ++i) v[n][i] = cadd(v[n][i], cadd(cscale(wS[i], es), cscale(wN[i], en)));
      }
    }
    for (int n = 0; n < a.n_gl; ++n) put(n, v[n][0], v[n][1]);
    return;
  }
  if (KER != PFMM_STOKES) {
    // Theorem south_thm_lap / south_thm: D^S, D^N = conj(D^S); w = fac D c (fac 2: the +-m pair)
    const dcx DS = lw::sn_scalar(a.d, a.xi, a.eta, al, chi, false);
    dcx cS{0, 0}, cN{0, 0};
    for (int n = 0; n < a.n_gl; ++n) {
      const double yb = a.gl[2 * n];
      const dcx Fn = F(0, n);
      cS = cadd(cS, cscale(Fn, exp(chi * yb)));
      cN = cadd(cN, cscale(Fn, exp(-chi * yb)));
    }
    const double fac = (m == 0) ? 1.0 : 2.0;
    const dcx wS = cscale(cmul(DS, cS), fac), wN = cscale(cmul(conj_(DS), cN), fac);
    dcx vx_prev{0, 0};
    for (int n = 0; n < a.n_gl; ++n) {
      const double yb = a.gl[2 * n];
      const double es = exp(-chi * yb), en = exp(chi * yb);
      const dcx v = cadd(cscale(wS, es), cscale(wN, en));
      const dcx vy = want_grad ? cscale(csub(cscale(wN, en), cscale(wS, es)), chi) : dcx{0, 0};
      put(n, v, vy);
      if (want_grad) {
        const dcx vx{-al * v.i, al * v.r};  // d/dx: multiply by i alpha
        if (n & 1)
          put(a.n_gl + n / 2, vx_prev, vx);
        else if (n == a.n_gl - 1)
          put(a.n_gl + n / 2, vx, {0, 0});
        vx_prev = vx;
      }
    }
    return;
  }
  // Stokes (Theorem south_thm_s): c_a = R f, c_b = R y' f for south (e^{+chi ybar}) and north (e^{-chi ybar})
  dcx caS[2] = {{0, 0}, {0, 0}}, cbS[2] = {{0, 0}, {0, 0}}, caN[2] = {{0, 0}, {0, 0}}, cbN[2] = {{0, 0}, {0, 0}};
  for (int n = 0; n < a.n_gl; ++n) {
    const double yb = a.gl[2 * n];
    const double ep = exp(chi * yb), em = exp(-chi * yb);
    for (int k = 0; k < 2; ++k) {
      const dcx fa = F(k, n), fb = F(2 + k, n);
      caS[k] = cadd(caS[k], cscale(fa, ep));
      cbS[k] = cadd(cbS[k], cscale(fb, ep));
      caN[k] = cadd(caN[k], cscale(fa, em));
      cbN[k] = cadd(cbN[k], cscale(fb, em));
    }
  }
  dcx Da[2][2], Db[2][2], waS[2], wbS[2], waN[2], wbN[2];
  lw::sn_stokes(a.d, a.xi, a.eta, al, false, Da, Db);
  lw::stokes_apply(Da, Db, caS, cbS, false, 2.0, waS, wbS);
  lw::sn_stokes(a.d, a.xi, a.eta, al, true, Da, Db);
  lw::stokes_apply(Da, Db, caN, cbN, true, 2.0, waN, wbN);
  for (int n = 0; n < a.n_gl; ++n) {
    const double yb = a.gl[2 * n];
    const double es = exp(-chi * yb), en = exp(chi * yb);
    dcx va[2], vb[2];
    for (int k = 0; k < 2; ++k) {
      va[k] = cadd(cscale(waS[k], es), cscale(waN[k], en));
      vb[k] = cadd(cscale(wbS[k], es), cscale(wbN[k], en));
    }
    put(n, va[0], va[1]);
    put(a.n_gl + n, vb[0], vb[1]);
  }
}

template <int KER>
__global__ void k_nufft_modes(const __grid_constant__ ModesArgs A) {
  k_nufft_modes_body<KER>(blockIdx, A);
}
template <int KER>
__global__ void k_nufft_modes_multi(const ModesArgs* __restrict__ cells, const int* __restrict__ off,
                                    const uint3* __restrict__ dims, int n) {
  const SubBlock s = sub_block(off, dims, n);
  k_nufft_modes_body<KER>(s.bid, cells[s.cell]);
}

// Inverse FFT of each packed line spectrum in place (bit-reversed load into
// smem).  out32 (mixed path): the line is written back as FP32 pairs into the
// first half of its own storage (float2 index i of the row), so that the
// interpolation reads FP32 values with no FP64 conversions; the row was read
// into shared memory in full before any write.
struct InvArgs {
  NufftArgs a;
  double2* spec;
  int out32;
};

__device__ __forceinline__ void k_nufft_inv_body(uint3 bid, const InvArgs& A) {
  const NufftArgs& a = A.a;
  double2* __restrict__ spec = A.spec;
  const int out32 = A.out32;
  extern __shared__ unsigned char smem_raw[];
  double2* s = reinterpret_cast<double2*>(smem_raw);
  double2* row = spec + (size_t)bid.x * a.nf;
  for (int i = threadIdx.x; i < a.nf; i += blockDim.x) s[bitrev(i, a.logn)] = row[i];
  __syncthreads();
  fft_smem(s, a.nf, a.tw, +1);
  if (out32) {
    float2* rf = reinterpret_cast<float2*>(row);
    for (int i = threadIdx.x; i < a.nf; i += blockDim.x) rf[i] = make_float2((float)s[i].x, (float)s[i].y);
  } else {
    for (int i = threadIdx.x; i < a.nf; i += blockDim.x) row[i] = s[i];
  }
}
PFMM_CELL_KERNELS(k_nufft_inv, InvArgs, )

// Interpolation at targets + barycentric combination over lines; adds the
// south/north field to pot / grad (input frame).  The lines are FP64 (FP32
// on the mixed path, converted once per grid value by k_nufft_inv); the
// mixed path interpolates in FP32 and sums over lines with compensation.  The
// ES and barycentric weights are computed once per target and serve every
// right-hand side; W, NGL as for the spreading kernel.
template <typename T>
struct InterpArgs {
  NufftArgs a;
  Geom g;
  const T* tx;
  const T* ty;
  const int* tU;
  const double2* spec;
  double* pot;
  double* grad;
};

template <typename T, int KER, int W, int NGL>
__device__ __forceinline__ void k_nufft_interp_body(uint3 bid, const InterpArgs<T>& A) {
  const NufftArgs& a = A.a;
  const Geom& g = A.g;
  const T* __restrict__ tx = A.tx;
  const T* __restrict__ ty = A.ty;
  const int* __restrict__ tU = A.tU;
  const double2* __restrict__ spec = A.spec;
  double* __restrict__ pot = A.pot;
  double* __restrict__ grad = A.grad;
  constexpr int WA = W ? W : 16, GA = NGL ? NGL : 32;
  const int w = W ? W : a.w, ngl = NGL ? NGL : a.n_gl;
  const int l = bid.x * blockDim.x + threadIdx.x;
  if (l >= a.nt) return;
  const T x = tx[l], y = ty[l];
  int gi;
  T gf, ker[WA], gam[GA];
  grid_pos(x, tU[l], a, &gi, &gf);
  const int l0 = es_weights<T, WA>(gi, gf, w, (T)a.es_beta, ker);
  bary<T, GA>(y, a, ngl, gam);
  if (a.rho) {
    const T rh = (T)rho_at(a, spread_coord(x, tU[l], a));
#pragma unroll
    for (int n = 0; n < GA; ++n) gam[n] *= rh;
  }
  int li[WA];
#pragma unroll
  for (int k = 0; k < WA; ++k) li[k] = (l0 + k) & (a.nf - 1);
  const double* R = g.rot;
  // value k of evaluation line `line` of rhs r: FP32 rows on the mixed path
  // (written by k_nufft_inv with out32, row stride 2 nf float2), FP64 otherwise
  struct V2 {
    T x, y;
  };
  auto val = [&](int r, int line, int k) -> V2 {
    if constexpr (sizeof(T) == 4) {
      const float2 v = reinterpret_cast<const float2*>(spec)[((size_t)r * a.npk + line) * 2 * a.nf + li[k]];
      return V2{v.x, v.y};
    } else {
      const double2 v = spec[((size_t)r * a.npk + line) * a.nf + li[k]];
      return V2{v.x, v.y};
    }
  };
  for (int r = 0; r < a.nrhs; ++r) {
    if (KER == PFMM_MSTOKES) {
      dm::KSum<T> ux, uy;
#pragma unroll 1
      for (int n = 0; n < ngl; ++n) {
        T sx = 0, sy = 0;
#pragma unroll
        for (int k = 0; k < WA; ++k) {
          if (k < w) {
            const V2 va = val(r, n, k);
            sx += ker[k] * va.x;
            sy += ker[k] * va.y;
          }
        }
        ux.add(gam[n] * sx);
        uy.add(gam[n] * sy);
      }
      const double uxd = ux.value(), uyd = uy.value();
      pot[((size_t)r * 2) * a.os + l] += R[0] * uxd + R[2] * uyd;
      pot[((size_t)r * 2 + 1) * a.os + l] += R[1] * uxd + R[3] * uyd;
      continue;
    }
    if (KER == PFMM_STOKES) {
      dm::KSum<T> ux, uy;
#pragma unroll 1
      for (int n = 0; n < ngl; ++n) {
        T sax = 0, say = 0, sbx = 0, sby = 0;
#pragma unroll
        for (int k = 0; k < WA; ++k) {
          if (k < w) {
            const V2 va = val(r, n, k), vb = val(r, ngl + n, k);
            sax += ker[k] * va.x;
            say += ker[k] * va.y;
            sbx += ker[k] * vb.x;
            sby += ker[k] * vb.y;
          }
        }
        ux.add(gam[n] * (sax + y * sbx));
        uy.add(gam[n] * (say + y * sby));
      }
      const double uxd = ux.value(), uyd = uy.value();
      pot[((size_t)r * 2) * a.os + l] += R[0] * uxd + R[2] * uyd;
      pot[((size_t)r * 2 + 1) * a.os + l] += R[1] * uxd + R[3] * uyd;
      continue;
    }
    dm::KSum<T> p, gx, gy;
#pragma unroll 1
    for (int n = 0; n < ngl; ++n) {
      T sp = 0, sy = 0, sx = 0;
#pragma unroll
      for (int k = 0; k < WA; ++k) {
        if (k < w) {
          const V2 v = val(r, n, k);
          sp += ker[k] * v.x;
          sy += ker[k] * v.y;
          if (grad) {
            const V2 vx = val(r, ngl + n / 2, k);
            sx += ker[k] * ((n & 1) ? vx.y : vx.x);
          }
        }
      }
      p.add(gam[n] * sp);
      gy.add(gam[n] * sy);
      gx.add(gam[n] * sx);
    }
    if (pot) pot[(size_t)r * a.os + l] += p.value();
    if (grad) {
      const double gxd = gx.value(), gyd = gy.value();
      grad[((size_t)r * 2) * a.os + l] += R[0] * gxd + R[2] * gyd;
      grad[((size_t)r * 2 + 1) * a.os + l] += R[1] * gxd + R[3] * gyd;
    }
  }
}

template <typename T, int KER, int W, int NGL>
__global__ void k_nufft_interp(const __grid_constant__ InterpArgs<T> A) {
  k_nufft_interp_body<T, KER, W, NGL>(blockIdx, A);
}
template <typename T, int KER, int W, int NGL>
__global__ void k_nufft_interp_multi(const InterpArgs<T>* __restrict__ cells, const int* __restrict__ off,
                                     const uint3* __restrict__ dims, int n) {
  const SubBlock s = sub_block(off, dims, n);
  k_nufft_interp_body<T, KER, W, NGL>(s.bid, cells[s.cell]);
}

// ---------------------------------------------------------------------------
// Singly periodic operator, west/east parts through the transforms (Sec. 6.1
// with x and y exchanged; Theorems west_thm, west_thm_lap, west_thm_s on the
// image row n = 0).  The plane waves e^{-+kappa_n x} e^{i lambda_n y} are
// smooth in x (GL lines xbar_k on [-d/2, d/2], barycentric weights in x) and
// oscillatory in y, at the piecewise-GL quadrature nodes lambda_n.  Per GL
// line the sums over sources S_k(lambda) = sum_j gamma(x'_j, k) q_j e^{-i lambda y'_j}
// are a type-3 transform: with psi the ES kernel in lambda (half-width
// alpha = w dl / 2, dl = 2 pi / Y) and Psi(y) its Fourier transform,
//   S_k(lambda) ~= dl sum_u psi(lambda - u dl) F_k(u),
//   F_k(u) = sum_j gamma(x'_j, k) (q_j / Psi(y'_j)) e^{-i u dl y'_j}
// (Poisson summation; the aliases Psi(y - p Y) / Psi(y), p != 0, are below the
// ES kernel's error for |y| <= Y/4), and F_k is the type-1 transform of the
// south/north path with y as the transform coordinate over the period Y.
// The evaluation is the adjoint: sum_n V(n) e^{i lambda_n y} ~= (1/Psi(y)) Re-part
// of the type-2 transform of H(u) = dl sum_n psi(lambda_n - u dl) V(n).
// ---------------------------------------------------------------------------

// Formation and weights at the nodes.  One thread per (node n = nq0 + j, rhs):
//   c^W_n = sum_k e^{ kappa_n xbar_k} S_k(lambda_n),  c^E_n = sum_k e^{-kappa_n xbar_k} S_k(lambda_n)
// (Stokes: the channels f_x, f_y, x' f_x, x' f_y give c_a and c_b), w = D c
// with the row-0 blocks of the direct path, and the evaluation lines
//   V_k(n) = w^W_n e^{-kappa_n xbar_k} + w^E_n e^{kappa_n xbar_k}
// with kappa_n (w^E e^{kappa xbar} - w^W e^{-kappa xbar}) the x-derivative line
// (scalar), or the a_x, a_y, b_x, b_y lines (Stokes), written to
// lines[r][line][j].  The ES weights are FP64 (the node count is small).
template <int KER>
__global__ void k_p1_modes(NufftArgs a, Geom g, const double* __restrict__ nodes, int nq0, int nnu, double dl,
                           double alpha, const double2* __restrict__ Fk, double2* __restrict__ lines) {
  constexpr int NCH = KER == PFMM_STOKES ? 4 : 1;
  constexpr int WU = 17;  // frequencies in a window of width 2 alpha = w dl, w <= 16
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (j >= nnu) return;
  const int n = nq0 + j;
  const double lam = nodes[2 * n], wq = nodes[2 * n + 1];
  const double kap = (KER == PFMM_MODHELM) ? sqrt(lam * lam + a.beta * a.beta) : lam;
  const int u0 = max(1, (int)ceil((lam - alpha) / dl));
  const int u1 = min(min(a.M, (int)floor((lam + alpha) / dl)), u0 + WU - 1);
  double psi[WU];
#pragma unroll
  for (int i = 0; i < WU; ++i) {
    const double z = (lam - (u0 + i) * dl) / alpha, t = 1.0 - z * z;
    psi[i] = (u0 + i <= u1 && t > 0.0) ? dl * exp(a.es_beta * (sqrt(t) - 1.0)) : 0.0;
  }
  dcx cW[NCH], cE[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) cW[c] = cE[c] = dcx{0, 0};
  for (int k = 0; k < a.n_gl; ++k) {
    const double xb = a.gl[2 * k];
    const double ep = exp(kap * xb), em = exp(-kap * xb);
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const double2* F = Fk + (((size_t)r * a.nch + c) * a.n_gl + k) * (a.M + 1);
      dcx sk{0, 0};
#pragma unroll
      for (int i = 0; i < WU; ++i)
        if (u0 + i <= u1) {
          const double2 f = F[u0 + i];
          sk = cadd(sk, dcx{psi[i] * f.x, psi[i] * f.y});
        }
      cW[c] = cadd(cW[c], cscale(sk, ep));
      cE[c] = cadd(cE[c], cscale(sk, em));
    }
  }
  const lw::WeFrame fr{g.wdx, g.wdy, g.wxr, g.wyr};
  const int ngl = a.n_gl;
  if (KER != PFMM_STOKES) {
    double2* out = lines + (size_t)r * 2 * ngl * nnu;
    const dcx wW = cmul(lw::we_scalar(fr, g.m0, lam, kap, wq, false, false), cW[0]);
    const dcx wE = cmul(lw::we_scalar(fr, g.m0, lam, kap, wq, true, false), cE[0]);
    for (int k = 0; k < ngl; ++k) {
      const double xb = a.gl[2 * k];
      const dcx vw = cscale(wW, exp(-kap * xb)), ve = cscale(wE, exp(kap * xb));
      const dcx v = cadd(vw, ve), vx = cscale(csub(ve, vw), kap);
      out[(size_t)k * nnu + j] = make_double2(v.r, v.i);
      out[(size_t)(ngl + k) * nnu + j] = make_double2(vx.r, vx.i);
    }
    return;
  }
  double2* out = lines + (size_t)r * 4 * ngl * nnu;
  dcx Da[2][2], Db[2][2], waW[2], wbW[2], waE[2], wbE[2];
  {
    const dcx ca[2] = {cW[0], cW[1]}, cb[2] = {cW[2], cW[3]};
    lw::we_stokes(fr, g.wc, g.ws, g.m0, lam, wq, false, Da, Db, false);
    lw::stokes_apply(Da, Db, ca, cb, false, 1.0, waW, wbW);
  }
  {
    const dcx ca[2] = {cE[0], cE[1]}, cb[2] = {cE[2], cE[3]};
    lw::we_stokes(fr, g.wc, g.ws, g.m0, lam, wq, true, Da, Db, false);
    lw::stokes_apply(Da, Db, ca, cb, true, 1.0, waE, wbE);
  }
  for (int k = 0; k < ngl; ++k) {
    const double xb = a.gl[2 * k];
    const double es = exp(-kap * xb), en = exp(kap * xb);
    for (int i = 0; i < 2; ++i) {
      const dcx va = cadd(cscale(waW[i], es), cscale(waE[i], en));
      const dcx vb = cadd(cscale(wbW[i], es), cscale(wbE[i], en));
      out[(size_t)(i * ngl + k) * nnu + j] = make_double2(va.r, va.i);
      out[(size_t)((2 + i) * ngl + k) * nnu + j] = make_double2(vb.r, vb.i);
    }
  }
}

// Evaluation-line spectra on the uniform frequencies u = 1..M:
//   H(u) = dl sum_n psi(lambda_n - u dl) V(n)   (nodes ascending: a binary
// search finds the window), deconvolved by the y-kernel's phihat and packed
// two real lines per complex line as in k_nufft_modes:
//   scalar: line k: V_k + i (x-derivative line k);  line n_gl + p: the
//           y-derivative lines (i lambda V) 2p and 2p + 1
//   Stokes: line k: a_x + i a_y;  line n_gl + k: b_x + i b_y.
// One thread per (u, packed line, rhs); spec was cleared before.
template <int KER>
__global__ void k_p1_gather(NufftArgs a, const double* __restrict__ nodes, int nq0, int nnu, double dl, double alpha,
                            const double2* __restrict__ lines, double2* __restrict__ spec, int want_grad) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int s = blockIdx.y, r = blockIdx.z;
  if (u > a.M) return;
  const int ngl = a.n_gl;
  const int nl = (KER == PFMM_STOKES ? 4 : 2) * ngl;
  const double2* L = lines + (size_t)r * nl * nnu;
  int la, lb;
  bool dy = false;  // multiply the node values by i lambda (y-derivative lines)
  if (KER == PFMM_STOKES) {
    la = s < ngl ? s : 2 * ngl + (s - ngl);
    lb = s < ngl ? ngl + s : 3 * ngl + (s - ngl);
  } else if (s < ngl) {
    la = s;
    lb = want_grad ? ngl + s : -1;
  } else {
    const int p = s - ngl;
    la = 2 * p;
    lb = 2 * p + 1 < ngl ? 2 * p + 1 : -1;
    dy = true;
  }
  const double uc = u * dl, lo = uc - alpha, hi = uc + alpha;
  int b = 0, e = nnu;  // first node with lambda > lo
  while (b < e) {
    const int m = (b + e) >> 1;
    if (nodes[2 * (nq0 + m)] <= lo) b = m + 1;
    else e = m;
  }
  dcx A{0, 0}, B{0, 0};
  for (int m = b; m < nnu; ++m) {
    const double lam = nodes[2 * (nq0 + m)];
    if (lam >= hi) break;
    const double z = (lam - uc) / alpha, t = 1.0 - z * z;
    if (t <= 0.0) continue;
    const double ps = exp(a.es_beta * (sqrt(t) - 1.0));
    const double f = dy ? ps * lam : ps;
    const double2 va = L[(size_t)la * nnu + m];
    A = cadd(A, dy ? dcx{-f * va.y, f * va.x} : dcx{f * va.x, f * va.y});
    if (lb >= 0) {
      const double2 vb = L[(size_t)lb * nnu + m];
      B = cadd(B, dy ? dcx{-f * vb.y, f * vb.x} : dcx{f * vb.x, f * vb.y});
    }
  }
  const double pre = dl * (2.0 / a.w) / a.phihat[u];
  double2* row = spec + ((size_t)r * a.npk + s) * a.nf;
  row[u] = {0.5 * pre * (A.r - B.i), 0.5 * pre * (A.i + B.r)};
  row[a.nf - u] = {0.5 * pre * (A.r + B.i), 0.5 * pre * (-A.i + B.r)};
}

// Raise a kernel's dynamic shared-memory limit once per device and size, so
// that executes after the first (including ones captured in a CUDA graph)
// make no attribute calls.  cudaFuncSetAttribute sets the limit (it may also
// lower it), so the call and the cache update happen under one lock and the
// value set is never below what an earlier call established: plans may
// execute from several host threads with different sizes.
static cudaError_t raise_smem(const void* fn, int slot, size_t bytes) {
  static std::mutex mu;
  static int done[32][16] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  const bool cached = dev >= 0 && dev < 32;
  if (cached && done[dev][slot] >= (int)bytes) return cudaSuccess;
  const int want = cached ? std::max(done[dev][slot], (int)bytes) : (int)bytes;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
  if (e == cudaSuccess && cached) done[dev][slot] = want;
  return e;
}

// (ES width, GL lines) compiled with the weight arrays in registers: the
// defaults at tol 1e-6, 1e-10 and 1e-12; other pairs take the general kernels.
static int nufft_spec(int w, int n_gl) {
  if (w == 8 && n_gl == 8) return 1;
  if (w == 12 && n_gl == 16) return 2;
  if (w == 14 && n_gl == 16) return 3;
  return 0;
}

template <typename T, int W, int NGL>
static cudaError_t spread_t(const NufftArgs& a, int nchunk, int chunk, const T* sx, const T* sy, const int* sU,
                            const T* qv, double* grid, int use_smem, int vg, size_t smem, int slot, cudaStream_t st) {
  if (!g_rec && smem > 48 * 1024) {
    cudaError_t e = raise_smem((const void*)k_nufft_spread<T, W, NGL>, slot, smem);
    if (e != cudaSuccess) return e;
  }
  const SpreadArgs<T> A{a, chunk, sx, sy, sU, qv, grid, use_smem, vg};
  return launch_or_record(k_nufft_spread<T, W, NGL>, k_nufft_spread_multi<T, W, NGL>, PH_SPREAD, dim3(nchunk),
                          kSpreadThreads, smem, st, A);
}

template <typename T, int KER>
static cudaError_t interp_k(int spec, int ni, const NufftArgs& a, const Geom& g, const T* tx, const T* ty,
                            const int* tU, const double2* sp, double* pot, double* grad, cudaStream_t st) {
  const InterpArgs<T> A{a, g, tx, ty, tU, sp, pot, grad};
  const dim3 gi(ni);
  switch (spec) {
    case 1:
      return launch_or_record(k_nufft_interp<T, KER, 8, 8>, k_nufft_interp_multi<T, KER, 8, 8>, PH_INTERP, gi, 128, 0,
                              st, A);
    case 2:
      return launch_or_record(k_nufft_interp<T, KER, 12, 16>, k_nufft_interp_multi<T, KER, 12, 16>, PH_INTERP, gi, 128,
                              0, st, A);
    case 3:
      return launch_or_record(k_nufft_interp<T, KER, 14, 16>, k_nufft_interp_multi<T, KER, 14, 16>, PH_INTERP, gi, 128,
                              0, st, A);
    default:
      return launch_or_record(k_nufft_interp<T, KER, 0, 0>, k_nufft_interp_multi<T, KER, 0, 0>, PH_INTERP, gi, 128, 0,
                              st, A);
  }
}

template <int KER>
static cudaError_t modes_k(const NufftArgs& a, dim3 gm, const double2* Fk, double2* spec, int wg, cudaStream_t st) {
  return launch_or_record(k_nufft_modes<KER>, k_nufft_modes_multi<KER>, PH_MODES, gm, 128, 0, st,
                          ModesArgs{a, Fk, spec, wg});
}

// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t run_nufft(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot,
                             double* grad, cudaStream_t st) {
  const Layout& L = p->lay;
  const bool mixed = sizeof(T) == 4;
  const int K = p->opts.kernel;
  NufftArgs a{};
  a.nf = p->nf;
  a.logn = 0;
  while ((1 << a.logn) < a.nf) ++a.logn;
  a.w = p->nufft_w;
  a.M = p->far.M;
  a.n_gl = p->n_gl;
  a.nrhs = p->opts.nrhs;
  a.ns = (int)ns;
  a.nt = (int)nt;
  a.kernel = K;
  a.nch = nufft_nch(K);
  a.npk = nufft_npk(K, a.n_gl);
  a.mlo = p->far.mode0 ? 0 : 1;
  a.os = p->o_stride;
  a.es_beta = p->es_beta;
  a.d = p->geom.d;
  a.eta = p->geom.eta;
  a.xi = p->geom.xi;
  a.beta = p->far.beta;
  a.gl = (const double*)(ws + L.nodes + off_gl(p));
  for (int i = 0; i < 2 * a.n_gl && i < 64; ++i) a.glf[i] = (float)p->gl_h[i];
  a.phihat = (const double*)(ws + L.nodes + off_phihat(p));
  a.tw = (const double*)(ws + L.nodes + off_twiddle(p));
  // workspace partition of the NUFFT scratch
  const int nline = a.nrhs * a.nch * a.n_gl;
  char* base = ws + L.nufft;
  double* grid = (double*)base;                                   // [nrhs][nch][n_gl][nf] double
  size_t off = (size_t)nline * a.nf * sizeof(double);
  double2* Fk = (double2*)(base + off);                           // [nrhs][nch][n_gl][M+1]
  off += (size_t)nline * (a.M + 1) * sizeof(double2);
  off = (off + 255) & ~size_t(255);
  double2* spec = (double2*)(base + off);                         // [nrhs][npk][nf]
  cudaError_t e = zero_or_record(grid, (size_t)nline * a.nf * sizeof(double), st);
  if (e != cudaSuccess) return e;
  e = zero_or_record(spec, (size_t)a.nrhs * a.npk * a.nf * sizeof(double2), st);
  if (e != cudaSuccess) return e;
  const T* sx = mixed ? (const T*)(ws + L.srcf) : (const T*)(ws + L.src64);
  const T* qv = mixed ? (const T*)(ws + L.qf) : (const T*)(ws + L.qc);
  int nchunk = std::max(1, std::min((int)((ns + 255) / 256), 2 * 152));
  int chunk = (int)((ns + nchunk - 1) / nchunk);
  nchunk = (int)((ns + chunk - 1) / chunk);
  // one shared grid per charge vector of a group; as many vectors per group
  // as fit in ~100 KB, so that the weights are computed once per group
  const size_t per_v = (size_t)a.n_gl * a.nf * sizeof(T);
  const int use_smem = per_v <= 96 * 1024;
  const int nv = a.nrhs * a.nch;
  const int vg = use_smem ? (int)std::max<size_t>(1, std::min<size_t>(nv, (100 * 1024) / per_v)) : nv;
  const size_t sm_spread = use_smem ? vg * per_v : 0;
  const int* sU = (const int*)(ws + L.srcU);
  const int wspec = nufft_spec(a.w, a.n_gl);
  const int slot = (sizeof(T) == 4 ? 0 : 4) + wspec;
  switch (wspec) {
    case 1: e = spread_t<T, 8, 8>(a, nchunk, chunk, sx, sx + ns, sU, qv, grid, use_smem, vg, sm_spread, slot, st); break;
    case 2: e = spread_t<T, 12, 16>(a, nchunk, chunk, sx, sx + ns, sU, qv, grid, use_smem, vg, sm_spread, slot, st); break;
    case 3: e = spread_t<T, 14, 16>(a, nchunk, chunk, sx, sx + ns, sU, qv, grid, use_smem, vg, sm_spread, slot, st); break;
    default: e = spread_t<T, 0, 0>(a, nchunk, chunk, sx, sx + ns, sU, qv, grid, use_smem, vg, sm_spread, slot, st); break;
  }
  if (e != cudaSuccess) return e;
  const int fth = std::min(512, std::max(32, a.nf / 2));
  const size_t sm_fft = (size_t)a.nf * sizeof(double2);
  if (!g_rec && sm_fft > 48 * 1024) {
    e = raise_smem((const void*)k_nufft_fwd, 8, sm_fft);
    if (e == cudaSuccess) e = raise_smem((const void*)k_nufft_inv, 9, sm_fft);
    if (e != cudaSuccess) return e;
  }
  e = launch_or_record(k_nufft_fwd, k_nufft_fwd_multi, PH_FWD, dim3((nline + 1) / 2), fth, sm_fft, st,
                       FwdArgs{a, grid, Fk});
  if (e != cudaSuccess) return e;
  const InvArgs inv{a, spec, mixed ? 1 : 0};
  const dim3 ginv(a.nrhs * a.npk);
  const int nmode = a.M - a.mlo + 1;
  dim3 gm((nmode + 127) / 128, a.nrhs);
  const T* tx = self ? sx : (mixed ? (const T*)(ws + L.trgf) : (const T*)(ws + L.trg64));
  const int* tU = self ? sU : (const int*)(ws + L.trgU);
  const int ni = (int)((nt + 127) / 128);
  const int wg = grad != nullptr;
  auto inv_k = [&]() {
    return launch_or_record(k_nufft_inv, k_nufft_inv_multi, PH_INV, ginv, fth, sm_fft, st, inv);
  };
  switch (K) {
    case PFMM_LAPLACE:
      e = modes_k<PFMM_LAPLACE>(a, gm, Fk, spec, wg, st);
      if (e == cudaSuccess) e = inv_k();
      if (e == cudaSuccess) e = interp_k<T, PFMM_LAPLACE>(wspec, ni, a, p->geom, tx, tx + nt, tU, spec, pot, grad, st);
      break;
    case PFMM_MODHELM:
      e = modes_k<PFMM_MODHELM>(a, gm, Fk, spec, wg, st);
      if (e == cudaSuccess) e = inv_k();
      if (e == cudaSuccess) e = interp_k<T, PFMM_MODHELM>(wspec, ni, a, p->geom, tx, tx + nt, tU, spec, pot, grad, st);
      break;
    case PFMM_MSTOKES:
      e = modes_k<PFMM_MSTOKES>(a, gm, Fk, spec, 0, st);
      if (e == cudaSuccess) e = inv_k();
      if (e == cudaSuccess)
        e = interp_k<T, PFMM_MSTOKES>(wspec, ni, a, p->geom, tx, tx + nt, tU, spec, pot, nullptr, st);
      break;
    default:
      e = modes_k<PFMM_STOKES>(a, gm, Fk, spec, 0, st);
      if (e == cudaSuccess) e = inv_k();
      if (e == cudaSuccess)
        e = interp_k<T, PFMM_STOKES>(wspec, ni, a, p->geom, tx, tx + nt, tU, spec, pot, nullptr, st);
      break;
  }
  if (e != cudaSuccess) return e;
  g_launches += 5;
  return launch_status();
}

// Singly periodic west/east nodes [p1_nq0, Nq) through the transforms (see
// k_p1_modes); adds to pot / grad, which the direct kernels wrote first.
template <typename T>
static cudaError_t run_p1_nufft(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot,
                                double* grad, cudaStream_t st) {
  const Layout& L = p->lay;
  const bool mixed = sizeof(T) == 4;
  const int K = p->opts.kernel;
  NufftArgs a{};
  a.nf = p->nf;
  a.logn = 0;
  while ((1 << a.logn) < a.nf) ++a.logn;
  a.w = p->nufft_w;
  a.M = p->p1_M;
  a.n_gl = p->n_gl;
  a.nrhs = p->opts.nrhs;
  a.ns = (int)ns;
  a.nt = (int)nt;
  a.kernel = K;
  a.nch = nufft_nch(K);
  a.npk = nufft_npk(K, a.n_gl);
  a.mlo = 1;
  a.os = p->o_stride;
  a.es_beta = p->es_beta;
  a.d = p->p1_Y;  // the transform's period
  a.eta = p->geom.d;
  a.xi = 0.0;
  a.beta = p->far.beta;
  const char* tab = ws + L.nodes;
  a.gl = (const double*)(tab + off_gl(p));
  for (int i = 0; i < 2 * a.n_gl && i < 64; ++i) a.glf[i] = (float)p->gl_h[i];
  a.phihat = (const double*)(tab + off_phihat(p));
  a.tw = (const double*)(tab + off_twiddle(p));
  a.rho = (const double*)(tab + off_rho(p));
  a.rho_c = 2.0 / p->geom.eta;
  const double* nodes = (const double*)tab;
  const int nq0 = p->p1_nq0, nnu = p->Nq - p->p1_nq0;
  const double dl = p->p1_dl, alpha = p->p1_alpha;
  const int nline = a.nrhs * a.nch * a.n_gl;
  char* base = ws + L.nufft;
  double* grid = (double*)base;  // [nrhs][nch][n_gl][nf]
  size_t off = (size_t)nline * a.nf * sizeof(double);
  double2* Fk = (double2*)(base + off);  // [nrhs][nch][n_gl][M+1]
  off += (size_t)nline * (a.M + 1) * sizeof(double2);
  off = (off + 255) & ~size_t(255);
  double2* spec = (double2*)(base + off);  // [nrhs][npk][nf]
  off += (size_t)a.nrhs * a.npk * a.nf * sizeof(double2);
  off = (off + 255) & ~size_t(255);
  double2* lines = (double2*)(base + off);  // [nrhs][p1_node_lines][nnu]
  cudaError_t e = cudaMemsetAsync(grid, 0, (size_t)nline * a.nf * sizeof(double), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(spec, 0, (size_t)a.nrhs * a.npk * a.nf * sizeof(double2), st);
  if (e != cudaSuccess) return e;
  // transform coordinate y, GL coordinate x, fixed-point phase of y
  const T* s64 = mixed ? (const T*)(ws + L.srcf) : (const T*)(ws + L.src64);
  const T* qv = mixed ? (const T*)(ws + L.qf) : (const T*)(ws + L.qc);
  const int* sV = (const int*)(ws + L.srcV);
  int nchunk = std::max(1, std::min((int)((ns + 255) / 256), 2 * 152));
  int chunk = (int)((ns + nchunk - 1) / nchunk);
  nchunk = (int)((ns + chunk - 1) / chunk);
  const size_t per_v = (size_t)a.n_gl * a.nf * sizeof(T);
  const int use_smem = per_v <= 96 * 1024;
  const int nv = a.nrhs * a.nch;
  const int vg = use_smem ? (int)std::max<size_t>(1, std::min<size_t>(nv, (100 * 1024) / per_v)) : nv;
  const size_t sm_spread = use_smem ? vg * per_v : 0;
  const int wspec = nufft_spec(a.w, a.n_gl);
  const int slot = (sizeof(T) == 4 ? 0 : 4) + wspec;
  const T* sy_ = s64 + ns;  // y
  switch (wspec) {
    case 1: e = spread_t<T, 8, 8>(a, nchunk, chunk, sy_, s64, sV, qv, grid, use_smem, vg, sm_spread, slot, st); break;
    case 2: e = spread_t<T, 12, 16>(a, nchunk, chunk, sy_, s64, sV, qv, grid, use_smem, vg, sm_spread, slot, st); break;
    case 3: e = spread_t<T, 14, 16>(a, nchunk, chunk, sy_, s64, sV, qv, grid, use_smem, vg, sm_spread, slot, st); break;
    default: e = spread_t<T, 0, 0>(a, nchunk, chunk, sy_, s64, sV, qv, grid, use_smem, vg, sm_spread, slot, st); break;
  }
  if (e != cudaSuccess) return e;
  const int fth = std::min(512, std::max(32, a.nf / 2));
  const size_t sm_fft = (size_t)a.nf * sizeof(double2);
  if (sm_fft > 48 * 1024) {
    e = raise_smem((const void*)k_nufft_fwd, 8, sm_fft);
    if (e == cudaSuccess) e = raise_smem((const void*)k_nufft_inv, 9, sm_fft);
    if (e != cudaSuccess) return e;
  }
  e = launch_or_record(k_nufft_fwd, k_nufft_fwd_multi, PH_FWD, dim3((nline + 1) / 2), fth, sm_fft, st,
                       FwdArgs{a, grid, Fk});
  if (e != cudaSuccess) return e;
  const int wg = grad != nullptr && K != PFMM_STOKES;
  const dim3 gm((nnu + 127) / 128, a.nrhs);
  const dim3 gg((a.M + 127) / 128, (K == PFMM_STOKES || wg) ? a.npk : a.n_gl, a.nrhs);
  const Geom& g = p->geom;
  if (K == PFMM_STOKES) {
    k_p1_modes<PFMM_STOKES><<<gm, 128, 0, st>>>(a, g, nodes, nq0, nnu, dl, alpha, Fk, lines);
    k_p1_gather<PFMM_STOKES><<<gg, 128, 0, st>>>(a, nodes, nq0, nnu, dl, alpha, lines, spec, 0);
  } else if (K == PFMM_MODHELM) {
    k_p1_modes<PFMM_MODHELM><<<gm, 128, 0, st>>>(a, g, nodes, nq0, nnu, dl, alpha, Fk, lines);
    k_p1_gather<PFMM_MODHELM><<<gg, 128, 0, st>>>(a, nodes, nq0, nnu, dl, alpha, lines, spec, wg);
  } else {
    k_p1_modes<PFMM_LAPLACE><<<gm, 128, 0, st>>>(a, g, nodes, nq0, nnu, dl, alpha, Fk, lines);
    k_p1_gather<PFMM_LAPLACE><<<gg, 128, 0, st>>>(a, nodes, nq0, nnu, dl, alpha, lines, spec, wg);
  }
  e = launch_or_record(k_nufft_inv, k_nufft_inv_multi, PH_INV, dim3(a.nrhs * a.npk), fth, sm_fft, st,
                       InvArgs{a, spec, mixed ? 1 : 0});
  if (e != cudaSuccess) return e;
  const T* t64 = self ? s64 : (mixed ? (const T*)(ws + L.trgf) : (const T*)(ws + L.trg64));
  const int* tV = self ? sV : (const int*)(ws + L.trgV);
  const int ni = (int)((nt + 127) / 128);
  if (K == PFMM_STOKES) {
    // velocity components are not coordinates: the plain frame
    e = interp_k<T, PFMM_STOKES>(wspec, ni, a, g, t64 + nt, t64, tV, spec, pot, nullptr, st);
    if (e != cudaSuccess) return e;
  } else {
    // the interpolation's "x" derivative is along its transform coordinate
    // (y here) and its "y" derivative along the GL lines (x): swap the
    // columns of the rotation that maps the canonical gradient back
    Geom gs = g;
    gs.rot[0] = g.rot[2];
    gs.rot[1] = g.rot[3];
    gs.rot[2] = g.rot[0];
    gs.rot[3] = g.rot[1];
    e = interp_k<T, PFMM_LAPLACE>(wspec, ni, a, gs, t64 + nt, t64, tV, spec, pot, wg ? grad : nullptr, st);
    if (e != cudaSuccess) return e;
  }
  g_launches += 6;
  return cudaGetLastError();
}

cudaError_t launch_far_nufft(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot,
                             double* grad, cudaStream_t st) {
  if (p->p1_nu) {
    // singly periodic: the nodes below the cut on the direct kernels (they
    // write the outputs), the rest through the transforms (they add)
    pfmm_plan q = *p;
    q.far.Nq = p->p1_nq0;
    q.far.nterm = 2 * p->p1_nq0;
    cudaError_t e = launch_far_direct(&q, ws, ns, nt, self, pot, grad, st);
    if (e != cudaSuccess) return e;
    return (p->opts.precision == PFMM_MIXED) ? run_p1_nufft<float>(p, ws, ns, nt, self, pot, grad, st)
                                             : run_p1_nufft<double>(p, ws, ns, nt, self, pot, grad, st);
  }
  // west/east terms and the m = 0 moment term on the direct kernels (their
  // number of nodes does not grow with the aspect ratio), south/north here.
  pfmm_plan q = *p;
  q.far.nsn = 0;
  q.far.M = 0;
  q.far.nterm = 2 * q.far.Nq;
  q.far2.nsn = 0;  // modified Stokes: the Laplace family's west/east terms
  q.far2.M = 0;
  q.far2.nterm = 2 * q.far2.Nq;
  cudaError_t e = launch_far_direct(&q, ws, ns, nt, self, pot, grad, st);
  if (e != cudaSuccess) return e;
  if (p->far.M > 0) {
    e = (p->opts.precision == PFMM_MIXED) ? run_nufft<float>(p, ws, ns, nt, self, pot, grad, st)
                                          : run_nufft<double>(p, ws, ns, nt, self, pot, grad, st);
  }
  return e;
}

}  // namespace pfmm
