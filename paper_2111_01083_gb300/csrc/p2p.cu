// Near-image P2P: u(t_l) += sum over the (2 m0 + 1) x 3 images l_mn of
// Lambda_near (Sec. 1) and sources j of G(t_l - s_j - l_mn) q_j, pairs at zero
// distance skipped (Eq. nearfarsplit: this is K^near q).
//
// Mixed kernel (k_p2p_mixed): FP32 pair arithmetic.  Coordinates enter as
// hi/lo float pairs: the target minus the image offset is formed in FP64 once
// per (target, image) and split, sources carry (x_hi, x_lo, y_hi, y_lo), and
// dx = (tx_hi - sx_hi) + (tx_lo - sx_lo) is the true difference to FP32
// rounding even for close pairs in a long cell.  Each source is read from
// shared memory once and applied to all images (target splits live in
// registers).  Pair terms are summed in FP32 over 8 sources x all images and
// those partial sums are added with Kahan compensation; the result is added
// into the FP64 output.  Logs and reciprocals use the MUFU approximations
// lg2.approx / rcp.approx (rel. error ~2^-22).
//
// FP64 kernel (k_p2p_f64): the same sum in double precision with log(),
// division and the FP64 Bessel routines.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include "pfmm_impl.h"
#include "p2p.h"
#include "sort.h"
#include "packed.cuh"
#include "bessel.cuh"

namespace pfmm {

constexpr int kP2PThreads = 128;
constexpr int kP2PTile = 128;
constexpr int kP2PSub = 16;    // sources per FP32 partial sum (then Kahan)
constexpr int kP2PUnroll = 4;

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct KahanF {
  float s, c;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// P2PArgs is declared in p2p.h

// Structure of the mixed kernels.  For each source j the contributions of all
// near images are first summed WITHOUT the strength (image sums such as
// L_j = sum_i log2 r_ij^2, Gx_j = sum_i dx_ij / r_ij^2), then multiplied by
// q_j once per rhs.  The image sums have no sign cancellation; the cancelling
// sum over sources (zero net charge) then has 9-15x fewer FP32 additions.
// The log terms of source j are combined through one logarithm of a product:
//   L_j = log2( prod_i r_ij^2 2^-e_i ) = sum_i log2 r_ij^2 - E,  E = sum_i e_i,
// with e_i an integer close to the mean of log2 r^2 over image i, so the
// product stays near 1 and L_j is small: its FP32 error is then a few 1e-7
// absolute whatever the cell size, and one MUFU lg2 serves all images of the
// pair (target, source).  With zero net charge sum_j q_j E cancels; the
// epilogue adds E sum_j q_j back in FP64 from the moments.  A skipped
// zero-distance pair enters the product as 1 * 2^-e_i, which the same
// add-back accounts for.  The Stokes velocity uses the per-source sums
// L, G1 = sum (dx^2 - dy^2)/r^2 and G2 = sum dx dy / r^2 (Axx = (n + G1)/2,
// Ayy = (n - G1)/2 with n the images used; the constant isotropic part is
// added back in FP64 like the log shift).
// Partial sums over kP2PSub sources are added with Kahan compensation.
//
// Laplace/Stokes kernel: two targets per thread packed in float2, so each
// pair-level FP32 operation is one FFMA2/FADD2/FMUL2 for two pairs; logs and
// reciprocals on the MUFU pipe (lg2.approx / rcp.approx).
//
// Output scaling constants:
//   Laplace: pot = -(ln2/4pi) sum q log2(r^2); grad = -(1/2pi) sum q (t-s)/r^2
//   Stokes : u = -(ln2/8pi) [ sum log2(r^2) f - (2/ln2) sum (r.f/r^2) r ]
//   modhelm: pot = (1/2pi) sum q K0;  grad = -(beta/2pi) sum q K1 (t-s)/r
// Hi/lo coordinates of the padding source at slot k of a tile: its subtile
// centre (so that the exact and the relative paths see the same point).
__device__ __forceinline__ float4 s_c_src(const P2PArgs& a, int jb, int k, int nb) {
  const int sub = k / kSubtile;
  return (sub * kSubtile < nb) ? a.s_sub[jb / kSubtile + sub] : make_float4(0.f, 0.f, 0.f, 0.f);
}

struct Kahan2 {
  float2 s, c;
  __device__ __forceinline__ void add(float2 v) {
    float2 y = add2(v, make_float2(-c.x, -c.y));
    float2 t = add2(s, y);
    c = add2(add2(t, make_float2(-s.x, -s.y)), make_float2(-y.x, -y.y));
    s = t;
  }
};

// Body of the Laplace/Stokes mixed kernel for one work item: target block bx
// (2 * kP2PThreads sorted targets), sorted sources [j0, j1), rhs r0 .. r0 + NR - 1.
//
// Coordinate differences.  Sources come in subtiles of 16 with a common centre
// c; per (target, image, subtile) the target minus image minus centre is
// formed once from its hi/lo parts, and per source one FP32 subtraction gives
// dx.  Its absolute error is a few ulp of the subtile extent h, so where a
// target lies within about h of the subtile (the expanded-box test below,
// rarely true since targets and sources are sorted) that subtile instead takes
// the exact path dx = (t_hi - s_hi) + (t_lo - s_lo).  Elsewhere r >= h and the
// relative error of dx stays near 1e-7.
template <int KER, int NIMG, int NR, bool GRAD>
__device__ __forceinline__ void p2p_mixed_body(const P2PArgs& a, int bx, int j0, int j1, int r0) {
  static_assert(KER != PFMM_MODHELM, "packed kernel is for Laplace/Stokes");
  constexpr int NC = (KER == PFMM_STOKES) ? 2 : 1;
  constexpr int CENTER = NIMG / 2;
  constexpr int NA = (KER == PFMM_STOKES) ? 2 : (GRAD ? 3 : 1);
  constexpr int NSUB = kP2PTile / kSubtile;
  __shared__ float2 s_p[kP2PTile];
  __shared__ float4 s_h[kP2PTile];
  __shared__ float4 s_c[NSUB];
  __shared__ float2 s_e[NSUB];
  __shared__ float s_q[NR * NC][kP2PTile];

  const int l0 = (bx * kP2PThreads + threadIdx.x) * 2;
  const bool inA = l0 < a.nt, inB = l0 + 1 < a.nt;
  const int nr = min(NR, a.nrhs - r0);
  float kimg[NIMG];
#pragma unroll
  for (int i = 0; i < NIMG; ++i) kimg[i] = a.kimg[i];

  float2 thx[NIMG], tlx[NIMG], thy[NIMG], tly[NIMG];
  {
    const int lA = inA ? l0 : 0, lB = inB ? l0 + 1 : lA;
    const double txA = a.trg64[lA], tyA = a.trg64[a.nt + lA];
    const double txB = a.trg64[lB], tyB = a.trg64[a.nt + lB];
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      const double ox = a.g.off[i][0], oy = a.g.off[i][1];
      const double vxA = txA - ox, vyA = tyA - oy, vxB = txB - ox, vyB = tyB - oy;
      thx[i] = make_float2((float)vxA, (float)vxB);
      tlx[i] = make_float2((float)(vxA - (double)thx[i].x), (float)(vxB - (double)thx[i].y));
      thy[i] = make_float2((float)vyA, (float)vyB);
      tly[i] = make_float2((float)(vyA - (double)thy[i].x), (float)(vyB - (double)thy[i].y));
    }
  }
  Kahan2 K[NR][NA];
  float2 S[NR][NA];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      K[r][k].s = K[r][k].c = f2(0.f);
      S[r][k] = f2(0.f);
    }
  constexpr float kStokesC = -2.0f / 0.69314718055994531f;  // -(1/4pi) / (ln2/8pi)

  // image sums of one source (dx, dy per image from `diff`), then one FMA per rhs
  auto source = [&](int jj, auto diff) {
    float2 P = f2(1.f), G1 = f2(0.f), G2 = f2(0.f), cnt = f2((float)NIMG);
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      float2 dx, dy;
      diff(i, dx, dy);
      float2 r2 = fma2(dx, dx, mul2(dy, dy));
      float2 msk = f2(1.0f);
      if (i == CENTER) {
        msk = make_float2(r2.x > 0.f ? 1.f : 0.f, r2.y > 0.f ? 1.f : 0.f);
        r2 = make_float2(r2.x > 0.f ? r2.x : 1.f, r2.y > 0.f ? r2.y : 1.f);
        cnt = add2(cnt, add2(msk, f2(-1.0f)));
      }
      float2 inv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
      if (i == CENTER) inv = mul2(inv, msk);
      P = mul2(P, mul2(r2, f2(kimg[i])));
      if (KER == PFMM_LAPLACE) {
        if (GRAD) {
          G1 = fma2(dx, inv, G1);
          G2 = fma2(dy, inv, G2);
        }
      } else {
        // G1 = sum (dx^2 - dy^2)/r^2 (= sum cos 2theta, centred), G2 = sum dx dy / r^2
        const float2 dx2 = mul2(dx, dx);
        const float2 t = fma2(make_float2(-dy.x, -dy.y), dy, dx2);
        G1 = fma2(t, inv, G1);
        G2 = fma2(mul2(dx, inv), dy, G2);
      }
    }
    const float2 L = make_float2(lg2_approx(P.x), lg2_approx(P.y));
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (KER == PFMM_LAPLACE) {
        const float2 q = f2(s_q[r][jj]);
        S[r][0] = fma2(q, L, S[r][0]);
        if (GRAD) {
          S[r][1 % NA] = fma2(q, G1, S[r][1 % NA]);
          S[r][2 % NA] = fma2(q, G2, S[r][2 % NA]);
        }
      } else {
        // Axx = (cnt + G1)/2, Ayy = (cnt - G1)/2; the isotropic part C nimg/2 is
        // moved into the FP64 add-back:  u_x += fx (Lx + C G1/2) + fy C G2,
        // u_y += fx C G2 + fy (Lx - C G1/2),  Lx = L + C (cnt - nimg)/2
        const float2 fx = f2(s_q[r * NC][jj]), fy = f2(s_q[r * NC + NC - 1][jj]);
        const float2 Lx = fma2(add2(cnt, f2(-(float)NIMG)), f2(0.5f * kStokesC), L);
        const float2 h1 = mul2(G1, f2(0.5f * kStokesC)), cxy = mul2(G2, f2(kStokesC));
        S[r][0] = fma2(fx, add2(Lx, h1), fma2(fy, cxy, S[r][0]));
        S[r][NA - 1] = fma2(fx, cxy, fma2(fy, add2(Lx, make_float2(-h1.x, -h1.y)), S[r][NA - 1]));
      }
    }
  };

  for (int jb = j0; jb < j1; jb += kP2PTile) {
    const int nb = min(kP2PTile, j1 - jb);
    __syncthreads();
    for (int k = threadIdx.x; k < kP2PTile; k += kP2PThreads) {
      // padding: a zero-strength source at its subtile centre (inside the cell:
      // finite r^2 in every image; a zero distance can only occur in the centre
      // image, which is masked)
      const bool v = k < nb;
      s_p[k] = v ? a.s_rel[jb + k] : make_float2(0.f, 0.f);
      s_h[k] = v ? a.s_hl[jb + k] : s_c_src(a, jb, k, nb);
      if (k < NSUB) {
        s_c[k] = (k * kSubtile < nb) ? a.s_sub[jb / kSubtile + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        s_e[k] = (k * kSubtile < nb) ? a.s_ext[jb / kSubtile + k] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2)
          s_q[r * NC + c2][k] = (v && r < nr) ? a.qs[((size_t)(r0 + r) * NC + c2) * a.ns + jb + k] : 0.f;
    }
    __syncthreads();
    for (int js = 0; js < nb; js += kP2PSub) {
      // target minus image minus subtile centre, from the hi/lo parts
      float2 txr[NIMG], tyr[NIMG];
      bool near = false;
      {
        const float4 c = s_c[js / kSubtile];
        const float2 e = s_e[js / kSubtile];
        const float bxe = 2.f * e.x + e.y, bye = e.x + 2.f * e.y;  // expanded half extents
        const float2 nch = f2(-c.x), ncl = f2(-c.y), nyh = f2(-c.z), nyl = f2(-c.w);
#pragma unroll
        for (int i = 0; i < NIMG; ++i) {
          txr[i] = add2(add2(thx[i], nch), add2(tlx[i], ncl));
          tyr[i] = add2(add2(thy[i], nyh), add2(tly[i], nyl));
          near |= (fabsf(txr[i].x) < bxe && fabsf(tyr[i].x) < bye) || (fabsf(txr[i].y) < bxe && fabsf(tyr[i].y) < bye);
        }
      }
      if (near) {
#pragma unroll 1
        for (int jj = js; jj < js + kP2PSub; ++jj) {
          const float4 h = s_h[jj];
          const float2 nxh = f2(-h.x), nxl = f2(-h.y), nyh = f2(-h.z), nyl = f2(-h.w);
          source(jj, [&](int i, float2& dx, float2& dy) {
            dx = add2(add2(thx[i], nxh), add2(tlx[i], nxl));
            dy = add2(add2(thy[i], nyh), add2(tly[i], nyl));
          });
        }
      } else {
#pragma unroll kP2PUnroll
        for (int jj = js; jj < js + kP2PSub; ++jj) {
          const float2 p = s_p[jj];
          const float2 nsx = f2(-p.x), nsy = f2(-p.y);
          source(jj, [&](int i, float2& dx, float2& dy) {
            dx = add2(txr[i], nsx);
            dy = add2(tyr[i], nsy);
          });
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          K[r][k].add(S[r][k]);
          S[r][k] = f2(0.f);
        }
    }
  }
  const double* R = a.g.rot;
  const double lgc = (double)a.lgc;  // = E (sum of the image exponents)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const bool in = h == 0 ? inA : inB;
    if (!in) continue;
    const int l = a.t_perm ? a.t_perm[l0 + h] : l0 + h;
    for (int r = 0; r < nr; ++r) {
      auto val = [&](int k) {
        const float2 s2 = K[r][k].s, c2 = K[r][k].c;
        return h == 0 ? (double)s2.x - (double)c2.x : (double)s2.y - (double)c2.y;
      };
      if (KER == PFMM_STOKES) {
        const double cst = -0.69314718055994531 / (8.0 * M_PI);
        double sx = val(0), sy = val(NA - 1);
        if (j0 == 0) {
          const double add = lgc + NIMG * 0.5 * (double)kStokesC;
          sx += add * a.mom[(r0 + r) * 8 + 0];
          sy += add * a.mom[(r0 + r) * 8 + 1];
        }
        const double ux = cst * sx, uy = cst * sy;
        atomicAdd(a.pot + ((size_t)(r0 + r) * 2) * a.os + l, R[0] * ux + R[2] * uy);
        atomicAdd(a.pot + ((size_t)(r0 + r) * 2 + 1) * a.os + l, R[1] * ux + R[3] * uy);
      } else {
        const double cp = -0.69314718055994531 / (4.0 * M_PI), cg = -1.0 / (2.0 * M_PI);
        double sp = val(0);
        if (j0 == 0) sp += lgc * a.mom[(r0 + r) * 8 + 0];
        if (a.pot) atomicAdd(a.pot + (size_t)(r0 + r) * a.os + l, cp * sp);
        if (GRAD && a.grad) {
          const double gx = cg * val(1 % NA), gy = cg * val(2 % NA);
          atomicAdd(a.grad + ((size_t)(r0 + r) * 2) * a.os + l, R[0] * gx + R[2] * gy);
          atomicAdd(a.grad + ((size_t)(r0 + r) * 2 + 1) * a.os + l, R[1] * gx + R[3] * gy);
        }
      }
    }
  }
}

template <int KER, int NIMG, int NR, bool GRAD>
__global__ void __launch_bounds__(kP2PThreads, 1) k_p2p_mixed(const __grid_constant__ P2PArgs a) {
  const int j0 = blockIdx.y * a.chunk;
  p2p_mixed_body<KER, NIMG, NR, GRAD>(a, blockIdx.x, j0, min(a.ns, j0 + a.chunk), a.r0 + blockIdx.z * NR);
}

// Modified Helmholtz mixed kernel: one target per thread, targets and sources
// in spatially sorted order, per-source image sums K0s = sum_i K0(beta r_i),
// K1x = sum_i K1(beta r_i) dx_i / r_i (and y), then one FMA per rhs (strengths
// read four at a time).  Pairs with beta r > x_c are skipped (plan: every skipped
// term below tol/10 / (images * ns)): per (target block, source
// tile, image) an FP64 test on the outward-rounded boxes classifies the image
// as skipped (boxes farther apart than x_c / beta, x_c from the plan: every
// skipped term below tol/10 / (images * ns)), complete (every pair within
// the cutoff: no per-pair test) or partial (pairs beyond the cutoff skipped).
// Two targets per thread in packed FP32 was measured slower here (register
// pressure halves the resident warps of this branch-heavy kernel).
template <int KER, int NIMG, int NR, bool GRAD>
__device__ __forceinline__ void p2p_mixed_mh_body(const P2PArgs& a, int bx, int j0, int j1, int r0) {
  constexpr int CENTER = NIMG / 2;
  constexpr int NA = GRAD ? 3 : 1;
  constexpr int NSUB = kP2PTile / kSubtile;
  __shared__ float2 s_p[kP2PTile];
  __shared__ float2 s_pb[kP2PTile];  // beta-scaled relative coordinates (far path)
  __shared__ float4 s_h[kP2PTile];
  __shared__ float4 s_c[NSUB];
  __shared__ float2 s_e[NSUB];
  constexpr int NQ4 = (NR + 3) / 4;
  __shared__ float4 s_q4[NQ4][kP2PTile];
  const int l = bx * kP2PThreads + threadIdx.x;
  const bool in = l < a.nt;
  const int nr = min(NR, a.nrhs - r0);
  // hi/lo target coordinates per image, one column per thread in shared
  // memory (read once per 16-source subtile; registers go to the pair loops)
  __shared__ float s_tc[4][NIMG][kP2PThreads];
  {
    const double tx = in ? a.trg64[l] : 0.0, ty = in ? a.trg64[a.nt + l] : 0.0;
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      double vx = tx - a.g.off[i][0], vy = ty - a.g.off[i][1];
      const float hx = (float)vx, hy = (float)vy;
      s_tc[0][i][threadIdx.x] = hx;
      s_tc[1][i][threadIdx.x] = (float)(vx - (double)hx);
      s_tc[2][i][threadIdx.x] = hy;
      s_tc[3][i][threadIdx.x] = (float)(vy - (double)hy);
    }
  }
  auto thx = [&](int i) { return s_tc[0][i][threadIdx.x]; };
  auto tlx = [&](int i) { return s_tc[1][i][threadIdx.x]; };
  auto thy = [&](int i) { return s_tc[2][i][threadIdx.x]; };
  auto tly = [&](int i) { return s_tc[3][i][threadIdx.x]; };
  KahanF K[NR][NA];
  float S[NR][NA];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      K[r][k].s = K[r][k].c = 0.f;
      S[r][k] = 0.f;
    }
  const float beta = a.beta_f;
  const float beta2 = beta * beta;
  const float cut2 = a.cut * a.cut;
  const float4 tb = a.t_box[bx];
  const float rsm = 2.0f / beta * 1.001f + 1e-6f;  // beta r <= 2 region, with margin
  float txr[NIMG], tyr[NIMG];

  // image sums of one source over the images in `any` (`all`: no per-pair
  // cutoff test), then one FMA per rhs
  auto source = [&](int jj, unsigned any, unsigned all, auto diff) {
    float K0s = 0.f, K1x = 0.f, K1y = 0.f;
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      if (!(any & (1u << i))) continue;
      float dx, dy;
      diff(i, dx, dy);
      float r2 = fmaf(dx, dx, dy * dy);
      float msk = 1.0f;
      if (i == CENTER) {
        msk = (r2 > 0.0f) ? 1.0f : 0.0f;
        r2 = (r2 > 0.0f) ? r2 : 1.0f;
      }
      // pairs beyond the cutoff x_c / beta of a partial image are
      // skipped (the branch is not taken at all when no lane of the warp needs it)
      if ((all & (1u << i)) || r2 < cut2) {
        const float x2 = beta2 * r2;
        if (GRAD) {
          float k0, k1ix;
          bes::k01f_x2(x2, &k0, &k1ix);  // k1ix = K1(x) / x
          K0s = fmaf(k0, msk, K0s);
          const float k1r = k1ix * beta * msk;  // K1(beta r) / r = beta K1(x) / x
          K1x = fmaf(k1r, dx, K1x);
          K1y = fmaf(k1r, dy, K1y);
        } else {
          K0s = fmaf(bes::k0f_x2(x2), msk, K0s);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < NQ4; ++g) {
      const float4 q4 = s_q4[g][jj];
      const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 4 * g + k;
        if (r >= NR) break;
        S[r][0] = fmaf(qv[k], K0s, S[r][0]);
        if (GRAD) {
          S[r][1 % NA] = fmaf(qv[k], K1x, S[r][1 % NA]);
          S[r][2 % NA] = fmaf(qv[k], K1y, S[r][2 % NA]);
        }
      }
    }
  };

  // Branch-free variant for subtiles where no pair of the warp can have
  // beta r <= 2: every image takes the large-argument fit (K0 at beta r > 88
  // underflows to 0), so the nine chains are independent and interleave.
  // Coordinates here are scaled by beta (beta txr, beta tyr per pair, the
  // source's in shared memory), so x^2 = dx^2 + dy^2 and K1(x)/x multiplies
  // the scaled difference directly; the fits' variable y = 2/x is folded into
  // their coefficients (c_k 2^k).  ALL: every image active, no per-image test.
  auto source_far = [&](int jj, unsigned any, auto diff, auto all_tag) {
    constexpr bool ALL = decltype(all_tag)::value;
    float K0s = 0.f, K1x = 0.f, K1y = 0.f;
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      if (!ALL && !(any & (1u << i))) continue;
      float dx, dy;
      diff(i, dx, dy);
      const float x2 = fmaf(dx, dx, dy * dy);
      const float ix = bes::mufu::rsqrt(x2);
      const float x = x2 * ix;
      const float e = bes::mufu::ex2(-1.4426950408889634f * x) * bes::mufu::rsqrt(x);
      const float k0 = e * (1.25331414f + ix * (-0.15664716f + ix * (0.08758272f + ix * (-0.08499568f + ix * (0.09405952f + ix * (-0.0804928f + ix * 0.03405312f))))));
      K0s += k0;
      if (GRAD) {
        const float k1ix = e * ix * (1.25331414f + ix * (0.46997238f + ix * (-0.1462248f + ix * (0.12034144f + ix * (-0.12485648f + ix * (0.10419648f + ix * (-0.0436768f)))))));
        K1x = fmaf(k1ix, dx, K1x);
        K1y = fmaf(k1ix, dy, K1y);
      }
    }
#pragma unroll
    for (int g = 0; g < NQ4; ++g) {
      const float4 q4 = s_q4[g][jj];
      const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 4 * g + k;
        if (r >= NR) break;
        S[r][0] = fmaf(qv[k], K0s, S[r][0]);
        if (GRAD) {
          S[r][1 % NA] = fmaf(qv[k], K1x, S[r][1 % NA]);
          S[r][2 % NA] = fmaf(qv[k], K1y, S[r][2 % NA]);
        }
      }
    }
  };

  // Packed form of source_far for subtiles where every image is active, on
  // the potential: the images go two per FADD2/FMUL2/FFMA2 (the MUFU
  // operations stay one per value), which halves the issue slots of the
  // arithmetic; bx2/by2 hold the beta-scaled target coordinates relative to
  // the subtile centre for the image pairs (2k, 2k + 1), (bxs, bys) those of
  // the last image (NIMG is odd).
  auto source_far_pk = [&](int jj, const float2* bx2, const float2* by2, float bxs, float bys) {
    const float2 p = s_pb[jj];
    const float2 npx = f2(-p.x), npy = f2(-p.y);
    float2 acc = f2(0.f);
#pragma unroll
    for (int k = 0; k < NIMG / 2; ++k) {
      const float2 dx = add2(bx2[k], npx), dy = add2(by2[k], npy);
      const float2 x2 = fma2(dx, dx, mul2(dy, dy));
      const float2 ix = make_float2(bes::mufu::rsqrt(x2.x), bes::mufu::rsqrt(x2.y));
      const float2 x = mul2(x2, ix);
      const float2 ar = mul2(x, f2(-1.4426950408889634f));
      const float2 e = mul2(make_float2(bes::mufu::ex2(ar.x), bes::mufu::ex2(ar.y)),
                            make_float2(bes::mufu::rsqrt(x.x), bes::mufu::rsqrt(x.y)));
      float2 pl = fma2(ix, f2(0.03405312f), f2(-0.0804928f));
      pl = fma2(ix, pl, f2(0.09405952f));
      pl = fma2(ix, pl, f2(-0.08499568f));
      pl = fma2(ix, pl, f2(0.08758272f));
      pl = fma2(ix, pl, f2(-0.15664716f));
      pl = fma2(ix, pl, f2(1.25331414f));
      acc = fma2(e, pl, acc);
    }
    float K0s;
    {
      const float dx = bxs - p.x, dy = bys - p.y;
      const float x2 = fmaf(dx, dx, dy * dy);
      const float ix = bes::mufu::rsqrt(x2);
      const float x = x2 * ix;
      const float e = bes::mufu::ex2(-1.4426950408889634f * x) * bes::mufu::rsqrt(x);
      const float k0 = e * (1.25331414f + ix * (-0.15664716f + ix * (0.08758272f + ix * (-0.08499568f + ix * (0.09405952f + ix * (-0.0804928f + ix * 0.03405312f))))));
      K0s = (acc.x + acc.y) + k0;
    }
#pragma unroll
    for (int g = 0; g < NQ4; ++g) {
      const float4 q4 = s_q4[g][jj];
      const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 4 * g + k;
        if (r >= NR) break;
        S[r][0] = fmaf(qv[k], K0s, S[r][0]);
      }
    }
  };

  // Tiles are classified kP2PThreads at a time, one thread per tile: per
  // image, some pair within the cutoff (any) or every pair within it (all).
  // FP32 on the outward-rounded boxes with a relative margin: a tile
  // misjudged at the margin only adds or drops terms below the cutoff's bound.
  // Culled tiles then cost no barrier.
  __shared__ unsigned s_tany[kP2PThreads], s_tall[kP2PThreads];
  const int ntile = (j1 - j0 + kP2PTile - 1) / kP2PTile;
  for (int g0 = 0; g0 < ntile; g0 += kP2PThreads) {
    __syncthreads();
    {
      const int t = g0 + threadIdx.x;
      unsigned many = 0u, mall = 0u;
      if (t < ntile) {
        const float4 sb = a.s_box[(j0 + t * kP2PTile) / kBoxTile];
        const float c2 = a.cut * a.cut;
        const float hx = tb.z + sb.z, hy = tb.w + sb.w;
#pragma unroll 1
        for (int i = 0; i < NIMG; ++i) {
          const float cx = fabsf(tb.x - a.offf[i][0] - sb.x), cy = fabsf(tb.y - a.offf[i][1] - sb.y);
          const float mx = 1e-5f * (fabsf(tb.x) + fabsf(sb.x) + fabsf(a.offf[i][0])) + 1e-6f * hx;
          const float my = 1e-5f * (fabsf(tb.y) + fabsf(sb.y) + fabsf(a.offf[i][1])) + 1e-6f * hy;
          const float ex = fmaxf(0.f, cx - hx - mx), ey = fmaxf(0.f, cy - hy - my);
          const float fx = cx + hx + mx, fy = cy + hy + my;
          if (ex * ex + ey * ey <= c2) many |= 1u << i;
          if (fx * fx + fy * fy < c2) mall |= 1u << i;
        }
        if (a.work && many) {
          const int nbt = min(kP2PTile, j1 - (j0 + t * kP2PTile));
          atomicAdd(a.work, (unsigned long long)__popc(many) * (unsigned long long)nbt *
                                (unsigned long long)min(kP2PThreads, a.nt - bx * kP2PThreads));
        }
      }
      s_tany[threadIdx.x] = many;
      s_tall[threadIdx.x] = mall;
    }
    __syncthreads();
    const int gn = min(kP2PThreads, ntile - g0);
  for (int tt = 0; tt < gn; ++tt) {
    const unsigned any = s_tany[tt], all = s_tall[tt];
    if (any == 0u) continue;
    const int jb = j0 + (g0 + tt) * kP2PTile;
    const int nb = min(kP2PTile, j1 - jb);
    __syncthreads();
    for (int k = threadIdx.x; k < kP2PTile; k += kP2PThreads) {
      // padding: zero strength at the subtile centre (finite distances)
      const bool v = k < nb;
      s_p[k] = v ? a.s_rel[jb + k] : make_float2(0.f, 0.f);
      s_pb[k] = make_float2(beta * s_p[k].x, beta * s_p[k].y);
      s_h[k] = v ? a.s_hl[jb + k] : s_c_src(a, jb, k, nb);
      if (k < NSUB) {
        s_c[k] = (k * kSubtile < nb) ? a.s_sub[jb / kSubtile + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        s_e[k] = (k * kSubtile < nb) ? a.s_ext[jb / kSubtile + k] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int g = 0; g < NQ4; ++g) {
        float qv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int r = 4 * g + t;
          qv[t] = (v && r < nr) ? a.qs[(size_t)(r0 + r) * a.ns + jb + k] : 0.f;
        }
        s_q4[g][k] = make_float4(qv[0], qv[1], qv[2], qv[3]);
      }
    }
    __syncthreads();
    for (int js = 0; js < nb; js += kP2PSub) {
      bool near = false, small = false;
      {
        const float4 c = s_c[js / kSubtile];
        const float2 e = s_e[js / kSubtile];
        const float bxe = 2.f * e.x + e.y, bye = e.x + 2.f * e.y;
        // beta r <= 2 possible: target within 2 / beta (+ margin) of the subtile box
        const float sxe = e.x + rsm, sye = e.y + rsm;
#pragma unroll
        for (int i = 0; i < NIMG; ++i) {
          txr[i] = (thx(i) - c.x) + (tlx(i) - c.y);
          tyr[i] = (thy(i) - c.z) + (tly(i) - c.w);
          const bool act = (any & (1u << i)) != 0u;
          near |= act && fabsf(txr[i]) < bxe && fabsf(tyr[i]) < bye;
          small |= act && fabsf(txr[i]) < sxe && fabsf(tyr[i]) < sye;
        }
      }
      if (!__any_sync(0xffffffffu, near || small)) {
        if (!GRAD && (NIMG & 1) && any == (1u << NIMG) - 1u) {
          float2 bx2[NIMG / 2], by2[NIMG / 2];
#pragma unroll
          for (int k = 0; k < NIMG / 2; ++k) {
            bx2[k] = make_float2(beta * txr[2 * k], beta * txr[2 * k + 1]);
            by2[k] = make_float2(beta * tyr[2 * k], beta * tyr[2 * k + 1]);
          }
          const float bxs = beta * txr[NIMG - 1], bys = beta * tyr[NIMG - 1];
#pragma unroll 2
          for (int jj = js; jj < js + kP2PSub; ++jj) source_far_pk(jj, bx2, by2, bxs, bys);
        } else if (any == (1u << NIMG) - 1u) {
#pragma unroll 2
          for (int jj = js; jj < js + kP2PSub; ++jj) {
            const float2 p = s_pb[jj];
            source_far(jj, any, [&](int i, float& dx, float& dy) {
              dx = fmaf(beta, txr[i], -p.x);
              dy = fmaf(beta, tyr[i], -p.y);
            },
                       std::true_type{});
          }
        } else {
#pragma unroll 2
          for (int jj = js; jj < js + kP2PSub; ++jj) {
            const float2 p = s_pb[jj];
            source_far(jj, any, [&](int i, float& dx, float& dy) {
              dx = fmaf(beta, txr[i], -p.x);
              dy = fmaf(beta, tyr[i], -p.y);
            },
                       std::false_type{});
          }
        }
      } else if (!__any_sync(0xffffffffu, small)) {
        // close pairs but none with beta r <= 2: exact differences (beta-scaled),
        // the branch-free large-argument fit
#pragma unroll 1
        for (int jj = js; jj < js + kP2PSub; ++jj) {
          const float4 h = s_h[jj];
          source_far(jj, any, [&](int i, float& dx, float& dy) {
            dx = beta * ((thx(i) - h.x) + (tlx(i) - h.y));
            dy = beta * ((thy(i) - h.z) + (tly(i) - h.w));
          }, std::false_type{});
        }
      } else {
        // close pairs or beta r <= 2 in reach: exact differences, both K0 fits
        // (one code path for both cases keeps the kernel small in the
        // instruction cache)
#pragma unroll 1
        for (int jj = js; jj < js + kP2PSub; ++jj) {
          const float4 h = s_h[jj];
          source(jj, any, all, [&](int i, float& dx, float& dy) {
            dx = (thx(i) - h.x) + (tlx(i) - h.y);
            dy = (thy(i) - h.z) + (tly(i) - h.w);
          });
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          K[r][k].add(S[r][k]);
          S[r][k] = 0.f;
        }
    }
  }
  }
  if (!in) return;
  const int lo = a.t_perm ? a.t_perm[l] : l;
  const double* R = a.g.rot;
  const double cp = 1.0 / (2.0 * M_PI), cg = -a.beta / (2.0 * M_PI);
  for (int r = 0; r < nr; ++r) {
    if (a.pot) atomicAdd(a.pot + (size_t)(r0 + r) * a.os + lo, cp * K[r][0].value());
    if (GRAD && a.grad) {
      const double gx = cg * K[r][1 % NA].value(), gy = cg * K[r][2 % NA].value();
      atomicAdd(a.grad + ((size_t)(r0 + r) * 2) * a.os + lo, R[0] * gx + R[2] * gy);
      atomicAdd(a.grad + ((size_t)(r0 + r) * 2 + 1) * a.os + lo, R[1] * gx + R[3] * gy);
    }
  }
}

// Six resident blocks per SM for the potential-only variants (80 registers,
// a small spill): measured 7 / 1 / 12 % faster on the 256-cell batch at
// beta = 1 / 10 / 100 than the unconstrained 121 registers, whose four blocks
// left the latency of the tile loop exposed.  The gradient variants keep
// their registers (six blocks would spill ~0.6 KB).
template <int KER, int NIMG, int NR, bool GRAD>
__global__ void __launch_bounds__(kP2PThreads, GRAD ? 1 : 6) k_p2p_mixed_mh(const __grid_constant__ P2PArgs a) {
  const int j0 = blockIdx.y * a.chunk;
  p2p_mixed_mh_body<KER, NIMG, NR, GRAD>(a, blockIdx.x, j0, min(a.ns, j0 + a.chunk), a.r0 + blockIdx.z * NR);
}

// Persistent batched kernel: blocks pull work items (cell, target block,
// source range, rhs group) from an atomic counter until the list is done.
// Items are sorted by decreasing cost on the host.  No block ever waits on
// another; the counter is the only shared state.
// P2PItem is declared in p2p.h

template <int NIMG, int NR>
__device__ __forceinline__ void p2p_ms_body(const P2PArgs& a, int bx, int j0, int j1, int r0);

template <int KER, int NIMG, int NR, bool GRAD>
__global__ void __launch_bounds__(kP2PThreads, (KER == PFMM_MODHELM && !GRAD) ? 6 : 1) k_p2p_batch(const P2PArgs* __restrict__ cells,
                                                           const P2PItem* __restrict__ items, int nitems,
                                                           int* __restrict__ counter) {
  __shared__ int s_item;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const P2PItem w = items[it];
    if constexpr (KER == PFMM_MODHELM)
      p2p_mixed_mh_body<KER, NIMG, NR, GRAD>(cells[w.cell], w.bx, w.j0, w.j1, w.r0);
    else if constexpr (KER == PFMM_MSTOKES)
      p2p_ms_body<NIMG, NR>(cells[w.cell], w.bx, w.j0, w.j1, w.r0);
    else
      p2p_mixed_body<KER, NIMG, NR, GRAD>(cells[w.cell], w.bx, w.j0, w.j1, w.r0);
  }
}

// Modified Stokeslet near-image sum (mixed precision).  Per (target, source)
// the image sum of the kernel is formed as one symmetric 2 x 2 matrix
//   G = sum_i (A_i I - B_i r_i r_i^T / r_i^2),  A = K0 + E,  B = K0 + 2E,
//   E = K1(x)/x - 1/x^2,  x = beta r   (times 1/2pi at the end),
// then applied to each rhs's force (4 FMAs).  Differences are the exact hi/lo
// form for every pair (there is no cutoff: the kernel decays like 1/r^2), so
// the target order does not matter; targets are still taken in the sorted
// order with outputs through the permutation.  Per-source terms are summed
// 16 at a time in FP32 and those partial sums Kahan-added.
template <int NIMG, int NR>
__device__ __forceinline__ void p2p_ms_body(const P2PArgs& a, int bx, int j0, int j1, int r0) {
  constexpr int CENTER = NIMG / 2;
  __shared__ float4 s_h[kP2PTile];
  __shared__ float2 s_f[NR][kP2PTile];
  const int l = bx * kP2PThreads + threadIdx.x;
  const bool in = l < a.nt;
  const int nr = min(NR, a.nrhs - r0);
  float thx[NIMG], tlx[NIMG], thy[NIMG], tly[NIMG];
  {
    const double tx = in ? a.trg64[l] : 0.0, ty = in ? a.trg64[a.nt + l] : 0.0;
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      const double vx = tx - a.g.off[i][0], vy = ty - a.g.off[i][1];
      thx[i] = (float)vx;
      tlx[i] = (float)(vx - (double)thx[i]);
      thy[i] = (float)vy;
      tly[i] = (float)(vy - (double)thy[i]);
    }
  }
  const float beta2 = a.beta_f * a.beta_f;
  KahanF K[NR][2];
  float S[NR][2];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      K[r][k].s = K[r][k].c = 0.f;
      S[r][k] = 0.f;
    }
  for (int jb = j0; jb < j1; jb += kP2PTile) {
    const int nb = min(kP2PTile, j1 - jb);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += kP2PThreads) {
      s_h[k] = a.s_hl[jb + k];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const bool v = r < nr;
        s_f[r][k] = make_float2(v ? a.qs[((size_t)(r0 + r) * 2) * a.ns + jb + k] : 0.f,
                                v ? a.qs[((size_t)(r0 + r) * 2 + 1) * a.ns + jb + k] : 0.f);
      }
    }
    __syncthreads();
    for (int js = 0; js < nb; js += kSubtile) {
      const int je = min(nb, js + kSubtile);
#pragma unroll 1
      for (int jj = js; jj < je; ++jj) {
        const float4 h = s_h[jj];
        float g11 = 0.f, g12 = 0.f, g22 = 0.f;
#pragma unroll
        for (int i = 0; i < NIMG; ++i) {
          const float dx = (thx[i] - h.x) + (tlx[i] - h.y);
          const float dy = (thy[i] - h.z) + (tly[i] - h.w);
          float r2 = fmaf(dx, dx, dy * dy);
          float msk = 1.0f;
          if (i == CENTER) {
            msk = (r2 > 0.0f) ? 1.0f : 0.0f;  // a target on a source: the pair is skipped
            r2 = (r2 > 0.0f) ? r2 : 1.0f;
          }
          float k0, e;
          bes::k0ef_x2(beta2 * r2, &k0, &e);
          const float A = (k0 + e) * msk;
          const float Bn = (k0 + 2.0f * e) * msk * bes::mufu::rcp(r2);
          const float bx = Bn * dx;
          g11 += A - bx * dx;
          g12 -= bx * dy;
          g22 += A - Bn * dy * dy;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float2 f = s_f[r][jj];
          S[r][0] = fmaf(g11, f.x, fmaf(g12, f.y, S[r][0]));
          S[r][1] = fmaf(g12, f.x, fmaf(g22, f.y, S[r][1]));
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          K[r][k].add(S[r][k]);
          S[r][k] = 0.f;
        }
    }
  }
  if (!in) return;
  const int lo = a.t_perm ? a.t_perm[l] : l;
  const double* R = a.g.rot;
  const double c = 1.0 / (2.0 * M_PI);
  for (int r = 0; r < nr; ++r) {
    const double ux = c * K[r][0].value(), uy = c * K[r][1].value();
    atomicAdd(a.pot + ((size_t)(r0 + r) * 2) * a.os + lo, R[0] * ux + R[2] * uy);
    atomicAdd(a.pot + ((size_t)(r0 + r) * 2 + 1) * a.os + lo, R[1] * ux + R[3] * uy);
  }
}

// Single-cell launch.  The same computation as p2p_ms_body, written out in
// the kernel: the device-function form, which reaches the arguments through
// a reference to the kernel parameter, measured 6 % slower here (162.2 vs
// 152.6 ms on the 1e5 + 1e5 skew-cell workload, same registers), so the
// batched kernel alone uses it.
template <int NIMG, int NR>
__global__ void __launch_bounds__(kP2PThreads) k_p2p_ms(const __grid_constant__ P2PArgs a) {
  constexpr int CENTER = NIMG / 2;
  __shared__ float4 s_h[kP2PTile];
  __shared__ float2 s_f[NR][kP2PTile];
  const int l = blockIdx.x * kP2PThreads + threadIdx.x;
  const bool in = l < a.nt;
  const int r0 = a.r0 + blockIdx.z * NR;
  const int nr = min(NR, a.nrhs - r0);
  float thx[NIMG], tlx[NIMG], thy[NIMG], tly[NIMG];
  {
    const double tx = in ? a.trg64[l] : 0.0, ty = in ? a.trg64[a.nt + l] : 0.0;
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      const double vx = tx - a.g.off[i][0], vy = ty - a.g.off[i][1];
      thx[i] = (float)vx;
      tlx[i] = (float)(vx - (double)thx[i]);
      thy[i] = (float)vy;
      tly[i] = (float)(vy - (double)thy[i]);
    }
  }
  const float beta2 = a.beta_f * a.beta_f;
  KahanF K[NR][2];
  float S[NR][2];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      K[r][k].s = K[r][k].c = 0.f;
      S[r][k] = 0.f;
    }
  const int j0 = blockIdx.y * a.chunk;
  const int j1 = min(a.ns, j0 + a.chunk);
  for (int jb = j0; jb < j1; jb += kP2PTile) {
    const int nb = min(kP2PTile, j1 - jb);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += kP2PThreads) {
      s_h[k] = a.s_hl[jb + k];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const bool v = r < nr;
        s_f[r][k] = make_float2(v ? a.qs[((size_t)(r0 + r) * 2) * a.ns + jb + k] : 0.f,
                                v ? a.qs[((size_t)(r0 + r) * 2 + 1) * a.ns + jb + k] : 0.f);
      }
    }
    __syncthreads();
    for (int js = 0; js < nb; js += kSubtile) {
      const int je = min(nb, js + kSubtile);
#pragma unroll 1
      for (int jj = js; jj < je; ++jj) {
        const float4 h = s_h[jj];
        float g11 = 0.f, g12 = 0.f, g22 = 0.f;
#pragma unroll
        for (int i = 0; i < NIMG; ++i) {
          const float dx = (thx[i] - h.x) + (tlx[i] - h.y);
          const float dy = (thy[i] - h.z) + (tly[i] - h.w);
          float r2 = fmaf(dx, dx, dy * dy);
          float msk = 1.0f;
          if (i == CENTER) {
            msk = (r2 > 0.0f) ? 1.0f : 0.0f;  // a target on a source: the pair is skipped
            r2 = (r2 > 0.0f) ? r2 : 1.0f;
          }
          float k0, e;
          bes::k0ef_x2(beta2 * r2, &k0, &e);
          const float A = (k0 + e) * msk;
          const float Bn = (k0 + 2.0f * e) * msk * bes::mufu::rcp(r2);
          const float bx = Bn * dx;
          g11 += A - bx * dx;
          g12 -= bx * dy;
          g22 += A - Bn * dy * dy;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float2 f = s_f[r][jj];
          S[r][0] = fmaf(g11, f.x, fmaf(g12, f.y, S[r][0]));
          S[r][1] = fmaf(g12, f.x, fmaf(g22, f.y, S[r][1]));
        }
      }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          K[r][k].add(S[r][k]);
          S[r][k] = 0.f;
        }
    }
  }
  if (!in) return;
  const int lo = a.t_perm ? a.t_perm[l] : l;
  const double* R = a.g.rot;
  const double c = 1.0 / (2.0 * M_PI);
  for (int r = 0; r < nr; ++r) {
    const double ux = c * K[r][0].value(), uy = c * K[r][1].value();
    atomicAdd(a.pot + ((size_t)(r0 + r) * 2) * a.os + lo, R[0] * ux + R[2] * uy);
    atomicAdd(a.pot + ((size_t)(r0 + r) * 2 + 1) * a.os + lo, R[1] * ux + R[3] * uy);
  }
}

// FP64 reference-precision kernel.
template <int KER, bool GRAD>
__global__ void __launch_bounds__(kP2PThreads) k_p2p_f64(P2PArgs a) {
  constexpr int NC = (KER == PFMM_STOKES || KER == PFMM_MSTOKES) ? 2 : 1;
  __shared__ double s_x[kP2PTile], s_y[kP2PTile];
  __shared__ double s_q[4][NC][kP2PTile];
  const int l = blockIdx.x * kP2PThreads + threadIdx.x;
  const bool in = l < a.nt;
  const int r0 = a.r0 + blockIdx.z * 4;
  const int nr = min(4, a.nrhs - r0);
  const double tx = in ? a.trg64[l] : 0.0, ty = in ? a.trg64[a.nt + l] : 0.0;
  double acc[4][3];
  for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
  const int j0 = blockIdx.y * a.chunk;
  const int j1 = min(a.ns, j0 + a.chunk);
  for (int jb = j0; jb < j1; jb += kP2PTile) {
    const int nb = min(kP2PTile, j1 - jb);
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += kP2PThreads) {
      s_x[k] = a.src64[jb + k];
      s_y[k] = a.src64[a.ns + jb + k];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < NC; ++c)
          s_q[r][c][k] = (r < nr) ? a.qc[((size_t)(r0 + r) * NC + c) * a.ns + jb + k] : 0.0;
    }
    __syncthreads();
    if (!in) continue;
    for (int i = 0; i < a.g.nimg; ++i) {
      const double ox = tx - a.g.off[i][0], oy = ty - a.g.off[i][1];
      for (int jj = 0; jj < nb; ++jj) {
        const double dx = ox - s_x[jj], dy = oy - s_y[jj];
        const double r2 = dx * dx + dy * dy;
        if (r2 == 0.0) continue;
        if (KER == PFMM_LAPLACE) {
          const double lg = -log(r2) / (4.0 * M_PI);
          const double f = -1.0 / (2.0 * M_PI * r2);
          for (int r = 0; r < nr; ++r) {
            const double q = s_q[r][0][jj];
            acc[r][0] += q * lg;
            if (GRAD) {
              acc[r][1] += q * f * dx;
              acc[r][2] += q * f * dy;
            }
          }
        } else if (KER == PFMM_STOKES) {
          const double lg = -log(r2) / (8.0 * M_PI);
          const double inv = 1.0 / (4.0 * M_PI * r2);
          for (int r = 0; r < nr; ++r) {
            const double fx = s_q[r][0][jj], fy = s_q[r][NC - 1][jj];
            const double s = (dx * fx + dy * fy) * inv;
            acc[r][0] += lg * fx + s * dx;
            acc[r][1] += lg * fy + s * dy;
          }
        } else if (KER == PFMM_MSTOKES) {
          // (1/2pi) (A I - B r r^T / r^2), A = K0 + E, B = K0 + 2E
          double k0, e;
          bes::k0ed(a.beta * sqrt(r2), &k0, &e);
          const double c = 1.0 / (2.0 * M_PI);
          const double A = c * (k0 + e), Bn = c * (k0 + 2.0 * e) / r2;
          for (int r = 0; r < nr; ++r) {
            const double fx = s_q[r][0][jj], fy = s_q[r][NC - 1][jj];
            const double s = (dx * fx + dy * fy) * Bn;
            acc[r][0] += A * fx - s * dx;
            acc[r][1] += A * fy - s * dy;
          }
        } else {
          const double rr = sqrt(r2);
          double k0, k1;
          bes::k01d(a.beta * rr, &k0, &k1);
          const double f = -a.beta * k1 / (2.0 * M_PI * rr);
          for (int r = 0; r < nr; ++r) {
            const double q = s_q[r][0][jj];
            acc[r][0] += q * k0 / (2.0 * M_PI);
            if (GRAD) {
              acc[r][1] += q * f * dx;
              acc[r][2] += q * f * dy;
            }
          }
        }
      }
    }
  }
  if (!in) return;
  const double* R = a.g.rot;
  for (int r = 0; r < nr; ++r) {
    if (KER == PFMM_STOKES || KER == PFMM_MSTOKES) {
      atomicAdd(a.pot + ((size_t)(r0 + r) * 2) * a.os + l, R[0] * acc[r][0] + R[2] * acc[r][1]);
      atomicAdd(a.pot + ((size_t)(r0 + r) * 2 + 1) * a.os + l, R[1] * acc[r][0] + R[3] * acc[r][1]);
    } else {
      if (a.pot) atomicAdd(a.pot + (size_t)(r0 + r) * a.os + l, acc[r][0]);
      if (GRAD && a.grad) {
        atomicAdd(a.grad + ((size_t)(r0 + r) * 2) * a.os + l, R[0] * acc[r][1] + R[2] * acc[r][2]);
        atomicAdd(a.grad + ((size_t)(r0 + r) * 2 + 1) * a.os + l, R[1] * acc[r][1] + R[3] * acc[r][2]);
      }
    }
  }
}

// ----------------------------------------------------------------------------
static inline int cdivl(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <int KER, int NIMG, int NR>
static void launch_mixed(P2PArgs a, bool grad, dim3 grid, cudaStream_t st) {
  ++g_launches;
  if constexpr (KER == PFMM_MODHELM) {
    if (grad)
      k_p2p_mixed_mh<KER, NIMG, NR, true><<<grid, kP2PThreads, 0, st>>>(a);
    else
      k_p2p_mixed_mh<KER, NIMG, NR, false><<<grid, kP2PThreads, 0, st>>>(a);
  } else {
    // two targets per thread (grid.x already counts 2 * kP2PThreads targets per block)
    if (grad)
      k_p2p_mixed<KER, NIMG, NR, true><<<grid, kP2PThreads, 0, st>>>(a);
    else
      k_p2p_mixed<KER, NIMG, NR, false><<<grid, kP2PThreads, 0, st>>>(a);
  }
}

template <int KER, int NIMG>
static void dispatch_nr(P2PArgs a, bool grad, int nrhs, int ntb, int nsc, cudaStream_t st) {
  // rhs processed in groups of NR in {4, 2, 1}
  int r = 0;
  while (r < nrhs) {
    int left = nrhs - r;
    a.r0 = r;
    if constexpr (KER == PFMM_MODHELM) {
      if (left >= 8) {
        int ng = left / 8;
        launch_mixed<KER, NIMG, 8>(a, grad, dim3(ntb, nsc, ng), st);
        r += 8 * ng;
        continue;
      }
    }
    if (left >= 4) {
      int ng = left / 4;
      launch_mixed<KER, NIMG, 4>(a, grad, dim3(ntb, nsc, ng), st);
      r += 4 * ng;
    } else if (left >= 2) {
      launch_mixed<KER, NIMG, 2>(a, grad, dim3(ntb, nsc, 1), st);
      r += 2;
    } else {
      launch_mixed<KER, NIMG, 1>(a, grad, dim3(ntb, nsc, 1), st);
      r += 1;
    }
  }
}

template <int KER>
static void dispatch_img(P2PArgs a, bool grad, int nrhs, int ntb, int nsc, cudaStream_t st) {
  // m0 <= 2 after lattice reduction (|xi| <= d/2), so 9 or 15 images; the
  // singly periodic strip has 3
  if (a.g.nimg == 9)
    dispatch_nr<KER, 9>(a, grad, nrhs, ntb, nsc, st);
  else if (a.g.nimg == 3)
    dispatch_nr<KER, 3>(a, grad, nrhs, ntb, nsc, st);
  else
    dispatch_nr<KER, 15>(a, grad, nrhs, ntb, nsc, st);
}

// Modified Stokes: rhs in groups of 4, 2, 1; 9 or 15 images.
template <int NIMG>
static void launch_ms_img(P2PArgs a, int nrhs, int ntb, int nsc, cudaStream_t st) {
  int r = 0;
  while (r < nrhs) {
    const int left = nrhs - r;
    a.r0 = r;
    ++g_launches;
    if (left >= 4) {
      const int ng = left / 4;
      k_p2p_ms<NIMG, 4><<<dim3(ntb, nsc, ng), kP2PThreads, 0, st>>>(a);
      r += 4 * ng;
    } else if (left >= 2) {
      k_p2p_ms<NIMG, 2><<<dim3(ntb, nsc, 1), kP2PThreads, 0, st>>>(a);
      r += 2;
    } else {
      k_p2p_ms<NIMG, 1><<<dim3(ntb, nsc, 1), kP2PThreads, 0, st>>>(a);
      r += 1;
    }
  }
}

static void launch_ms(const P2PArgs& a, int nrhs, int ntb, int nsc, cudaStream_t st) {
  if (a.g.nimg == 9)
    launch_ms_img<9>(a, nrhs, ntb, nsc, st);
  else
    launch_ms_img<15>(a, nrhs, ntb, nsc, st);
}

void fill_p2p_args(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot, double* grad,
                   P2PArgs* out) {
  const Layout& L = p->lay;
  P2PArgs a{};
  a.g = p->geom;
  a.nt = (int)nt;
  a.ns = (int)ns;
  a.os = p->o_stride;
  a.nrhs = p->opts.nrhs;
  a.trg64 = self ? (const double*)(ws + L.src64) : (const double*)(ws + L.trg64);
  if (p->opts.precision == PFMM_MIXED) {
    a.s_rel = (const float2*)(ws + L.s_rel);
    a.s_hl = (const float4*)(ws + L.s_hl);
    a.s_sub = (const float4*)(ws + L.s_sub);
    a.s_ext = (const float2*)(ws + L.s_ext);
    a.s_box = (const float4*)(ws + L.s_box);
    a.qs = (const float*)(ws + L.qs);
    // targets in sorted order too; outputs go back through the permutation
    a.trg64 = self ? (const double*)(ws + L.s_sorted) : (const double*)(ws + L.t_sorted);
    a.t_perm = self ? (const int*)(ws + L.s_perm) : (const int*)(ws + L.t_perm);
    a.t_box = self ? (const float4*)(ws + L.s_box) : (const float4*)(ws + L.t_box);
  }
  a.cut = (float)(p->mh_cut / std::max(p->far.beta, 1e-300));
  for (int i = 0; i < p->geom.nimg; ++i) {
    a.offf[i][0] = (float)p->geom.off[i][0];
    a.offf[i][1] = (float)p->geom.off[i][1];
  }
  a.src64 = (const double*)(ws + L.src64);
  a.qc = (const double*)(ws + L.qc);
  a.beta = p->far.beta;
  a.beta_f = (float)p->far.beta;
  a.pot = pot;
  a.grad = grad;
  a.mom = (const double*)(ws + L.moments);
  {
    // e_i = nearest integer to the mean of log2 |t - s - l_i|^2 over t, s on a
    // 16 x 16 lattice of fractional positions in the cell (deterministic)
    const Geom& g = p->geom;
    double E = 0.0;
    for (int i = 0; i < g.nimg; ++i) {
      double acc = 0.0;
      int cntp = 0;
      for (int a1 = 0; a1 < 16; ++a1)
        for (int a2 = 0; a2 < 16; ++a2)
          for (int b1 = 0; b1 < 16; b1 += 3)
            for (int b2 = 0; b2 < 16; b2 += 3) {
              double u1 = (a1 + 0.5) / 16 - 0.5 - ((b1 + 0.5) / 16 - 0.5);
              double u2 = (a2 + 0.5) / 16 - 0.5 - ((b2 + 0.5) / 16 - 0.5);
              double dx = u1 * g.d + u2 * g.xi - g.off[i][0], dy = u2 * g.eta - g.off[i][1];
              double r2 = dx * dx + dy * dy;
              if (r2 > 0) { acc += std::log2(r2); ++cntp; }
            }
      double e = std::nearbyint(acc / std::max(1, cntp));
      a.kimg[i] = (float)std::ldexp(1.0, -(int)e);
      E += e;
    }
    a.lgc = (float)E;
  }
  *out = a;
}

int p2p_targets_per_block(int kernel) {
  return kP2PThreads * ((kernel == PFMM_LAPLACE || kernel == PFMM_STOKES) ? 2 : 1);
}

int fill_sort_cells(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, int64_t off_s, int64_t off_t,
                    SortCell* out) {
  const Layout& L = p->lay;
  SortCell c{};
  c.n = (int)ns;
  c.off = off_s;
  c.xy = (const double*)(ws + L.src64);
  sort_grid(p->geom, (int)ns, &c);
  c.q_in = (const float*)(ws + L.qf);
  c.nq = p->opts.nrhs * p->ncomp;
  c.q_out = (float*)(ws + L.qs);
  c.rel = (float2*)(ws + L.s_rel);
  c.hl = (float4*)(ws + L.s_hl);
  c.sub = (float4*)(ws + L.s_sub);
  c.ext = (float2*)(ws + L.s_ext);
  c.box = (float4*)(ws + L.s_box);
  c.perm = (int*)(ws + L.s_perm);
  c.xy_sorted = self ? (double*)(ws + L.s_sorted) : nullptr;
  out[0] = c;
  if (self) return 1;
  SortCell t{};
  t.n = (int)nt;
  t.off = off_t;
  t.xy = (const double*)(ws + L.trg64);
  sort_grid(p->geom, (int)nt, &t);
  t.box = (float4*)(ws + L.t_box);
  t.perm = (int*)(ws + L.t_perm);
  t.xy_sorted = (double*)(ws + L.t_sorted);
  out[1] = t;
  return 2;
}

cudaError_t launch_p2p(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot, double* grad,
                       bool accumulate, cudaStream_t st) {
  (void)accumulate;
  const bool mixed = p->opts.precision == PFMM_MIXED;
  int sort_launches = 0;
  if (mixed) {
    // spatial sort of the sources (and modified Helmholtz targets) of this cell
    const int nc = fill_sort_cells(p, ws, ns, nt, self, 0, ns, p->sort_h);
    SortCell* dcells = (SortCell*)(ws + p->lay.sortd);
    // the descriptors depend only on (workspace, ns, nt, self): under stream
    // capture they must be the ones an eager execute uploaded (a copy from
    // pageable host memory cannot be captured)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    cudaError_t e = cudaSuccess;
    if (cap != cudaStreamCaptureStatusNone) {
      if (!(p->sort_ws == ws && p->sort_ns == ns && p->sort_nt == nt && p->sort_self == self))
        return cudaErrorStreamCaptureUnsupported;
    } else {
      e = cudaMemcpyAsync(dcells, p->sort_h, nc * sizeof(SortCell), cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return e;
      p->sort_ws = ws;
      p->sort_ns = ns;
      p->sort_nt = nt;
      p->sort_self = self;
    }
    e = sort_cells(dcells, p->sort_h, nc, ns + (nc > 1 ? nt : 0), ws + p->lay.sortscr, st, &sort_launches);
    if (e != cudaSuccess) return e;
  }
  P2PArgs a;
  fill_p2p_args(p, ws, ns, nt, self, pot, grad, &a);
  set_work_counter(p, ws, p->prof, &a);
  const bool packed = mixed && (p->opts.kernel == PFMM_LAPLACE || p->opts.kernel == PFMM_STOKES);  // two targets per thread
  const int ntb = cdivl(nt, kP2PThreads * (packed ? 2 : 1));
  const int nrg = mixed ? 1 : cdivl(a.nrhs, 4);
  // split the sources so that the grid holds >= ~32 blocks per SM
  int nsc = std::max(1, std::min(cdivl(ns, kP2PTile), cdivl(32 * 152, (int64_t)ntb * nrg)));
  // deterministic mode: one source chunk per target block, so each output
  // receives exactly one addition from the P2P
  if (p->opts.flags & PFMM_DETERMINISTIC) nsc = 1;
  a.chunk = cdivl(cdivl(ns, nsc), kP2PTile) * kP2PTile;
  nsc = cdivl(ns, a.chunk);
  const bool g = grad != nullptr;
  g_launches = (mixed ? 0 : 1) + sort_launches;
  if (mixed) {
    switch (p->opts.kernel) {
      case PFMM_LAPLACE: dispatch_img<PFMM_LAPLACE>(a, g, a.nrhs, ntb, nsc, st); break;
      case PFMM_MODHELM: dispatch_img<PFMM_MODHELM>(a, g, a.nrhs, ntb, nsc, st); break;
      case PFMM_MSTOKES: launch_ms(a, a.nrhs, ntb, nsc, st); break;
      default: dispatch_img<PFMM_STOKES>(a, false, a.nrhs, ntb, nsc, st); break;
    }
  } else {
    dim3 grid(ntb, nsc, nrg);
    a.r0 = 0;
    switch (p->opts.kernel) {
      case PFMM_LAPLACE:
        if (g) k_p2p_f64<PFMM_LAPLACE, true><<<grid, kP2PThreads, 0, st>>>(a);
        else k_p2p_f64<PFMM_LAPLACE, false><<<grid, kP2PThreads, 0, st>>>(a);
        break;
      case PFMM_MODHELM:
        if (g) k_p2p_f64<PFMM_MODHELM, true><<<grid, kP2PThreads, 0, st>>>(a);
        else k_p2p_f64<PFMM_MODHELM, false><<<grid, kP2PThreads, 0, st>>>(a);
        break;
      case PFMM_MSTOKES: k_p2p_f64<PFMM_MSTOKES, false><<<grid, kP2PThreads, 0, st>>>(a); break;
      default: k_p2p_f64<PFMM_STOKES, false><<<grid, kP2PThreads, 0, st>>>(a); break;
    }
  }
  return cudaGetLastError();
}


template <int KER, int NIMG, int NR, bool GRAD>
static cudaError_t launch_batch_t(const P2PArgs* cells, const P2PItem* items, int nitems, int* counter, int grid,
                                  cudaStream_t st) {
  k_p2p_batch<KER, NIMG, NR, GRAD><<<grid, kP2PThreads, 0, st>>>(cells, items, nitems, counter);
  return cudaGetLastError();
}

template <int KER, int NIMG, int NR, bool GRAD>
static int grid_t() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_p2p_batch<KER, NIMG, NR, GRAD>, kP2PThreads, 0);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, nb) * std::max(1, sms);
}

// dispatch over (kernel, nimg in {9, 15}, nr in {1, 2, 4}, grad); Stokes has no grad variant
#define PFMM_P2P_BATCH_DISPATCH(FN, ...)                                                          \
  do {                                                                                            \
    const int ki = kernel == PFMM_LAPLACE ? 0 : (kernel == PFMM_MODHELM ? 1 : 2);                 \
    const int ii = nimg == 9 ? 0 : 1, ri = nr == 4 ? 2 : (nr == 2 ? 1 : 0), gi = grad ? 1 : 0;    \
    const int code = nr == 8 ? 1000 + ii * 2 + gi : ((ki * 2 + ii) * 3 + ri) * 2 + gi;            \
    switch (code) {                                                                               \
      PFMM_P2P_CASES(FN, __VA_ARGS__)                                                             \
      case 1000: return FN<PFMM_MODHELM, 9, 8, false>(__VA_ARGS__);                               \
      case 1001: return FN<PFMM_MODHELM, 9, 8, true>(__VA_ARGS__);                                \
      case 1002: return FN<PFMM_MODHELM, 15, 8, false>(__VA_ARGS__);                              \
      case 1003: return FN<PFMM_MODHELM, 15, 8, true>(__VA_ARGS__);                               \
      default: return FN<PFMM_STOKES, 15, 1, false>(__VA_ARGS__);                                 \
    }                                                                                             \
  } while (0)
#define PFMM_P2P_CASE(FN, K, KI, NI, II, R, RI, G, GI, ...) \
  case ((KI * 2 + II) * 3 + RI) * 2 + GI: return FN<K, NI, R, G>(__VA_ARGS__);
#define PFMM_P2P_CASES_KI(FN, K, KI, ...)                                   \
  PFMM_P2P_CASE(FN, K, KI, 9, 0, 1, 0, false, 0, __VA_ARGS__)               \
  PFMM_P2P_CASE(FN, K, KI, 9, 0, 1, 0, true, 1, __VA_ARGS__)                \
  PFMM_P2P_CASE(FN, K, KI, 9, 0, 2, 1, false, 0, __VA_ARGS__)               \
  PFMM_P2P_CASE(FN, K, KI, 9, 0, 2, 1, true, 1, __VA_ARGS__)                \
  PFMM_P2P_CASE(FN, K, KI, 9, 0, 4, 2, false, 0, __VA_ARGS__)               \
  PFMM_P2P_CASE(FN, K, KI, 9, 0, 4, 2, true, 1, __VA_ARGS__)                \
  PFMM_P2P_CASE(FN, K, KI, 15, 1, 1, 0, false, 0, __VA_ARGS__)              \
  PFMM_P2P_CASE(FN, K, KI, 15, 1, 1, 0, true, 1, __VA_ARGS__)               \
  PFMM_P2P_CASE(FN, K, KI, 15, 1, 2, 1, false, 0, __VA_ARGS__)              \
  PFMM_P2P_CASE(FN, K, KI, 15, 1, 2, 1, true, 1, __VA_ARGS__)               \
  PFMM_P2P_CASE(FN, K, KI, 15, 1, 4, 2, false, 0, __VA_ARGS__)              \
  PFMM_P2P_CASE(FN, K, KI, 15, 1, 4, 2, true, 1, __VA_ARGS__)
#define PFMM_P2P_CASES(FN, ...)                                  \
  PFMM_P2P_CASES_KI(FN, PFMM_LAPLACE, 0, __VA_ARGS__)            \
  PFMM_P2P_CASES_KI(FN, PFMM_MODHELM, 1, __VA_ARGS__)            \
  PFMM_P2P_CASES_KI(FN, PFMM_STOKES, 2, __VA_ARGS__)

// modified Stokes: velocity only, nimg in {9, 15}, nr in {1, 2, 4}
#define PFMM_P2P_MS_DISPATCH(FN, ...)                                           \
  do {                                                                          \
    switch ((nimg == 9 ? 0 : 3) + (nr == 4 ? 2 : (nr == 2 ? 1 : 0))) {          \
      case 0: return FN<PFMM_MSTOKES, 9, 1, false>(__VA_ARGS__);                \
      case 1: return FN<PFMM_MSTOKES, 9, 2, false>(__VA_ARGS__);                \
      case 2: return FN<PFMM_MSTOKES, 9, 4, false>(__VA_ARGS__);                \
      case 3: return FN<PFMM_MSTOKES, 15, 1, false>(__VA_ARGS__);               \
      case 4: return FN<PFMM_MSTOKES, 15, 2, false>(__VA_ARGS__);               \
      default: return FN<PFMM_MSTOKES, 15, 4, false>(__VA_ARGS__);              \
    }                                                                           \
  } while (0)

cudaError_t launch_p2p_batch(int kernel, int nimg, int nr, bool grad, const P2PArgs* cells, const P2PItem* items,
                             int nitems, int* counter, int grid, cudaStream_t st) {
  if (kernel == PFMM_MSTOKES) PFMM_P2P_MS_DISPATCH(launch_batch_t, cells, items, nitems, counter, grid, st);
  if (kernel == PFMM_STOKES) grad = false;
  PFMM_P2P_BATCH_DISPATCH(launch_batch_t, cells, items, nitems, counter, grid, st);
}

int p2p_batch_grid(int kernel, int nimg, int nr, bool grad) {
  if (kernel == PFMM_MSTOKES) PFMM_P2P_MS_DISPATCH(grid_t);
  if (kernel == PFMM_STOKES) grad = false;
  PFMM_P2P_BATCH_DISPATCH(grid_t);
}

}  // namespace pfmm
