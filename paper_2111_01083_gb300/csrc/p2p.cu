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
#include "devmath.cuh"

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
  __device__ __forceinline__ double value() const { return dm::f2d(s) - dm::f2d(c); }
};

// (h + l) - (oh + ol) as an unevaluated FP32 pair (sh, sl): two-sum of the
// high parts, the low parts added to its error
__device__ __forceinline__ void shift_two(float h, float l, float oh, float ol, float& sh, float& sl) {
  const float sm = h - oh;
  const float bb = sm - h;
  const float err = (h - (sm - bb)) + (-oh - bb);
  sh = sm;
  sl = err + (l - ol);
}

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
// in spatially sorted order, per (target, source) the image sums
// K0s = sum_i K0(beta r_i), K1x = sum_i K1(beta r_i) dx_i / r_i (and y), then
// one FMA per rhs.  Two sources go through each packed FP32 instruction
// (FFMA2 / FADD2 / FMUL2 on the source pair), four per step.
//
// Culling: pairs with beta r > x_c are skipped (x_c from the plan: every
// skipped term below tol/10 / (images * ns)).  Per (target block, source tile)
// one thread classifies each image with an FP32 test on the outward-rounded
// boxes: an image with no pair within the cutoff is skipped for the tile.
//
// Per 16-source subtile and image, warp-uniform routing:
//  - exact: some lane of the warp lies within about two subtile extents of
//    the subtile (close pairs: differences from the hi/lo coordinates), or
//    within 2 / beta of it (beta r <= 2 possible).  K0 from the small- or the
//    large-argument fit per pair; a warp vote decides which fits run, so a
//    warp whose pairs all fall on one side evaluates one fit only.
//  - fast: every other active image.  Every pair of the warp has beta r > 2,
//    so only the large-argument fit runs, on beta-scaled coordinates relative
//    to the subtile centre; the image list is compacted per thread in shared
//    memory, so the loop runs over the active images only.
// Pairs of the exact images beyond the cutoff are evaluated as well (their
// terms lie below the cutoff's bound).
template <int KER, int NIMG, int NR, bool GRAD>
__device__ __forceinline__ void p2p_mixed_mh_body(const P2PArgs& a, int bx, int j0, int j1, int r0) {
  constexpr int CENTER = NIMG / 2;
  constexpr int NA = GRAD ? 3 : 1;
  constexpr int NSUB = kP2PTile / kSubtile;
  constexpr unsigned kFull = 0xffffffffu;
  static_assert(kP2PTile == kP2PThreads, "one thread loads one source of the tile");
  // the source tile, component-major: consecutive sources are the two lanes
  // of a packed operation
  __shared__ __align__(16) float s_bs[2][kP2PTile];  // beta (s - subtile centre)
  __shared__ __align__(16) float s_hs[4][kP2PTile];  // x_hi, x_lo, y_hi, y_lo
  __shared__ __align__(16) float s_q[NR][kP2PTile];
  __shared__ float4 s_c[NSUB];
  __shared__ float2 s_e[NSUB];
  // hi/lo target coordinates per image, one column per thread
  __shared__ float s_tc[4][NIMG][kP2PThreads];
  // the fast images of the current subtile: beta (target - image - centre)
  __shared__ float2 s_bt[NIMG][kP2PThreads];
  __shared__ unsigned s_tany[kP2PThreads];
  const int tid = threadIdx.x;
  const int l = bx * kP2PThreads + tid;
  const bool in = l < a.nt;
  const int nr = min(NR, a.nrhs - r0);
  {
    // the target's hi/lo split (read with targets = sources, else from FP64),
    // shifted by each image offset (hi/lo) with an FP32 two-sum: no FP64
    // arithmetic per image (FP64 runs at 1/64 of the FP32 rate here)
    float4 t;
    if (a.t_hl) {
      t = in ? a.t_hl[l] : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const double tx = in ? a.trg64[l] : 0.0, ty = in ? a.trg64[a.nt + l] : 0.0;
      const float hx = (float)tx, hy = (float)ty;
      t = make_float4(hx, (float)(tx - (double)hx), hy, (float)(ty - (double)hy));
    }
#pragma unroll
    for (int i = 0; i < NIMG; ++i) {
      float h, lo;
      shift_two(t.x, t.y, a.offf[i][0], a.offl[i][0], h, lo);
      s_tc[0][i][tid] = h;
      s_tc[1][i][tid] = lo;
      shift_two(t.z, t.w, a.offf[i][1], a.offl[i][1], h, lo);
      s_tc[2][i][tid] = h;
      s_tc[3][i][tid] = lo;
    }
  }
  KahanF K[NR][NA];
  float2 S[NR][NA];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      K[r][k].s = K[r][k].c = 0.f;
      S[r][k] = f2(0.f);
    }
  const float beta = a.beta_f;
  const float beta2 = beta * beta;
  const float4 tb = a.t_box[bx];
  const float rsm = 2.0f / beta * 1.001f + 1e-6f;  // beta r <= 2 region, with margin

  // large-argument fit on beta-scaled differences of a source pair: K0 and
  // K1(x) / x times the scaled difference; the fit variable y = 2/x folded
  // into the coefficients (c_k 2^k)
  auto far_pair = [&](float2 dx, float2 dy, float2& k0, float2& gx, float2& gy) {
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
    k0 = fma2(e, pl, k0);
    if (GRAD) {
      float2 p1 = fma2(ix, f2(-0.0436768f), f2(0.10419648f));
      p1 = fma2(ix, p1, f2(-0.12485648f));
      p1 = fma2(ix, p1, f2(0.12034144f));
      p1 = fma2(ix, p1, f2(-0.1462248f));
      p1 = fma2(ix, p1, f2(0.46997238f));
      p1 = fma2(ix, p1, f2(1.25331414f));
      const float2 k1ix = mul2(mul2(e, ix), p1);
      gx = fma2(k1ix, dx, gx);
      gy = fma2(k1ix, dy, gy);
    }
  };

  const int ntile = (j1 - j0 + kP2PTile - 1) / kP2PTile;
  for (int g0 = 0; g0 < ntile; g0 += kP2PThreads) {
    __syncthreads();
    {
      // per tile and image: some pair within the cutoff (FP32 on the
      // outward-rounded boxes with a relative margin: a tile misjudged at the
      // margin only adds or drops terms below the cutoff's bound)
      const int t = g0 + tid;
      unsigned many = 0u;
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
          if (ex * ex + ey * ey <= c2) many |= 1u << i;
        }
        if (a.work && many) {
          const int nbt = min(kP2PTile, j1 - (j0 + t * kP2PTile));
          atomicAdd(a.work, (unsigned long long)__popc(many) * (unsigned long long)nbt *
                                (unsigned long long)min(kP2PThreads, a.nt - bx * kP2PThreads));
        }
      }
      s_tany[tid] = many;
    }
    __syncthreads();
    const int gn = min(kP2PThreads, ntile - g0);
    for (int tt = 0; tt < gn; ++tt) {
      const unsigned any = s_tany[tt];
      if (any == 0u) continue;
      const int jb = j0 + (g0 + tt) * kP2PTile;
      const int nb = min(kP2PTile, j1 - jb);
      __syncthreads();
      {
        // padding: zero strength at the subtile centre (finite distances)
        const int k = tid;
        const bool v = k < nb;
        const float2 p = v ? a.s_rel[jb + k] : make_float2(0.f, 0.f);
        s_bs[0][k] = beta * p.x;
        s_bs[1][k] = beta * p.y;
        const float4 h = v ? a.s_hl[jb + k] : s_c_src(a, jb, k, nb);
        s_hs[0][k] = h.x;
        s_hs[1][k] = h.y;
        s_hs[2][k] = h.z;
        s_hs[3][k] = h.w;
        if (k < NSUB) {
          s_c[k] = (k * kSubtile < nb) ? a.s_sub[jb / kSubtile + k] : make_float4(0.f, 0.f, 0.f, 0.f);
          s_e[k] = (k * kSubtile < nb) ? a.s_ext[jb / kSubtile + k] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) s_q[r][k] = (v && r < nr) ? a.qs[(size_t)(r0 + r) * a.ns + jb + k] : 0.f;
      }
      __syncthreads();
      for (int js = 0; js < nb; js += kP2PSub) {
        // routing of the active images for this subtile (warp-uniform)
        unsigned slow = 0u;
        int nf = 0;
        {
          const float4 c = s_c[js / kSubtile];
          const float2 e = s_e[js / kSubtile];
          const float bxe = 2.f * e.x + e.y, bye = e.x + 2.f * e.y;
          const float sxe = e.x + rsm, sye = e.y + rsm;
          float bxr[NIMG], byr[NIMG];
          unsigned mine = 0u;
#pragma unroll
          for (int i = 0; i < NIMG; ++i) {
            bxr[i] = byr[i] = 0.f;
            if (!(any & (1u << i))) continue;
            const float xr = (s_tc[0][i][tid] - c.x) + (s_tc[1][i][tid] - c.y);
            const float yr = (s_tc[2][i][tid] - c.z) + (s_tc[3][i][tid] - c.w);
            bxr[i] = beta * xr;
            byr[i] = beta * yr;
            const float ax = fabsf(xr), ay = fabsf(yr);
            if (in && ((ax < bxe && ay < bye) || (ax < sxe && ay < sye))) mine |= 1u << i;
          }
          slow = any & __reduce_or_sync(kFull, mine);
          const unsigned fast = any & ~slow;
#pragma unroll
          for (int i = 0; i < NIMG; ++i)
            if (fast & (1u << i)) s_bt[nf++][tid] = make_float2(bxr[i], byr[i]);
        }
        for (int jj = js; jj < js + kP2PSub; jj += 4) {
          float2 kA = f2(0.f), kB = f2(0.f), gxA = f2(0.f), gyA = f2(0.f), gxB = f2(0.f), gyB = f2(0.f);
          if (nf) {
            const float4 px = *reinterpret_cast<const float4*>(&s_bs[0][jj]);
            const float4 py = *reinterpret_cast<const float4*>(&s_bs[1][jj]);
            const float2 npxA = make_float2(-px.x, -px.y), npxB = make_float2(-px.z, -px.w);
            const float2 npyA = make_float2(-py.x, -py.y), npyB = make_float2(-py.z, -py.w);
#pragma unroll 3
            for (int k = 0; k < nf; ++k) {
              const float2 bt = s_bt[k][tid];
              far_pair(add2(f2(bt.x), npxA), add2(f2(bt.y), npyA), kA, gxA, gyA);
              far_pair(add2(f2(bt.x), npxB), add2(f2(bt.y), npyB), kB, gxB, gyB);
            }
          }
          if (slow) {
            const float4 hx = *reinterpret_cast<const float4*>(&s_hs[0][jj]);
            const float4 lx = *reinterpret_cast<const float4*>(&s_hs[1][jj]);
            const float4 hy = *reinterpret_cast<const float4*>(&s_hs[2][jj]);
            const float4 ly = *reinterpret_cast<const float4*>(&s_hs[3][jj]);
#pragma unroll 1
            for (unsigned m = slow; m; m &= m - 1u) {
              const int i = __ffs(m) - 1;
              const float thx = s_tc[0][i][tid], tlx = s_tc[1][i][tid];
              const float thy = s_tc[2][i][tid], tly = s_tc[3][i][tid];
              // exact differences (t_hi - s_hi) + (t_lo - s_lo)
              const float2 dxA = add2(add2(f2(thx), make_float2(-hx.x, -hx.y)), add2(f2(tlx), make_float2(-lx.x, -lx.y)));
              const float2 dxB = add2(add2(f2(thx), make_float2(-hx.z, -hx.w)), add2(f2(tlx), make_float2(-lx.z, -lx.w)));
              const float2 dyA = add2(add2(f2(thy), make_float2(-hy.x, -hy.y)), add2(f2(tly), make_float2(-ly.x, -ly.y)));
              const float2 dyB = add2(add2(f2(thy), make_float2(-hy.z, -hy.w)), add2(f2(tly), make_float2(-ly.z, -ly.w)));
              float2 r2A = fma2(dxA, dxA, mul2(dyA, dyA)), r2B = fma2(dxB, dxB, mul2(dyB, dyB));
              float2 mA = f2(1.f), mB = f2(1.f);
              if (i == CENTER) {
                // a zero distance (the target itself) is skipped
                mA = make_float2(r2A.x > 0.f ? 1.f : 0.f, r2A.y > 0.f ? 1.f : 0.f);
                mB = make_float2(r2B.x > 0.f ? 1.f : 0.f, r2B.y > 0.f ? 1.f : 0.f);
                r2A = make_float2(r2A.x > 0.f ? r2A.x : 1.f, r2A.y > 0.f ? r2A.y : 1.f);
                r2B = make_float2(r2B.x > 0.f ? r2B.x : 1.f, r2B.y > 0.f ? r2B.y : 1.f);
              }
              const float2 x2A = mul2(r2A, f2(beta2)), x2B = mul2(r2B, f2(beta2));
              const bool sml = fminf(fminf(x2A.x, x2A.y), fminf(x2B.x, x2B.y)) <= 4.0f;
              const bool lrg = fmaxf(fmaxf(x2A.x, x2A.y), fmaxf(x2B.x, x2B.y)) > 4.0f;
              const bool doS = __any_sync(kFull, sml), doL = __any_sync(kFull, lrg);
              float2 k0A = f2(0.f), k0B = f2(0.f), k1A = f2(0.f), k1B = f2(0.f);
              if (doS) {
                if (GRAD) {
                  bes::pk::k01_small(x2A, &k0A, &k1A);
                  bes::pk::k01_small(x2B, &k0B, &k1B);
                } else {
                  k0A = bes::pk::k0_small(x2A);
                  k0B = bes::pk::k0_small(x2B);
                }
              }
              if (doL) {
                float2 l0A, l0B, l1A = f2(0.f), l1B = f2(0.f);
                if (GRAD) {
                  bes::pk::k01_large(x2A, &l0A, &l1A);
                  bes::pk::k01_large(x2B, &l0B, &l1B);
                } else {
                  l0A = bes::pk::k0_large(x2A);
                  l0B = bes::pk::k0_large(x2B);
                }
                if (x2A.x > 4.0f) { k0A.x = l0A.x; k1A.x = l1A.x; }
                if (x2A.y > 4.0f) { k0A.y = l0A.y; k1A.y = l1A.y; }
                if (x2B.x > 4.0f) { k0B.x = l0B.x; k1B.x = l1B.x; }
                if (x2B.y > 4.0f) { k0B.y = l0B.y; k1B.y = l1B.y; }
              }
              kA = fma2(k0A, mA, kA);
              kB = fma2(k0B, mB, kB);
              if (GRAD) {
                // K1(beta r) / r = beta K1(x) / x
                const float2 k1rA = mul2(mul2(k1A, f2(beta)), mA), k1rB = mul2(mul2(k1B, f2(beta)), mB);
                gxA = fma2(k1rA, dxA, gxA);
                gyA = fma2(k1rA, dyA, gyA);
                gxB = fma2(k1rB, dxB, gxB);
                gyB = fma2(k1rB, dyB, gyB);
              }
            }
          }
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const float4 q = *reinterpret_cast<const float4*>(&s_q[r][jj]);
            const float2 qA = make_float2(q.x, q.y), qB = make_float2(q.z, q.w);
            S[r][0] = fma2(qB, kB, fma2(qA, kA, S[r][0]));
            if (GRAD) {
              S[r][1 % NA] = fma2(qB, gxB, fma2(qA, gxA, S[r][1 % NA]));
              S[r][2 % NA] = fma2(qB, gyB, fma2(qA, gyA, S[r][2 % NA]));
            }
          }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int k = 0; k < NA; ++k) {
            K[r][k].add(S[r][k].x + S[r][k].y);
            S[r][k] = f2(0.f);
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
  for (int i = 0; i < p->geom.nimg; ++i)
    for (int k = 0; k < 2; ++k) {
      a.offf[i][k] = (float)p->geom.off[i][k];
      a.offl[i][k] = (float)(p->geom.off[i][k] - (double)a.offf[i][k]);
    }
  a.t_hl = (p->opts.precision == PFMM_MIXED && self) ? (const float4*)(ws + L.s_hl) : nullptr;
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
