// Lattice weights D of the low-rank factorizations of the far part of the
// periodizing operator (FP64).  Shared by the direct far-field kernels and the
// NUFFT south/north path so that both apply one set of formulas.
//
//   scalar south/north   Theorem south_thm (modified Helmholtz, chi = sqrt(alpha^2 + beta^2))
//                        and Theorem south_thm_lap (Laplace, chi = |alpha|)
//   scalar west/east     Theorem west_thm / west_thm_lap, general m0
//   Stokes south/north   Theorem south_thm_s (Eq. pssm)
//   Stokes west/east     Theorem west_thm_s (Eq. pssw0), general m0
//   mod. Stokes          Theorems south_thm_ms, west_thm_ms (Eqs. pmss1, pmsw0)
//
// North is the complex conjugate of south (coordinate terms change sign for
// Stokes), east the conjugate of west.
//
// West/east frame (WeFrame): the plane waves decay along x~ of a frame in
// which the image column m is shifted by m (dx, dy) and the row n by
// n (xr, yr).  Along e1 (the paper's main text): (d, 0) and (xi, eta).  Along
// e2-perp (App. A, Eq. k0west2): (d c, d s) and (0, |e2|) with c = eta/|e2|,
// s = xi/|e2|.  The geometric sum over the columns m <= -(m0+1) then has the
// complex ratio e^{-(kappa dx - i lambda dy)}.
#pragma once
#include <cuda_runtime.h>

namespace pfmm {

struct dcx {
  double r, i;
};
__device__ __forceinline__ dcx cmul(dcx a, dcx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ dcx cadd(dcx a, dcx b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ dcx csub(dcx a, dcx b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ dcx cscale(dcx a, double s) { return {a.r * s, a.i * s}; }
__device__ __forceinline__ dcx cexp_(dcx z) {
  double e = exp(z.r), s, c;
  sincos(z.i, &s, &c);
  return {e * c, e * s};
}
__device__ __forceinline__ dcx cdiv(dcx a, dcx b) {
  double den = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / den, (a.i * b.r - a.r * b.i) / den};
}
__device__ __forceinline__ dcx conj_(dcx a) { return {a.r, -a.i}; }

namespace lw {

// Scalar south (north: conj): D = e^{-2Q} / (2 d chi (1 - e^{-Q})), Q = chi eta - i alpha xi.
__device__ __forceinline__ dcx sn_scalar(double d, double xi, double eta, double alpha, double chi, bool north) {
  dcx Q{chi * eta, -alpha * xi};
  dcx e1 = cexp_({-Q.r, -Q.i});
  dcx e2 = cmul(e1, e1);
  dcx D = cdiv(e2, cscale({1.0 - e1.r, -e1.i}, 2.0 * d * chi));
  return north ? conj_(D) : D;
}

struct WeFrame {
  double dx, dy;  // image column step in the frame
  double xr, yr;  // image row step in the frame
};

// 1 - e^{-g} for complex g = gr + i gi, without cancellation for small |g|:
// 1 - e^{-gr} (cos gi - i sin gi) = -expm1(-gr) + e^{-gr} 2 sin^2(gi/2) + i e^{-gr} sin gi.
__device__ __forceinline__ dcx one_minus_exp_neg(double gr, double gi) {
  const double e = exp(-gr), sh = sin(0.5 * gi);
  return {-expm1(-gr) + 2.0 * e * sh * sh, e * sin(gi)};
}

// Scalar west (east: conj), quadrature node (lambda, kappa) with weight w:
//   D = (w / (2 pi kappa)) e^{-(m0+1) g} / (1 - e^{-g}) B,   g = kappa dx - i lambda dy,
//   B = e^{kappa xr - i lambda yr} + 1 + e^{-kappa xr + i lambda yr}.
//   rows3 = false (singly periodic P1): only the row n = 0, B = 1.
__device__ __forceinline__ dcx we_scalar(const WeFrame& fr, int m0, double lam, double kap, double w, bool east,
                                         bool rows3 = true) {
  const double gr = kap * fr.dx, gi = -lam * fr.dy;
  const dcx F = cdiv(cexp_({-(m0 + 1) * gr, -(m0 + 1) * gi}), one_minus_exp_neg(gr, gi));
  dcx B = rows3 ? cadd(cadd(cexp_({kap * fr.xr, -lam * fr.yr}), {1.0, 0.0}), cexp_({-kap * fr.xr, lam * fr.yr}))
                : dcx{1.0, 0.0};
  dcx D = cscale(cmul(B, F), w / (2.0 * M_PI * kap));
  return east ? conj_(D) : D;
}

// Stokes south (m != 0): z = e^{-Q}, Q = |alpha| eta - i alpha xi,
//   Db = z^2/(4d(1-z)) S,  Da = z^2/(4d(1-z)) [ I/|alpha| - eta (2 - z)/(1 - z) S ],
//   S = [[1, i], [i, -1]].  North: Q and S conjugated.
__device__ __forceinline__ void sn_stokes(double d, double xi, double eta, double alpha, bool north, dcx Da[2][2],
                                          dcx Db[2][2]) {
  double aa = fabs(alpha);
  dcx Q{aa * eta, -alpha * xi};
  if (north) Q = conj_(Q);
  dcx z = cexp_({-Q.r, -Q.i});
  dcx omz{1.0 - z.r, -z.i};
  dcx pre = cdiv(cmul(z, z), cscale(omz, 4.0 * d));
  dcx S[2][2] = {{{1, 0}, {0, 1}}, {{0, 1}, {-1, 0}}};
  if (north) {
    S[0][1] = conj_(S[0][1]);
    S[1][0] = conj_(S[1][0]);
  }
  dcx q2 = cscale(cdiv({2.0 - z.r, -z.i}, omz), eta);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      Db[i][j] = cmul(pre, S[i][j]);
      dcx id = (i == j) ? dcx{1.0 / aa, 0.0} : dcx{0.0, 0.0};
      Da[i][j] = cmul(pre, csub(id, cmul(q2, S[i][j])));
    }
}

// Stokes west (east: conj), node (lambda, w), P = m0 + 1, z = e^{-lambda dx + i lambda dy}:
//   pref = (w / 4 pi) z^P / (1 - z),  phi_r = e^{r (lambda xr - i lambda yr)},  B = phi_1 + 1 + phi_-1,
//   Db = pref B S',  Da = pref [ B (I/lambda - (P dx + dx z/(1 - z)) S') + xr (phi_1 - phi_-1) S' ],
//   S' = [[-1, i], [i, 1]], all in the west/east frame.
//   rows3 = false (singly periodic P1): only the row n = 0, B = 1 and no xr term.
//   c, s: the frame's rotation (canonical -> frame).  The blocks are returned
//   as Q^T D Q, Q = [[c, -s], [s, c]], so that they act on canonical forces
//   and give canonical velocities (the coordinate factors stay the frame's x~).
__device__ __forceinline__ void we_stokes(const WeFrame& fr, double c, double s, int m0, double lam, double w,
                                          bool east, dcx Da[2][2], dcx Db[2][2], bool rows3 = true) {
  const double gr = lam * fr.dx, gi = -lam * fr.dy;  // z = e^{-(gr + i gi)}
  const dcx z = cexp_({-gr, -gi});
  const dcx omz = one_minus_exp_neg(gr, gi);
  const int P = m0 + 1;
  const dcx pref = cscale(cdiv(cexp_({-P * gr, -P * gi}), omz), w / (4.0 * M_PI));
  dcx ph1 = cexp_({lam * fr.xr, -lam * fr.yr}), phm = cexp_({-lam * fr.xr, lam * fr.yr});
  dcx B = rows3 ? cadd(cadd(ph1, phm), {1.0, 0.0}) : dcx{1.0, 0.0};
  dcx Sp[2][2] = {{{-1, 0}, {0, 1}}, {{0, 1}, {1, 0}}};
  const dcx kx = cadd({P * fr.dx, 0.0}, cscale(cdiv(z, omz), fr.dx));
  dcx dph = rows3 ? cscale(csub(ph1, phm), fr.xr) : dcx{0.0, 0.0};
  dcx A[2][2], Bb[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      Bb[i][j] = cmul(cmul(B, Sp[i][j]), pref);
      dcx id = (i == j) ? dcx{1.0 / lam, 0.0} : dcx{0.0, 0.0};
      dcx t1 = cmul(B, csub(id, cmul(Sp[i][j], kx)));
      A[i][j] = cmul(cadd(t1, cmul(dph, Sp[i][j])), pref);
      if (east) {
        Bb[i][j] = conj_(Bb[i][j]);
        A[i][j] = conj_(A[i][j]);
      }
    }
  // Q^T X Q
  const double Q[2][2] = {{c, -s}, {s, c}};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      dcx a = {0, 0}, b = {0, 0};
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) {
          const double qq = Q[k][i] * Q[l][j];
          a = cadd(a, cscale(A[k][l], qq));
          b = cadd(b, cscale(Bb[k][l], qq));
        }
      Da[i][j] = a;
      Db[i][j] = b;
    }
}

// Modified Stokes south (north: conj), mode m with alpha = a, decay b:
//   beta family (fam 0, b = chi):      D = F [[chi, i a], [i a, -a^2/chi]],
//   Laplace family (fam 1, b = |a|):   D = F [[-|a|, -i a], [-i a, |a|]],
//   F = e^{-2Q} / ((1 - e^{-Q}) 2 beta^2 d),  Q = b eta - i a xi.
__device__ __forceinline__ void ms_sn(double d, double xi, double eta, double a, double b, double beta, int fam,
                                      bool north, dcx D[2][2]) {
  const dcx e1 = cexp_({-b * eta, a * xi});
  const dcx F = cdiv(cmul(e1, e1), cscale({1.0 - e1.r, -e1.i}, 2.0 * beta * beta * d));
  dcx M[2][2];
  if (fam == 0) {
    M[0][0] = {b, 0.0};
    M[0][1] = M[1][0] = {0.0, a};
    M[1][1] = {-a * a / b, 0.0};
  } else {
    M[0][0] = {-b, 0.0};
    M[0][1] = M[1][0] = {0.0, -a};
    M[1][1] = {b, 0.0};
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      D[i][j] = cmul(F, M[i][j]);
      if (north) D[i][j] = conj_(D[i][j]);
    }
}

// Modified Stokes west (east: conj), node (lambda, w), decay kappa, in the
// west/east frame (rotation c, s; blocks returned as Q^T D Q):
//   D = (w / (2 pi beta^2)) e^{-(m0+1) g} / (1 - e^{-g}) B  Mat,  g = kappa dx - i lambda dy,
//   B = e^{kappa xr - i lambda yr} + 1 + e^{-kappa xr + i lambda yr},
//   Mat = [[-lambda^2/kappa, i lambda], [i lambda, kappa]] (fam 0) or
//         [[lambda, -i lambda], [-i lambda, -lambda]] (fam 1, kappa = lambda).
__device__ __forceinline__ void ms_we(const WeFrame& fr, double c, double s, int m0, double lam, double kap,
                                      double w, double beta, int fam, bool east, dcx D[2][2]) {
  const double gr = kap * fr.dx, gi = -lam * fr.dy;
  const dcx F = cdiv(cexp_({-(m0 + 1) * gr, -(m0 + 1) * gi}), one_minus_exp_neg(gr, gi));
  const dcx B = cadd(cadd(cexp_({kap * fr.xr, -lam * fr.yr}), {1.0, 0.0}), cexp_({-kap * fr.xr, lam * fr.yr}));
  const dcx pre = cscale(cmul(F, B), w / (2.0 * M_PI * beta * beta));
  dcx M[2][2];
  if (fam == 0) {
    M[0][0] = {-lam * lam / kap, 0.0};
    M[0][1] = M[1][0] = {0.0, lam};
    M[1][1] = {kap, 0.0};
  } else {
    M[0][0] = {lam, 0.0};
    M[0][1] = M[1][0] = {0.0, -lam};
    M[1][1] = {-lam, 0.0};
  }
  dcx A[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      A[i][j] = cmul(pre, M[i][j]);
      if (east) A[i][j] = conj_(A[i][j]);
    }
  const double Q[2][2] = {{c, -s}, {s, c}};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      dcx v = {0, 0};
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) v = cadd(v, cscale(A[k][l], Q[k][i] * Q[l][j]));
      D[i][j] = v;
    }
}

// Stokes weights from the coefficients c_a = R f, c_b = R coord f:
//   south/west:  Wa = fac (Da c_a + Db c_b),  Wb = -fac Db c_a
//   north/east:  Wa = fac (Da c_a - Db c_b),  Wb = +fac Db c_a
// (the coordinate terms of the kernel change sign with the direction).
__device__ __forceinline__ void stokes_apply(const dcx Da[2][2], const dcx Db[2][2], const dcx ca[2], const dcx cb[2],
                                             bool flip, double fac, dcx wa[2], dcx wb[2]) {
  const double sg = flip ? -1.0 : 1.0;
  for (int i = 0; i < 2; ++i) {
    dcx a = {0, 0}, b = {0, 0};
    for (int j = 0; j < 2; ++j) {
      a = cadd(a, cadd(cmul(Da[i][j], ca[j]), cscale(cmul(Db[i][j], cb[j]), sg)));
      b = cadd(b, cscale(cmul(Db[i][j], ca[j]), -sg));
    }
    wa[i] = cscale(a, fac);
    wb[i] = cscale(b, fac);
  }
}

}  // namespace lw
}  // namespace pfmm
