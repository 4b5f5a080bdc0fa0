// Host side of the library: plan construction (canonical cell, near block,
// modes, west/east quadrature, NUFFT sizes), workspace layout, argument
// validation and the order of kernel launches.  No device memory is ever
// allocated here.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "multi.cuh"
#include "pfmm_impl.h"
#include "sort.h"

using namespace pfmm;

namespace pfmm {
thread_local int g_launches = 0;
thread_local Recorder* g_rec = nullptr;
}

namespace {

thread_local std::string g_err;

pfmm_status fail(pfmm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

pfmm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(PFMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Sec. 1: canonical cell.  Lagrange-Gauss reduction (same lattice), longer
// reduced vector -> e1 rotated onto +x, shorter -> e2 flipped to eta > 0.
bool canonicalize(const double e1[2], const double e2[2], Geom* g) {
  double b1[2] = {e1[0], e1[1]}, b2[2] = {e2[0], e2[1]};
  auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1]; };
  double cross = b1[0] * b2[1] - b1[1] * b2[0];
  if (!std::isfinite(cross) || std::fabs(cross) <= 1e-14 * (dot(b1, b1) + dot(b2, b2))) return false;
  for (int it = 0; it < 200; ++it) {
    if (dot(b1, b1) > dot(b2, b2)) std::swap(b1, b2);
    double mu = std::floor(dot(b1, b2) / dot(b1, b1) + 0.5);
    if (mu == 0.0) break;
    b2[0] -= mu * b1[0];
    b2[1] -= mu * b1[1];
  }
  const double* a = b2;  // longer
  const double* b = b1;  // shorter
  double d = std::hypot(a[0], a[1]);
  double c = a[0] / d, s = a[1] / d;
  g->rot[0] = c; g->rot[1] = s; g->rot[2] = -s; g->rot[3] = c;
  double bx = c * b[0] + s * b[1], by = -s * b[0] + c * b[1];
  if (by < 0) { bx = -bx; by = -by; }
  g->d = d; g->xi = bx; g->eta = by;
  // fractional coordinates: canonical = [[d, xi],[0, eta]] u
  g->ainv[0] = 1.0 / d; g->ainv[1] = -bx / (d * by); g->ainv[2] = 0.0; g->ainv[3] = 1.0 / by;
  return true;
}

// Singly periodic (P1) strip: e1 rotated onto +x (no lattice reduction: e1 is
// the period), eta = |e1 x e2| / |e1| the strip width, xi = 0 (only the
// period matters along x).  Fractional coordinates u1 = x / d, u2 = y / eta.
bool canonicalize_strip(const double e1[2], const double e2[2], Geom* g) {
  const double d = std::hypot(e1[0], e1[1]);
  const double cross = e1[0] * e2[1] - e1[1] * e2[0];
  if (!std::isfinite(cross) || !(d > 0) || std::fabs(cross) <= 1e-14 * (d * d + e2[0] * e2[0] + e2[1] * e2[1]))
    return false;
  const double c = e1[0] / d, s = e1[1] / d;
  g->rot[0] = c; g->rot[1] = s; g->rot[2] = -s; g->rot[3] = c;
  g->d = d; g->xi = 0.0; g->eta = std::fabs(cross) / d;
  g->ainv[0] = 1.0 / d; g->ainv[1] = 0.0; g->ainv[2] = 0.0; g->ainv[3] = 1.0 / g->eta;
  return true;
}

// Proof after Eq. pylw02: west/east images need x - x' - m d - n xi >= margin > 0;
// the smallest gap over the parallelogram is m0 d - 2|xi|.  The paper uses
// margin = d; here margin = d/4 (any positive gap keeps the west/east
// integrands decaying; a smaller gap only costs quadrature nodes), so m0 = 1
// unless |xi| > 3d/8 and the near block stays 3 x 3 cells for most cells.
int choose_m0(double d, double xi) {
  return std::max(1, (int)std::ceil((0.25 * d + 2.0 * std::fabs(xi)) / d - 1e-12));
}

// Eq. mpk0s.
int mpk0s(double d, double eta, double eps) {
  double r = 2.0 * M_PI * eta / d;
  return (int)std::ceil((d / (2.0 * M_PI * eta)) * std::log(1.0 / ((1.0 - std::exp(-r)) * eps)));
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    if (n == 1) { p1 = z; p0 = 1.0; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// West/east frame.  Axis (the paper's main text): x along e1, columns step
// (d, 0), rows (xi, eta).  Rotated (App. A, Eq. k0west2): x~ along e2-perp,
// (x~, y~) = (c x - s y, s x + c y) with c = eta/|e2|, s = xi/|e2|, so that
// e2 -> (0, |e2|) and e1 -> (d c, d s); a point's x~ spans exactly d c, and
// m0 = 1 leaves the gap d c > 0 for every parallelogram.
void set_we_frame(Geom* g, bool rotated) {
  g->we_rot = rotated ? 1 : 0;
  if (!rotated) {
    g->wc = 1.0; g->ws = 0.0;
    g->wdx = g->d; g->wdy = 0.0; g->wxr = g->xi; g->wyr = g->eta;
    return;
  }
  const double h = std::hypot(g->xi, g->eta);
  g->wc = g->eta / h; g->ws = g->xi / h;
  g->wdx = g->d * g->wc; g->wdy = g->d * g->ws; g->wxr = 0.0; g->wyr = h;
}

// West/east quadrature for int_0^inf (.) d lambda (own composite GL rule in
// lambda' = lambda d): panels of width 2 (narrower when the integrand's
// lambda-frequency exceeds 2d, so that each panel sees at most ~4 radians),
// 8/12/16 points for tol >= 1e-7 /
// >= 1e-11 / smaller, dyadic panels toward 0 when 0 < beta d < 2, truncated
// where exp(-kappa' x_min') < tol/10 with x_min' the smallest scaled gap
// between a point and a far image column: (m0 d - 2|xi|)/d on the axis,
// m0 d c / d rotated.
// nsrc: sources the plan admits.  For the modified Helmholtz decay the
// truncation and the decision to drop the whole west/east part use the bound
// per unit charge times sqrt(nsrc): the dropped field of nsrc random-sign
// charges grows like their l2 norm, while the short-range potential it is
// compared with does not (a per-unit-charge tol/10 left 4e-6 relative error
// on a 4.7e4-point cell at beta = 10).
void we_quadrature(const Geom& g, int kernel, double beta, double tol, double nsrc, std::vector<double>& nodes) {
  nodes.clear();
  // largest lambda-frequency of the integrand, over d: axis: |y - y'| < eta
  // plus the row shifts +-eta (eta alone for the singly periodic row);
  // rotated: |y~ - y~'| < |e2| + d|s|, row shifts +-|e2|, and the first far
  // column's phase (m0 + 1) d|s|
  const double yspan = g.we_rot ? (2.0 * g.wyr + (g.m0 + 2) * std::fabs(g.wdy)) / g.d
                                : (g.p1 ? 1.0 : 2.0) * g.eta / g.d;
  const double pw = yspan > 2.0 ? 4.0 / yspan : 2.0;
  double xmin = g.we_rot ? g.m0 * g.wdx / g.d : (g.m0 * g.d - 2.0 * std::fabs(g.xi)) / g.d;
  double bt = (kernel == PFMM_MODHELM) ? beta * g.d : 0.0;
  const double tol_t = kernel == PFMM_MODHELM ? tol / std::sqrt(std::max(1.0, nsrc)) : tol;
  double top = std::log(10.0 / tol_t) / xmin;
  if (top <= bt) return;
  double lmax = std::sqrt(top * top - bt * bt);
  int npts = tol >= 1e-7 ? 8 : (tol >= 1e-11 ? 12 : 16);
  std::vector<double> edges{0.0};
  if (bt > 0 && bt < 2.0) {
    for (double e = bt / 8; e < 2.0 && e < lmax; e *= 2) edges.push_back(e);
  }
  double e = edges.back();
  while (e < lmax - 1e-12) { e = std::min(lmax, e + pw); edges.push_back(e); }
  std::vector<double> gx, gw;
  gauss_legendre(npts, gx, gw);
  for (size_t i = 0; i + 1 < edges.size(); ++i) {
    double a = edges[i], b = edges[i + 1];
    for (int k = 0; k < npts; ++k) {
      nodes.push_back((0.5 * (b - a) * (gx[k] + 1.0) + a) / g.d);
      nodes.push_back(0.5 * (b - a) * gw[k] / g.d);
    }
  }
}

// Exponential-of-semicircle kernel phi(z) = exp(b (sqrt(1 - z^2) - 1)), |z| <= 1,
// and its Fourier transform phihat(k) = int_{-1}^{1} phi(z) cos(k z) dz by
// Gauss-Legendre quadrature (the kernel is from the NUFFT reference the paper
// cites for its NUFFTs).
double es_phihat(double b, double k) {
  static thread_local std::vector<double> x, w;
  if (x.size() != 96) gauss_legendre(96, x, w);
  double s = 0.0;
  for (int i = 0; i < 96; ++i) s += w[i] * std::exp(b * (std::sqrt(1.0 - x[i] * x[i]) - 1.0)) * std::cos(k * x[i]);
  return s;
}

}  // namespace

namespace pfmm {
pfmm_status set_error(pfmm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

// Copy the plan's host tables (west/east nodes, GL lines, ES transform) into
// the workspace.
cudaError_t upload_tables(const pfmm_plan* p, char* ws, cudaStream_t st) {
  char* base = ws + p->lay.nodes;
  cudaError_t e = cudaSuccess;
  if (p->Nq > 0) e = cudaMemcpyAsync(base, p->nodes_h, p->Nq * 2 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + off_gl(p), p->gl_h, p->n_gl * 2 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + off_phihat(p), p->phihat_h, p->nphihat * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && p->tw_h)
    e = cudaMemcpyAsync(base + off_twiddle(p), p->tw_h, p->nf * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && p->rho_h)
    e = cudaMemcpyAsync(base + off_rho(p), p->rho_h, kRhoCheb * sizeof(double), cudaMemcpyHostToDevice, st);
  return e;
}

// One cell: clear accumulators, (optionally) upload tables, prep, far field,
// (optionally) near-image P2P.  Arguments were validated by the caller, which
// also set p->s_stride / t_stride / o_stride.
// The tree code's second stream and its fork/join events, created at the
// first execute outside stream capture (nothing is created while capturing;
// a capture before any eager execute runs the phases in sequence).
static bool side_setup(pfmm_plan* p, cudaStream_t st) {
  if (p->side_ready) return true;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return false;
  if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    cudaStreamDestroy(p->side);
    p->side = nullptr;
    p->fork_ev = nullptr;
    return false;
  }
  p->side_ready = true;
  return true;
}

pfmm_status execute_cell(pfmm_plan* p, char* ws, int64_t ns, const double* src, const double* q, int64_t nt,
                         const double* trg, double* pot, double* grad, cudaStream_t st, bool self, bool upload,
                         bool near) {
  cudaError_t e;
  e = zero_or_record(ws + p->lay.status, p->lay.nodes - p->lay.status, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  e = zero_or_record(ws + p->lay.coef, p->lay.wts - p->lay.coef, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (upload) {
    // Under stream capture the tables must already be in this workspace (an
    // eager execute on it put them there): a copy from pageable host memory
    // cannot be captured.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
    if (cap != cudaStreamCaptureStatusNone) {
      if (p->tables_ws != ws)
        return fail(PFMM_ERR_INVALID_ARG, "stream capture: execute once on this workspace before capturing");
    } else {
      e = upload_tables(p, ws, st);
      if (e != cudaSuccess) return cuda_fail(e, "upload tables");
      p->tables_ws = ws;
    }
  }
  p->nlaunch = 0;
  p->npairs = 0;
  auto rec = [&](int i) { if (p->prof && !g_rec) record_event(p->ev[i], st); };
  rec(0);
  if (nt == 0) {
    rec(1); rec(2); rec(3);
    return PFMM_OK;
  }
  if (ns > 0) {
    e = launch_prep(p, ws, ns, src, q, nt, trg, self, st);
    if (e != cudaSuccess) return cuda_fail(e, "prep kernel");
    p->nlaunch += g_launches;
  }
  rec(1);
  unsigned fl = p->opts.flags;
  bool do_far = !(fl & PFMM_NEAR_ONLY) && ns > 0;
  bool do_near = near && ns > 0;
  // tree code beside the far field: fork its stream after the preparation
  p->near_overlap = do_near && do_far && p->fmm.on && !g_rec && side_setup(p, st);
  if (p->near_overlap) {
    e = cudaEventRecord(p->fork_ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->fork_ev, 0);
    if (e != cudaSuccess) return cuda_fail(e, "fork");
  }
  if (do_far) {
    e = (p->path == PFMM_PATH_NUFFT) ? launch_far_nufft(p, ws, ns, nt, self, pot, grad, st)
                                     : launch_far_direct(p, ws, ns, nt, self, pot, grad, st);
    if (e != cudaSuccess) return cuda_fail(e, "far-field kernels");
    p->nlaunch += g_launches;
  } else {
    e = launch_zero_out(p, nt, pot, grad, st);
    if (e != cudaSuccess) return cuda_fail(e, "zero outputs");
  }
  rec(2);
  p->near_fmm_ran = do_near && p->fmm.on;
  if (do_near) {
    e = p->fmm.on ? (p->near_overlap ? launch_fmm_near(p, ws, ns, nt, self, pot, grad, st, p->side, p->join_ev)
                                     : launch_fmm_near(p, ws, ns, nt, self, pot, grad, st))
                  : launch_p2p(p, ws, ns, nt, self, pot, grad, true, st);
    if (e != cudaSuccess) return cuda_fail(e, p->fmm.on ? "near-field tree code" : "p2p kernel");
    p->nlaunch += g_launches;
    p->npairs = (int64_t)ns * nt * p->geom.nimg;
  }
  rec(3);
  return PFMM_OK;
}
}  // namespace pfmm

extern "C" {

const char* pfmm_last_error(void) { return g_err.c_str(); }
const char* pfmm_version(void) { return "pfmm-gb300 0.1 (sm_103a)"; }

pfmm_status pfmm_plan_create(const pfmm_opts* o, int64_t ns_max, int64_t nt_max, pfmm_plan** out) {
  if (!o || !out) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (o->kernel < 0 || o->kernel > 3) return fail(PFMM_ERR_INVALID_ARG, "bad kernel %d", o->kernel);
  if (o->precision < 0 || o->precision > 1) return fail(PFMM_ERR_INVALID_ARG, "bad precision %d", o->precision);
  if (o->path < 0 || o->path > 2) return fail(PFMM_ERR_INVALID_ARG, "bad path %d", o->path);
  if (o->nrhs < 1 || o->nrhs > 64) return fail(PFMM_ERR_INVALID_ARG, "nrhs must be in [1, 64]");
  if (ns_max < 0 || nt_max < 0 || ns_max > (int64_t(1) << 31) || nt_max > (int64_t(1) << 31))
    return fail(PFMM_ERR_INVALID_ARG, "ns_max/nt_max out of range");
  if (!(o->tol >= 1e-14 && o->tol <= 1e-2)) return fail(PFMM_ERR_TOLERANCE, "tol must be in [1e-14, 1e-2]");
  if ((o->kernel == PFMM_MODHELM || o->kernel == PFMM_MSTOKES) && !(o->beta > 0 && std::isfinite(o->beta)))
    return fail(PFMM_ERR_INVALID_ARG, "beta must be > 0 for the modified Helmholtz and modified Stokes kernels");
  if (o->kernel == PFMM_MSTOKES) {
    if (o->flags & PFMM_SINGLY_PERIODIC)
      return fail(PFMM_ERR_INVALID_ARG, "the modified Stokes kernel is doubly periodic only");
  }
  if (o->flags & ~1023u) return fail(PFMM_ERR_INVALID_ARG, "unknown flag bits 0x%x", o->flags & ~1023u);
  if ((o->flags & PFMM_DETERMINISTIC) && (o->flags & PFMM_NEAR_FMM))
    return fail(PFMM_ERR_INVALID_ARG, "DETERMINISTIC uses the direct near sum (not NEAR_FMM)");
  if ((o->flags & PFMM_DETERMINISTIC) && o->path == PFMM_PATH_NUFFT)
    return fail(PFMM_ERR_INVALID_ARG, "DETERMINISTIC uses the direct far-field path (not NUFFT)");
  if ((o->flags & PFMM_NEAR_DIRECT) && (o->flags & PFMM_NEAR_FMM))
    return fail(PFMM_ERR_INVALID_ARG, "NEAR_DIRECT and NEAR_FMM are exclusive");
  if (o->near_order != 0 && (o->near_order < 8 || o->near_order > 32))
    return fail(PFMM_ERR_INVALID_ARG, "near_order in [8, 32]");
  if (o->near_leaf != 0 && (o->near_leaf < 8 || o->near_leaf > 1024))
    return fail(PFMM_ERR_INVALID_ARG, "near_leaf in [8, 1024]");
  if ((o->flags & PFMM_FAR_ONLY) && (o->flags & PFMM_NEAR_ONLY))
    return fail(PFMM_ERR_INVALID_ARG, "FAR_ONLY and NEAR_ONLY are exclusive");
  if (o->nufft_w != 0 && (o->nufft_w < 2 || o->nufft_w > 16)) return fail(PFMM_ERR_INVALID_ARG, "nufft_w in [2,16]");
  if (o->n_gl != 0 && (o->n_gl < 4 || o->n_gl > 32)) return fail(PFMM_ERR_INVALID_ARG, "n_gl in [4,32]");

  Geom g{};
  const bool p1 = (o->flags & PFMM_SINGLY_PERIODIC) != 0;
  if (p1) {
    if (!canonicalize_strip(o->e1, o->e2, &g)) return fail(PFMM_ERR_LATTICE, "degenerate strip vectors");
    g.p1 = 1;
    g.m0 = 1;  // |x - x'| < d after wrapping: images |m| >= 2 are separated by >= d
  } else {
    if (!canonicalize(o->e1, o->e2, &g)) return fail(PFMM_ERR_LATTICE, "degenerate lattice vectors");
    g.m0 = choose_m0(g.d, g.xi);
  }
  {
    const bool want_rot = (o->flags & PFMM_WE_ROTATED) != 0, want_axis = (o->flags & PFMM_WE_AXIS) != 0;
    if (want_rot && want_axis) return fail(PFMM_ERR_INVALID_ARG, "WE_ROTATED and WE_AXIS are exclusive");
    if (p1 && want_rot) return fail(PFMM_ERR_INVALID_ARG, "the singly periodic operator uses the axis direction");
    const bool rot = !p1 && (want_rot || (!want_axis && g.m0 >= 2));
    if (rot) g.m0 = 1;
    set_we_frame(&g, rot);
  }
  if ((2 * g.m0 + 1) * 3 > kMaxNear) return fail(PFMM_ERR_INTERNAL, "near block too large");
  g.nimg = 0;
  for (int n = p1 ? 0 : -1; n <= (p1 ? 0 : 1); ++n)
    for (int m = -g.m0; m <= g.m0; ++m) {
      if (m == 0 && n == 0) g.center = g.nimg;
      g.off[g.nimg][0] = m * g.d + n * g.xi;
      g.off[g.nimg][1] = n * g.eta;
      ++g.nimg;
    }

  pfmm_plan* p = new pfmm_plan();
  p->sort_h = new pfmm::SortCell[2]();
  p->opts = *o;
  p->geom = g;
  p->ns_max = ns_max;
  p->nt_max = nt_max;
  p->ncomp = (o->kernel == PFMM_STOKES || o->kernel == PFMM_MSTOKES) ? 2 : 1;
  p->nout = p->ncomp;

  // ---- south/north modes (Eq. mpk0s with eps = tol/10; for beta > 0 modes
  // whose per-unit-charge bound e^{-chi eta}/(d chi (1 - e^{-chi eta})) is below
  // tol/10 are dropped from the top: chi_m grows with m, so the bound decreases).
  double eps = o->tol * 0.1;
  int M = p1 ? 0 : mpk0s(g.d, g.eta, eps);  // P1: no south/north parts
  // m = 0 is a regular term only for modhelm; for Laplace/Stokes it is the
  // moment term -(1/(2 d eta)) y sum q y' (Eq. phis3, Eq. pss0) added separately.
  int mode0 = (o->kernel == PFMM_MODHELM && !p1) ? 1 : 0;
  if (o->kernel == PFMM_MODHELM && !p1) {
    // drop threshold: the per-unit-charge bound times sqrt(ns_max) (see
    // we_quadrature: the dropped field of many charges grows like their l2
    // norm, the short-range potential does not)
    const double eps_drop = eps / std::sqrt(std::max<double>(1.0, (double)ns_max));
    auto bound = [&](int m) {
      double al = 2 * M_PI * m / g.d, chi = std::sqrt(al * al + o->beta * o->beta);
      double e = std::exp(-chi * g.eta);
      return e / (g.d * chi * (1 - e));
    };
    while (M >= 1 && bound(M) < eps_drop) --M;
    if (bound(0) < eps_drop) { mode0 = 0; M = 0; }
  }
  // modified Stokes (Theorem south_thm_ms): the beta family has an m = 0 term
  // (its block [[beta, 0], [0, 0]]); the Laplace family has none (each image
  // row is Poisson-summed on its own and the row integral of grad grad^T log r
  // vanishes).  No pruning: the Laplace family decays like Eq. mpk0s assumes.
  const bool ms = o->kernel == PFMM_MSTOKES;
  if (ms) mode0 = 1;
  Far& f = p->far;
  f.kernel = o->kernel;
  f.beta = (o->kernel == PFMM_MODHELM || ms) ? o->beta : 0.0;
  f.M = M;
  f.mode0 = mode0;
  f.nsn = mode0 ? (M + 1) : M;
  f.nrhs = o->nrhs;
  f.nch = (o->kernel == PFMM_STOKES) ? 4 : (ms ? 2 : 1);
  f.rows3 = p1 ? 0 : 1;
  f.msfam = 0;

  std::vector<double> nodes, nodes2;
  // the modified Stokes beta family integrates in kappa = sqrt(lambda^2 + beta^2)
  // like modified Helmholtz, the Laplace family in |lambda| like Laplace
  we_quadrature(g, ms ? PFMM_MODHELM : o->kernel, f.beta, o->tol, (double)ns_max, nodes);
  f.Nq = (int)(nodes.size() / 2);
  f.nterm = 2 * f.nsn + 2 * f.Nq;
  p->far2 = f;
  p->far2.nterm = 0;
  p->far2.Nq = 0;
  if (ms) {
    we_quadrature(g, PFMM_LAPLACE, 0.0, o->tol, (double)ns_max, nodes2);
    Far& f2 = p->far2;
    f2.msfam = 1;
    f2.mode0 = 0;
    f2.nsn = M;
    f2.Nq = (int)(nodes2.size() / 2);
    f2.nterm = 2 * f2.nsn + 2 * f2.Nq;
  }
  nodes.insert(nodes.end(), nodes2.begin(), nodes2.end());
  p->Nq = (int)(nodes.size() / 2);
  p->nodes_h = (double*)std::malloc(std::max<size_t>(1, nodes.size()) * sizeof(double));
  if (!nodes.empty()) std::memcpy(p->nodes_h, nodes.data(), nodes.size() * sizeof(double));

  // ---- NUFFT parameters (Sec. 6): GL lines, ES width, fine grid (sigma = 2,
  // power of two for the radix-2 FFT).
  p->n_gl = o->n_gl ? o->n_gl : (o->tol >= 1e-7 ? 8 : 16);
  int w = o->nufft_w ? o->nufft_w : std::min(16, std::max(2, (int)std::ceil(std::log10(1.0 / o->tol)) + 2));
  p->nufft_w = w;
  p->es_beta = 2.30 * w;
  // Singly periodic operator on the NUFFT path (Sec. 6.1 with the roles of x
  // and y exchanged: a fast algorithm is needed when eta >> d, where the
  // west/east rank grows like eta/d).  The nodes lambda_n are piecewise GL, not
  // uniform, so each GL line's transform in y is a type-3 one: a type-1
  // transform onto the uniform frequencies u dl (dl = 2 pi / Y, Y = 2 eta, so
  // that |y| <= Y/4 like the modes of a sigma = 2 grid) of the strengths divided
  // by Psi(y), then ES interpolation in lambda (width w, half-width
  // alpha = w dl / 2; Psi is the kernel's Fourier transform).  Nodes below
  // alpha + 2 dl stay on the direct kernels: they would need frequencies
  // u <= 0, and their lattice weight grows like 1/lambda^2.
  int p1_M = 0, p1_nq0 = p->Nq;
  double p1_Y = 0, p1_dl = 0, p1_alpha = 0;
  if (p1 && p->Nq > 0 && o->path != PFMM_PATH_DIRECT) {
    p1_Y = 2.0 * g.eta;
    p1_dl = 2.0 * M_PI / p1_Y;
    p1_alpha = 0.5 * w * p1_dl;
    const double lcut = p1_alpha + 2.0 * p1_dl;
    p1_nq0 = 0;
    while (p1_nq0 < p->Nq && nodes[2 * p1_nq0] < lcut) ++p1_nq0;
    if (p1_nq0 < p->Nq) p1_M = (int)std::ceil((nodes[2 * (p->Nq - 1)] + p1_alpha) / p1_dl) + 1;
  }
  const int p1_nnu = p->Nq - p1_nq0;
  const int Mt = p1 ? p1_M : M;  // uniform modes of the transforms
  int nf = 16;
  while (nf < 2 * (2 * Mt + 1) || nf < 2 * w) nf *= 2;
  p->nf = nf;
  int path = o->path;
  // the single-block shared-memory FFT handles fine grids up to 8192 points
  if (path == PFMM_PATH_AUTO) {
    const bool big = p1 ? p1_nnu >= 128 : M >= 64;
    path = (big && nf <= 8192 && !(o->flags & PFMM_DETERMINISTIC)) ? PFMM_PATH_NUFFT : PFMM_PATH_DIRECT;
  }
  if (path == PFMM_PATH_NUFFT && nf > 8192) {
    pfmm_plan_destroy(p);
    return fail(PFMM_ERR_INVALID_ARG, "NUFFT fine grid of %d points exceeds 8192 (use the direct path)", nf);
  }
  if (p1 ? p1_nnu == 0 : M == 0) path = PFMM_PATH_DIRECT;
  p->path = path;
  p->p1_nu = p1 && path == PFMM_PATH_NUFFT;
  p->p1_nq0 = p->p1_nu ? p1_nq0 : p->Nq;
  p->p1_M = p->p1_nu ? p1_M : 0;
  p->p1_Y = p1_Y;
  p->p1_dl = p1_dl;
  p->p1_alpha = p1_alpha;
  p->rho_h = nullptr;
  {
    std::vector<double> gx, gw;
    gauss_legendre(p->n_gl, gx, gw);
    p->gl_h = (double*)std::malloc(2 * p->n_gl * sizeof(double));
    // GL lines across the non-oscillatory direction: y in [-eta/2, eta/2]
    // (south/north), x in [-d/2, d/2] (singly periodic west/east)
    const double ext = p->p1_nu ? g.d : g.eta;
    for (int i = 0; i < p->n_gl; ++i) {
      double s = 1.0;  // barycentric weight 1/prod_{j != i}(t_i - t_j) (Eq. baryweights), scaled node
      for (int j = 0; j < p->n_gl; ++j)
        if (j != i) s /= (gx[i] - gx[j]);
      p->gl_h[2 * i] = 0.5 * ext * gx[i];
      p->gl_h[2 * i + 1] = s;
    }
    p->nphihat = Mt + 1;
    p->phihat_h = (double*)std::malloc((Mt + 1) * sizeof(double));
    for (int m = 0; m <= Mt; ++m) p->phihat_h[m] = es_phihat(p->es_beta, 2.0 * M_PI * m * (w * 0.5) / nf);
    if (p->p1_nu) {
      // 1/Psi(y), Psi(y) = alpha phihat(alpha y), on |y| <= eta/2 as a
      // Chebyshev series in t = 2 y / eta (64-point interpolation; the
      // coefficients beyond 40 are at rounding level for w <= 16)
      constexpr int N = 64;
      double f[N];
      for (int i = 0; i < N; ++i) {
        const double t = std::cos(M_PI * (i + 0.5) / N);
        f[i] = 1.0 / (p1_alpha * es_phihat(p->es_beta, p1_alpha * 0.5 * g.eta * t));
      }
      p->rho_h = (double*)std::malloc(kRhoCheb * sizeof(double));
      for (int k = 0; k < kRhoCheb; ++k) {
        double c = 0.0;
        for (int i = 0; i < N; ++i) c += f[i] * std::cos(k * M_PI * (i + 0.5) / N);
        p->rho_h[k] = (k == 0 ? 1.0 : 2.0) * c / N;
      }
    }
    p->tw_h = nullptr;
    if (path == PFMM_PATH_NUFFT) {
      // FP64 twiddles for the shared-memory FFT: (cos, sin)(2 pi k / nf), k < nf/2
      p->tw_h = (double*)std::malloc(nf * sizeof(double));
      for (int k = 0; k < nf / 2; ++k) {
        p->tw_h[2 * k] = std::cos(2.0 * M_PI * k / nf);
        p->tw_h[2 * k + 1] = std::sin(2.0 * M_PI * k / nf);
      }
    }
  }

  // ---- workspace layout
  Layout& L = p->lay;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = align256(off + std::max<size_t>(bytes, 1)); return r; };
  int nrhs = o->nrhs;
  L.status = take(kStatusWords * sizeof(int));
  L.moments = take(nrhs * 8 * sizeof(double));
  L.work = take(sizeof(unsigned long long));
  L.nodes = take(pfmm::node_region_bytes(p));
  L.src64 = take(2 * ns_max * sizeof(double));
  L.trg64 = take(2 * nt_max * sizeof(double));
  L.srcf = take(2 * ns_max * sizeof(float));
  L.trgf = take(2 * nt_max * sizeof(float));
  L.srcU = take(ns_max * sizeof(int));
  L.trgU = take(nt_max * sizeof(int));
  L.srcV = take(p->p1_nu ? ns_max * sizeof(int) : 0);
  L.trgV = take(p->p1_nu ? nt_max * sizeof(int) : 0);
  L.qc = take((size_t)nrhs * p->ncomp * ns_max * sizeof(double));
  L.qf = take((size_t)nrhs * p->ncomp * ns_max * sizeof(float));
  {
    // sorted-source arrays of the mixed P2P (sort.h)
    // (targets are sorted as well: with targets = sources they share the order)
    const bool mixed = o->precision == PFMM_MIXED;
    const size_t ns_m = mixed ? (size_t)ns_max : 0, nt_m = mixed ? (size_t)nt_max : 0;
    const size_t nsub = (ns_m + pfmm::kSubtile - 1) / pfmm::kSubtile;
    L.s_rel = take(ns_m * sizeof(float2));
    L.s_hl = take(ns_m * sizeof(float4));
    L.s_sub = take(nsub * sizeof(float4));
    L.s_ext = take(nsub * sizeof(float2));
    L.s_box = take((ns_m + pfmm::kBoxTile - 1) / pfmm::kBoxTile * sizeof(float4));
    L.qs = take((size_t)nrhs * p->ncomp * ns_m * sizeof(float));
    L.s_perm = take(ns_m * sizeof(int));
    L.s_sorted = take(ns_m * 2 * sizeof(double));
    L.t_sorted = take(nt_m * 2 * sizeof(double));
    L.t_perm = take(nt_m * sizeof(int));
    L.t_box = take((nt_m + pfmm::kBoxTile - 1) / pfmm::kBoxTile * sizeof(float4));
    L.sortd = take(2 * sizeof(pfmm::SortCell));
    L.sortscr = take(mixed ? pfmm::sort_scratch_bytes((int64_t)ns_m + (int64_t)nt_m, 2) : 0);
  }
  // (modified Stokes: both families' coefficients and weights, one after the other)
  L.coef = take((size_t)nrhs * f.nch * std::max(1, f.nterm + p->far2.nterm) * 2 * sizeof(double));
  L.wts = take((size_t)nrhs * 4 * std::max(1, f.nterm + p->far2.nterm) * 2 * sizeof(double));
  size_t nuf = 0;
  if (path == PFMM_PATH_NUFFT) {
    // FP64 spread grid [nrhs][nch][n_gl][nf], FP64 spectra F_n(k) [nrhs][nch][n_gl][M+1],
    // evaluation spectra [nrhs][npk][nf] complex (float2 for mixed, double2 for fp64)
    size_t cplx = 16;  // FFTs and spectra are FP64 on both precision paths
    size_t nline = (size_t)nrhs * pfmm::nufft_nch(o->kernel) * p->n_gl;
    nuf = nline * nf * 8 + nline * (Mt + 1) * 16 + 256 +
          (size_t)nrhs * pfmm::nufft_npk(o->kernel, p->n_gl) * nf * cplx + 256;
    // singly periodic: evaluation lines at the nodes [nrhs][lines][nodes] complex
    if (p->p1_nu) nuf += (size_t)nrhs * pfmm::p1_node_lines(o->kernel, p->n_gl) * p1_nnu * cplx + 256;
  }
  L.nufft = take(nuf);
  // adjoint scratch: dL/dpot projected as strengths is handled in place; the
  // gradient of the adjoint field at the sources needs [nrhs][2][max n]
  L.adj = take((size_t)nrhs * 2 * std::max(ns_max, nt_max) * sizeof(double) +
               (size_t)nrhs * p->ncomp * std::max(ns_max, nt_max) * sizeof(double));
  // modified Helmholtz near field: pairs with beta r > x_c are skipped, x_c
  // chosen so that every skipped term is below tol/10 / (images * ns_max):
  // even if all the terms a target skips had one sign and that bound, they
  // would stay below tol/10 in total (K0(x) < sqrt(pi/(2x)) e^-x; fixed point
  // of x = ln(sqrt(pi/(2x)) / thr)); between 10 and 50.
  {
    const double thr = o->tol * 0.1 / ((double)g.nimg * std::max<double>(1.0, (double)ns_max));
    double x = 30.0;
    for (int it = 0; it < 30; ++it) x = std::log(std::sqrt(M_PI / (2.0 * x)) / thr);
    p->mh_cut = std::min(50.0, std::max(10.0, x + 0.5));
  }
  pfmm::fmm_setup(p);
  L.fmm = take(p->fmm.bytes);
  {
    // deterministic mode: per-warp moment partials (k_prep_q / k_net, whole
    // blocks of 8 warps) and per-chunk formation partials, one use at a time
    size_t det = 0;
    if (o->flags & PFMM_DETERMINISTIC) {
      const size_t warps = (size_t)((ns_max + 255) / 256) * 8;
      const size_t prep = warps * nrhs * 4 * sizeof(double);
      const size_t form = (size_t)kDetChunks * nrhs * f.nch * std::max(f.nterm, p->far2.nterm) * 2 * sizeof(double);
      det = std::max(prep, form);
    }
    L.det = take(det);
  }
  L.total = off;
  size_t ncq = (size_t)nrhs * p->ncomp;
  L.stage = off;
  size_t stage = 2 * ns_max * 8 + 2 * nt_max * 8 + ncq * ns_max * 8 + (size_t)nrhs * p->nout * nt_max * 8 +
                 (size_t)nrhs * 2 * nt_max * 8 + 5 * 256;
  L.total_host = off + stage;
  f.nodes = nullptr;
  *out = p;
  return PFMM_OK;
}

void pfmm_plan_destroy(pfmm_plan* p) {
  if (!p) return;
  if (p->prof)
    for (int i = 0; i < kPlanEvents; ++i) cudaEventDestroy(p->ev[i]);
  if (p->side_ready) {
    cudaStreamDestroy(p->side);
    cudaEventDestroy(p->fork_ev);
    cudaEventDestroy(p->join_ev);
  }
  std::free(p->nodes_h);
  std::free(p->gl_h);
  std::free(p->phihat_h);
  std::free(p->tw_h);
  std::free(p->rho_h);
  delete[] p->sort_h;
  delete p;
}

pfmm_status pfmm_workspace_size(const pfmm_plan* p, size_t* bytes) {
  if (!p || !bytes) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
  *bytes = p->lay.total;
  return PFMM_OK;
}

pfmm_status pfmm_workspace_size_host(const pfmm_plan* p, size_t* bytes) {
  if (!p || !bytes) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
  *bytes = p->lay.total_host;
  return PFMM_OK;
}

pfmm_status pfmm_plan_describe(const pfmm_plan* p, pfmm_plan_desc* d) {
  if (!p || !d) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
  d->d = p->geom.d; d->xi = p->geom.xi; d->eta = p->geom.eta;
  for (int i = 0; i < 4; ++i) d->rot[i] = p->geom.rot[i];
  d->m0 = p->geom.m0;
  d->we_rotated = p->geom.we_rot;
  d->we_dir[0] = p->geom.wc;
  d->we_dir[1] = p->geom.ws;
  d->M = p->far.M;
  d->mode0 = (p->opts.kernel == PFMM_MODHELM || p->opts.kernel == PFMM_MSTOKES) ? p->far.mode0 : 1;
  d->Nq = p->Nq;
  d->path = p->path;
  d->n_gl = p->n_gl; d->nf = p->nf; d->nufft_w = p->nufft_w; d->es_beta = p->es_beta;
  d->nlaunch = p->nlaunch;
  d->npairs = p->npairs;
  d->near_fmm = p->fmm.on;
  d->near_order = p->fmm.p;
  d->near_leaf = p->fmm.nleaf;
  d->near_theta = p->fmm.theta;
  d->p1_nufft_nodes = p->p1_nu ? p->Nq - p->p1_nq0 : 0;
  return PFMM_OK;
}

pfmm_status pfmm_near_stats(pfmm_plan* p, const void* workspace, void* stream, int64_t out[5]) {
  if (!p || !workspace || !out) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
  if (!p->fmm.on) return fail(PFMM_ERR_INVALID_ARG, "the plan does not use the near-field tree code");
  cudaError_t e = fmm_stats(p, (const char*)workspace, (cudaStream_t)stream, out);
  if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, "read tree-code statistics: %s", cudaGetErrorString(e));
  return PFMM_OK;
}

pfmm_status pfmm_profile_enable(pfmm_plan* p, int on) {
  if (!p) return fail(PFMM_ERR_INVALID_ARG, "NULL plan");
  if (on && !p->prof) {
    for (int i = 0; i < kPlanEvents; ++i) {
      cudaError_t e = cudaEventCreate(&p->ev[i]);
      if (e != cudaSuccess) {
        for (int k = 0; k < i; ++k) cudaEventDestroy(p->ev[k]);
        return fail(PFMM_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
      }
    }
    p->prof = true;
  } else if (!on && p->prof) {
    for (int i = 0; i < kPlanEvents; ++i) cudaEventDestroy(p->ev[i]);
    p->prof = false;
  }
  return PFMM_OK;
}

pfmm_status pfmm_profile_read(pfmm_plan* p, float* ms, int n) {
  if (!p || !ms || n < 0) return fail(PFMM_ERR_INVALID_ARG, "bad argument");
  if (!p->prof) return fail(PFMM_ERR_INVALID_ARG, "profiling not enabled");
  cudaError_t e = cudaEventSynchronize(p->ev[3]);
  if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
  for (int i = 0; i < n && i < 3; ++i) {
    e = cudaEventElapsedTime(&ms[i], p->ev[i], p->ev[i + 1]);
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e));
  }
  // tree-code sub-phases of the near field: tree, upward pass, traversal and
  // grouping, downward pass, leaves (events 2, 4, 5, 6, 7, 3)
  // (with the tree phases beside the far field, the tree starts after the
  // preparation, event 1)
  const int from[5] = {p->near_overlap ? 1 : 2, 4, 5, 6, 7}, to[5] = {4, 5, 6, 7, 3};
  for (int i = 3; i < n && i < 8; ++i) {
    ms[i] = 0.0f;
    if (!p->near_fmm_ran) continue;
    e = cudaEventElapsedTime(&ms[i], p->ev[from[i - 3]], p->ev[to[i - 3]]);
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e));
  }
  return PFMM_OK;
}

pfmm_status pfmm_profile_pairs(pfmm_plan* p, const void* workspace, void* stream, double* pairs) {
  if (!p || !workspace || !pairs) return fail(PFMM_ERR_INVALID_ARG, "NULL argument");
  if (!p->prof) return fail(PFMM_ERR_INVALID_ARG, "profiling not enabled");
  *pairs = (double)p->npairs;
  if (p->fmm.on) {
    int64_t st[5];
    cudaError_t e = fmm_stats(p, (const char*)workspace, (cudaStream_t)stream, st);
    if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, "read pair count: %s", cudaGetErrorString(e));
    *pairs = (double)st[3];
    return PFMM_OK;
  }
  if (p->opts.kernel != PFMM_MODHELM || p->opts.precision != PFMM_MIXED) return PFMM_OK;
  unsigned long long w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, (const char*)workspace + p->lay.work, sizeof w, cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return fail(PFMM_ERR_CUDA, "read pair count: %s", cudaGetErrorString(e));
  *pairs = (double)w;
  return PFMM_OK;
}

pfmm_status pfmm_execute(pfmm_plan* p, void* workspace, size_t ws_bytes, int64_t ns, const double* src,
                         const double* q, int64_t nt, const double* trg, double* pot, double* grad,
                         void* stream) {
  if (!p) return fail(PFMM_ERR_INVALID_ARG, "NULL plan");
  if (ns < 0 || nt < 0 || ns > p->ns_max || nt > p->nt_max)
    return fail(PFMM_ERR_INVALID_ARG, "ns=%lld nt=%lld outside plan maxima (%lld, %lld)", (long long)ns,
                (long long)nt, (long long)p->ns_max, (long long)p->nt_max);
  if (!workspace || ws_bytes < p->lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(PFMM_ERR_WORKSPACE, "workspace NULL, misaligned or smaller than %zu bytes", p->lay.total);
  bool stokes = p->opts.kernel == PFMM_STOKES || p->opts.kernel == PFMM_MSTOKES;
  if (stokes && grad) return fail(PFMM_ERR_INVALID_ARG, "grad must be NULL for the Stokes kernels");
  if (p->opts.flags & PFMM_NO_GRAD) grad = nullptr;
  if (nt > 0 && !pot && !grad) return fail(PFMM_ERR_INVALID_ARG, "no output requested");
  if (nt > 0 && !trg) return fail(PFMM_ERR_INVALID_ARG, "NULL targets");
  if (ns > 0 && (!src || !q)) return fail(PFMM_ERR_INVALID_ARG, "NULL sources/strengths");
  bool self = (trg == src) && (nt == ns);
  if (trg == src && nt != ns) return fail(PFMM_ERR_INVALID_ARG, "targets alias sources but nt != ns");
  p->s_stride = ns;
  p->t_stride = nt;
  p->o_stride = nt;
  return pfmm::execute_cell(p, (char*)workspace, ns, src, q, nt, trg, pot, grad, (cudaStream_t)stream, self, true,
                            !(p->opts.flags & PFMM_FAR_ONLY));
}

pfmm_status pfmm_execute_host(pfmm_plan* p, void* workspace, size_t ws_bytes, int64_t ns, const double* src,
                              const double* q, int64_t nt, const double* trg, double* pot, double* grad,
                              void* stream) {
  if (!p) return fail(PFMM_ERR_INVALID_ARG, "NULL plan");
  if (!workspace || ws_bytes < p->lay.total_host || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(PFMM_ERR_WORKSPACE, "workspace NULL, misaligned or smaller than %zu bytes", p->lay.total_host);
  if (ns < 0 || nt < 0 || ns > p->ns_max || nt > p->nt_max) return fail(PFMM_ERR_INVALID_ARG, "sizes");
  if ((p->opts.kernel == PFMM_STOKES || p->opts.kernel == PFMM_MSTOKES) && grad)
    return fail(PFMM_ERR_INVALID_ARG, "grad must be NULL for the Stokes kernels");
  if (p->opts.flags & PFMM_NO_GRAD) grad = nullptr;
  bool self = (trg == src) && (nt == ns);
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)workspace + p->lay.stage;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* r = base + off; off = align256(off + bytes); return r; };
  int nrhs = p->opts.nrhs;
  double* d_src = (double*)take(2 * ns * 8);
  double* d_trg = self ? d_src : (double*)take(2 * nt * 8);
  double* d_q = (double*)take((size_t)nrhs * p->ncomp * ns * 8);
  double* d_pot = pot ? (double*)take((size_t)nrhs * p->nout * nt * 8) : nullptr;
  double* d_grad = grad ? (double*)take((size_t)nrhs * 2 * nt * 8) : nullptr;
  cudaError_t e = cudaSuccess;
  if (ns) e = cudaMemcpyAsync(d_src, src, 2 * ns * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !self && nt) e = cudaMemcpyAsync(d_trg, trg, 2 * nt * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ns) e = cudaMemcpyAsync(d_q, q, (size_t)nrhs * p->ncomp * ns * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "stage inputs");
  pfmm_status s = pfmm_execute(p, workspace, p->lay.total, ns, d_src, d_q, nt, d_trg, d_pot, d_grad, stream);
  if (s != PFMM_OK) return s;
  if (pot) e = cudaMemcpyAsync(pot, d_pot, (size_t)nrhs * p->nout * nt * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, d_grad, (size_t)nrhs * 2 * nt * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "read back outputs");
  return PFMM_OK;
}

pfmm_status pfmm_stokes_pressure(pfmm_plan* p, void* workspace, size_t ws_bytes, int64_t ns, const double* src,
                                 const double* f, int64_t nt, const double* trg, double* pres, void* stream) {
  if (!p) return fail(PFMM_ERR_INVALID_ARG, "NULL plan");
  if (p->opts.kernel != PFMM_LAPLACE || (p->opts.nrhs & 1))
    return fail(PFMM_ERR_INVALID_ARG, "the pressure needs a Laplace plan with an even nrhs (2 per Stokes rhs)");
  if (p->opts.flags & (PFMM_FAR_ONLY | PFMM_NEAR_ONLY | PFMM_NO_GRAD))
    return fail(PFMM_ERR_INVALID_ARG, "the pressure is defined for the full operator with the gradient");
  if (ns < 0 || nt < 0 || ns > p->ns_max || nt > p->nt_max)
    return fail(PFMM_ERR_INVALID_ARG, "ns=%lld nt=%lld outside plan maxima", (long long)ns, (long long)nt);
  if (!workspace || ws_bytes < p->lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(PFMM_ERR_WORKSPACE, "workspace NULL, misaligned or smaller than %zu bytes", p->lay.total);
  if ((ns > 0 && (!src || !f)) || (nt > 0 && (!trg || !pres))) return fail(PFMM_ERR_INVALID_ARG, "NULL inputs");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const bool self = (trg == src) && (nt == ns);
  // gradient of the nrhs Laplace fields into the adjoint scratch [nrhs][2][nt]
  double* g = (double*)(ws + p->lay.adj);
  p->s_stride = ns;
  p->t_stride = nt;
  p->o_stride = nt;
  pfmm_status s = pfmm::execute_cell(p, ws, ns, src, f, nt, trg, nullptr, g, st, self, true, true);
  if (s != PFMM_OK) return s;
  cudaError_t e = pfmm::launch_pressure(p->opts.nrhs / 2, nt, g, pres, st);
  if (e != cudaSuccess) return cuda_fail(e, "pressure kernel");
  return PFMM_OK;
}

pfmm_status pfmm_execute_adjoint(pfmm_plan* p, void* workspace, size_t ws_bytes, int64_t ns, const double* src,
                                 const double* q, int64_t nt, const double* trg, const double* g,
                                 const double* grad_fwd, double* dq, double* dsrc, double* dtrg, void* stream) {
  if (!p) return fail(PFMM_ERR_INVALID_ARG, "NULL plan");
  if (ns < 0 || nt < 0 || nt > p->ns_max || ns > p->nt_max || ns > p->ns_max || nt > p->nt_max)
    return fail(PFMM_ERR_INVALID_ARG, "adjoint needs nt <= ns_max and ns <= nt_max (ns=%lld nt=%lld)", (long long)ns,
                (long long)nt);
  if (!workspace || ws_bytes < p->lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(PFMM_ERR_WORKSPACE, "workspace NULL, misaligned or smaller than %zu bytes", p->lay.total);
  // Stokes kernels: strengths only.  Modified Stokes: G^MS(r) is a symmetric
  // matrix and even in r, and the image-row sum is symmetric under l -> -l, so
  // the operator is its own transpose; no gauge, so g is used as given (the
  // neutral projection below applies to Laplace and Stokes only).
  const bool stokes = p->opts.kernel == PFMM_STOKES || p->opts.kernel == PFMM_MSTOKES;
  if (stokes && (dsrc || dtrg)) return fail(PFMM_ERR_INVALID_ARG, "Stokes adjoint: strengths only (dq)");
  if (dtrg && !grad_fwd) return fail(PFMM_ERR_INVALID_ARG, "dtrg needs the forward gradient grad_fwd");
  if (p->opts.flags & (PFMM_FAR_ONLY | PFMM_NEAR_ONLY))
    return fail(PFMM_ERR_INVALID_ARG, "the adjoint is defined for the full operator");
  if ((ns > 0 && (!src || !q)) || (nt > 0 && (!trg || !g))) return fail(PFMM_ERR_INVALID_ARG, "NULL inputs");
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  const bool self = (trg == src) && (nt == ns);
  const int nrhs = p->opts.nrhs;
  const int64_t nmax = std::max(p->ns_max, p->nt_max);
  double* adj_grad = (double*)(ws + p->lay.adj);             // [nrhs][2][ns]
  double* adj_pot = adj_grad + (size_t)nrhs * 2 * nmax;      // [nrhs][ncomp][ns]
  cudaError_t e;
  if (dq || dsrc) {
    // sources = targets of the forward call with strengths g, targets = forward sources
    const unsigned saved = p->opts.flags;
    p->opts.flags = saved | PFMM_PROJECT_NEUTRAL;
    p->s_stride = nt;
    p->t_stride = ns;
    p->o_stride = ns;
    double* pot_out = dq ? dq : adj_pot;
    pfmm_status s = pfmm::execute_cell(p, ws, nt, self ? src : trg, g, ns, src, pot_out, dsrc ? adj_grad : nullptr,
                                       st, self, true, true);
    p->opts.flags = saved;
    if (s != PFMM_OK) return s;
    if (dsrc) {
      // targets = sources with dsrc == dtrg: one array receives both roles
      const bool both = self && dtrg == dsrc;
      e = launch_contract(nrhs, ns, q, ns, adj_grad, ns, both ? g : nullptr, both ? grad_fwd : nullptr, dsrc, st);
      if (e != cudaSuccess) return cuda_fail(e, "contract");
      if (both) return PFMM_OK;
    }
  }
  if (dtrg) {
    e = launch_contract(nrhs, nt, g, nt, grad_fwd, nt, nullptr, nullptr, dtrg, st);
    if (e != cudaSuccess) return cuda_fail(e, "contract");
  }
  return PFMM_OK;
}

pfmm_status pfmm_get_status(pfmm_plan* p, void* workspace, void* stream) {
  if (!p) return fail(PFMM_ERR_INVALID_ARG, "NULL plan");
  if (!workspace) {
    // the status word of pfmm_execute_static's scratch array on this device
    pfmm_status s = static_scratch(&workspace);
    if (s != PFMM_OK) return s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int h[kStatusWords];
  cudaError_t e = cudaMemcpyAsync(h, (char*)workspace + p->lay.status, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  e = cudaMemsetAsync((char*)workspace + p->lay.status, 0, sizeof h, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear status");
  if (h[0] & ST_NONFINITE) return fail(PFMM_ERR_NONFINITE, "non-finite coordinates or strengths");
  if (h[0] & ST_TIMEOUT) return fail(PFMM_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h[0] & ST_NOT_NEUTRAL) return fail(PFMM_ERR_NOT_NEUTRAL, "net charge / net force is not zero");
  if (h[0] & ST_OUTSIDE) return fail(PFMM_ERR_INVALID_ARG, "points outside the singly periodic strip |y| < eta/2");
  return PFMM_OK;
}

}  // extern "C"
