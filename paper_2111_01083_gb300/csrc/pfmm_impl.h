// Internal declarations shared by the host plan code and the CUDA kernels.
#pragma once
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>
#include "../../include/pfmm.h"

namespace pfmm {

constexpr int kMaxNear = 32;      // (2 m0 + 1) * 3 images; m0 <= 3 after reduction
constexpr int kPlanEvents = 8;    // profiling events of a plan
constexpr int kRhoCheb = 40;      // Chebyshev terms of the singly periodic NUFFT deconvolution 1/Psi(y)
constexpr int kDetChunks = 128;   // deterministic mode: source chunks of the coefficient formation
constexpr int kStatusWords = 8;   // status word region (ints)

// device status bits (combined with atomicOr; mapped to pfmm_status by the host)
enum : int { ST_NONFINITE = 1, ST_NOT_NEUTRAL = 2, ST_TIMEOUT = 4, ST_OUTSIDE = 8 };

// Geometry of the canonical cell, passed by value to kernels.
struct Geom {
  double d, xi, eta;      // e1 = (d, 0), e2 = (xi, eta)
  double rot[4];          // canonical = rot * input (row-major)
  double ainv[4];         // fractional coordinates u = ainv * canonical
  int m0;
  int nimg;               // (2 m0 + 1) * 3
  double off[kMaxNear][2];// image offsets l_mn = m e1 + n e2 (canonical)
  int center;             // index of the (0, 0) image in off[]
  int p1;                 // singly periodic (along e1 only): no wrap across the strip
  // west/east frame: (x~, y~) = (wc x - ws y, ws x + wc y); image column step
  // (wdx, wdy) and row step (wxr, wyr) in it.  Axis: (1, 0), (d, 0), (xi, eta).
  int we_rot;
  double wc, ws, wdx, wdy, wxr, wyr;
};

// Far-field parameters (direct path).  Terms are ordered
//   [ south m = m_lo..M | north m = m_lo..M | west n = 0..Nq-1 | east n = 0..Nq-1 ]
// with m_lo = 0 if mode0 else 1.
struct Far {
  int kernel;        // pfmm_kernel
  double beta;
  int M, mode0, Nq;
  int nsn;           // terms per south/north block = M - m_lo + 1
  int nterm;         // 2 nsn + 2 Nq
  int nrhs;
  int nch;           // coefficient channels per rhs: 1 (scalar) or 4 (Stokes: a_x, a_y, b_x, b_y)
  int rows3;         // west/east over the image rows n = -1, 0, 1 (doubly periodic) or n = 0 only (P1)
  int msfam;         // modified Stokes: 0 the beta family (decay chi, kappa), 1 the Laplace family (|alpha|, |lambda|)
  const double* nodes;  // device [Nq][2] (lambda_n, w_n), in workspace
  // FP32 term decoding of the mixed kernels (set at launch): 2 pi / d, beta
  float alpha1f = 0.f, beta_f = 0.f;
};

// NUFFT path: charge channels per rhs (scalar q; Stokes f_x, f_y, y' f_x,
// y' f_y; modified Stokes f_x, f_y) and complex evaluation-spectrum lines per
// rhs (scalar: potential + y-derivative per GL line, x-derivatives two lines
// per spectrum; Stokes: the a and b weight lines per GL line; modified
// Stokes: one line u_x + i u_y per GL line).
inline int nufft_nch(int kernel) { return kernel == PFMM_STOKES ? 4 : (kernel == PFMM_MSTOKES ? 2 : 1); }
// singly periodic NUFFT: evaluation lines per rhs at the nodes (scalar: value
// and x-derivative per GL line; Stokes: a_x, a_y, b_x, b_y per GL line)
inline int p1_node_lines(int kernel, int n_gl) { return (kernel == PFMM_STOKES ? 4 : 2) * n_gl; }
inline int nufft_npk(int kernel, int n_gl) {
  return kernel == PFMM_STOKES ? 2 * n_gl : (kernel == PFMM_MSTOKES ? n_gl : n_gl + (n_gl + 1) / 2);
}

// Workspace layout (byte offsets from the workspace base, all 256-aligned).
struct Layout {
  size_t status, moments;
  size_t work;             // uint64: near-image pairs evaluated (counted while profiling)
  size_t nodes;
  size_t src64, trg64;     // double [2][n] canonical coordinates
  size_t srcf, trgf;       // float  [2][n] canonical coordinates (mixed far field)
  size_t srcU, trgU;       // int32 [n] fixed-point x/d phase (mixed south/north)
  size_t srcV, trgV;       // int32 [n] fixed-point y/Y phase (singly periodic NUFFT, mixed)
  // mixed P2P: spatially sorted sources (and, for modified Helmholtz, targets)
  size_t s_rel;            // float2 [ns] coordinates relative to the subtile centre
  size_t s_hl;             // float4 [ns] sorted (x_hi, x_lo, y_hi, y_lo)
  size_t s_sub;            // float4 [ceil(ns/16)] subtile centres (hi/lo)
  size_t s_ext;            // float2 [ceil(ns/16)] subtile half extents
  size_t s_box;            // float4 [ceil(ns/128)] source tile boxes
  size_t qs;               // float [nrhs][ncomp][ns] strengths in sorted order
  size_t s_perm;           // int [ns] input index of sorted source p
  size_t s_sorted;         // double [2][ns] sorted coordinates (targets = sources)
  size_t t_sorted;         // double [2][nt] sorted target coordinates (separate targets)
  size_t t_perm;           // int [nt]
  size_t t_box;            // float4 [ceil(nt/128)]
  size_t sortd;            // SortCell [2] device descriptors
  size_t sortscr;          // radix-sort scratch
  size_t qc;               // strengths in canonical frame: double [nrhs][ncomp][ns]
  size_t qf;               // float copy of qc (mixed P2P and far field)
  size_t coef;             // double2 [nrhs][nch][nterm]
  size_t wts;              // weights for evaluation: double2 or float2 [nrhs][nwch][nterm]
  size_t nufft;            // NUFFT scratch (grids, spectra)
  size_t adj;              // adjoint scratch (gradient of the adjoint field, potential if dq is not wanted)
  size_t fmm;              // near-field tree code (FmmPlan offsets are relative to this)
  size_t det;              // deterministic mode: partial sums reduced in a fixed order
  size_t stage;            // host-staging region (pfmm_execute_host only)
  size_t total, total_host;
};

// Near field by the tree code of fmm.cu (see there): sizes and byte offsets
// of its region of the workspace, fixed at plan creation from ns_max, nt_max.
constexpr int kFmmL = 11;                  // finest tree level: boxes of side s0 / 2^11
constexpr int kFmmIter = 2 * (kFmmL + 1);  // traversal sweeps (each descends at least one tree)
constexpr int kFmmMaxP = 32;               // expansion terms are lanes of a warp
struct FmmPlan {
  int on;              // 1: the near field runs through the tree code
  int p;               // expansion terms (coefficients 0 .. p-1)
  int nleaf;           // a box with more points than this is split (down to level kFmmL)
  double theta;        // a (target box, source box, image) triple is expanded when r_t + r_s <= theta |c_t - c_s - l|
  int ncol;            // root boxes (squares of side s0) along x
  double x0, y0, s0;   // lower-left corner of the root row, root side
  int nchan;           // complex expansions per source box: nrhs (Laplace), 4 nrhs (Stokes)
  int64_t npts;        // ns_max + nt_max
  int64_t node_cap;    // bound on tree boxes of both point sets (never exceeded)
  int64_t exp_cap;     // boxes with expansions; more boxes, or longer lists, switch to the direct fallback
  int64_t m2l_cap, p2p_cap, front_cap;
  // byte offsets inside the region
  size_t o_ctl, o_key, o_val, o_key2, o_val2, o_hist, o_xy, o_hl, o_perm, o_qd, o_qf, o_cnt, o_lf, o_off,
      o_bsum, o_lo, o_hi, o_lev, o_par, o_nend, o_nch, o_done, o_ctr, o_half, o_rad, o_scl, o_mult, o_loc, o_front,
      o_m2l, o_p2p, o_gcnt, o_gcur, o_glist, o_gtgt, o_roots;
  size_t bytes;
};

}  // namespace pfmm

namespace pfmm {
struct SortCell;
}

// pfmm_plan is an opaque C type; its definition is here so that all
// translation units of the library see the same layout.
struct pfmm_plan {
  pfmm_opts opts;
  pfmm::Geom geom;
  pfmm::Far far;
  pfmm::Far far2;           // modified Stokes: the Laplace family (far: the beta family); nterm 0 otherwise
  int64_t ns_max, nt_max;
  int nout;                 // output components per rhs for 'pot' (1 scalar, 2 Stokes)
  int ncomp;                // strength components (1 scalar, 2 Stokes)
  int path;                 // resolved path
  // west/east quadrature (host copy); modified Stokes: the beta family's
  // far.Nq nodes, then the Laplace family's far2.Nq
  int Nq;
  double* nodes_h;          // [Nq][2]
  // NUFFT parameters
  int n_gl, nf, nufft_w;
  double es_beta;
  double* gl_h;             // [n_gl][2] (ybar_n, sigma_n) on [-eta/2, eta/2]
  double* phihat_h;         // [M+1] ES kernel Fourier transform at modes 0..M
  double* tw_h;             // [nf/2][2] FFT twiddles (cos, sin)(2 pi k / nf), NUFFT path only
  int nphihat;              // entries of phihat_h (M + 1; singly periodic NUFFT: p1_M + 1)
  // singly periodic operator on the NUFFT path (west/east parts through the
  // transforms with the roles of x and y exchanged): west/east nodes
  // [0, p1_nq0) stay on the direct kernels, [p1_nq0, Nq) go through a type-1
  // transform in y over the virtual period p1_Y = 2 eta (uniform frequencies
  // u p1_dl, u = 0..p1_M) and ES interpolation in lambda (half-width p1_alpha);
  // gl_h then holds GL nodes in x on [-d/2, d/2]
  int p1_nu;                // 1: on
  int p1_nq0, p1_M;
  double p1_Y, p1_dl, p1_alpha;
  double* rho_h;            // [kRhoCheb] Chebyshev coefficients of 1/Psi(y) on |y| <= eta/2
  pfmm::Layout lay;
  pfmm::FmmPlan fmm;        // near field by the tree code (fmm.on)
  double mh_cut;            // modified Helmholtz P2P: pairs with beta r > mh_cut are skipped
  // what the last eager execute left in a workspace (a captured execute
  // reuses it instead of uploading from pageable host memory): the node
  // tables, and the P2P sort descriptors for (workspace, ns, nt, self)
  mutable const char* tables_ws;
  mutable const char* sort_ws;
  mutable int64_t sort_ns, sort_nt;
  mutable bool sort_self;
  // host copies of the sort descriptors of the last execute (sources, targets);
  // kept in the plan so that the asynchronous upload reads live memory
  pfmm::SortCell* sort_h;
  // row strides of the caller's arrays for the current execute: sources
  // (src [2][*], q [nrhs][comp][*]), targets (trg [2][*]) and outputs
  // (pot/grad [nrhs][comp][*]); equal to ns / nt for a single cell, to the
  // concatenated totals for a batch
  int64_t s_stride, t_stride, o_stride;
  // tracing / bookkeeping
  bool prof;
  cudaEvent_t ev[pfmm::kPlanEvents];  // phase boundaries (0-3), tree-code sub-phases (4-7)
  bool near_fmm_ran;                  // the last execute ran the tree code
  // tree-code executes: the tree phases (sort, build, upward pass, traversal,
  // downward pass) run on a second stream beside the far field, which they
  // do not touch; the leaf kernels, which add into the outputs, join back
  // (created at the first execute outside stream capture)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool side_ready = false;
  bool near_overlap = false;          // the last execute overlapped them
  int nlaunch;
  int64_t npairs;
};

namespace pfmm {
// Byte offsets inside the node-table region (L.nodes): west/east nodes
// [max(1,Nq)][2], GL lines [n_gl][2], phihat [nphihat], then (16-aligned) the
// FFT twiddles [nf/2][2] and the singly periodic NUFFT's Chebyshev table.
inline size_t off_gl(const pfmm_plan* p) { return (size_t)(p->Nq > 0 ? p->Nq : 1) * 2 * sizeof(double); }
inline size_t off_phihat(const pfmm_plan* p) { return off_gl(p) + (size_t)p->n_gl * 2 * sizeof(double); }
inline size_t off_twiddle(const pfmm_plan* p) {
  return (off_phihat(p) + (size_t)p->nphihat * sizeof(double) + 15) & ~size_t(15);
}
inline size_t off_rho(const pfmm_plan* p) {
  return off_twiddle(p) + (p->tw_h ? (size_t)p->nf * sizeof(double) : 0);
}
inline size_t node_region_bytes(const pfmm_plan* p) {
  return off_rho(p) + (p->rho_h ? (size_t)kRhoCheb * sizeof(double) : 0);
}

// Record a profiling event on st; under stream capture as an external event
// node, so that every replay of the graph records it (a plain record during
// capture only orders the graph's nodes).
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
  return cap != cudaStreamCaptureStatusNone ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
                                            : cudaEventRecord(ev, st);
}

// kernels.cu entry points (host-side launchers)
cudaError_t launch_prep(const pfmm_plan* p, char* ws, int64_t ns, const double* src, const double* q,
                        int64_t nt, const double* trg, bool self, cudaStream_t st);
cudaError_t launch_far_direct(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self,
                              double* pot, double* grad, cudaStream_t st);
cudaError_t launch_far_nufft(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self,
                             double* pot, double* grad, cudaStream_t st);
cudaError_t launch_p2p(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self,
                       double* pot, double* grad, bool accumulate, cudaStream_t st);
// near field through the tree code (fmm.cu); adds to pot/grad like launch_p2p
// Tree code: its tree phases on st_tree; the leaf kernels on st (after
// st_tree's work, through `join`, when the two differ).
cudaError_t launch_fmm_near(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot,
                            double* grad, cudaStream_t st, cudaStream_t st_tree = nullptr, cudaEvent_t join = nullptr);
// sizes and offsets of the tree code's workspace region (p->fmm.bytes = 0 when it is off)
void fmm_setup(pfmm_plan* p);
// statistics of the last tree-code execute (see pfmm_near_stats); synchronises st
cudaError_t fmm_stats(const pfmm_plan* p, const char* ws, cudaStream_t st, int64_t out[5]);
// records a thread-local error message (pfmm_last_error) and returns s
pfmm_status set_error(pfmm_status s, const char* fmt, ...);
cudaError_t upload_tables(const pfmm_plan* p, char* ws, cudaStream_t st);
pfmm_status execute_cell(pfmm_plan* p, char* ws, int64_t ns, const double* src, const double* q, int64_t nt,
                         const double* trg, double* pot, double* grad, cudaStream_t st, bool self, bool upload,
                         bool near);
// device address of pfmm_execute_static's scratch array on the current device
pfmm_status static_scratch(void** out);
// kernels launched by the most recent launch_* call (set by each launcher)
extern thread_local int g_launches;
cudaError_t launch_zero_out(const pfmm_plan* p, int64_t nt, double* pot, double* grad, cudaStream_t st);
// pres[r][l] = -(g[2r][0][l] + g[2r+1][1][l]): the Stokes pressure from the
// gradients of the Laplace fields of the force components.
cudaError_t launch_pressure(int nrhs, int64_t nt, const double* g, double* pres, cudaStream_t st);
cudaError_t launch_contract(int nrhs, int64_t n, const double* a, int64_t sa, const double* b, int64_t sb,
                            const double* c, const double* d, double* out, cudaStream_t st);
}  // namespace pfmm
