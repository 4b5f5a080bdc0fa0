// Arguments of the near-image P2P kernels (shared by the single-cell and
// batched launchers).
#pragma once
#include "pfmm_impl.h"
#include "sort.h"

namespace pfmm {

struct P2PArgs {
  Geom g;
  int nt, ns, chunk;
  int64_t os;            // output row stride
  int r0, nrhs;          // rhs group start, total rhs
  const double* trg64;   // [2][nt] canonical (sorted on the mixed path, see t_perm)
  const int* t_perm;     // output index of target l (NULL: l itself)
  const float4* t_box;   // [ceil(nt/128)] boxes of target blocks (modified Helmholtz culling)
  // mixed kernels: sources in spatially sorted order (sort.h)
  const float2* s_rel;   // [ns] coordinates relative to the subtile centre
  const float4* s_hl;    // [ns] (x_hi, x_lo, y_hi, y_lo)
  const float4* s_sub;   // [ceil(ns/16)] subtile centres (x_hi, x_lo, y_hi, y_lo)
  const float2* s_ext;   // [ceil(ns/16)] subtile half extents
  const float4* s_box;   // [ceil(ns/128)] source tile boxes
  const float* qs;       // [nrhs][ncomp][ns] FP32 strengths in sorted order
  float cut;             // modified Helmholtz: pairs with r > cut = x_c / beta are skipped (x_c from the plan)
  const double* src64;   // [2][ns] (FP64 kernel)
  const double* qc;      // [nrhs][ncomp][ns] (FP64 kernel)
  float beta_f;
  double beta;
  float lgc;             // log2(r^2) shift (Laplace/Stokes, FP64 add-back), see below
  float kimg[kMaxNear];  // per-image scale 2^-e_i of r^2 (exact powers of two)
  float offf[kMaxNear][2];  // image offsets in FP32 (tile culling; the high parts of the hi/lo split)
  float offl[kMaxNear][2];  // low parts: offset = offf + offl to ~2^-48 relative
  const float4* t_hl;       // [nt] target (x_hi, x_lo, y_hi, y_lo) when targets = sources (mixed), else NULL
  const double* mom;     // FP64 moments: mom[r*8+0] = sum q (Stokes: sum f_x), [1] = sum f_y
  double* pot;
  double* grad;
  unsigned long long* work;  // evaluated-pair counter (profiling), NULL otherwise
};

// One unit of work of the persistent batched P2P kernel: target block bx of
// cell `cell`, sources [j0, j1), rhs r0 .. r0 + NR - 1.
struct P2PItem {
  int cell, bx, j0, j1, r0;
};

// Fill the P2P arguments of one cell (pointers into its workspace and the
// caller's outputs, image offsets, log-product exponents).
void fill_p2p_args(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, double* pot, double* grad,
                   P2PArgs* a);
// Launch the persistent batched kernel over `nitems` items (device arrays).
cudaError_t launch_p2p_batch(int kernel, int nimg, int nr, bool grad, const P2PArgs* cells, const P2PItem* items,
                             int nitems, int* counter, int grid, cudaStream_t st);
// Blocks of the persistent batched kernel that fit on the GPU at once.
int p2p_batch_grid(int kernel, int nimg, int nr, bool grad);
// Targets per block of the mixed P2P kernels (2 per thread for Laplace/Stokes).
int p2p_targets_per_block(int kernel);
// Sort descriptors of one cell (mixed path): sources, and for modified
// Helmholtz with separate targets also the targets.  off_s / off_t: first
// slot of each set in the concatenated sort arrays.  Returns 1 or 2.
// Set or clear the evaluated-pair counter of a cell's P2P arguments.
inline void set_work_counter(const pfmm_plan* p, char* ws, bool on, P2PArgs* a) {
  a->work = on ? (unsigned long long*)(ws + p->lay.work) : nullptr;
}
int fill_sort_cells(const pfmm_plan* p, char* ws, int64_t ns, int64_t nt, bool self, int64_t off_s, int64_t off_t,
                    SortCell* out);

}  // namespace pfmm
