// Arguments of the near-image P2P kernels (shared by the single-cell and
// batched launchers).
#pragma once
#include "pfmm_impl.h"

namespace pfmm {

struct P2PArgs {
  Geom g;
  int nt, ns, chunk;
  int64_t os;            // output row stride
  int r0, nrhs;          // rhs group start, total rhs
  const double* trg64;   // [2][nt] canonical
  const float4* src_hl;  // [ns]
  const float* qf;       // [nrhs][ncomp][ns]
  const double* src64;   // [2][ns] (FP64 kernel)
  const double* qc;      // [nrhs][ncomp][ns] (FP64 kernel)
  float beta_f;
  double beta;
  float lgc;             // log2(r^2) shift (Laplace/Stokes, FP64 add-back), see below
  float kimg[kMaxNear];  // per-image scale 2^-e_i of r^2 (exact powers of two)
  const double* mom;     // FP64 moments: mom[r*8+0] = sum q (Stokes: sum f_x), [1] = sum f_y
  double* pot;
  double* grad;
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

}  // namespace pfmm
