// Spatial sort of point sets for the mixed-precision near-image P2P.
//
// The points of a cell are ordered along a Morton (Z) curve over a grid of
// bins covering the canonical cell, by a stable radix sort, so that 16
// consecutive sorted points (a subtile) and 128 consecutive points (a tile)
// are close together in the plane.  The P2P then forms coordinate
// differences against the subtile centre in FP32 (one subtraction per
// coordinate instead of a hi/lo pair), and the modified Helmholtz kernel
// skips (target block, source tile, image) triples beyond the K0 cutoff.
// The sort is deterministic: equal keys keep their input order.
#pragma once
#include <cstdint>
#include "pfmm_impl.h"

namespace pfmm {

constexpr int kSubtile = 16;   // sources per subtile (common centre)
constexpr int kBoxTile = 128;  // points per culling box

// One cell's point set.  Inputs are the canonical FP64 coordinates (and
// FP32 strengths for sources); outputs are written in sorted order.
struct SortCell {
  int n;                 // points
  int64_t off;           // first key/value slot of this cell in the concatenated arrays
  const double* xy;      // [2][n] canonical FP64 coordinates (row stride n)
  double x0, y0;         // lower-left corner of the bin grid
  double ibx, iby;       // inverse bin widths
  int nbx, nby;          // bins per axis (<= 256)
  const float* q_in;     // [nq][n] FP32 strengths, NULL for a target set
  int nq;
  float* q_out;          // [nq][n] strengths in sorted order
  float2* rel;           // [n] (x, y) - subtile centre, FP32 (NULL for a target set)
  float4* hl;            // [n] (x_hi, x_lo, y_hi, y_lo) sorted (sources)
  float4* sub;           // [ceil(n/16)] subtile centres (x_hi, x_lo, y_hi, y_lo)
  float2* ext;           // [ceil(n/16)] subtile half extents, outward-rounded
  float4* box;           // [ceil(n/128)] tile boxes (cx, cy, half width, half height), outward-rounded
  int* perm;             // [n] cell-local input index of sorted position p
  double* xy_sorted;     // [2][n] sorted FP64 coordinates (NULL if not needed)
};

// Bin grid for n points in the canonical cell (x in [-(d+|xi|)/2, (d+|xi|)/2],
// y in [-eta/2, eta/2]): about 8 points per bin, at most 256 bins per axis.
void sort_grid(const Geom& g, int n, SortCell* c);

// Scratch bytes for sorting `total` points of `ncell` cells.
size_t sort_scratch_bytes(int64_t total, int ncell);

// Sort every cell of the device descriptor array `cells` (host copy `hcells`
// gives the sizes): keys, radix sort over the concatenated slots, gather.
// scratch: sort_scratch_bytes(total, ncell) bytes, 256-aligned.
cudaError_t sort_cells(const SortCell* cells, const SortCell* hcells, int ncell, int64_t total, char* scratch,
                       cudaStream_t st, int* nlaunch);

// Stable LSD radix sort of n (key, value) pairs on the low `bits` bits of the
// keys, 8 bits per pass.  After an even number of passes the sorted pairs are
// in (ka, va), after an odd number in (kb, vb); *in_b tells which.  hist:
// radix_hist_ints(n) ints of scratch.
int64_t radix_hist_ints(int64_t n);
cudaError_t radix_sort_pairs(uint32_t* ka, int* va, uint32_t* kb, int* vb, int* hist, int64_t n, int bits,
                             cudaStream_t st, bool* in_b, int* nlaunch);
// Exclusive scan of m ints in place by one block of 1024 threads (for m up
// to a few times 1e5).
cudaError_t scan_small(int* a, int m, cudaStream_t st);

}  // namespace pfmm
